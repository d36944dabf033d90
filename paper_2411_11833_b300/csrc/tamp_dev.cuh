// Device-side data layout shared by the host compiler (tamp_api.cu) and the
// kernels (tamp_kernels.cu).  Everything a CTA needs is packed by the host into
// two word arrays -- the scene blob and the problem blob -- that the kernel
// stages into shared memory with one TMA bulk copy each.
#pragma once
#include <cstdint>

namespace tamp {

constexpr int MAXJ = 8;        // joints per arm
constexpr int NB = 5;          // spheres per register batch (arm table padded per link)
constexpr int MAX_NBS = 8;     // spheres per box model
constexpr int MAX_BOX = 32;
constexpr int MAX_OBS = 256;
constexpr int MAX_SPH = 512;   // padded arm sphere table
constexpr int MAX_CFG = 128;   // arm configurations per skeleton (knots included)
constexpr int MAX_D = 1024;

// ---- scene blob (32-bit words) ----------------------------------------------
enum SceneHdr {
  SH_NJ = 0, SH_NSPH, SH_O, SH_OPAD, SH_B, SH_NBS, SH_NSURF, SH_WORDS,
  SH_LINK0 = 8,                 // link_start[0..MAXJ+1]: 10 entries (words 8..17)
  SH_OFF_ARM = 18, SH_OFF_SPH, SH_OFF_OBS, SH_OFF_BOX, SH_OFF_BLOC, SH_OFF_BINIT, SH_OFF_SPHB,
  SH_OFF_SURF,
  SH_OFF_SELF,                  // self-collision masks: word l (l = 0..MAXJ) = the lower links j tested against
                                // link l (bit j); word MAXJ + 1 = the links the held box is tested against
  SH_OFF_OBS2,                  // the obstacles again, two per OBS2_W-word record (broad phase)
  SH_HDR_WORDS = 32
};
// arm section: base frame (12), tool frame (12), then per joint ARM_JW words
// frame = R row-major (9) + t (3)
constexpr int ARM_JW = 8;       // a, d, cos(alpha), sin(alpha), offset, q_lo, q_hi, pad
// sphere table: float4 (x, y, z, r) per padded slot; padding slots sit far away
// with r = -1 (unused).  Per batch of NB slots, a bounding sphere (centre in the
// link frame, radius) for the broad phase.
constexpr float DUMMY_FAR = 1.0e4f;
// obstacles: 20 floats each -- t' = R^T t (3), R row-major (9), half extents (3),
// pad; the 80-byte stride puts the records of 8 consecutive obstacles in
// disjoint shared-memory banks when the lanes of a warp read different ones
constexpr int OBS_W = 20;
// obstacles 2i and 2i + 1 interleaved for the broad phase's paired FP32 math:
// per axis k the R column (R[0k] pair, R[3+k] pair, R[6+k] pair) and -t'_k pair,
// then the half extents (hx, hx', hy, hy', hz, hz', pad, pad); an odd count is
// padded with an obstacle far away that nothing touches
constexpr int OBS2_W = 32;
// box record: half x,y,z, bounding radius of its spheres about its centre,
// init x,y,z,yaw, cos(yaw), sin(yaw), then the half extents (box frame, about
// the centre) of a box that holds every sphere of the model, pad
constexpr int BOX_W = 16;
// box spheres: local (x, y, z, r) per box, and the same at the initial pose in the world
// surface record: cx, cy, yaw, hx, hy, z_top, cos(yaw), sin(yaw)
constexpr int SURF_W = 8;

// ---- problem blob ------------------------------------------------------------
enum ProbHdr {
  PH_D = 0, PH_K, PH_NT, PH_NCON, PH_GOAL_T, PH_NGOAL, PH_OFF_CFG, PH_OFF_ENV, PH_OFF_TERMS,
  PH_OFF_GOAL, PH_OFF_LR, PH_OFF_SAMP, PH_WORDS, PH_NSLOT, PH_OFF_SLOT, PH_NSEG, PH_OFF_SEG,
  PH_GRASP6,                    // 1: grasps are (x, y, z, yaw, roll, pitch)
  PH_NTAB, PH_OFF_TAB,          // configurations with rows in the per-iteration (cos, sin) table: count, list
  PH_HDR_WORDS = 20
};
// Configuration kinds: a Pick's, a Place's, or a knot of the trajectory
// between two of them (MoveFree / MoveHold).
enum CfgKind { CK_PICK = 0, CK_PLACE = 1, CK_KNOT = 2 };
constexpr int CFG_W = 32;
enum CfgField {
  CF_KIND = 0, CF_BOX, CF_QOFF, CF_GOFF, CF_TSRC, CF_SURF, CF_NENV, CF_ENVOFF,
  CF_T_KP, CF_T_KR, CF_T_X, CF_T_CF, CF_T_CP, CF_T_JL, CF_PSRC,
  CF_CP_SRC,                    // placement offset of the CFreePlace spheres this configuration tests (-1: none)
  CF_TX, CF_TY, CF_TZ, CF_TYAW,  // floats: target pose if CF_TSRC < 0, else CF_TZ = surface z + h_z
  CF_PZ,                        // float: z of that placed box
  CF_CP_FIRST, CF_CP_COUNT,     // its spheres [first, first + count)
  CF_CP_T,                      // CFreePlace term index
  CF_T_SLOT,                    // placement slot of the Kin target if CF_TSRC >= 0, else -1
  CF_CP_SLOT,                   // placement slot of CF_CP_SRC (-1: none)
  CF_TCOS, CF_TSIN,             // floats: cos, sin of CF_TYAW
  CF_HOLD,                      // 1: the hand holds box CF_BOX with the grasp at CF_GOFF (Pick, Place, MoveHold knot)
  CF_T_SELF,                    // SelfCollision term index (-1: none)
  CF_TG                         // row of the per-iteration (cos, sin) table (-1: a knot, whose angles
                                // the kernel computes where it needs them)
};
// Motion segments between consecutive Pick/Place configurations (only with
// knots): q offsets of the start and end configurations, of the first knot
// (the knots' q are consecutive), the number of knots, the TrajLength term.
constexpr int SEG_W = 8;
enum SegField { SG_QA = 0, SG_QB, SG_QK, SG_M, SG_T };
// Per iteration the optimisation kernel tabulates, for every particle of its
// tile, (cos, sin) of each configuration's joint angles (plus the joint
// offsets) followed by its grasp yaw (and, with 6-DOF grasps, roll and pitch):
// K x (n_joints + 1 (+ 2)) entries, so that the kinematics, the reverse sweep
// and Kin read them instead of evaluating them.
// The problem blob ends with the sampler's per-component records; the
// optimisation kernel stages only the words before them (PH_OFF_SAMP).
// A Place's CFreePlace spheres are split between the Place and the Pick right
// before it (same box, same environment), which evens the work of their warps.
constexpr int ENV_W = 4;        // box, src (-1 = initial pose, else placement offset), slot, pad
constexpr int SLOT_W = 4;       // placement slot (one per Place): box, placement offset, z (float), pad
constexpr int MAX_SLOT = 16;
constexpr int TERM_W = 4;       // kind, weight (float), tol (float), is_constraint
constexpr int GOAL_W = 4;       // box, src, z (float), pad
constexpr int SAMP_W = 4;       // per component: kind, a (float), b (float), surface
enum SampKind { SK_LINEAR = 0, SK_PLACE_X = 1, SK_PLACE_Y = 2 };
// Proposal-sampler row record (one per Pick/Place action, in action order):
// word 0 kind (0 Pick, 1 Place), word 1 offset of the grasp / placement in the
// particle, words 4.. floats: Pick h_x, h_y, h_z of the box; Place the surface's
// centre x, y, cos yaw, sin yaw, half x, half y.
constexpr int PROW_W = 12;
constexpr int PROP_NF = 48, PROP_NT = 16;   // network inputs, target slots (outputs = 2 * PROP_NT)

enum TermKind {
  TK_KIN_POS = 0, TK_KIN_ROT, TK_GRASP, TK_STABLE, TK_CFREE_HOLD, TK_CFREE_PLACE, TK_JOINT_LIMIT,
  TK_OBJ_DIST, TK_CFREE_TRAJ, TK_TRAJ_LEN, TK_SELF, TK_N
};

// device error word bits
enum ErrBits { ERR_TMA_TIMEOUT = 1, ERR_BAD_BLOB = 2 };

// One problem of a launch (an array of these lives in device memory).
struct ProbDesc {
  const uint32_t* prob; int prob_words;
  const float* x_in;                  // [D][stride]
  float* x_out; float* m; float* v;   // state (may be null in evaluation mode)
  int stride; int P;
  float* out_cost; float* out_terms; uint8_t* out_flags; float* out_grad; int* out_counts;
  int* first_iter;
  unsigned long long* work;           // optional [2]: cuboid / box candidates resolved exactly
  const int* t_dev;                   // if set, the Adam step count before the launch is read here
  int t0;                             // else this one
  int n_steps;
  float gscale;                       // 1/N_b (Eq. 4) or 1
  float beta1, beta2, eps;
  int load_mv;                        // read m, v from memory (else zeros)
  int pad;
  // optional best-satisfying record (all four set or all null): per particle the
  // state with the lowest Eq. 2 cost among the Eq. 3 checks it satisfied
  float* best_x;                      // [D][stride]
  float* best_cost;                   // [stride]; kNoBestCost: none yet
  int* best_iter;                     // [stride]; the check index of best_x, -1: none
  float* stage_x;                     // 2 x [tiles][D][PT] (2 * D * ceil(P / 32) * 32 floats, 16-byte
                                      // aligned): x_t of each tile, by iteration parity
};
// byte-uniform sentinel of best_cost (so that a memset clears it): 0x7f7f7f7f = 3.39e38
constexpr unsigned kNoBestCostBits = 0x7f7f7f7fu;

// One launch of the persistent optimisation kernel: CTAs take work items
// (problem << 20 | tile) from a shared counter until the list is exhausted.
struct LaunchArgs {
  const uint32_t* scene; int scene_words;
  const ProbDesc* probs;
  const uint32_t* items; int n_items;
  int* item_counter;                  // zero before the launch
  int* err;
  int scratch_offset;                 // bytes from the start of dynamic shared memory to the warp scratch
  const int* stop;                    // optional: a non-zero value makes the launch return at once
  int mv_global;                      // 1: Adam moments used in place in global memory (not staged)
  int feat;                           // the optional terms of the launch's problems: 0 or a KernelFeat
  int rec;                            // 1: every problem's best-satisfying record is kept (ProbDesc best_*)
};
// Feature sets of the optimisation kernel's instantiations (0: none of the
// optional terms): SelfCollision alone; 6-DOF grasps; knots with 4-DOF grasps;
// knots with 6-DOF grasps -- each with or without SelfCollision.
enum KernelFeat { FEAT_SELF = 1, FEAT_EXT = 2, FEAT_KNOT = 3, FEAT_KNOT6 = 4, N_FEAT = 5 };
constexpr int ITEM_TILE_BITS = 20;

}  // namespace tamp

namespace tamp {
// the kernels read box records, environment entries and joint records as float4 / int4
static_assert(BOX_W % 4 == 0 && ENV_W == 4 && ARM_JW % 4 == 0, "16-byte records");
}  // namespace tamp
