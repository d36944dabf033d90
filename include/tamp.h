/*
 * tamp.h -- C ABI of the B300 particle-optimisation library (libtamp.so).
 *
 * What it computes: the continuous half of a sequence-then-satisfy TAMP planner
 * (arXiv 2411.11833, "cuTAMP").  A plan skeleton induces a constraint
 * satisfaction problem over continuous parameters (Sec. V); a batch of
 * "particles" -- candidate assignments -- is optimised in parallel by Adam on
 * the batch-mean penalty objective (Eq. 2, Eq. 4, Sec. V-B) and a particle is a
 * solution when every constraint is within its tolerance (Eq. 3).
 *
 * Conventions for every call:
 *   - every function returns a tamp_status and never aborts; on failure the
 *     outputs are left untouched and tamp_last_error() describes the cause;
 *   - geometry is in metres and radians, z up; 4x4 poses are row-major;
 *   - host pointers are owned by the caller and only read/written during the
 *     call; the library owns all device memory it allocates for a scene -- by
 *     cudaMalloc on the scene's device, or from the caller's tamp_allocator --
 *     and gives it back at the latest in tamp_destroy_scene;
 *   - all GPU work of a scene is issued on the stream given at creation, in call
 *     order; calls on one scene must not be made from two threads at once;
 *   - particle arrays are structure-of-arrays: component c of particle i is at
 *     index c * stride + i (stride = number of particles unless stated).
 *
 * Particle layout of a skeleton (tamp_set_skeleton): the actions are walked in
 * order; a Pick adds its grasp (x, y, z, yaw: end-effector pose in the object
 * frame, top-down) and then its arm configuration (n_joints angles); a Place
 * adds its placement (x, y, yaw of the box on the surface; z follows from the
 * surface height) and then its configuration; the goal action adds nothing.
 * This is the paper's stacking of each continuous variable across the batch
 * (Sec. V-B, "Parallelizing on GPUs").
 *
 * Term layout of a skeleton: per action, in order, Pick -> [KIN_POS, KIN_ROT,
 * GRASP, CFREE_HOLD, JOINT_LIMIT]; Place -> [KIN_POS, KIN_ROT, STABLE_PLACE,
 * CFREE_HOLD, CFREE_PLACE, JOINT_LIMIT]; goal -> [OBJ_DIST].  OBJ_DIST is a
 * cost (Eq. 1 objective), every other term a constraint with a tolerance.
 */
#ifndef TAMP_H
#define TAMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TAMP_OK = 0,
  TAMP_ERR_INVALID_ARG = 1,   /* a pointer, size or index is out of range        */
  TAMP_ERR_STATE = 2,         /* call order violated (e.g. optimise before sample) */
  TAMP_ERR_OOM = 3,           /* device allocation failed                         */
  TAMP_ERR_CUDA = 4,          /* a CUDA runtime call failed                        */
  TAMP_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up                */
  TAMP_ERR_DEVICE_CHECK = 6   /* a device-side bounds check fired                  */
} tamp_status;

/* Action kinds (Listing 1; appendix "Actions"). */
enum { TAMP_PICK = 0, TAMP_PLACE = 1, TAMP_GOAL_MIN_OBJ_DIST = 2 };

/* Constraint / cost kinds (appendix "Constraints"; appendix cost listing). */
enum {
  TAMP_TERM_KIN_POS = 0,      /* Kin: ||t_EE - t_target||, m                          */
  TAMP_TERM_KIN_ROT = 1,      /* Kin: geodesic angle between EE and target, rad       */
  TAMP_TERM_GRASP = 2,        /* Grasp: bound distance of the grasp position          */
  TAMP_TERM_STABLE_PLACE = 3, /* StablePlace: footprint corners outside the surface   */
  TAMP_TERM_CFREE_HOLD = 4,   /* CFreeHold: arm + held box penetration depth, m       */
  TAMP_TERM_CFREE_PLACE = 5,  /* CFreePlace: placed box penetration depth, m          */
  TAMP_TERM_JOINT_LIMIT = 6,  /* Motion (limits part): bound distance of q            */
  TAMP_TERM_OBJ_DIST = 7,     /* MinimizeObjDist goal cost: sum of pairwise distances */
  TAMP_TERM_CFREE_TRAJ = 8,   /* CFreeTraj(Hold): penetration depth at a knot, m       */
  TAMP_TERM_TRAJ_LEN = 9,     /* TrajLength cost: joint-space length of a motion, rad  */
  TAMP_TERM_SELF_COLLISION = 10, /* robot self-collision penetration depth, m          */
  TAMP_N_TERM_KINDS = 11
};

typedef struct tamp_scene tamp_scene;   /* opaque, library-owned */

/* Scene Pi = (robot, movable boxes, static cuboids, surfaces) (Sec. III; the
 * appendix's collision representation: spheres for robot and objects,
 * oriented boxes for static obstacles).  All arrays are read during
 * tamp_create_scene only. */
typedef struct {
  int n_joints;                 /* 1..8 revolute joints                                   */
  const double *dh_a, *dh_d, *dh_alpha, *dh_offset;   /* [n_joints], standard DH:
                                   A_i = Rz(q_i + offset_i) Tz(d_i) Tx(a_i) Rx(alpha_i)   */
  const double *q_lo, *q_hi;    /* [n_joints] joint limits                                */
  double base[16];              /* world <- frame 0                                       */
  double tool[16];              /* frame n <- end effector                                */
  int n_spheres;                /* arm collision spheres                                  */
  const int *sphere_link;       /* [n_spheres] frame index 0..n_joints the sphere is on   */
  const double *sphere_xyzr;    /* [n_spheres][4] centre in that frame, radius            */
  int n_boxes;                  /* movable boxes, <= 32                                   */
  const double *box_half;       /* [n_boxes][3] half extents                              */
  const double *box_init;       /* [n_boxes][4] initial centre x, y, z and yaw            */
  int spheres_per_box;          /* spheres per box model, 1..8                            */
  const double *box_spheres;    /* [n_boxes][spheres_per_box][4] centre in box frame, r   */
  int n_obs;                    /* static cuboids, 0..256                                 */
  const double *obs_center;     /* [n_obs][3]                                             */
  const double *obs_rot;        /* [n_obs][3][3] row-major, columns = cuboid axes         */
  const double *obs_half;       /* [n_obs][3]                                             */
  int n_surf;                   /* placement surfaces, >= 1 if the skeleton places        */
  const double *surf;           /* [n_surf][6] centre x, y, yaw, half x, half y, top z    */
} tamp_scene_desc;

/* One skeleton action (Listing 1): Pick(box), Place(box, surface), or the goal
 * MinimizeObjDist over every box the skeleton has placed so far. */
typedef struct {
  int kind;
  int box;
  int surface;
} tamp_action;

/* Weights lambda_c (Eq. 2), tolerances eps_c (Eq. 3) and Adam settings (Sec.
 * V-B).  tamp_default_options fills the appendix's values: weights 1 except
 * kinematic rotation 5 and stable placement 2, goal 0.25; tolerances 5 mm /
 * 0.05 rad (Kin), 1 mm (collisions, containment, grasp bounds), 0 (joint
 * limits); beta1 0.9, beta2 0.999, eps 1e-8; lr 1e-2 (joints, yaws), 3e-3 (m);
 * no knots.  Knots (Listing 1 MoveFree / MoveHold; Sec. VIII: trajectories as
 * knot points): with n_knots > 0 the motion between two consecutive Pick /
 * Place configurations is a trajectory of n_knots knot configurations whose
 * joint positions sit in the particle just before the variables of the action
 * the motion leads to (there is no motion before the first action).  Each
 * knot carries CFreeTraj -- the CFreeHold penetration depth of the arm, plus
 * the held box on a MoveHold (between a Pick and its Place), against the
 * static cuboids and every box not in the hand -- (weight 1, tolerance 1 mm)
 * and its joint limits (Motion); each motion carries the TrajLength cost, the
 * joint-space length of the polyline start, knots, end (weight 0.01: the paper
 * gives none; never a constraint).  Self-collision (the CFree constraints'
 * "does not cause robot self-collisions"; appendix tolerance 0 penetration):
 * with self_collision = 1 every configuration, knots included, carries
 * SelfCollision = sum of max(0, r_a + r_b - ||c_a - c_b||) over the arm's
 * sphere pairs on links i > j + 1 whose spheres do not already overlap at q = 0
 * (such links always touch: the scene's ignore list), plus the held box's
 * spheres against the spheres of links 0..n-2 (not the wrist and the gripper
 * that hold it); weight 1, tolerance 0.  6-DOF grasps (Sec. VIII setup: grasps
 * are "top-down 4-DOF or 6-DOF poses"): with grasp_dof = 6 a grasp is (x, y, z,
 * yaw, roll, pitch) in the box frame, G(g) = Trans(x, y, z) Rz(yaw) Ry(pitch)
 * Rx(roll) Rx(pi) (roll = pitch = 0 is the top-down grasp), Grasp bounds the
 * position by the whole box [-h, h] (any side may be held), and the uniform
 * sampler draws roll and pitch in [-pi/2, pi/2). */
typedef struct {
  float w[TAMP_N_TERM_KINDS];
  float tol[TAMP_N_TERM_KINDS];
  float lr_joint, lr_pos, lr_yaw;
  float beta1, beta2, eps;
  int optimize_grasp;           /* 0: grasps keep their sampled values (lr 0)            */
  int scale_by_batch;           /* 1: gradient of the batch mean (Eq. 4), i.e. / N_b      */
  int lanes;                    /* threads per (particle, configuration): 0 = tuned, 1,2,4,8 */
  int n_knots;                  /* knot configurations per motion between actions (0: none) */
  int self_collision;           /* 1: every configuration carries SelfCollision             */
  int grasp_dof;                /* 4 (0 reads as 4): top-down grasps; 6: 6-DOF grasps         */
  int keep_best;                /* 1: every optimisation launch keeps the best-satisfying
                                   record (tamp_query_best); the stop modes keep it anyway */
} tamp_options;

void tamp_default_options(tamp_options *opt);

/* A caller-supplied device allocator (optional; not part of the paper's
 * method).  alloc returns `bytes` bytes of device memory on `device`, to be
 * used on `stream` (the scene's stream), or NULL when it cannot (the library
 * call then fails with TAMP_ERR_OOM or TAMP_ERR_CUDA); free gives back a block
 * that alloc returned, with the same device and stream.  ctx is passed through
 * unchanged.  Both callbacks are called on the thread that makes the library
 * call, during that call.  A host framework that pools device memory (e.g.
 * PyTorch's caching allocator) can so back every buffer of a scene. */
typedef struct {
  void *(*alloc)(size_t bytes, int device, void *stream, void *ctx);
  void (*free)(void *ptr, int device, void *stream, void *ctx);
  void *ctx;
} tamp_allocator;

/* Copy a scene to the device.  device: CUDA ordinal; stream: a cudaStream_t
 * (NULL = legacy default stream).  allocator: NULL = cudaMalloc / cudaFree;
 * otherwise (copied; alloc and free both set, else TAMP_ERR_INVALID_ARG) every
 * device buffer of the scene, of its problems, graphs and autotuner trials
 * comes from it.  *out receives the handle. */
tamp_status tamp_create_scene(const tamp_scene_desc *desc, int device, void *stream,
                              const tamp_allocator *allocator, tamp_scene **out);
tamp_status tamp_destroy_scene(tamp_scene *scene);

/* Compile a skeleton (Sec. V: con(pi), cost(pi), the particle layout above).
 * Preconditions of the actions are checked (Pick needs an empty hand, Place
 * the box in hand); a violation returns TAMP_ERR_INVALID_ARG.  opt may be NULL
 * (defaults).  *problem_id receives an index valid for the scene's lifetime. */
tamp_status tamp_set_skeleton(tamp_scene *scene, const tamp_action *actions, int n_actions,
                              const tamp_options *opt, int *problem_id);

/* Particle dimension D and number of terms of a compiled skeleton.  term_kinds
 * (may be NULL) receives the kind of every term, in term order. */
tamp_status tamp_problem_info(const tamp_scene *scene, int problem_id, int *D, int *n_terms,
                              int *term_kinds);

/* Sampler flags of tamp_sample_particles (combine with |). */
enum {
  TAMP_SAMPLE_UNIFORM = 0,   /* every component uniform within its bounds                 */
  TAMP_SAMPLE_LEARNED = 1,   /* grasps and placements from the attached proposal network  */
  TAMP_SAMPLE_IK = 2         /* joint configurations by parallel IK on the sampled targets */
};
/* Parameters of the IK configuration sampler: iterations, damping lambda, the
 * largest entry of one step (rad). */
#define TAMP_IK_ITERS 64
#define TAMP_IK_DAMPING 0.05f
#define TAMP_IK_MAX_STEP 0.4f

/* Initialise a batch of n_particles (InitializeParticles, Alg. 1).  Knots,
 * whatever the sampler, are then placed evenly on the joint-space line between
 * their motion's start and end configurations (Sec. VIII).  sampler 0:
 * uniform within bounds (the paper's "Optimization" initialisation, Sec. VIII):
 * component c of particle i takes u = (w >> 8) * 2^-24 where w is the first
 * output word of Philox4x32-10 (Salmon et al., SC'11) with counter (i, c, 0, 0)
 * and key (seed & 0xffffffff, seed >> 32); joints map u onto [q_lo, q_hi],
 * grasp positions onto [-h_x, h_x] x [-h_y, h_y] x [h_z - 0.02, h_z], yaws onto
 * [-pi, pi), a placement's (x, y) onto the surface rectangle in the surface
 * frame.  sampler is a combination of the TAMP_SAMPLE_* flags, applied in
 * this order:
 * TAMP_SAMPLE_LEARNED (learned proposals, Sec. V-A; needs tamp_set_proposal):
 * joint configurations as sampler 0; the attached network maps each Pick /
 * Place row's features (tamp_proposal_rows) to means mu_k and log standard
 * deviations s_k of the row's target slots, and slot k of row r of particle i
 * takes t = mu_k + exp(clamp(s_k, -8, 3)) xi with xi = sqrt(-2 ln u1)
 * cos(2 pi u2), u1 = ((w0 >> 8) + 1) 2^-24, u2 = (w1 >> 8) 2^-24 from the
 * Philox4x32-10 words w0, w1 at counter (i, 16 r + k, 1, 0); positions are
 * clamped to [-1, 1] and mapped back through the target normalisation, yaws
 * are atan2(sin slot, cos slot); without a network the flag returns
 * TAMP_ERR_STATE.
 * TAMP_SAMPLE_IK (the conditional configuration sampler of Sec. VI): every
 * configuration, in skeleton order, gets the joint positions that put the end
 * effector on its Kin target P_box G(g) given the sampled grasp / placement,
 * with one free yaw -- a Pick's grasp yaw, a Place's placement yaw -- solved
 * along: TAMP_IK_ITERS damped-least-squares steps from the uniform q on
 * r = [t* - t_EE ; log(R* R_EE^T)] over (q, yaw), A = [J_q | -d(t*, R*)/dyaw]
 * (J_q the geometric Jacobian; d(t*, R*)/dyaw = [z x (t* - box centre) ; z] for a
 * Place, [0 ; z] for a Pick), step = A^T (A A^T + lambda^2 I)^-1 r scaled to
 * a largest entry <= TAMP_IK_MAX_STEP, q clamped to its limits.
 * Adam state and the iteration counter are reset. */
tamp_status tamp_sample_particles(tamp_scene *scene, int problem_id, int n_particles,
                                  uint64_t seed, int sampler);

/* Subgraph caching (Sec. VI, reusing samples across skeletons): as
 * tamp_sample_particles, except that the particle components of the longest
 * action prefix that problem_id shares with src_problem_id (the same actions
 * in the same order: the same variables, constraints and environment, at the
 * same components) are copied from src_problem_id's current batch -- the
 * sampler's output as long as that batch has not been optimised -- instead of
 * being drawn, and TAMP_SAMPLE_IK solves only the configurations after the
 * prefix (they read the copied grasps and placements).  With no shared prefix
 * this is tamp_sample_particles.  src_problem_id must hold a batch of exactly
 * n_particles when a prefix is shared (else TAMP_ERR_STATE) and differ from
 * problem_id.  *shared_components (host, may be NULL) receives the number of
 * components copied. */
tamp_status tamp_sample_particles_from(tamp_scene *scene, int problem_id, int n_particles, uint64_t seed,
                                       int sampler, int src_problem_id, int *shared_components);

/* For every term of a compiled skeleton (term order, as tamp_problem_info),
 * the index of the action of the skeleton that introduced it (host array of
 * n_terms entries).  Constraint c of the per-constraint counts is the c-th
 * term whose kind is not TAMP_TERM_OBJ_DIST. */
tamp_status tamp_term_actions(const tamp_scene *scene, int problem_id, int *action_index);

/* Load a batch [D][n_particles] (host or device pointer, is_device says which)
 * with optional Adam moments m, v (NULL = zeros) and step count t0. */
tamp_status tamp_set_particles(tamp_scene *scene, int problem_id, int n_particles,
                               const float *x, const float *m, const float *v, int t0,
                               int is_device);

/* Read back the batch state [D][n_particles] to host or device memory (any
 * pointer may be NULL); *t receives the Adam step count.  Synchronises. */
tamp_status tamp_get_particles(tamp_scene *scene, int problem_id, float *x, float *m, float *v,
                               int *t, int is_device);

/* OptimizeParticles (Alg. 1; Sec. V-B): n_steps Adam updates of each listed
 * problem's batch.  At x_t before every update, and once more after the last
 * update, every particle is checked against Eq. 3; the first check index with a
 * satisfying particle is recorded per problem.
 * stop_on_first_satisfying = 0: all n_steps run, asynchronously on the stream.
 * stop_on_first_satisfying = k > 0 (the stopping criterion of Alg. 1 and Sec.
 * V-B): the steps run in chunks of k (the last one shorter), and every chunk
 * after the first one whose checks found a satisfying particle in any listed
 * problem is skipped on the device, without a host round trip; the call then
 * synchronises to read back how many steps ran (tamp_get_particles reports the
 * step count).  The results of the last check (tamp_query_satisfied) are those
 * of the last chunk that ran. */
tamp_status tamp_optimize_steps(tamp_scene *scene, const int *problem_ids, int n_problems,
                                int n_steps, int stop_on_first_satisfying);

/* A CUDA graph of the optimisation loop (OptimizeParticles, Alg. 1; Sec. V-B):
 * n_chunks chunks of steps_per_chunk fused iterations of the listed problems,
 * each chunk followed by a one-thread control kernel that advances the step
 * counts and -- if stop_on_first -- raises a stop flag once any problem has a
 * satisfying particle (Eq. 3, the stopping criterion of Sec. V-B), after which
 * the remaining chunks return at once.  The graph records the problems' batch
 * buffers: it is valid while each batch keeps its size.  Created on a private
 * capture stream; run on the scene's stream. */
typedef struct tamp_graph tamp_graph;
tamp_status tamp_graph_create(tamp_scene *scene, const int *problem_ids, int n_problems, int steps_per_chunk,
                              int n_chunks, int stop_on_first, tamp_graph **out);
/* Replay a graph and wait for it; *steps_run (may be NULL) receives the number
 * of iterations actually run (a multiple of steps_per_chunk). */
tamp_status tamp_graph_run(tamp_graph *graph, int *steps_run);
tamp_status tamp_graph_destroy(tamp_graph *graph);

/* Results of the last check of a problem (IsGoalSatisfied, Alg. 1; Eq. 3; the
 * Eq. 5 per-constraint satisfied counts, in constraint order = term order with
 * the OBJ_DIST term left out).  Host pointers, each may be NULL: mask[P],
 * particles[D][P], cost[P] (Eq. 2 value), counts[n_constraints]; *first_iter is
 * -1 if no check has found a satisfying particle.  Synchronises. */
tamp_status tamp_query_satisfied(tamp_scene *scene, int problem_id, uint8_t *mask,
                                 int *n_satisfied, int *first_iter, float *particles,
                                 float *cost, int *counts);

/* Best satisfying state of each particle (Alg. 1 returns a particle that
 * satisfies Eq. 3; the soft-cost experiments of Sec. VIII and the appendix
 * keep the lowest-cost one).  Every Eq. 3 check of an optimisation launch that
 * keeps the record -- at x_t before each update and after the last -- compares
 * each satisfying particle's Eq. 2 cost with its record and keeps the state if
 * the cost is lower, so a satisfying particle is not lost when later updates
 * move it out of the feasible set (the state tamp_query_satisfied reports
 * after a stop on the first satisfying particle is the one after the chunk's
 * last update).  Launches that keep it: tamp_optimize_steps with
 * stop_on_first_satisfying > 0, graphs created with stop_on_first, and every
 * launch that includes a problem whose options set keep_best (the other
 * problems of such a launch keep theirs too); other launches skip this work
 * (about 1.5% of an iteration).  The record starts empty with each batch
 * (tamp_sample_particles*, tamp_set_particles) and runs across calls and graph
 * replays; tamp_autotune's trial launches leave it alone.  Host pointers, each
 * may be NULL: found[P] (1: the particle satisfied some check), particles[D][P]
 * (the recorded state; unspecified where found is 0), cost[P] (its Eq. 2 cost,
 * +inf where found is 0), iter[P] (the check index, the Adam step count at that
 * check, as first_iter counts; -1 where found is 0); *n_found = number of found
 * particles.  A batch not checked yet is checked once first.  Synchronises.
 * Errors: TAMP_ERR_INVALID_ARG for an unknown problem, TAMP_ERR_STATE without a
 * batch. */
tamp_status tamp_query_best(tamp_scene *scene, int problem_id, uint8_t *found, int *n_found,
                            float *particles, float *cost, int *iter);

/* Evaluate a caller batch on the device without touching the problem's state:
 * x_dev [D][n] (stride n), outputs (device, each may be NULL) cost[n] (Eq. 2),
 * terms[n_terms][n] (unweighted J_c), flags[n] (Eq. 3) and grad[D][n]
 * (dJ/dx of Eq. 2 for each particle, not divided by n). */
tamp_status tamp_eval(tamp_scene *scene, int problem_id, int n, const float *x_dev,
                      float *cost_dev, float *terms_dev, uint8_t *flags_dev, float *grad_dev);

/* tamp_eval for callers that cannot allocate device memory while they run --
 * for example a control loop whose device-memory budget is frozen after
 * start-up, or a host framework that serves every device byte from its own
 * pool and does not let libraries call cudaMalloc.  It evaluates exactly what
 * tamp_eval does, with the same arguments, but never allocates: the launch's
 * work-item list, problem descriptor and work counter live in one static
 * device array of 16.5 KB compiled into the library (each GPU that loads the
 * library keeps its copy until the process exits).
 *   - The first call on a device sets the array up (resolves its address,
 *     writes the work-item list and waits for the device to finish that copy,
 *     so the kernel may then run on any stream).  A set-up that fails returns
 *     TAMP_ERR_CUDA and the next call tries it again.
 *   - Batches are limited to 4096 tiles of 32/L particles (131072 particles at
 *     one lane per particle-configuration); a larger n returns
 *     TAMP_ERR_INVALID_ARG with the limit in tamp_last_error.
 *   - Every call, on any scene, shares the array and leaves its contents in
 *     place; the counter is cleared on the scene's stream at the start of each
 *     call.  Calls whose work overlaps on the GPU (different streams, or
 *     different scenes on one device without ordering) race on the array.
 * The paper has no counterpart: this is an interface convenience. */
tamp_status tamp_eval_static_scratch(tamp_scene *scene, int problem_id, int n, const float *x_dev,
                                     float *cost_dev, float *terms_dev, uint8_t *flags_dev,
                                     float *grad_dev);

/* Work counters of a problem since its batch was last sampled or set:
 * out[0] = (sphere batch, cuboid) pairs and out[1] = (sphere batch, box) pairs
 * that the collision broad phase passed on to the exact test (the exact work is
 * data-dependent; everything else per iteration is fixed by the skeleton).
 * Synchronises.  Not part of the paper's method: performance accounting only. */
tamp_status tamp_work_counters(tamp_scene *scene, int problem_id, uint64_t out[2]);

/* Autotuner of the persistent launch (not part of the paper's method: it only
 * picks how the same work is laid out).  For the listed problems with their
 * current batches, times every launch shape that fits -- lanes L in {1, 2, 4,
 * 8} per (particle, configuration) (32 / L particles per CTA) and W <= 16 warps
 * per CTA (1..8 work items per warp; a configuration is two items) -- with
 * trial_steps fused iterations on scratch copies of the batches (the problems'
 * state is left untouched), three times each in interleaved rounds, and keeps
 * the shape with the best time for later launches of exactly these problems at
 * these batch sizes whose options have lanes = 0.  Outputs (host, each may be
 * NULL): the chosen L, W and its best trial time in ms.  Synchronises. */
tamp_status tamp_autotune(tamp_scene *scene, const int *problem_ids, int n_problems, int trial_steps,
                          int *lanes, int *warps, float *ms);
/* Install a known launch shape for the listed problems at their current batch
 * sizes (e.g. one tamp_autotune found earlier on the same GPU); lanes 0
 * removes the entry.  A shape that does not fit returns TAMP_ERR_INVALID_ARG. */
tamp_status tamp_set_tuning(tamp_scene *scene, const int *problem_ids, int n_problems, int lanes, int warps);

/* Text of the last error on this scene ("" if none); valid until the next call. */
const char *tamp_last_error(const tamp_scene *scene);

/* Measurement utility, not part of the method: times independent FFMA chains
 * filling every SM of `device` on the legacy default stream and returns the
 * achieved FP32 rate (2 FLOP per FFMA) in *tflops and the kernel time in *ms
 * (may be NULL) -- the measured counterpart of the FP32 peak the roofline of
 * the optimisation kernel is quoted against.  Synchronises. */
tamp_status tamp_measure_fp32_peak(int device, double *tflops, double *ms);

/* ---------------------------------------------------------------------------
 * Learned particle proposals (Sec. V-A and Sec. VIII: particles may be seeded
 * from learned samplers instead of uniformly).  The paper leaves the sampler
 * open; this library provides one small conditional density network that runs
 * on the tensor cores:
 *   4 dense layers 48 -> 256 -> 256 -> 256 -> 32, exact GELU between layers;
 *   weights and inter-layer activations BF16, products accumulated in FP32;
 *   output k < 16 is the predicted mean of target k, output 16 + k its log
 *   standard deviation; trained by Adam (beta 0.9 / 0.999, eps 1e-8) on FP32
 *   master weights with the Gaussian negative log-likelihood
 *     L = mean over rows of sum_k mask_k ((y_k - mu_k)^2 exp(-2 s_k) / 2 + s_k).
 * Parameter vector (FP32, tamp_mlp_param_count() entries), in order:
 *   W1 [256][48], b1 [256], W2 [256][256], b2 [256], W3 [256][256], b3 [256],
 *   W4 [32][256], b4 [32]   (row-major; W maps inputs to outputs: z = W a + b).
 * All batch arrays are device pointers, row-major: x [B][48], y and mask
 * [B][16], out [B][32].  Every call is asynchronous on the network's stream
 * unless it says it synchronises.  A tensor-core completion wait that gives up
 * on the device makes the next synchronising call return TAMP_ERR_TIMEOUT.
 * --------------------------------------------------------------------------- */
typedef struct tamp_mlp tamp_mlp;   /* opaque, library-owned */

/* Create a network with zero parameters on `device`, issuing work on `stream`
 * (a cudaStream_t, NULL = legacy default); max_batch bounds the batch of the
 * training calls (activations for max_batch rows are kept on the device). */
tamp_status tamp_mlp_create(int device, void *stream, int max_batch, tamp_mlp **out);
tamp_status tamp_mlp_destroy(tamp_mlp *net);
int tamp_mlp_param_count(void);
/* Host parameter vector in the layout above; set also resets Adam's moments
 * and step count.  Both synchronise. */
tamp_status tamp_mlp_set_params(tamp_mlp *net, const float *host_params, int count);
tamp_status tamp_mlp_get_params(tamp_mlp *net, float *host_params, int count);
/* out = network(x) for B >= 1 rows (any B; no training state is touched). */
tamp_status tamp_mlp_forward(tamp_mlp *net, const float *x_dev, int B, float *out_dev);
/* Gradient of L at the current parameters (1 <= B <= max_batch): grad_dev
 * (device, param_count floats, may be NULL) and *loss (host, may be NULL).
 * The sums over rows are accumulated by floating-point atomic additions, so
 * two calls on the same batch agree to rounding, not bit for bit.
 * Synchronises. */
tamp_status tamp_mlp_gradient(tamp_mlp *net, const float *x_dev, const float *y_dev, const float *mask_dev,
                              int B, float *grad_dev, float *loss);
/* One Adam step on L with learning rate lr (the gradient as tamp_mlp_gradient
 * forms it).  *loss (host, may be NULL) gets the loss before the step; asking
 * for it synchronises. */
tamp_status tamp_mlp_train_step(tamp_mlp *net, const float *x_dev, const float *y_dev, const float *mask_dev,
                                int B, float lr, float *loss);
const char *tamp_mlp_last_error(const tamp_mlp *net);

/* Attach a proposal network to a scene (NULL detaches); tamp_sample_particles
 * with sampler 1 then seeds grasps and placements from it.  The scene does not
 * own the network: keep it alive while it is attached.  Both must be on the
 * same device. */
tamp_status tamp_set_proposal(tamp_scene *scene, tamp_mlp *net);

/* Proposal rows of a skeleton: one per Pick or Place action, in action order
 * (*n_rows receives R).  Features (48 floats per row):
 *   [0:3] the box's half extents; [3:8] its initial pose x, y, z, cos yaw,
 *   sin yaw; [8:15] the surface it is placed on -- a Place's own, for a Pick the
 *   next Place of the same box (zeros if none) -- centre x, y, cos yaw, sin yaw,
 *   half x, half y, top z; [15:17] one-hot Pick / Place; [17] action index /
 *   number of actions; [18] 1 if the skeleton has a goal; [19:27] DH a,
 *   [27:35] DH d, [35:43] DH alpha / (pi/2) of joints 1..8 (zero past the
 *   arm); [43] joints / 8; [44:48] zero.
 * Targets (16 slots, mask 1 where used), normalised so that the sampling
 * bounds map to [-1, 1]:
 *   Pick  slots 0..4: g_x / h_x, g_y / h_y, (g_z - h_z + 0.02) / 0.01 - 1,
 *         cos g_yaw, sin g_yaw;
 *   Place slots 5..8: u / H_x, v / H_y (placement centre in the surface frame
 *         over the surface half sizes), cos p_yaw, sin p_yaw.
 * For training data: x is a host batch [D][n] (stride n); feat [n*R][48],
 * y [n*R][16] and mask [n*R][16] are host arrays (each may be NULL; all NULL
 * only returns R); row i*R + r belongs to particle i, action row r. */
tamp_status tamp_proposal_rows(tamp_scene *scene, int problem_id, int n, const float *x, float *feat,
                               float *y, float *mask, int *n_rows);

#ifdef __cplusplus
}
#endif

#endif /* TAMP_H */
