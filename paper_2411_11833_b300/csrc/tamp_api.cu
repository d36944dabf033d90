// C ABI of libtamp.so: scene and skeleton compilation on the host, device
// buffers, and the launches of the sampler and the fused optimisation kernel.
// The declarations, argument meanings and error behaviour are in include/tamp.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <vector>

#include "tamp.h"
#include "tamp_dev.cuh"

namespace tamp {
cudaError_t launch_optimize(const LaunchArgs& a, int L, int warps, int grid, size_t smem, cudaStream_t st);
cudaError_t optimize_set_smem(int L, size_t smem);
cudaError_t launch_chunk_control(int* t_dev, const int* const* first_iters, int* const* counts, const int* n_counts,
                                 int n_problems, int steps, int stop_on_first, int* stop, int* chunks_run, int last,
                                 cudaStream_t st);
size_t optimize_tile_bytes(int prob_words, int D, int NT, int NSLOT, int NANG, int L, bool mv_global);
size_t optimize_scratch_bytes(int warps);
int optimize_blocks_per_sm(int L, int warps, size_t smem);
cudaError_t launch_sample(const uint32_t* pb, const uint32_t* sc, float* x, float* m, float* v, int stride, int P,
                          int D, uint64_t seed, cudaStream_t st);
int optimize_warps(int K);
cudaError_t launch_sample_proposal(const uint32_t* rows, int R, const float* out, float* x, int stride, int P,
                                   uint64_t seed, cudaStream_t st);
cudaError_t launch_ik(const uint32_t* pb, const uint32_t* sc, float* x, int stride, int P, int iters, float lam,
                      float dmax, const int* chains, int n_chains, int chain_w, int keep, cudaStream_t st);
cudaError_t launch_ffma_probe(float* out, int blocks, int iters, cudaStream_t st);
cudaError_t launch_knots(const uint32_t* pb, float* x, int stride, int P, int n_seg, int nj, int keep,
                         cudaStream_t st);
}  // namespace tamp

tamp_status mlp_forward_on_stream(tamp_mlp* n, const float* x_dev, int B, float* out_dev, cudaStream_t st,
                                  int device);

using namespace tamp;

namespace {

struct Problem {
  int id = -1;
  int D = 0, K = 0, NT = 0, NCON = 0, NSLOT = 0;
  int NANG = 0;       // entries of the kernel's per-iteration (cos, sin) table per particle
  int n_seg = 0;      // motions with knots
  bool self = false;  // configurations carry SelfCollision
  bool grasp6 = false;  // 6-DOF grasps
  std::vector<uint32_t> blob;
  int opt_words = 0;  // leading words of the blob that the optimisation kernel stages
  uint32_t* d_blob = nullptr;
  std::vector<int> term_kinds;
  std::vector<int> term_actions;          // the action that introduced each term
  std::vector<tamp_action> acts;          // the skeleton as given
  std::vector<int> act_off;               // first particle component of each action; [n] = D
  tamp_options opt{};
  // batch state
  int P = 0, cap = 0, t = 0;
  float *d_x = nullptr, *d_m = nullptr, *d_v = nullptr, *d_cost = nullptr;
  uint8_t* d_flags = nullptr;
  int* d_counts = nullptr;
  int* d_first = nullptr;
  unsigned long long* d_work = nullptr;  // [2] broad-phase candidates resolved exactly
  // best-satisfying record of the batch (tamp_query_best) and the kernel's staging of x_t
  float *d_best_x = nullptr, *d_best_cost = nullptr, *d_stage = nullptr;
  int* d_best_iter = nullptr;
  bool has_batch = false, checked = false;
  // learned proposals: one row per Pick/Place action (features, decode record)
  int R = 0;
  std::vector<float> pfeat;               // [R][PROP_NF]
  std::vector<uint32_t> prow;             // [R][PROW_W]
  std::vector<int> prow_box, prow_kind, prow_off, prow_surf;
  uint32_t* d_prow = nullptr;
  float* d_pfeat = nullptr;
  float* d_pout = nullptr;                // [R][2 * PROP_NT]
  // IK sampler: per box its configurations in order ([n_chain][1 + K]: length, indices)
  int n_chain = 0;
  std::vector<int> chains;
  int* d_chains = nullptr;
};

}  // namespace

struct tamp_scene {
  int device = 0;
  cudaStream_t stream = nullptr;
  tamp_allocator alloc{};                 // the caller's device allocator (alloc == NULL: cudaMalloc)
  int nj = 0, S = 0, B = 0, NBS = 0, O = 0, NS = 0;
  std::vector<double> box_half, box_init, surf;
  std::vector<double> dh_a, dh_d, dh_alpha;
  tamp_mlp* proposal = nullptr;           // attached proposal network (not owned)
  // launch shapes chosen by tamp_autotune / tamp_set_tuning, keyed by the
  // sorted (problem id, batch size) list of a launch: lanes L and warps W
  std::map<std::vector<long long>, std::pair<int, int>> tuning;
  std::vector<uint32_t> blob;
  uint32_t* d_blob = nullptr;
  int* d_err = nullptr;
  int* d_scratch_first = nullptr;
  int sm_count = 148;
  // launch tables of the persistent kernel (library-owned, grown on demand)
  ProbDesc* d_descs = nullptr;
  int descs_cap = 0;
  uint32_t* d_items = nullptr;
  int items_cap = 0;
  int* d_item_counter = nullptr;
  // control block of tamp_optimize_steps when it stops on the first satisfying
  // particle (library-owned, grown on demand)
  unsigned char* d_ctl = nullptr;
  size_t ctl_cap = 0;
  std::vector<Problem*> probs;
  std::string err;
};

namespace {

tamp_status fail(tamp_scene* s, tamp_status st, const char* fmt, ...) {
  if (s) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    s->err = buf;
  }
  return st;
}

#define CUDA_TRY(s, call)                                                                 \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail((s), e_ == cudaErrorMemoryAllocation ? TAMP_ERR_OOM : TAMP_ERR_CUDA,    \
                  "%s: %s", #call, cudaGetErrorString(e_));                               \
  } while (0)

inline uint32_t fbits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}
inline void align4(std::vector<uint32_t>& v) {
  while (v.size() % 4) v.push_back(0);
}
inline void push_f(std::vector<uint32_t>& v, double x) { v.push_back(fbits(static_cast<float>(x))); }

// Device memory of a scene: from the caller's allocator when tamp_create_scene
// was given one, else cudaMalloc / cudaFree.
cudaError_t dalloc_raw(tamp_scene* s, void** p, size_t bytes) {
  if (s->alloc.alloc) {
    *p = s->alloc.alloc(bytes, s->device, s->stream, s->alloc.ctx);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}
template <class T>
cudaError_t dalloc(tamp_scene* s, T** p, size_t bytes) {
  void* v = nullptr;
  const cudaError_t e = dalloc_raw(s, &v, bytes);
  *p = static_cast<T*>(v);
  return e;
}
void dfree(tamp_scene* s, void* p) {
  if (!p) return;
  if (s->alloc.alloc) s->alloc.free(p, s->device, s->stream, s->alloc.ctx);
  else cudaFree(p);
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Pack the scene blob (layout in tamp_dev.cuh).
tamp_status build_scene_blob(tamp_scene* s, const tamp_scene_desc* d) {
  const int nj = d->n_joints;
  std::vector<uint32_t>& v = s->blob;
  v.assign(SH_HDR_WORDS, 0);
  // arm
  v[SH_OFF_ARM] = static_cast<uint32_t>(v.size());
  auto push_frame = [&](const double* T) {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) push_f(v, T[4 * i + j]);
    for (int i = 0; i < 3; ++i) push_f(v, T[4 * i + 3]);
  };
  push_frame(d->base);
  push_frame(d->tool);
  for (int j = 0; j < nj; ++j) {
    push_f(v, d->dh_a[j]);
    push_f(v, d->dh_d[j]);
    push_f(v, std::cos(d->dh_alpha[j]));
    push_f(v, std::sin(d->dh_alpha[j]));
    push_f(v, d->dh_offset[j]);
    push_f(v, d->q_lo[j]);
    push_f(v, d->q_hi[j]);
    v.push_back(0);
  }
  align4(v);
  // spheres grouped by link, each group padded to a multiple of SB with far, zero-radius slots
  v[SH_OFF_SPH] = static_cast<uint32_t>(v.size());
  int slot = 0;
  for (int l = 0; l <= nj; ++l) {
    v[SH_LINK0 + l] = static_cast<uint32_t>(slot);
    int cnt = 0;
    for (int i = 0; i < d->n_spheres; ++i)
      if (d->sphere_link[i] == l) {
        for (int c = 0; c < 4; ++c) push_f(v, d->sphere_xyzr[4 * i + c]);
        ++cnt;
      }
    while (cnt % NB) {
      push_f(v, DUMMY_FAR); push_f(v, DUMMY_FAR); push_f(v, DUMMY_FAR); push_f(v, -1.0);
      ++cnt;
    }
    slot += cnt;
  }
  for (int l = nj + 1; l <= MAXJ + 1; ++l) v[SH_LINK0 + l] = static_cast<uint32_t>(slot);
  if (slot > MAX_SPH) return fail(s, TAMP_ERR_INVALID_ARG, "too many arm spheres after padding (%d > %d)", slot, MAX_SPH);
  v[SH_NSPH] = static_cast<uint32_t>(slot);
  align4(v);
  // bounding sphere of every batch of NB slots (link frame), from its real spheres
  {
    const uint32_t base = v[SH_OFF_SPH];
    std::vector<float> bounds;
    for (int b0 = 0; b0 < slot; b0 += NB) {
      double lo[3] = {1e30, 1e30, 1e30}, hi[3] = {-1e30, -1e30, -1e30};
      auto rd = [&](int k, int c) { float f; std::memcpy(&f, &v[base + 4 * k + c], 4); return static_cast<double>(f); };
      int nreal = 0;
      for (int k = b0; k < b0 + NB; ++k)
        if (rd(k, 3) >= 0.0) {
          ++nreal;
          for (int c = 0; c < 3; ++c) { lo[c] = std::min(lo[c], rd(k, c)); hi[c] = std::max(hi[c], rd(k, c)); }
        }
      double cen[3] = {0, 0, 0}, R = -1.0;
      if (nreal) {
        for (int c = 0; c < 3; ++c) cen[c] = 0.5 * (lo[c] + hi[c]);
        for (int k = b0; k < b0 + NB; ++k)
          if (rd(k, 3) >= 0.0) {
            const double dx = rd(k, 0) - cen[0], dy = rd(k, 1) - cen[1], dz = rd(k, 2) - cen[2];
            R = std::max(R, std::sqrt(dx * dx + dy * dy + dz * dz) + rd(k, 3));
          }
        R = R * (1.0 + 1e-5) + 1e-5;  // cover FP32 rounding of the transformed centre
      }
      for (int c = 0; c < 3; ++c) bounds.push_back(static_cast<float>(cen[c]));
      bounds.push_back(static_cast<float>(R));
    }
    v[SH_OFF_SPHB] = static_cast<uint32_t>(v.size());
    for (float f : bounds) v.push_back(fbits(f));
    if (bounds.empty())
      for (int c = 0; c < 4; ++c) v.push_back(0);
    align4(v);
  }
  // obstacles: t' = R^T t, R row-major, half extents, pad (OBS_W words each)
  const int O = d->n_obs;
  v[SH_OFF_OBS] = static_cast<uint32_t>(v.size());
  for (int o = 0; o < O; ++o) {
    const double* Rm = d->obs_rot + 9 * o;
    const double* c = d->obs_center + 3 * o;
    for (int j = 0; j < 3; ++j) push_f(v, Rm[0 + j] * c[0] + Rm[3 + j] * c[1] + Rm[6 + j] * c[2]);
    for (int k = 0; k < 9; ++k) push_f(v, Rm[k]);
    for (int j = 0; j < 3; ++j) push_f(v, d->obs_half[3 * o + j]);
    for (int k = 15; k < OBS_W; ++k) v.push_back(0);
  }
  if (O == 0)
    for (int k = 0; k < OBS_W; ++k) v.push_back(0);
  v[SH_O] = static_cast<uint32_t>(O);
  align4(v);
  // the same obstacles in pairs (broad phase): the values of the records above
  v[SH_OFF_OBS2] = static_cast<uint32_t>(v.size());
  {
    const size_t rec0 = v[SH_OFF_OBS];
    auto word = [&](int o, int k) -> uint32_t {  // word k of obstacle o's record; o == O: far away
      if (o < O) return v[rec0 + static_cast<size_t>(o) * OBS_W + k];
      if (k < 3) return fbits(DUMMY_FAR);
      if (k < 12) return fbits((k - 3) % 4 == 0 ? 1.f : 0.f);  // identity rotation
      return 0;
    };
    auto neg = [](uint32_t w) { return w ^ 0x80000000u; };
    for (int p = 0; 2 * p < std::max(O, 1); ++p) {
      const int a = 2 * p, b = 2 * p + 1;
      for (int ax = 0; ax < 3; ++ax) {
        // R[ax], R[3 + ax], R[6 + ax] (record words 3 + ...), then -t'[ax]
        const uint32_t r[8] = {word(a, 3 + ax), word(b, 3 + ax), word(a, 6 + ax),  word(b, 6 + ax),
                               word(a, 9 + ax), word(b, 9 + ax), neg(word(a, ax)), neg(word(b, ax))};
        v.insert(v.end(), r, r + 8);
      }
      const uint32_t h[8] = {word(a, 12), word(b, 12), word(a, 13), word(b, 13), word(a, 14), word(b, 14), 0, 0};
      v.insert(v.end(), h, h + 8);
    }
  }
  align4(v);
  // boxes
  const int B = d->n_boxes, NBS = d->spheres_per_box;
  v[SH_OFF_BOX] = static_cast<uint32_t>(v.size());
  for (int b = 0; b < B; ++b) {
    const double* h = d->box_half + 3 * b;
    const double* p = d->box_init + 4 * b;
    double rb = 0.0;  // radius about the centre that bounds every sphere of the box model
    for (int e = 0; e < NBS; ++e) {
      const double* l = d->box_spheres + (b * NBS + e) * 4;
      rb = std::max(rb, std::sqrt(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]) + l[3]);
    }
    double hull[3] = {0.0, 0.0, 0.0};  // box-frame half extents holding every (real) sphere
    for (int e = 0; e < NBS; ++e) {
      const double* l = d->box_spheres + (b * NBS + e) * 4;
      if (l[3] < 0.0) continue;
      for (int a = 0; a < 3; ++a) hull[a] = std::max(hull[a], std::fabs(l[a]) + l[3]);
    }
    push_f(v, h[0]); push_f(v, h[1]); push_f(v, h[2]); push_f(v, rb * (1.0 + 1e-5) + 1e-5);
    push_f(v, p[0]); push_f(v, p[1]); push_f(v, p[2]); push_f(v, p[3]);
    push_f(v, std::cos(p[3])); push_f(v, std::sin(p[3]));
    for (int a = 0; a < 3; ++a) push_f(v, hull[a] * (1.0 + 1e-5) + 1e-5);
    for (int k = 13; k < BOX_W; ++k) v.push_back(0);
  }
  align4(v);
  v[SH_OFF_BLOC] = static_cast<uint32_t>(v.size());
  for (int b = 0; b < B; ++b)
    for (int e = 0; e < NBS; ++e)
      for (int c = 0; c < 4; ++c) push_f(v, d->box_spheres[(b * NBS + e) * 4 + c]);
  align4(v);
  v[SH_OFF_BINIT] = static_cast<uint32_t>(v.size());
  for (int b = 0; b < B; ++b) {
    const double* p = d->box_init + 4 * b;
    const double c = std::cos(p[3]), sn = std::sin(p[3]);
    for (int e = 0; e < NBS; ++e) {
      const double* l = d->box_spheres + (b * NBS + e) * 4;
      push_f(v, p[0] + c * l[0] - sn * l[1]);
      push_f(v, p[1] + sn * l[0] + c * l[1]);
      push_f(v, p[2] + l[2]);
      push_f(v, l[3]);
    }
  }
  align4(v);
  v[SH_OFF_SURF] = static_cast<uint32_t>(v.size());
  for (int k = 0; k < d->n_surf; ++k) {
    const double* f = d->surf + 6 * k;
    for (int c = 0; c < 6; ++c) push_f(v, f[c]);
    push_f(v, std::cos(f[2]));
    push_f(v, std::sin(f[2]));
  }
  if (d->n_surf == 0)
    for (int c = 0; c < SURF_W; ++c) v.push_back(0);
  align4(v);
  // self-collision masks: link pairs i > j + 1 whose spheres do not overlap at
  // q = 0 (FP64 kinematics: T_{j+1} = T_j Rz(offset) Tz(d) Tx(a) Rx(alpha)),
  // and the links 0..n-2 for the held box
  {
    auto mul = [](const double* A, const double* B, double* C) {
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
          double acc = 0.0;
          for (int k = 0; k < 4; ++k) acc += A[4 * i + k] * B[4 * k + j];
          C[4 * i + j] = acc;
        }
    };
    std::vector<double> T(static_cast<size_t>(nj + 1) * 16);
    std::copy(d->base, d->base + 16, T.begin());
    for (int j = 0; j < nj; ++j) {
      const double th = d->dh_offset[j], ct = std::cos(th), st = std::sin(th);
      const double ca = std::cos(d->dh_alpha[j]), sa = std::sin(d->dh_alpha[j]);
      const double A[16] = {ct, -st * ca, st * sa, d->dh_a[j] * ct,
                            st, ct * ca, -ct * sa, d->dh_a[j] * st,
                            0.0, sa, ca, d->dh_d[j],
                            0.0, 0.0, 0.0, 1.0};
      mul(&T[16 * j], A, &T[16 * (j + 1)]);
    }
    std::vector<double> c(3 * static_cast<size_t>(d->n_spheres));
    for (int i = 0; i < d->n_spheres; ++i) {
      const double* M = &T[16 * d->sphere_link[i]];
      const double* l = d->sphere_xyzr + 4 * i;
      for (int r = 0; r < 3; ++r) c[3 * i + r] = M[4 * r] * l[0] + M[4 * r + 1] * l[1] + M[4 * r + 2] * l[2] + M[4 * r + 3];
    }
    uint32_t mask[MAXJ + 2] = {0};
    for (int li = 0; li <= nj; ++li)
      for (int lj = 0; lj + 1 < li; ++lj) {
        bool any_i = false, any_j = false, touch = false;
        for (int a = 0; a < d->n_spheres; ++a) {
          if (d->sphere_link[a] != li) continue;
          any_i = true;
          for (int b = 0; b < d->n_spheres; ++b) {
            if (d->sphere_link[b] != lj) continue;
            any_j = true;
            const double dx = c[3 * a] - c[3 * b], dy = c[3 * a + 1] - c[3 * b + 1], dz = c[3 * a + 2] - c[3 * b + 2];
            if (std::sqrt(dx * dx + dy * dy + dz * dz) < d->sphere_xyzr[4 * a + 3] + d->sphere_xyzr[4 * b + 3])
              touch = true;
          }
        }
        if (any_i && any_j && !touch) mask[li] |= 1u << lj;
      }
    for (int lj = 0; lj <= nj - 2; ++lj) mask[MAXJ + 1] |= 1u << lj;
    v[SH_OFF_SELF] = static_cast<uint32_t>(v.size());
    v.insert(v.end(), mask, mask + MAXJ + 2);
  }
  align4(v);
  v[SH_NJ] = static_cast<uint32_t>(nj);
  v[SH_B] = static_cast<uint32_t>(B);
  v[SH_NBS] = static_cast<uint32_t>(NBS);
  v[SH_NSURF] = static_cast<uint32_t>(d->n_surf);
  v[SH_WORDS] = static_cast<uint32_t>(v.size());
  return TAMP_OK;
}

struct PoseSrc {
  int kind = 0;   // 0 = initial pose, 1 = placement variable, 2 = held
  int off = -1;
  int surf = -1;
  int slot = -1;  // placement slot (index of the Place action among the Places)
};

// Walk the skeleton (Listing 1 preconditions / effects) and pack the problem blob.
tamp_status compile_problem(tamp_scene* s, const tamp_action* acts, int n, const tamp_options& opt, Problem& pr) {
  const int nj = s->nj, B = s->B;
  if (opt.grasp_dof != 0 && opt.grasp_dof != 4 && opt.grasp_dof != 6)
    return fail(s, TAMP_ERR_INVALID_ARG, "grasp_dof %d (4 or 6)", opt.grasp_dof);
  const bool g6 = opt.grasp_dof == 6;
  std::vector<PoseSrc> pose(B);
  int held = -1, held_g = -1;
  int off = 0;
  struct Cfg {
    int kind, box, qo, go, tsrc, surf, ai;
    int hold = 1;                   // the hand holds `box` with the grasp at `go`
    int t_self = -1;                // SelfCollision term
    int t_slot = -1, cp_slot = -1;  // placement slots of the Kin target and of the CFreePlace box
    std::vector<std::pair<int, PoseSrc>> env;
    int t_kp, t_kr, t_x, t_cf, t_cp, t_jl;
    float tx, ty, tz, tyaw, pz;
    int cp_src = -1, cp_first = 0, cp_count = 0, cp_t = -1;
    float cp_z = 0.f;
  };
  std::vector<Cfg> cfgs;
  struct Seg { int qa, qb, qk, m, t; };   // motion: start / end q offsets, first knot q offset, knots, term
  std::vector<Seg> segs;
  struct Term { int kind, ai; };
  std::vector<Term> terms;
  int cur_ai = 0;
  std::vector<int> comp_kind;  // 0 q, 1 grasp pos, 2 grasp yaw, 3 place pos, 4 place yaw
  struct Samp { int kind; float a, b; int surf; };
  std::vector<Samp> samp;
  int goal_t = -1;
  std::vector<std::pair<int, PoseSrc>> goal;
  struct Slot { int box, off; float z; };
  std::vector<Slot> slots;
  auto add_term = [&](int kind) {
    terms.push_back({kind, cur_ai});
    return static_cast<int>(terms.size()) - 1;
  };
  pr.act_off.assign(static_cast<size_t>(n) + 1, 0);
  for (int ai = 0; ai < n; ++ai) {
    cur_ai = ai;
    pr.act_off[ai] = off;
    const int kind = acts[ai].kind, b = acts[ai].box, sf = acts[ai].surface;
    if (kind == TAMP_PICK || kind == TAMP_PLACE) {
      if (b < 0 || b >= B) return fail(s, TAMP_ERR_INVALID_ARG, "action %d: box %d out of range", ai, b);
      // the motion from the previous configuration into this action's (Listing 1
      // MoveFree / MoveHold): n_knots knots, their q before this action's variables
      if (opt.n_knots > 0 && !cfgs.empty()) {
        int prev = static_cast<int>(cfgs.size()) - 1;
        while (cfgs[prev].kind == CK_KNOT) --prev;
        Seg sg{cfgs[prev].qo, -1, off, opt.n_knots, -1};
        for (int j = 0; j < opt.n_knots; ++j) {
          Cfg c{};
          c.kind = CK_KNOT; c.box = held; c.hold = held >= 0 ? 1 : 0; c.go = held >= 0 ? held_g : 0; c.ai = ai;
          c.qo = off;
          off += nj;
          for (int d = 0; d < nj; ++d) {
            samp.push_back({SK_LINEAR, 0.f, 0.f, 0});
            comp_kind.push_back(0);
          }
          for (int jb = 0; jb < B; ++jb)
            if (jb != held) c.env.push_back({jb, pose[jb]});
          c.tsrc = -1; c.surf = -1;
          c.t_cf = add_term(TK_CFREE_TRAJ); c.t_jl = add_term(TK_JOINT_LIMIT);
          c.t_self = opt.self_collision ? add_term(TK_SELF) : -1;
          c.t_kp = c.t_kr = c.t_x = c.t_cf;  // never read for a knot
          c.t_cp = -1;
          cfgs.push_back(c);
        }
        sg.t = add_term(TK_TRAJ_LEN);
        segs.push_back(sg);
      }
    }
    if (kind == TAMP_PICK) {
      if (held >= 0) return fail(s, TAMP_ERR_INVALID_ARG, "action %d: Pick while holding box %d", ai, held);
      Cfg c{};
      c.kind = 0; c.box = b; c.go = off; c.ai = ai;
      const double* h = &s->box_half[3 * b];
      samp.push_back({SK_LINEAR, static_cast<float>(-h[0]), static_cast<float>(h[0]), 0});
      samp.push_back({SK_LINEAR, static_cast<float>(-h[1]), static_cast<float>(h[1]), 0});
      if (g6)  // a 6-DOF grasp may hold any side: the whole box
        samp.push_back({SK_LINEAR, static_cast<float>(-h[2]), static_cast<float>(h[2]), 0});
      else
        samp.push_back({SK_LINEAR, static_cast<float>(h[2] - 0.02), static_cast<float>(h[2]), 0});
      samp.push_back({SK_LINEAR, static_cast<float>(-M_PI), static_cast<float>(M_PI), 0});
      comp_kind.insert(comp_kind.end(), {1, 1, 1, 2});
      if (g6) {  // roll, pitch in [-pi/2, pi/2): from above to the side
        samp.push_back({SK_LINEAR, static_cast<float>(-M_PI / 2), static_cast<float>(M_PI / 2), 0});
        samp.push_back({SK_LINEAR, static_cast<float>(-M_PI / 2), static_cast<float>(M_PI / 2), 0});
        comp_kind.insert(comp_kind.end(), {2, 2});
      }
      off += g6 ? 6 : 4;
      c.qo = off;
      off += nj;
      for (int j = 0; j < B; ++j)
        if (j != b) c.env.push_back({j, pose[j]});
      if (pose[b].kind == 1) {
        c.tsrc = pose[b].off;
        c.t_slot = pose[b].slot;
        c.tz = static_cast<float>(s->surf[6 * pose[b].surf + 5] + s->box_half[3 * b + 2]);
      } else {
        c.tsrc = -1;
        const double* p = &s->box_init[4 * b];
        c.tx = static_cast<float>(p[0]); c.ty = static_cast<float>(p[1]);
        c.tz = static_cast<float>(p[2]); c.tyaw = static_cast<float>(p[3]);
      }
      c.surf = -1;
      c.t_kp = add_term(TK_KIN_POS); c.t_kr = add_term(TK_KIN_ROT); c.t_x = add_term(TK_GRASP);
      c.t_cf = add_term(TK_CFREE_HOLD); c.t_cp = -1; c.t_jl = add_term(TK_JOINT_LIMIT);
      c.t_self = opt.self_collision ? add_term(TK_SELF) : -1;
      cfgs.push_back(c);
      held = b; held_g = c.go;
      pose[b].kind = 2;
    } else if (kind == TAMP_PLACE) {
      if (held != b) return fail(s, TAMP_ERR_INVALID_ARG, "action %d: Place of box %d that is not held", ai, b);
      if (sf < 0 || sf >= s->NS) return fail(s, TAMP_ERR_INVALID_ARG, "action %d: surface %d out of range", ai, sf);
      Cfg c{};
      c.kind = 1; c.box = b; c.go = held_g; c.surf = sf; c.ai = ai;
      const int po = off;
      samp.push_back({SK_PLACE_X, 0.f, 0.f, sf});
      samp.push_back({SK_PLACE_Y, 0.f, 0.f, sf});
      samp.push_back({SK_LINEAR, static_cast<float>(-M_PI), static_cast<float>(M_PI), 0});
      comp_kind.insert(comp_kind.end(), {3, 3, 4});
      off += 3;
      c.qo = off;
      off += nj;
      for (int j = 0; j < B; ++j)
        if (j != b) c.env.push_back({j, pose[j]});
      c.tsrc = po;
      c.t_slot = static_cast<int>(slots.size());
      c.tz = static_cast<float>(s->surf[6 * sf + 5] + s->box_half[3 * b + 2]);
      c.pz = c.tz;
      c.t_kp = add_term(TK_KIN_POS); c.t_kr = add_term(TK_KIN_ROT); c.t_x = add_term(TK_STABLE);
      c.t_cf = add_term(TK_CFREE_HOLD); c.t_cp = add_term(TK_CFREE_PLACE); c.t_jl = add_term(TK_JOINT_LIMIT);
      c.t_self = opt.self_collision ? add_term(TK_SELF) : -1;
      cfgs.push_back(c);
      pose[b].kind = 1; pose[b].off = po; pose[b].surf = sf;
      pose[b].slot = static_cast<int>(slots.size());
      slots.push_back({b, po, static_cast<float>(s->surf[6 * sf + 5] + s->box_half[3 * b + 2])});
      held = -1; held_g = -1;
    } else if (kind == TAMP_GOAL_MIN_OBJ_DIST) {
      goal.clear();
      for (int j = 0; j < B; ++j)
        if (pose[j].kind == 1) goal.push_back({j, pose[j]});
      goal_t = add_term(TK_OBJ_DIST);
    } else {
      return fail(s, TAMP_ERR_INVALID_ARG, "action %d: unknown kind %d", ai, kind);
    }
    // q of the new configuration is sampled uniformly within the joint limits
    if (kind == TAMP_PICK || kind == TAMP_PLACE) {
      for (int j = 0; j < nj; ++j) {
        samp.push_back({SK_LINEAR, 0.f, 0.f, 0});
        comp_kind.push_back(0);
      }
    }
  }
  if (cfgs.empty()) return fail(s, TAMP_ERR_INVALID_ARG, "skeleton has no Pick/Place action");
  // each motion ends at the configuration right after its knots
  for (Seg& sg : segs)
    for (size_t k = 0; k < cfgs.size(); ++k)
      if (cfgs[k].kind != CK_KNOT && cfgs[k].qo > sg.qk) {
        sg.qb = cfgs[k].qo;
        break;
      }
  // CFreePlace of a Place: first half of the box's spheres on the preceding Pick
  // (the hand holds one box, so that Pick is the configuration right before),
  // second half on the Place itself
  for (size_t i = 0; i < cfgs.size(); ++i) {
    Cfg& c = cfgs[i];
    if (c.kind != 1) continue;
    const int half = (i > 0 && cfgs[i - 1].kind == 0 && cfgs[i - 1].box == c.box) ? s->NBS / 2 : 0;
    c.cp_src = c.tsrc; c.cp_z = c.pz; c.cp_t = c.t_cp; c.cp_first = half; c.cp_count = s->NBS - half;
    c.cp_slot = c.t_slot;
    if (half > 0) {
      Cfg& pk = cfgs[i - 1];
      pk.cp_src = c.tsrc; pk.cp_z = c.pz; pk.cp_t = c.t_cp; pk.cp_first = 0; pk.cp_count = half;
      pk.cp_slot = c.t_slot;
    }
  }
  if (static_cast<int>(cfgs.size()) > MAX_CFG) return fail(s, TAMP_ERR_INVALID_ARG, "too many configurations");
  if (off > MAX_D) return fail(s, TAMP_ERR_INVALID_ARG, "particle dimension %d exceeds %d", off, MAX_D);
  if (static_cast<int>(slots.size()) > MAX_SLOT) return fail(s, TAMP_ERR_INVALID_ARG, "too many Place actions");
  pr.D = off;
  pr.act_off[n] = off;
  pr.acts.assign(acts, acts + n);
  pr.K = static_cast<int>(cfgs.size());
  // learned-proposal rows: features of what each Pick/Place acts on, and the
  // record the sampler decodes with (Sec. V-A; the layouts are in tamp.h)
  bool has_goal = false;
  for (int ai = 0; ai < n; ++ai) has_goal = has_goal || acts[ai].kind == TAMP_GOAL_MIN_OBJ_DIST;
  // the IK sampler's chains: each box's configurations, in skeleton order
  {
    std::vector<int> box_chain(B, -1);
    std::vector<std::vector<int>> ch;
    for (int k = 0; k < static_cast<int>(cfgs.size()); ++k) {
      if (cfgs[k].kind == CK_KNOT) continue;  // knots are interpolated, not solved
      const int b = cfgs[k].box;
      if (box_chain[b] < 0) {
        box_chain[b] = static_cast<int>(ch.size());
        ch.emplace_back();
      }
      ch[box_chain[b]].push_back(k);
    }
    const int w = 1 + static_cast<int>(cfgs.size());
    pr.n_chain = static_cast<int>(ch.size());
    pr.chains.assign(static_cast<size_t>(pr.n_chain) * w, 0);
    for (int c = 0; c < pr.n_chain; ++c) {
      pr.chains[static_cast<size_t>(c) * w] = static_cast<int>(ch[c].size());
      for (size_t e = 0; e < ch[c].size(); ++e) pr.chains[static_cast<size_t>(c) * w + 1 + e] = ch[c][e];
    }
  }
  std::vector<int> acfg;  // the Pick / Place configurations (one proposal row each)
  for (size_t k = 0; k < cfgs.size(); ++k)
    if (cfgs[k].kind != CK_KNOT) acfg.push_back(static_cast<int>(k));
  pr.R = static_cast<int>(acfg.size());
  pr.pfeat.assign(static_cast<size_t>(pr.R) * PROP_NF, 0.f);
  pr.prow.assign(static_cast<size_t>(pr.R) * PROW_W, 0u);
  pr.prow_box.clear(); pr.prow_kind.clear(); pr.prow_off.clear(); pr.prow_surf.clear();
  for (int r = 0; r < pr.R; ++r) {
    const Cfg& c = cfgs[acfg[r]];
    int sf = c.surf;
    if (c.kind == 0) {
      sf = -1;
      for (int aj = c.ai + 1; aj < n && sf < 0; ++aj)
        if (acts[aj].kind == TAMP_PLACE && acts[aj].box == c.box) sf = acts[aj].surface;
    }
    const int poff = c.kind == 0 ? c.go : c.tsrc;
    pr.prow_box.push_back(c.box); pr.prow_kind.push_back(c.kind);
    pr.prow_off.push_back(poff); pr.prow_surf.push_back(sf);
    float* f = &pr.pfeat[static_cast<size_t>(r) * PROP_NF];
    const double* h = &s->box_half[3 * c.box];
    const double* p0 = &s->box_init[4 * c.box];
    f[0] = static_cast<float>(h[0]); f[1] = static_cast<float>(h[1]); f[2] = static_cast<float>(h[2]);
    f[3] = static_cast<float>(p0[0]); f[4] = static_cast<float>(p0[1]); f[5] = static_cast<float>(p0[2]);
    f[6] = static_cast<float>(std::cos(p0[3])); f[7] = static_cast<float>(std::sin(p0[3]));
    if (sf >= 0) {
      const double* q = &s->surf[6 * sf];
      f[8] = static_cast<float>(q[0]); f[9] = static_cast<float>(q[1]);
      f[10] = static_cast<float>(std::cos(q[2])); f[11] = static_cast<float>(std::sin(q[2]));
      f[12] = static_cast<float>(q[3]); f[13] = static_cast<float>(q[4]); f[14] = static_cast<float>(q[5]);
    }
    f[15 + c.kind] = 1.f;
    f[17] = static_cast<float>(static_cast<double>(c.ai) / n);
    f[18] = has_goal ? 1.f : 0.f;
    for (int j = 0; j < nj; ++j) {
      f[19 + j] = static_cast<float>(s->dh_a[j]);
      f[27 + j] = static_cast<float>(s->dh_d[j]);
      f[35 + j] = static_cast<float>(s->dh_alpha[j] / (M_PI / 2));
    }
    f[43] = static_cast<float>(nj / 8.0);
    uint32_t* w = &pr.prow[static_cast<size_t>(r) * PROW_W];
    w[0] = static_cast<uint32_t>(c.kind);
    w[1] = static_cast<uint32_t>(poff);
    float* wf = reinterpret_cast<float*>(w + 4);
    if (c.kind == 0) {
      wf[0] = f[0]; wf[1] = f[1]; wf[2] = f[2];
    } else {
      const double* q = &s->surf[6 * sf];
      wf[0] = static_cast<float>(q[0]); wf[1] = static_cast<float>(q[1]);
      wf[2] = static_cast<float>(std::cos(q[2])); wf[3] = static_cast<float>(std::sin(q[2]));
      wf[4] = static_cast<float>(q[3]); wf[5] = static_cast<float>(q[4]);
    }
  }
  pr.NT = static_cast<int>(terms.size());
  // pack
  std::vector<uint32_t>& v = pr.blob;
  v.assign(PH_HDR_WORDS, 0);
  v[PH_OFF_CFG] = static_cast<uint32_t>(v.size());
  int env_count = 0, n_tab = 0;
  for (const Cfg& c : cfgs) {
    uint32_t rec[CFG_W] = {0};
    // knots have no row in the kernel's table: with several knots per motion
    // the table would crowd the particle tile out of shared memory
    rec[CF_TG] = c.kind == CK_KNOT ? static_cast<uint32_t>(-1) : static_cast<uint32_t>(n_tab++);
    rec[CF_KIND] = c.kind; rec[CF_BOX] = c.box; rec[CF_QOFF] = c.qo; rec[CF_GOFF] = c.go;
    rec[CF_TSRC] = static_cast<uint32_t>(c.tsrc); rec[CF_SURF] = static_cast<uint32_t>(c.surf);
    rec[CF_NENV] = static_cast<uint32_t>(c.env.size()); rec[CF_ENVOFF] = static_cast<uint32_t>(env_count);
    rec[CF_T_KP] = c.t_kp; rec[CF_T_KR] = c.t_kr; rec[CF_T_X] = c.t_x; rec[CF_T_CF] = c.t_cf;
    rec[CF_T_CP] = static_cast<uint32_t>(c.t_cp); rec[CF_T_JL] = c.t_jl;
    rec[CF_PSRC] = static_cast<uint32_t>(c.tsrc);
    rec[CF_TX] = fbits(c.tx); rec[CF_TY] = fbits(c.ty); rec[CF_TZ] = fbits(c.tz); rec[CF_TYAW] = fbits(c.tyaw);
    rec[CF_PZ] = fbits(c.cp_z);
    rec[CF_CP_SRC] = static_cast<uint32_t>(c.cp_src);
    rec[CF_CP_FIRST] = static_cast<uint32_t>(c.cp_first);
    rec[CF_CP_COUNT] = static_cast<uint32_t>(c.cp_count);
    rec[CF_CP_T] = static_cast<uint32_t>(c.cp_t);
    rec[CF_T_SLOT] = static_cast<uint32_t>(c.t_slot);
    rec[CF_CP_SLOT] = static_cast<uint32_t>(c.cp_slot);
    rec[CF_TCOS] = fbits(static_cast<float>(std::cos(static_cast<double>(c.tyaw))));
    rec[CF_TSIN] = fbits(static_cast<float>(std::sin(static_cast<double>(c.tyaw))));
    rec[CF_HOLD] = static_cast<uint32_t>(c.hold);
    rec[CF_T_SELF] = static_cast<uint32_t>(c.t_self);
    v.insert(v.end(), rec, rec + CFG_W);
    env_count += static_cast<int>(c.env.size());
  }
  align4(v);
  v[PH_OFF_ENV] = static_cast<uint32_t>(v.size());
  for (const Cfg& c : cfgs)
    for (const auto& e : c.env) {
      const PoseSrc& ps = e.second;
      v.push_back(static_cast<uint32_t>(e.first));
      if (ps.kind == 1) {
        v.push_back(static_cast<uint32_t>(ps.off));
        v.push_back(static_cast<uint32_t>(ps.slot));
      } else {
        v.push_back(static_cast<uint32_t>(-1));
        v.push_back(static_cast<uint32_t>(-1));
      }
      v.push_back(0);
    }
  if (env_count == 0)
    for (int i = 0; i < ENV_W; ++i) v.push_back(0);
  align4(v);
  v[PH_OFF_TERMS] = static_cast<uint32_t>(v.size());
  int ncon = 0;
  pr.term_kinds.clear();
  pr.term_actions.clear();
  for (const Term& t : terms) {
    pr.term_actions.push_back(t.ai);
    v.push_back(static_cast<uint32_t>(t.kind));
    v.push_back(fbits(opt.w[t.kind]));
    v.push_back(fbits(opt.tol[t.kind]));
    const bool cost = t.kind == TK_OBJ_DIST || t.kind == TK_TRAJ_LEN;  // costs never constrain (Eq. 3)
    v.push_back(cost ? static_cast<uint32_t>(-1) : static_cast<uint32_t>(ncon++));
    pr.term_kinds.push_back(t.kind);
  }
  pr.NCON = ncon;
  align4(v);
  v[PH_OFF_GOAL] = static_cast<uint32_t>(v.size());
  for (const auto& g : goal) {
    v.push_back(static_cast<uint32_t>(g.first));
    v.push_back(static_cast<uint32_t>(g.second.off));
    v.push_back(fbits(static_cast<float>(s->surf[6 * g.second.surf + 5] + s->box_half[3 * g.first + 2])));
    v.push_back(0);
  }
  if (goal.empty())
    for (int i = 0; i < GOAL_W; ++i) v.push_back(0);
  align4(v);
  v[PH_OFF_LR] = static_cast<uint32_t>(v.size());
  for (int ck : comp_kind) {
    float lr = 0.f;
    switch (ck) {
      case 0: lr = opt.lr_joint; break;
      case 1: lr = opt.optimize_grasp ? opt.lr_pos : 0.f; break;
      case 2: lr = opt.optimize_grasp ? opt.lr_yaw : 0.f; break;
      case 3: lr = opt.lr_pos; break;
      case 4: lr = opt.lr_yaw; break;
    }
    v.push_back(fbits(lr));
  }
  align4(v);
  v[PH_OFF_SLOT] = static_cast<uint32_t>(v.size());
  for (const Slot& sl : slots) {
    v.push_back(static_cast<uint32_t>(sl.box));
    v.push_back(static_cast<uint32_t>(sl.off));
    v.push_back(fbits(sl.z));
    v.push_back(0);
  }
  if (slots.empty())
    for (int i = 0; i < SLOT_W; ++i) v.push_back(0);
  align4(v);
  v[PH_OFF_SEG] = static_cast<uint32_t>(v.size());
  v[PH_NSEG] = static_cast<uint32_t>(segs.size());
  pr.n_seg = static_cast<int>(segs.size());
  pr.self = opt.self_collision != 0;
  for (const Seg& sg : segs) {
    const uint32_t rec[SEG_W] = {static_cast<uint32_t>(sg.qa), static_cast<uint32_t>(sg.qb),
                                 static_cast<uint32_t>(sg.qk), static_cast<uint32_t>(sg.m),
                                 static_cast<uint32_t>(sg.t), 0, 0, 0};
    v.insert(v.end(), rec, rec + SEG_W);
  }
  align4(v);
  v[PH_OFF_TAB] = static_cast<uint32_t>(v.size());
  v[PH_NTAB] = static_cast<uint32_t>(n_tab);
  for (int k = 0; k < pr.K; ++k)
    if (cfgs[k].kind != CK_KNOT) v.push_back(static_cast<uint32_t>(k));
  align4(v);
  // the sampler's records last: the optimisation kernel stages the words before them
  v[PH_OFF_SAMP] = static_cast<uint32_t>(v.size());
  pr.opt_words = static_cast<int>(v.size());
  for (const Cfg& c : cfgs)
    for (int j = 0; j < nj; ++j) {
      // q ~ U[q_lo, q_hi]: bounds from the scene blob's joint records
      const float* jr = reinterpret_cast<const float*>(&s->blob[s->blob[SH_OFF_ARM] + 24 + j * ARM_JW]);
      samp[c.qo + j] = {SK_LINEAR, jr[5], jr[6], 0};
    }
  for (const Samp& sp : samp) {
    v.push_back(static_cast<uint32_t>(sp.kind));
    v.push_back(fbits(sp.a));
    v.push_back(fbits(sp.b));
    v.push_back(static_cast<uint32_t>(sp.surf));
  }
  align4(v);
  pr.NANG = n_tab * (nj + 1 + (g6 ? 2 : 0));
  pr.grasp6 = g6;
  pr.NSLOT = static_cast<int>(slots.size());
  v[PH_NSLOT] = static_cast<uint32_t>(pr.NSLOT);
  v[PH_D] = pr.D; v[PH_K] = pr.K; v[PH_NT] = pr.NT; v[PH_NCON] = pr.NCON;
  v[PH_GOAL_T] = static_cast<uint32_t>(goal_t); v[PH_NGOAL] = static_cast<uint32_t>(goal.size());
  v[PH_GRASP6] = g6 ? 1u : 0u;
  v[PH_WORDS] = static_cast<uint32_t>(v.size());
  return TAMP_OK;
}

// dynamic shared memory of one CTA, below the 227 KB opt-in limit with room for
// the kernel's static shared variables
constexpr size_t kMaxDynSmem = 227 * 1024 - 256;

// Threads per (particle, configuration) when neither the options nor a tuned
// shape say otherwise.  More lanes split each configuration's environment
// (shorter critical path, more CTAs for small batches) but repeat its
// kinematics; one lane keeps 32 particles per CTA, which is fastest as soon as
// the batch gives every SM a tile or more (tamp_autotune measures it).
int preferred_lanes(int requested, long total_particles) {
  if (requested == 1 || requested == 2 || requested == 4 || requested == 8) return requested;
  return total_particles >= 148L * 16 ? 1 : (total_particles >= 148L * 8 ? 2 : 4);
}

// The kernel instantiation for problems that need knots, 6-DOF grasps and
// self-collision (any of them): the smallest feature set that holds them.
int feat_of(bool knots, bool g6, bool self) {
  if (knots) return g6 ? FEAT_KNOT6 : FEAT_KNOT;
  if (g6) return FEAT_EXT;
  return self ? FEAT_SELF : 0;
}
int problem_feat(const Problem& pr) { return feat_of(pr.n_seg > 0, pr.grasp6, pr.self); }

void free_batch(tamp_scene* s, Problem& pr) {
  dfree(s, pr.d_x); dfree(s, pr.d_m); dfree(s, pr.d_v); dfree(s, pr.d_cost);
  dfree(s, pr.d_flags); dfree(s, pr.d_counts); dfree(s, pr.d_first); dfree(s, pr.d_work);
  dfree(s, pr.d_best_x); dfree(s, pr.d_best_cost); dfree(s, pr.d_stage); dfree(s, pr.d_best_iter);
  pr.d_x = pr.d_m = pr.d_v = pr.d_cost = nullptr;
  pr.d_flags = nullptr; pr.d_counts = nullptr; pr.d_first = nullptr; pr.d_work = nullptr;
  pr.d_best_x = pr.d_best_cost = pr.d_stage = nullptr; pr.d_best_iter = nullptr;
  pr.cap = 0;
}

tamp_status ensure_batch(tamp_scene* s, Problem& pr, int P) {
  if (P > pr.cap) {
    free_batch(s, pr);
    const size_t n = static_cast<size_t>(pr.D) * P;
    CUDA_TRY(s, dalloc(s, &pr.d_x, n * 4));
    CUDA_TRY(s, dalloc(s, &pr.d_m, n * 4));
    CUDA_TRY(s, dalloc(s, &pr.d_v, n * 4));
    CUDA_TRY(s, dalloc(s, &pr.d_cost, static_cast<size_t>(P) * 4));
    CUDA_TRY(s, dalloc(s, &pr.d_flags, static_cast<size_t>(P)));
    CUDA_TRY(s, dalloc(s, &pr.d_counts, static_cast<size_t>(std::max(pr.NCON, 1)) * 4));
    CUDA_TRY(s, dalloc(s, &pr.d_first, 4));
    CUDA_TRY(s, dalloc(s, &pr.d_work, 2 * sizeof(unsigned long long)));
    CUDA_TRY(s, dalloc(s, &pr.d_best_x, n * 4));
    CUDA_TRY(s, dalloc(s, &pr.d_stage, 2 * static_cast<size_t>(pr.D) * ((P + 31) & ~31) * 4));
    CUDA_TRY(s, dalloc(s, &pr.d_best_cost, static_cast<size_t>(P) * 4));
    CUDA_TRY(s, dalloc(s, &pr.d_best_iter, static_cast<size_t>(P) * 4));
    pr.cap = P;
  }
  CUDA_TRY(s, cudaMemsetAsync(pr.d_work, 0, 2 * sizeof(unsigned long long), s->stream));
  // a new batch starts with no best-satisfying record: cost kNoBestCostBits, check index -1
  CUDA_TRY(s, cudaMemsetAsync(pr.d_best_cost, kNoBestCostBits & 0xff, static_cast<size_t>(P) * 4, s->stream));
  CUDA_TRY(s, cudaMemsetAsync(pr.d_best_iter, 0xff, static_cast<size_t>(P) * 4, s->stream));
  pr.P = P;
  const int big = INT_MAX;
  CUDA_TRY(s, cudaMemcpyAsync(pr.d_first, &big, 4, cudaMemcpyHostToDevice, s->stream));
  pr.t = 0;
  pr.has_batch = true;
  pr.checked = false;
  return TAMP_OK;
}

struct Job {
  Problem* pr;
  ProbDesc d;
};

// Launch plan of the persistent kernel over several problems: the lane split
// and shared memory sized for the largest problem, the work-item list (longest
// skeletons first) and the grid that fills the SMs (CTAs then pull items until
// the list is empty).
struct Plan {
  int L = 1, warps = 1, grid = 0;
  bool mv_global = false;  // Adam moments in global memory: the tile fits shared memory only that way
  int feat = 0;            // optional terms of the problems: 0 or the KernelFeat that holds all of them
  size_t smem = 0;
  std::vector<ProbDesc> descs;
  std::vector<uint32_t> items;
};

std::vector<long long> job_key(const std::vector<Job>& jobs) {
  std::vector<long long> key;
  for (const Job& j : jobs) key.push_back((static_cast<long long>(j.pr->id) << 32) | static_cast<long long>(j.d.P));
  std::sort(key.begin(), key.end());
  return key;
}

// forced_L / forced_W > 0 pin the launch shape (the autotuner's trials);
// otherwise a tuned shape for this set of problems and batch sizes is used
// when the options leave the lane count to the library.
tamp_status plan_jobs(tamp_scene* s, std::vector<Job>& jobs, int requested_lanes, Plan* plan, int forced_L = 0,
                      int forced_W = 0) {
  long total = 0;
  int warps = 1;
  for (const Job& j : jobs) {
    total += j.d.P;
    warps = std::max(warps, optimize_warps(j.pr->K));
  }
  int L = preferred_lanes(requested_lanes, total);
  if (forced_L > 0) {
    L = forced_L;
    warps = std::max(1, std::min(forced_W, warps));
  } else if (requested_lanes == 0) {
    auto it = s->tuning.find(job_key(jobs));
    if (it != s->tuning.end()) {
      L = it->second.first;
      warps = std::max(1, std::min(it->second.second, warps));
    }
  }
  size_t smem = 0;
  // the first lane split that fits, with the Adam moments staged in shared
  // memory if possible, else used in place in global memory
  bool mvg = false;
  for (; L <= 8; L *= 2) {
    for (int g = 0; g < 2; ++g) {
      size_t tile = 0;
      for (const Job& j : jobs)
        tile = std::max(tile, optimize_tile_bytes(j.pr->opt_words, j.pr->D, j.pr->NT, j.pr->NSLOT, j.pr->NANG, L,
                                                  g == 1));
      smem = 4 * ((s->blob.size() + 3) & ~static_cast<size_t>(3)) + tile + optimize_scratch_bytes(warps);
      mvg = g == 1;
      if (smem <= kMaxDynSmem) break;
    }
    if (smem <= kMaxDynSmem) break;
  }
  if (L > 8) return fail(s, TAMP_ERR_INVALID_ARG, "problem does not fit in shared memory");
  if (forced_L > 0 && L != forced_L) return fail(s, TAMP_ERR_INVALID_ARG, "lane split %d does not fit", forced_L);
  const int PT = 32 / L;
  std::vector<int> order(jobs.size());
  for (size_t i = 0; i < jobs.size(); ++i) order[i] = static_cast<int>(i);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return jobs[a].pr->K > jobs[b].pr->K; });
  plan->items.clear();
  for (int i : order) {
    const int tiles = (jobs[i].d.P + PT - 1) / PT;
    if (tiles >= (1 << ITEM_TILE_BITS)) return fail(s, TAMP_ERR_INVALID_ARG, "batch too large");
    for (int t = 0; t < tiles; ++t)
      plan->items.push_back(static_cast<uint32_t>(i) << ITEM_TILE_BITS | static_cast<uint32_t>(t));
  }
  plan->descs.clear();
  for (const Job& j : jobs) plan->descs.push_back(j.d);
  plan->L = L;
  plan->warps = warps;
  plan->smem = smem;
  plan->mv_global = mvg;
  bool knots = false, g6 = false, self = false;
  for (const Job& j : jobs) {
    knots = knots || j.pr->n_seg > 0;
    g6 = g6 || j.pr->grasp6;
    self = self || j.pr->self;
  }
  plan->feat = feat_of(knots, g6, self);
  const int per_sm = std::max(1, optimize_blocks_per_sm(L, warps, smem));
  plan->grid = std::min(static_cast<int>(plan->items.size()), s->sm_count * per_sm);
  return TAMP_OK;
}

LaunchArgs plan_args(const tamp_scene* s, const Plan& plan, ProbDesc* d_descs, uint32_t* d_items, int* d_counter) {
  LaunchArgs a{};
  a.scene = s->d_blob;
  a.scene_words = static_cast<int>(s->blob.size());
  a.probs = d_descs;
  a.items = d_items;
  a.n_items = static_cast<int>(plan.items.size());
  a.item_counter = d_counter;
  a.err = s->d_err;
  a.scratch_offset = static_cast<int>(plan.smem - optimize_scratch_bytes(plan.warps));
  a.mv_global = plan.mv_global ? 1 : 0;
  a.feat = plan.feat;
  a.rec = plan.descs.empty() || plan.descs[0].best_x == nullptr ? 0 : 1;
  return a;
}

tamp_status launch_jobs(tamp_scene* s, std::vector<Job>& jobs, int requested_lanes, int forced_L = 0,
                        int forced_W = 0) {
  if (jobs.empty()) return TAMP_OK;
  Plan plan;
  tamp_status st = plan_jobs(s, jobs, requested_lanes, &plan, forced_L, forced_W);
  if (st != TAMP_OK) return st;
  if (static_cast<int>(jobs.size()) > s->descs_cap) {
    dfree(s, s->d_descs);
    s->d_descs = nullptr;
    s->descs_cap = 0;
    CUDA_TRY(s, dalloc(s, &s->d_descs, jobs.size() * sizeof(ProbDesc)));
    s->descs_cap = static_cast<int>(jobs.size());
  }
  if (static_cast<int>(plan.items.size()) > s->items_cap) {
    dfree(s, s->d_items);
    s->d_items = nullptr;
    s->items_cap = 0;
    CUDA_TRY(s, dalloc(s, &s->d_items, plan.items.size() * 4));
    s->items_cap = static_cast<int>(plan.items.size());
  }
  CUDA_TRY(s, cudaMemcpyAsync(s->d_descs, plan.descs.data(), plan.descs.size() * sizeof(ProbDesc),
                              cudaMemcpyHostToDevice, s->stream));
  CUDA_TRY(s, cudaMemcpyAsync(s->d_items, plan.items.data(), plan.items.size() * 4, cudaMemcpyHostToDevice,
                              s->stream));
  CUDA_TRY(s, cudaMemsetAsync(s->d_item_counter, 0, 4, s->stream));
  const LaunchArgs a = plan_args(s, plan, s->d_descs, s->d_items, s->d_item_counter);
  CUDA_TRY(s, launch_optimize(a, plan.L, plan.warps, plan.grid, plan.smem, s->stream));
  return TAMP_OK;
}

// The launch keeps this problem's best-satisfying record (tamp_query_best).
void keep_record(ProbDesc& d, Problem& pr) {
  d.best_x = pr.d_best_x; d.best_cost = pr.d_best_cost; d.best_iter = pr.d_best_iter; d.stage_x = pr.d_stage;
}

// Whether a launch of these problems keeps the records: always in the stop
// modes, otherwise if one of them asks for it (tamp_options.keep_best).
bool wants_record(const std::vector<Problem*>& prs, bool stop_mode) {
  if (stop_mode) return true;
  for (const Problem* pr : prs)
    if (pr->opt.keep_best) return true;
  return false;
}

ProbDesc state_desc(Problem& pr, int n_steps) {
  ProbDesc d{};
  d.prob = pr.d_blob;
  d.prob_words = pr.opt_words;
  d.x_in = pr.d_x; d.x_out = pr.d_x; d.m = pr.d_m; d.v = pr.d_v; d.load_mv = 1;
  d.stride = pr.P; d.P = pr.P;
  d.out_cost = pr.d_cost; d.out_flags = pr.d_flags; d.out_counts = pr.d_counts;
  d.first_iter = pr.d_first;
  d.work = pr.d_work;
  d.t0 = pr.t;
  d.n_steps = n_steps;
  d.gscale = pr.opt.scale_by_batch ? 1.f / static_cast<float>(pr.P) : 1.f;
  d.beta1 = pr.opt.beta1; d.beta2 = pr.opt.beta2; d.eps = pr.opt.eps;
  return d;
}

tamp_status run_state(tamp_scene* s, std::vector<Problem*> prs, int n_steps) {
  std::vector<Job> jobs;
  int lanes = 0;
  const bool rec = wants_record(prs, false);
  for (Problem* pr : prs) {
    CUDA_TRY(s, cudaMemsetAsync(pr->d_counts, 0, static_cast<size_t>(std::max(pr->NCON, 1)) * 4, s->stream));
    jobs.push_back({pr, state_desc(*pr, n_steps)});
    if (rec) keep_record(jobs.back().d, *pr);
    lanes = pr->opt.lanes;
  }
  tamp_status st = launch_jobs(s, jobs, lanes);
  if (st != TAMP_OK) return st;
  for (Problem* pr : prs) {
    pr->t += n_steps;
    pr->checked = true;
  }
  return TAMP_OK;
}

tamp_status check_device_error(tamp_scene* s);

// tamp_optimize_steps stopping on the first satisfying particle: the steps run
// as chunks of `chunk` fused iterations (the last one shorter), each followed
// by the control kernel, which advances the step counts on the device and
// raises the stop flag once a listed problem's Eq. 3 check has found a
// satisfying particle; every later chunk returns at once.  The host then reads
// the step counts back (this synchronises).
tamp_status run_state_stopping(tamp_scene* s, const std::vector<Problem*>& prs, int n_steps, int chunk) {
  const int n = static_cast<int>(prs.size());
  const int full = n_steps / chunk, rem = n_steps % chunk, n_chunks = full + (rem ? 1 : 0);
  // control block: ints [item counter, stop, chunks run, step counts [n], count sizes [n]], then pointers
  // [first-satisfying records [n], count arrays [n]], then the descriptors of a full and of the last chunk
  const size_t off_ptr = (4 * (3 + 2 * static_cast<size_t>(n)) + 15) & ~static_cast<size_t>(15);
  const size_t off_desc = (off_ptr + 2 * n * sizeof(void*) + 15) & ~static_cast<size_t>(15);
  const size_t bytes = off_desc + 2 * n * sizeof(ProbDesc);
  if (bytes > s->ctl_cap) {
    dfree(s, s->d_ctl);
    s->d_ctl = nullptr;
    s->ctl_cap = 0;
    CUDA_TRY(s, dalloc(s, &s->d_ctl, bytes));
    s->ctl_cap = bytes;
  }
  int* ints = reinterpret_cast<int*>(s->d_ctl);
  void** ptrs = reinterpret_cast<void**>(s->d_ctl + off_ptr);
  ProbDesc* descs = reinterpret_cast<ProbDesc*>(s->d_ctl + off_desc);
  std::vector<unsigned char> host(bytes, 0);
  int* hi = reinterpret_cast<int*>(host.data());
  void** hp = reinterpret_cast<void**>(host.data() + off_ptr);
  std::vector<Job> jobs;
  for (int i = 0; i < n; ++i) {
    Problem* pr = prs[i];
    hi[3 + i] = pr->t;
    hi[3 + n + i] = std::max(pr->NCON, 1);
    hp[i] = pr->d_first;
    hp[n + i] = pr->d_counts;
    ProbDesc d = state_desc(*pr, chunk);
    d.t_dev = ints + 3 + i;
    keep_record(d, *pr);  // a stop must not lose the satisfying particle it stopped on
    jobs.push_back({pr, d});
    CUDA_TRY(s, cudaMemsetAsync(pr->d_counts, 0, static_cast<size_t>(std::max(pr->NCON, 1)) * 4, s->stream));
  }
  Plan plan;
  tamp_status st = plan_jobs(s, jobs, prs[0]->opt.lanes, &plan);
  if (st != TAMP_OK) return st;
  ProbDesc* hd = reinterpret_cast<ProbDesc*>(host.data() + off_desc);
  for (int i = 0; i < n; ++i) {
    hd[i] = plan.descs[i];
    hd[n + i] = plan.descs[i];
    hd[n + i].n_steps = rem;
  }
  if (static_cast<int>(plan.items.size()) > s->items_cap) {
    dfree(s, s->d_items);
    s->d_items = nullptr;
    s->items_cap = 0;
    CUDA_TRY(s, dalloc(s, &s->d_items, plan.items.size() * 4));
    s->items_cap = static_cast<int>(plan.items.size());
  }
  CUDA_TRY(s, cudaMemcpyAsync(s->d_ctl, host.data(), bytes, cudaMemcpyHostToDevice, s->stream));
  CUDA_TRY(s, cudaMemcpyAsync(s->d_items, plan.items.data(), plan.items.size() * 4, cudaMemcpyHostToDevice,
                              s->stream));
  for (int c = 0; c < n_chunks; ++c) {
    const bool short_chunk = c == full;
    LaunchArgs a = plan_args(s, plan, short_chunk ? descs + n : descs, s->d_items, ints);
    a.stop = ints + 1;
    CUDA_TRY(s, cudaMemsetAsync(ints, 0, sizeof(int), s->stream));
    CUDA_TRY(s, launch_optimize(a, plan.L, plan.warps, plan.grid, plan.smem, s->stream));
    CUDA_TRY(s, launch_chunk_control(ints + 3, reinterpret_cast<const int* const*>(ptrs),
                                     reinterpret_cast<int* const*>(ptrs + n), ints + 3 + n, n,
                                     short_chunk ? rem : chunk, 1, ints + 1, ints + 2, c == n_chunks - 1,
                                     s->stream));
  }
  std::vector<int> t(3 + n, 0);
  CUDA_TRY(s, cudaMemcpyAsync(t.data(), ints, t.size() * sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  st = check_device_error(s);  // synchronises
  if (st != TAMP_OK) return st;
  for (int i = 0; i < n; ++i) {
    prs[i]->t = t[3 + i];
    prs[i]->checked = true;
  }
  return TAMP_OK;
}

Problem* get_problem(tamp_scene* s, int id) {
  if (!s || id < 0 || id >= static_cast<int>(s->probs.size())) return nullptr;
  return s->probs[id];
}

tamp_status check_device_error(tamp_scene* s) {
  int e = 0;
  CUDA_TRY(s, cudaMemcpyAsync(&e, s->d_err, 4, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(s, cudaStreamSynchronize(s->stream));
  if (e & ERR_TMA_TIMEOUT) return fail(s, TAMP_ERR_TIMEOUT, "a shared-memory staging wait timed out on the device");
  if (e) return fail(s, TAMP_ERR_DEVICE_CHECK, "device check word 0x%x", e);
  return TAMP_OK;
}

}  // namespace

extern "C" {

void tamp_default_options(tamp_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  const float w[TAMP_N_TERM_KINDS] = {1.f, 5.f, 1.f, 2.f, 1.f, 1.f, 1.f, 0.25f, 1.f, 0.01f, 1.f};
  const float tol[TAMP_N_TERM_KINDS] = {5e-3f, 0.05f, 1e-3f, 1e-3f, 1e-3f, 1e-3f, 0.f, INFINITY, 1e-3f, INFINITY, 0.f};
  for (int i = 0; i < TAMP_N_TERM_KINDS; ++i) {
    o->w[i] = w[i];
    o->tol[i] = tol[i];
  }
  o->lr_joint = 1e-2f; o->lr_pos = 3e-3f; o->lr_yaw = 1e-2f;
  o->beta1 = 0.9f; o->beta2 = 0.999f; o->eps = 1e-8f;
  o->optimize_grasp = 1; o->scale_by_batch = 1; o->lanes = 0;
  o->grasp_dof = 4;
}

tamp_status tamp_create_scene(const tamp_scene_desc* d, int device, void* stream, const tamp_allocator* allocator,
                              tamp_scene** out) {
  if (!d || !out) return TAMP_ERR_INVALID_ARG;
  *out = nullptr;
  if (allocator && (!allocator->alloc || !allocator->free)) return TAMP_ERR_INVALID_ARG;
  tamp_scene* s = new tamp_scene();
  auto bad = [&](const char*) {
    delete s;
    return TAMP_ERR_INVALID_ARG;
  };
  if (d->n_joints < 1 || d->n_joints > MAXJ) return bad("n_joints");
  if (!d->dh_a || !d->dh_d || !d->dh_alpha || !d->dh_offset || !d->q_lo || !d->q_hi) return bad("arm arrays");
  if (d->n_spheres < 0 || (d->n_spheres > 0 && (!d->sphere_link || !d->sphere_xyzr))) return bad("spheres");
  for (int i = 0; i < d->n_spheres; ++i)
    if (d->sphere_link[i] < 0 || d->sphere_link[i] > d->n_joints || d->sphere_xyzr[4 * i + 3] < 0) return bad("sphere");
  if (d->n_boxes < 0 || d->n_boxes > MAX_BOX) return bad("n_boxes");
  if (d->n_boxes > 0 && (!d->box_half || !d->box_init || !d->box_spheres)) return bad("box arrays");
  if (d->spheres_per_box < 1 || d->spheres_per_box > MAX_NBS) return bad("spheres_per_box");
  if (d->n_obs < 0 || d->n_obs > MAX_OBS) return bad("n_obs");
  if (d->n_obs > 0 && (!d->obs_center || !d->obs_rot || !d->obs_half)) return bad("obstacle arrays");
  if (d->n_surf < 0 || (d->n_surf > 0 && !d->surf)) return bad("surfaces");
  if (!finite_all(d->dh_a, d->n_joints) || !finite_all(d->dh_d, d->n_joints) || !finite_all(d->base, 16) ||
      !finite_all(d->tool, 16))
    return bad("non-finite arm");
  s->device = device;
  s->stream = static_cast<cudaStream_t>(stream);
  if (allocator) s->alloc = *allocator;
  s->nj = d->n_joints; s->S = d->n_spheres; s->B = d->n_boxes; s->NBS = d->spheres_per_box;
  s->O = d->n_obs; s->NS = d->n_surf;
  s->box_half.assign(d->box_half, d->box_half + 3 * d->n_boxes);
  s->dh_a.assign(d->dh_a, d->dh_a + d->n_joints);
  s->dh_d.assign(d->dh_d, d->dh_d + d->n_joints);
  s->dh_alpha.assign(d->dh_alpha, d->dh_alpha + d->n_joints);
  s->box_init.assign(d->box_init, d->box_init + 4 * d->n_boxes);
  if (d->n_surf) s->surf.assign(d->surf, d->surf + 6 * d->n_surf);
  tamp_status st = build_scene_blob(s, d);
  if (st != TAMP_OK) {
    delete s;
    return st;
  }
  DeviceGuard g(device);
  cudaError_t e = dalloc(s, &s->d_blob, s->blob.size() * 4);
  if (e == cudaSuccess) e = dalloc(s, &s->d_err, 4);
  if (e == cudaSuccess) e = dalloc(s, &s->d_scratch_first, 4);
  if (e == cudaSuccess) e = dalloc(s, &s->d_item_counter, 4);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_blob, s->blob.data(), s->blob.size() * 4, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_err, 0, 4, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    dfree(s, s->d_blob); dfree(s, s->d_err); dfree(s, s->d_scratch_first); dfree(s, s->d_item_counter);
    delete s;
    return e == cudaErrorMemoryAllocation ? TAMP_ERR_OOM : TAMP_ERR_CUDA;
  }
  *out = s;
  return TAMP_OK;
}

tamp_status tamp_destroy_scene(tamp_scene* s) {
  if (!s) return TAMP_ERR_INVALID_ARG;
  DeviceGuard g(s->device);
  cudaStreamSynchronize(s->stream);
  for (Problem* p : s->probs) {
    free_batch(s, *p);
    dfree(s, p->d_blob);
    dfree(s, p->d_prow); dfree(s, p->d_pfeat); dfree(s, p->d_pout); dfree(s, p->d_chains);
    delete p;
  }
  dfree(s, s->d_blob); dfree(s, s->d_err); dfree(s, s->d_scratch_first); dfree(s, s->d_item_counter);
  dfree(s, s->d_descs); dfree(s, s->d_items); dfree(s, s->d_ctl);
  delete s;
  return TAMP_OK;
}

tamp_status tamp_set_skeleton(tamp_scene* s, const tamp_action* acts, int n, const tamp_options* opt, int* pid) {
  if (!s) return TAMP_ERR_INVALID_ARG;
  if (!acts || n <= 0 || !pid) return fail(s, TAMP_ERR_INVALID_ARG, "empty skeleton or null output");
  Problem* pr = new Problem();
  if (opt) pr->opt = *opt; else tamp_default_options(&pr->opt);
  tamp_status st = compile_problem(s, acts, n, pr->opt, *pr);
  if (st != TAMP_OK) {
    delete pr;
    return st;
  }
  DeviceGuard g(s->device);
  cudaError_t e = dalloc(s, &pr->d_blob, pr->blob.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pr->d_blob, pr->blob.data(), pr->blob.size() * 4, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    dfree(s, pr->d_blob);
    delete pr;
    return fail(s, TAMP_ERR_CUDA, "skeleton upload: %s", cudaGetErrorString(e));
  }
  s->probs.push_back(pr);
  *pid = static_cast<int>(s->probs.size()) - 1;
  pr->id = *pid;
  s->err.clear();
  return TAMP_OK;
}

tamp_status tamp_problem_info(const tamp_scene* sc, int id, int* D, int* n_terms, int* kinds) {
  tamp_scene* s = const_cast<tamp_scene*>(sc);
  Problem* pr = get_problem(s, id);
  if (!pr) return fail(s, TAMP_ERR_INVALID_ARG, "unknown problem %d", id);
  if (D) *D = pr->D;
  if (n_terms) *n_terms = pr->NT;
  if (kinds) std::copy(pr->term_kinds.begin(), pr->term_kinds.end(), kinds);
  return TAMP_OK;
}

tamp_status tamp_term_actions(const tamp_scene* sc, int id, int* action_index) {
  tamp_scene* s = const_cast<tamp_scene*>(sc);
  Problem* pr = get_problem(s, id);
  if (!pr) return fail(s, TAMP_ERR_INVALID_ARG, "unknown problem %d", id);
  if (!action_index) return fail(s, TAMP_ERR_INVALID_ARG, "null output");
  std::copy(pr->term_actions.begin(), pr->term_actions.end(), action_index);
  return TAMP_OK;
}

namespace {
// Components of the longest action prefix two skeletons share: the same
// actions in the same order give the same sub-CSP (same variables, same
// constraints, same environment), laid out at the same particle components.
int shared_prefix_components(const Problem& a, const Problem& b) {
  size_t k = 0;
  while (k < a.acts.size() && k < b.acts.size() && a.acts[k].kind == b.acts[k].kind &&
         a.acts[k].box == b.acts[k].box && a.acts[k].surface == b.acts[k].surface)
    ++k;
  return a.act_off[k];
}
}  // namespace

static tamp_status sample_batch(tamp_scene* s, Problem* pr, int P, uint64_t seed, int sampler, const Problem* src,
                                int keep);

tamp_status tamp_sample_particles(tamp_scene* s, int id, int P, uint64_t seed, int sampler) {
  Problem* pr = get_problem(s, id);
  if (!pr) return fail(s, TAMP_ERR_INVALID_ARG, "unknown problem %d", id);
  return sample_batch(s, pr, P, seed, sampler, nullptr, 0);
}

tamp_status tamp_sample_particles_from(tamp_scene* s, int id, int P, uint64_t seed, int sampler, int src_id,
                                       int* shared) {
  Problem* pr = get_problem(s, id);
  if (!pr) return fail(s, TAMP_ERR_INVALID_ARG, "unknown problem %d", id);
  Problem* src = get_problem(s, src_id);
  if (!src) return fail(s, TAMP_ERR_INVALID_ARG, "unknown source problem %d", src_id);
  if (src == pr) return fail(s, TAMP_ERR_INVALID_ARG, "a problem cannot be its own source");
  const int keep = shared_prefix_components(*pr, *src);
  if (keep > 0 && (!src->has_batch || src->P != P))
    return fail(s, TAMP_ERR_STATE, "source problem %d holds no batch of %d particles", src_id, P);
  tamp_status st = sample_batch(s, pr, P, seed, sampler, keep > 0 ? src : nullptr, keep);
  if (st == TAMP_OK && shared) *shared = keep;
  return st;
}

static tamp_status sample_batch(tamp_scene* s, Problem* pr, int P, uint64_t seed, int sampler, const Problem* src,
                                int keep) {
  if (P <= 0 || P > (1 << 24)) return fail(s, TAMP_ERR_INVALID_ARG, "n_particles %d out of range", P);
  if (sampler < 0 || sampler > 3) return fail(s, TAMP_ERR_INVALID_ARG, "sampler %d not available", sampler);
  if ((sampler & TAMP_SAMPLE_LEARNED) && !s->proposal)
    return fail(s, TAMP_ERR_STATE, "the learned sampler needs a proposal network attached");
  DeviceGuard g(s->device);
  tamp_status st = ensure_batch(s, *pr, P);
  if (st != TAMP_OK) return st;
  CUDA_TRY(s, launch_sample(pr->d_blob, s->d_blob, pr->d_x, pr->d_m, pr->d_v, P, P, pr->D, seed, s->stream));
  if (sampler & TAMP_SAMPLE_LEARNED) {
    if (!pr->d_prow) {
      CUDA_TRY(s, dalloc(s, &pr->d_prow, pr->prow.size() * 4));
      CUDA_TRY(s, dalloc(s, &pr->d_pfeat, pr->pfeat.size() * 4));
      CUDA_TRY(s, dalloc(s, &pr->d_pout, static_cast<size_t>(pr->R) * 2 * PROP_NT * 4));
      CUDA_TRY(s, cudaMemcpyAsync(pr->d_prow, pr->prow.data(), pr->prow.size() * 4, cudaMemcpyHostToDevice, s->stream));
      CUDA_TRY(s, cudaMemcpyAsync(pr->d_pfeat, pr->pfeat.data(), pr->pfeat.size() * 4, cudaMemcpyHostToDevice,
                                  s->stream));
    }
    st = mlp_forward_on_stream(s->proposal, pr->d_pfeat, pr->R, pr->d_pout, s->stream, s->device);
    if (st != TAMP_OK) return fail(s, st, "proposal network forward: %s", tamp_mlp_last_error(s->proposal));
    CUDA_TRY(s, launch_sample_proposal(pr->d_prow, pr->R, pr->d_pout, pr->d_x, P, P, seed, s->stream));
  }
  // the shared prefix: the source's components (rows of the [D][P] layout) as they stand
  if (src && keep > 0)
    CUDA_TRY(s, cudaMemcpyAsync(pr->d_x, src->d_x, static_cast<size_t>(keep) * P * 4, cudaMemcpyDeviceToDevice,
                                s->stream));
  if (sampler & TAMP_SAMPLE_IK) {
    if (!pr->d_chains) {
      CUDA_TRY(s, dalloc(s, &pr->d_chains, pr->chains.size() * 4));
      CUDA_TRY(s, cudaMemcpyAsync(pr->d_chains, pr->chains.data(), pr->chains.size() * 4, cudaMemcpyHostToDevice,
                                  s->stream));
    }
    CUDA_TRY(s, launch_ik(pr->d_blob, s->d_blob, pr->d_x, P, P, TAMP_IK_ITERS, TAMP_IK_DAMPING, TAMP_IK_MAX_STEP,
                          pr->d_chains, pr->n_chain, 1 + pr->K, keep, s->stream));
  }
  // knots on the joint-space line between their motion's ends (Sec. VIII)
  CUDA_TRY(s, launch_knots(pr->d_blob, pr->d_x, P, P, pr->n_seg, s->nj, keep, s->stream));
  return TAMP_OK;
}

tamp_status tamp_set_proposal(tamp_scene* s, tamp_mlp* net) {
  if (!s) return TAMP_ERR_INVALID_ARG;
  s->proposal = net;
  return TAMP_OK;
}

tamp_status tamp_proposal_rows(tamp_scene* s, int id, int n, const float* x, float* feat, float* y, float* mask,
                               int* n_rows) {
  Problem* pr = get_problem(s, id);
  if (!pr) return fail(s, TAMP_ERR_INVALID_ARG, "unknown problem %d", id);
  if (n_rows) *n_rows = pr->R;
  if (!feat && !y && !mask) return TAMP_OK;
  if (n <= 0 || !x) return fail(s, TAMP_ERR_INVALID_ARG, "bad particle batch");
  const int R = pr->R;
  for (int i = 0; i < n; ++i) {
    for (int r = 0; r < R; ++r) {
      const size_t row = static_cast<size_t>(i) * R + r;
      if (feat) std::copy(&pr->pfeat[static_cast<size_t>(r) * PROP_NF], &pr->pfeat[static_cast<size_t>(r + 1) * PROP_NF],
                          feat + row * PROP_NF);
      float* yy = y ? y + row * PROP_NT : nullptr;
      float* mm = mask ? mask + row * PROP_NT : nullptr;
      if (yy) std::fill(yy, yy + PROP_NT, 0.f);
      if (mm) std::fill(mm, mm + PROP_NT, 0.f);
      const int off = pr->prow_off[r], b = pr->prow_box[r];
      auto X = [&](int c) { return static_cast<double>(x[static_cast<size_t>(off + c) * n + i]); };
      if (pr->prow_kind[r] == 0) {
        const double* h = &s->box_half[3 * b];
        const double t[5] = {X(0) / h[0], X(1) / h[1], (X(2) - (h[2] - 0.02)) / 0.01 - 1.0, std::cos(X(3)),
                             std::sin(X(3))};
        for (int k = 0; k < 5; ++k) {
          if (yy) yy[k] = static_cast<float>(t[k]);
          if (mm) mm[k] = 1.f;
        }
      } else {
        const double* q = &s->surf[6 * pr->prow_surf[r]];
        const double dx = X(0) - q[0], dy = X(1) - q[1];
        const double u = std::cos(q[2]) * dx + std::sin(q[2]) * dy, v = -std::sin(q[2]) * dx + std::cos(q[2]) * dy;
        const double t[4] = {u / q[3], v / q[4], std::cos(X(2)), std::sin(X(2))};
        for (int k = 0; k < 4; ++k) {
          if (yy) yy[5 + k] = static_cast<float>(t[k]);
          if (mm) mm[5 + k] = 1.f;
        }
      }
    }
  }
  return TAMP_OK;
}

tamp_status tamp_set_particles(tamp_scene* s, int id, int P, const float* x, const float* m, const float* v, int t0,
                               int is_device) {
  Problem* pr = get_problem(s, id);
  if (!pr) return fail(s, TAMP_ERR_INVALID_ARG, "unknown problem %d", id);
  if (P <= 0 || P > (1 << 24) || !x || t0 < 0) return fail(s, TAMP_ERR_INVALID_ARG, "bad batch arguments");
  DeviceGuard g(s->device);
  tamp_status st = ensure_batch(s, *pr, P);
  if (st != TAMP_OK) return st;
  const size_t n = static_cast<size_t>(pr->D) * P * 4;
  const cudaMemcpyKind kd = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CUDA_TRY(s, cudaMemcpyAsync(pr->d_x, x, n, kd, s->stream));
  if (m) CUDA_TRY(s, cudaMemcpyAsync(pr->d_m, m, n, kd, s->stream));
  else CUDA_TRY(s, cudaMemsetAsync(pr->d_m, 0, n, s->stream));
  if (v) CUDA_TRY(s, cudaMemcpyAsync(pr->d_v, v, n, kd, s->stream));
  else CUDA_TRY(s, cudaMemsetAsync(pr->d_v, 0, n, s->stream));
  pr->t = t0;
  if (!is_device) CUDA_TRY(s, cudaStreamSynchronize(s->stream));
  return TAMP_OK;
}

tamp_status tamp_get_particles(tamp_scene* s, int id, float* x, float* m, float* v, int* t, int is_device) {
  Problem* pr = get_problem(s, id);
  if (!pr) return fail(s, TAMP_ERR_INVALID_ARG, "unknown problem %d", id);
  if (!pr->has_batch) return fail(s, TAMP_ERR_STATE, "problem %d has no particles", id);
  DeviceGuard g(s->device);
  const size_t n = static_cast<size_t>(pr->D) * pr->P * 4;
  const cudaMemcpyKind kd = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (x) CUDA_TRY(s, cudaMemcpyAsync(x, pr->d_x, n, kd, s->stream));
  if (m) CUDA_TRY(s, cudaMemcpyAsync(m, pr->d_m, n, kd, s->stream));
  if (v) CUDA_TRY(s, cudaMemcpyAsync(v, pr->d_v, n, kd, s->stream));
  if (t) *t = pr->t;
  return check_device_error(s);
}

tamp_status tamp_optimize_steps(tamp_scene* s, const int* ids, int n, int n_steps, int stop_on_first_satisfying) {
  if (!s) return TAMP_ERR_INVALID_ARG;
  if (!ids || n <= 0 || n_steps < 0 || stop_on_first_satisfying < 0)
    return fail(s, TAMP_ERR_INVALID_ARG, "bad optimize arguments");
  DeviceGuard g(s->device);
  for (int i = 0; i < n; ++i) {
    Problem* pr = get_problem(s, ids[i]);
    if (!pr) return fail(s, TAMP_ERR_INVALID_ARG, "unknown problem %d", ids[i]);
    if (!pr->has_batch) return fail(s, TAMP_ERR_STATE, "problem %d has no particles", ids[i]);
  }
  std::vector<Problem*> prs;
  for (int i = 0; i < n; ++i) {
    Problem* pr = s->probs[ids[i]];
    if (std::find(prs.begin(), prs.end(), pr) != prs.end())
      return fail(s, TAMP_ERR_INVALID_ARG, "problem %d listed twice", ids[i]);
    prs.push_back(pr);
  }
  if (stop_on_first_satisfying > 0 && n_steps > 0) return run_state_stopping(s, prs, n_steps, stop_on_first_satisfying);
  return run_state(s, prs, n_steps);
}

tamp_status tamp_query_satisfied(tamp_scene* s, int id, uint8_t* mask, int* n_sat, int* first_iter, float* particles,
                                 float* cost, int* counts) {
  Problem* pr = get_problem(s, id);
  if (!pr) return fail(s, TAMP_ERR_INVALID_ARG, "unknown problem %d", id);
  if (!pr->has_batch) return fail(s, TAMP_ERR_STATE, "problem %d has no particles", id);
  DeviceGuard g(s->device);
  if (!pr->checked) {
    tamp_status st = run_state(s, {pr}, 0);
    if (st != TAMP_OK) return st;
  }
  std::vector<uint8_t> fl(pr->P);
  int first = INT_MAX;
  CUDA_TRY(s, cudaMemcpyAsync(fl.data(), pr->d_flags, pr->P, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(s, cudaMemcpyAsync(&first, pr->d_first, 4, cudaMemcpyDeviceToHost, s->stream));
  if (particles)
    CUDA_TRY(s, cudaMemcpyAsync(particles, pr->d_x, static_cast<size_t>(pr->D) * pr->P * 4, cudaMemcpyDeviceToHost, s->stream));
  if (cost) CUDA_TRY(s, cudaMemcpyAsync(cost, pr->d_cost, static_cast<size_t>(pr->P) * 4, cudaMemcpyDeviceToHost, s->stream));
  if (counts && pr->NCON)
    CUDA_TRY(s, cudaMemcpyAsync(counts, pr->d_counts, static_cast<size_t>(pr->NCON) * 4, cudaMemcpyDeviceToHost, s->stream));
  tamp_status st = check_device_error(s);
  if (st != TAMP_OK) return st;
  int ns = 0;
  for (int i = 0; i < pr->P; ++i) ns += fl[i] ? 1 : 0;
  if (mask) std::copy(fl.begin(), fl.end(), mask);
  if (n_sat) *n_sat = ns;
  if (first_iter) *first_iter = first == INT_MAX ? -1 : first;
  return TAMP_OK;
}

tamp_status tamp_query_best(tamp_scene* s, int id, uint8_t* found, int* n_found, float* particles, float* cost,
                            int* iter) {
  Problem* pr = get_problem(s, id);
  if (!pr) return fail(s, TAMP_ERR_INVALID_ARG, "unknown problem %d", id);
  if (!pr->has_batch) return fail(s, TAMP_ERR_STATE, "problem %d has no particles", id);
  DeviceGuard g(s->device);
  if (!pr->checked) {  // the batch as set has not been checked yet: check it once
    tamp_status st = run_state(s, {pr}, 0);
    if (st != TAMP_OK) return st;
  }
  std::vector<int> it(pr->P);
  CUDA_TRY(s, cudaMemcpyAsync(it.data(), pr->d_best_iter, static_cast<size_t>(pr->P) * 4, cudaMemcpyDeviceToHost,
                              s->stream));
  if (particles)
    CUDA_TRY(s, cudaMemcpyAsync(particles, pr->d_best_x, static_cast<size_t>(pr->D) * pr->P * 4,
                                cudaMemcpyDeviceToHost, s->stream));
  if (cost)
    CUDA_TRY(s, cudaMemcpyAsync(cost, pr->d_best_cost, static_cast<size_t>(pr->P) * 4, cudaMemcpyDeviceToHost,
                                s->stream));
  tamp_status st = check_device_error(s);
  if (st != TAMP_OK) return st;
  int nf = 0;
  for (int i = 0; i < pr->P; ++i) {
    const bool f = it[i] >= 0;
    nf += f ? 1 : 0;
    if (found) found[i] = f ? 1 : 0;
    if (cost && !f) cost[i] = INFINITY;
  }
  if (iter) std::copy(it.begin(), it.end(), iter);
  if (n_found) *n_found = nf;
  return TAMP_OK;
}

tamp_status tamp_eval(tamp_scene* s, int id, int n, const float* x, float* cost, float* terms, uint8_t* flags,
                      float* grad) {
  Problem* pr = get_problem(s, id);
  if (!pr) return fail(s, TAMP_ERR_INVALID_ARG, "unknown problem %d", id);
  if (n <= 0 || !x) return fail(s, TAMP_ERR_INVALID_ARG, "bad eval arguments");
  DeviceGuard g(s->device);
  ProbDesc d{};
  d.prob = pr->d_blob;
  d.prob_words = pr->opt_words;
  d.x_in = x; d.stride = n; d.P = n;
  d.out_cost = cost; d.out_terms = terms; d.out_flags = flags; d.out_grad = grad;
  d.n_steps = 0;
  d.gscale = 1.f; d.beta1 = pr->opt.beta1; d.beta2 = pr->opt.beta2; d.eps = pr->opt.eps;
  std::vector<Job> jobs{{pr, d}};
  return launch_jobs(s, jobs, pr->opt.lanes);
}

tamp_status tamp_autotune(tamp_scene* s, const int* ids, int n, int trial_steps, int* lanes_out, int* warps_out,
                          float* ms_out) {
  if (!s) return TAMP_ERR_INVALID_ARG;
  if (!ids || n <= 0 || trial_steps <= 0 || trial_steps > 100000) return fail(s, TAMP_ERR_INVALID_ARG, "bad arguments");
  std::vector<Problem*> prs;
  for (int i = 0; i < n; ++i) {
    Problem* pr = get_problem(s, ids[i]);
    if (!pr) return fail(s, TAMP_ERR_INVALID_ARG, "unknown problem %d", ids[i]);
    if (!pr->has_batch) return fail(s, TAMP_ERR_STATE, "problem %d has no particles", ids[i]);
    for (Problem* q : prs)
      if (q == pr) return fail(s, TAMP_ERR_INVALID_ARG, "problem %d listed twice", ids[i]);
    prs.push_back(pr);
  }
  DeviceGuard g(s->device);
  // scratch copies of every batch: the trials must leave the problems' state alone
  struct Scratch { float *x = nullptr, *m = nullptr, *v = nullptr, *cost = nullptr; uint8_t* flags = nullptr;
                   int *counts = nullptr, *first = nullptr; unsigned long long* work = nullptr; };
  std::vector<Scratch> sc(prs.size());
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto release = [&]() {
    for (Scratch& b : sc) {
      dfree(s, b.x); dfree(s, b.m); dfree(s, b.v); dfree(s, b.cost); dfree(s, b.flags);
      dfree(s, b.counts); dfree(s, b.first); dfree(s, b.work);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (size_t i = 0; i < prs.size() && e == cudaSuccess; ++i) {
    const size_t nb = static_cast<size_t>(prs[i]->D) * prs[i]->P * 4;
    e = dalloc(s, &sc[i].x, nb);
    if (e == cudaSuccess) e = dalloc(s, &sc[i].m, nb);
    if (e == cudaSuccess) e = dalloc(s, &sc[i].v, nb);
    if (e == cudaSuccess) e = dalloc(s, &sc[i].cost, static_cast<size_t>(prs[i]->P) * 4);
    if (e == cudaSuccess) e = dalloc(s, &sc[i].flags, static_cast<size_t>(prs[i]->P));
    if (e == cudaSuccess) e = dalloc(s, &sc[i].counts, static_cast<size_t>(std::max(prs[i]->NCON, 1)) * 4);
    if (e == cudaSuccess) e = dalloc(s, &sc[i].first, 4);
    if (e == cudaSuccess) e = dalloc(s, &sc[i].work, 16);
  }
  if (e != cudaSuccess) {
    release();
    return fail(s, e == cudaErrorMemoryAllocation ? TAMP_ERR_OOM : TAMP_ERR_CUDA, "autotune scratch: %s",
                cudaGetErrorString(e));
  }
  std::vector<Job> jobs;
  for (size_t i = 0; i < prs.size(); ++i) {
    ProbDesc d = state_desc(*prs[i], trial_steps);
    d.x_in = d.x_out = sc[i].x; d.m = sc[i].m; d.v = sc[i].v;
    d.out_cost = sc[i].cost; d.out_flags = sc[i].flags; d.out_counts = sc[i].counts;
    d.first_iter = sc[i].first; d.work = sc[i].work;
    // trial launches run on copies and keep no best-satisfying record
    jobs.push_back({prs[i], d});
  }
  auto restore = [&]() {
    cudaError_t r = cudaSuccess;
    for (size_t i = 0; i < prs.size() && r == cudaSuccess; ++i) {
      const size_t nb = static_cast<size_t>(prs[i]->D) * prs[i]->P * 4;
      r = cudaMemcpyAsync(sc[i].x, prs[i]->d_x, nb, cudaMemcpyDeviceToDevice, s->stream);
      if (r == cudaSuccess) r = cudaMemcpyAsync(sc[i].m, prs[i]->d_m, nb, cudaMemcpyDeviceToDevice, s->stream);
      if (r == cudaSuccess) r = cudaMemcpyAsync(sc[i].v, prs[i]->d_v, nb, cudaMemcpyDeviceToDevice, s->stream);
    }
    return r;
  };
  int max_w = 1;
  for (Problem* pr : prs) max_w = std::max(max_w, optimize_warps(pr->K));
  std::vector<int> wc;
  for (int per : {1, 2, 3, 4, 6, 8}) {  // work items (two per configuration) per warp
    int kmax = 0;
    for (Problem* pr : prs) kmax = std::max(kmax, pr->K);
    const int w = std::min(max_w, (2 * kmax + per - 1) / per);
    if (std::find(wc.begin(), wc.end(), w) == wc.end()) wc.push_back(w);
  }
  // the shapes that fit, each timed in kTuneRounds interleaved rounds (its best
  // time counts), so that clock drift during the tuning treats them alike
  constexpr int kTuneRounds = 3;
  const std::string saved = s->err;
  std::vector<std::pair<int, int>> shapes;
  for (int L = 1; L <= 8; L *= 2)
    for (int W : wc) {
      Plan probe;
      if (plan_jobs(s, jobs, 0, &probe, L, W) == TAMP_OK) shapes.push_back({L, W});  // else: does not fit
    }
  std::vector<float> best_ms(shapes.size(), -1.f);
  for (int round = 0; round < kTuneRounds; ++round)
    for (size_t c = 0; c < shapes.size(); ++c) {
      const int L = shapes[c].first, W = shapes[c].second;
      e = restore();
      if (round == 0 && e == cudaSuccess && launch_jobs(s, jobs, 0, L, W) != TAMP_OK)  // warm-up
        e = cudaErrorLaunchFailure;
      if (round == 0 && e == cudaSuccess) e = restore();
      if (e == cudaSuccess) e = cudaEventRecord(e0, s->stream);
      if (e == cudaSuccess && launch_jobs(s, jobs, 0, L, W) != TAMP_OK) e = cudaErrorLaunchFailure;
      if (e == cudaSuccess) e = cudaEventRecord(e1, s->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        release();
        return fail(s, TAMP_ERR_CUDA, "autotune trial L=%d W=%d: %s", L, W, cudaGetErrorString(e));
      }
      if (best_ms[c] < 0.f || ms < best_ms[c]) best_ms[c] = ms;
    }
  float best = -1.f;
  int bL = 0, bW = 0;
  for (size_t c = 0; c < shapes.size(); ++c)
    if (best < 0.f || best_ms[c] < best) {
      best = best_ms[c]; bL = shapes[c].first; bW = shapes[c].second;
    }
  s->err = saved;
  release();
  if (best < 0.f) return fail(s, TAMP_ERR_INVALID_ARG, "no launch shape fits these problems");
  tamp_status st = check_device_error(s);
  if (st != TAMP_OK) return st;
  s->tuning[job_key(jobs)] = {bL, bW};
  if (lanes_out) *lanes_out = bL;
  if (warps_out) *warps_out = bW;
  if (ms_out) *ms_out = best;
  return TAMP_OK;
}

tamp_status tamp_set_tuning(tamp_scene* s, const int* ids, int n, int lanes, int warps) {
  if (!s) return TAMP_ERR_INVALID_ARG;
  if (!ids || n <= 0) return fail(s, TAMP_ERR_INVALID_ARG, "bad arguments");
  std::vector<Job> jobs;
  for (int i = 0; i < n; ++i) {
    Problem* pr = get_problem(s, ids[i]);
    if (!pr) return fail(s, TAMP_ERR_INVALID_ARG, "unknown problem %d", ids[i]);
    if (!pr->has_batch) return fail(s, TAMP_ERR_STATE, "problem %d has no particles", ids[i]);
    jobs.push_back({pr, state_desc(*pr, 1)});
  }
  if (lanes == 0) {
    s->tuning.erase(job_key(jobs));
    return TAMP_OK;
  }
  if (lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8) return fail(s, TAMP_ERR_INVALID_ARG, "lanes %d", lanes);
  if (warps < 1 || warps > 16) return fail(s, TAMP_ERR_INVALID_ARG, "warps %d", warps);
  Plan probe;
  tamp_status st = plan_jobs(s, jobs, 0, &probe, lanes, warps);
  if (st != TAMP_OK) return st;
  s->tuning[job_key(jobs)] = {lanes, warps};
  return TAMP_OK;
}

tamp_status tamp_measure_fp32_peak(int device, double* tflops, double* ms) {
  if (!tflops) return TAMP_ERR_INVALID_ARG;
  DeviceGuard g(device);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return TAMP_ERR_CUDA;
  const int blocks = sms * 8, iters = 4096;  // 8 x 256 threads per SM, 8 chains each
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&out, static_cast<size_t>(blocks) * 256 * 4);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch_ffma_probe(out, blocks, iters, nullptr);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, nullptr);
  if (e == cudaSuccess) e = launch_ffma_probe(out, blocks, iters, nullptr);
  if (e == cudaSuccess) e = cudaEventRecord(e1, nullptr);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return TAMP_ERR_CUDA;
  const double flop = 2.0 * blocks * 256.0 * iters * 16.0 * 8.0;
  *tflops = flop / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return TAMP_OK;
}

tamp_status tamp_work_counters(tamp_scene* s, int id, uint64_t out[2]) {
  Problem* pr = get_problem(s, id);
  if (!pr) return fail(s, TAMP_ERR_INVALID_ARG, "unknown problem %d", id);
  if (!out) return fail(s, TAMP_ERR_INVALID_ARG, "null output");
  if (!pr->has_batch) return fail(s, TAMP_ERR_STATE, "problem %d has no particles", id);
  DeviceGuard g(s->device);
  unsigned long long w[2] = {0, 0};
  CUDA_TRY(s, cudaMemcpyAsync(w, pr->d_work, sizeof w, cudaMemcpyDeviceToHost, s->stream));
  tamp_status st = check_device_error(s);
  if (st != TAMP_OK) return st;
  out[0] = w[0];
  out[1] = w[1];
  return TAMP_OK;
}

const char* tamp_last_error(const tamp_scene* s) { return s ? s->err.c_str() : "null scene"; }

}  // extern "C"

// ---------------------------------------------------------------- CUDA graphs of the optimisation loop
struct tamp_graph {
  tamp_scene* s = nullptr;
  std::vector<Problem*> prs;
  std::vector<int> sizes;  // batch sizes the graph was built for
  int steps = 0, chunks = 0;
  ProbDesc* d_descs = nullptr;
  uint32_t* d_items = nullptr;
  int* d_ints = nullptr;  // [0] item counter, [1] stop, [2] chunks run, [3, 3 + n) per-problem step
                          // counts, [3 + n, 3 + 2n) per-problem constraint counts (Eq. 5 array sizes)
  void** d_first = nullptr;  // [0, n) first-satisfying records, [n, 2n) Eq. 5 count arrays
  cudaStream_t capture = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {
void free_graph(tamp_graph* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->capture) cudaStreamDestroy(g->capture);
  dfree(g->s, g->d_descs); dfree(g->s, g->d_items); dfree(g->s, g->d_ints); dfree(g->s, g->d_first);
  delete g;
}
}  // namespace

extern "C" tamp_status tamp_graph_create(tamp_scene* s, const int* ids, int n, int steps_per_chunk, int n_chunks,
                                         int stop_on_first, tamp_graph** out) {
  if (!s) return TAMP_ERR_INVALID_ARG;
  if (!ids || n <= 0 || steps_per_chunk <= 0 || n_chunks <= 0 || !out)
    return fail(s, TAMP_ERR_INVALID_ARG, "bad graph arguments");
  DeviceGuard dg(s->device);
  tamp_graph* g = new tamp_graph();
  g->s = s;
  g->steps = steps_per_chunk;
  g->chunks = n_chunks;
  std::vector<Job> jobs;
  auto bail = [&](tamp_status st) {
    free_graph(g);
    return st;
  };
  cudaError_t e = dalloc(s, &g->d_ints, (3 + 2 * n) * sizeof(int));
  if (e == cudaSuccess) e = dalloc(s, &g->d_first, 2 * n * sizeof(void*));
  if (e != cudaSuccess) return bail(fail(s, TAMP_ERR_OOM, "graph buffers: %s", cudaGetErrorString(e)));
  std::vector<void*> firsts(2 * n, nullptr);
  std::vector<int> ncons(n, 0);
  for (int i = 0; i < n; ++i) {
    Problem* pr = get_problem(s, ids[i]);
    if (!pr) return bail(fail(s, TAMP_ERR_INVALID_ARG, "unknown problem %d", ids[i]));
    if (!pr->has_batch) return bail(fail(s, TAMP_ERR_STATE, "problem %d has no particles", ids[i]));
    if (std::find(g->prs.begin(), g->prs.end(), pr) != g->prs.end())
      return bail(fail(s, TAMP_ERR_INVALID_ARG, "problem %d listed twice", ids[i]));
    g->prs.push_back(pr);
    g->sizes.push_back(pr->P);
    ProbDesc d = state_desc(*pr, steps_per_chunk);
    d.t_dev = g->d_ints + 3 + i;
    jobs.push_back({pr, d});
    firsts[i] = pr->d_first;
    firsts[n + i] = pr->d_counts;
    ncons[i] = std::max(pr->NCON, 1);
  }
  if (wants_record(g->prs, stop_on_first != 0))
    for (Job& j : jobs) keep_record(j.d, *j.pr);
  Plan plan;
  tamp_status st = plan_jobs(s, jobs, g->prs[0]->opt.lanes, &plan);
  if (st != TAMP_OK) return bail(st);
  e = dalloc(s, &g->d_descs, plan.descs.size() * sizeof(ProbDesc));
  if (e == cudaSuccess) e = dalloc(s, &g->d_items, plan.items.size() * 4);
  if (e == cudaSuccess)
    e = cudaMemcpy(g->d_descs, plan.descs.data(), plan.descs.size() * sizeof(ProbDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_items, plan.items.data(), plan.items.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_first, firsts.data(), 2 * n * sizeof(void*), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_ints + 3 + n, ncons.data(), n * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = optimize_set_smem(plan.L, plan.smem);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(fail(s, TAMP_ERR_CUDA, "graph set-up: %s", cudaGetErrorString(e)));
  LaunchArgs a = plan_args(s, plan, g->d_descs, g->d_items, g->d_ints);
  a.stop = g->d_ints + 1;
  // capture: clear the counts; per chunk, clear the item counter, optimise, control (which clears the
  // counts again for the next chunk's final check unless the loop stops)
  e = cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeThreadLocal);
  for (Problem* pr : g->prs)
    if (e == cudaSuccess)
      e = cudaMemsetAsync(pr->d_counts, 0, static_cast<size_t>(std::max(pr->NCON, 1)) * 4, g->capture);
  for (int c = 0; c < n_chunks && e == cudaSuccess; ++c) {
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_ints, 0, sizeof(int), g->capture);
    if (e == cudaSuccess) e = launch_optimize(a, plan.L, plan.warps, plan.grid, plan.smem, g->capture);
    if (e == cudaSuccess)
      e = launch_chunk_control(g->d_ints + 3, reinterpret_cast<const int* const*>(g->d_first),
                               reinterpret_cast<int* const*>(g->d_first + n), g->d_ints + 3 + n, n,
                               steps_per_chunk, stop_on_first, g->d_ints + 1, g->d_ints + 2, c == n_chunks - 1,
                               g->capture);
  }
  cudaError_t e2 = cudaStreamEndCapture(g->capture, &g->graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) return bail(fail(s, TAMP_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e)));
  *out = g;
  return TAMP_OK;
}

extern "C" tamp_status tamp_graph_run(tamp_graph* g, int* steps_run) {
  if (!g) return TAMP_ERR_INVALID_ARG;
  tamp_scene* s = g->s;
  DeviceGuard dg(s->device);
  const int n = static_cast<int>(g->prs.size());
  std::vector<int> host(3 + n, 0);  // the control words and step counts (the count sizes stay)
  for (int i = 0; i < n; ++i) {
    if (g->prs[i]->P != g->sizes[i] || !g->prs[i]->has_batch)
      return fail(s, TAMP_ERR_STATE, "batch of a graph's problem changed size; rebuild the graph");
    host[3 + i] = g->prs[i]->t;
  }
  CUDA_TRY(s, cudaMemcpyAsync(g->d_ints, host.data(), host.size() * sizeof(int), cudaMemcpyHostToDevice, s->stream));
  CUDA_TRY(s, cudaGraphLaunch(g->exec, s->stream));
  CUDA_TRY(s, cudaMemcpyAsync(host.data(), g->d_ints, host.size() * sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  tamp_status st = check_device_error(s);  // synchronises
  if (st != TAMP_OK) return st;
  for (int i = 0; i < n; ++i) {
    g->prs[i]->t = host[3 + i];
    g->prs[i]->checked = true;
  }
  if (steps_run) *steps_run = host[2] * g->steps;
  return TAMP_OK;
}

extern "C" tamp_status tamp_graph_destroy(tamp_graph* g) {
  if (!g) return TAMP_ERR_INVALID_ARG;
  DeviceGuard dg(g->s->device);
  cudaStreamSynchronize(g->s->stream);
  free_graph(g);
  return TAMP_OK;
}

// ---------------------------------------------------------------- evaluation with static scratch
// tamp_eval keeps its launch tables (work-item list, problem descriptor, work
// counter) in device memory it allocates on demand.  Callers that may not
// allocate device memory once they are running -- a control loop whose memory
// budget is fixed after start-up, a host framework that hands every device
// byte out of its own pool and forbids library allocations -- use
// tamp_eval_static_scratch instead, which keeps those tables in the array below.
// The array is a file-scope device variable: every GPU that loads the library
// holds one copy until the process exits.  In host code its name only stands in
// for the symbol; the device address comes from cudaGetSymbolAddress, resolved
// once per device on that device's first call.
namespace {

constexpr int kStaticTiles = 4096;                 // largest batch: 4096 tiles of 32/L particles
constexpr size_t kStaticCounterOff = 0;            // int work-item counter
constexpr size_t kStaticDescOff = 256;             // one ProbDesc
constexpr size_t kStaticItemsOff = 512;            // uint32 work items 0 .. kStaticTiles - 1
constexpr size_t kStaticBytes = kStaticItemsOff + 4 * kStaticTiles;
static_assert(sizeof(ProbDesc) <= kStaticItemsOff - kStaticDescOff, "descriptor slot too small");

__device__ __align__(256) unsigned char g_eval_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
unsigned char* g_scratch_dev[kMaxDevices];   // non-null once the device's set-up has succeeded

// With `device` current: resolve the array's device address and write the
// work-item list (tile i of problem 0), which never changes afterwards.  The
// copy is finished on the device before the address is published, so a first
// call whose kernel runs on any stream reads the complete list.  Only a set-up
// that succeeded is kept: after a failure the next call tries again.
cudaError_t static_scratch(int device, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_eval_scratch);
    if (e != cudaSuccess) return e;
    static uint32_t items[kStaticTiles];
    for (int i = 0; i < kStaticTiles; ++i) items[i] = static_cast<uint32_t>(i);
    e = cudaMemcpy(static_cast<unsigned char*>(p) + kStaticItemsOff, items, sizeof items, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    g_scratch_dev[device] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_dev[device];
  return cudaSuccess;
}

}  // namespace

extern "C" tamp_status tamp_eval_static_scratch(tamp_scene* s, int id, int n, const float* x, float* cost,
                                                float* terms, uint8_t* flags, float* grad) {
  Problem* pr = get_problem(s, id);
  if (!pr) return fail(s, TAMP_ERR_INVALID_ARG, "unknown problem %d", id);
  if (n <= 0 || !x) return fail(s, TAMP_ERR_INVALID_ARG, "bad eval arguments");
  if (s->device < 0 || s->device >= kMaxDevices) return fail(s, TAMP_ERR_INVALID_ARG, "device %d", s->device);
  DeviceGuard g(s->device);
  unsigned char* scratch = nullptr;
  cudaError_t e = static_scratch(s->device, &scratch);
  if (e != cudaSuccess)
    return fail(s, TAMP_ERR_CUDA, "static scratch set-up: %s", cudaGetErrorString(e));
  // lane split and shared memory as for tamp_eval
  const int warps = optimize_warps(pr->K);
  int L = preferred_lanes(pr->opt.lanes, n);
  size_t smem = 0;
  for (; L <= 8; L *= 2) {
    smem = 4 * ((s->blob.size() + 3) & ~static_cast<size_t>(3)) +
           optimize_tile_bytes(pr->opt_words, pr->D, pr->NT, pr->NSLOT, pr->NANG, L, false) +
           optimize_scratch_bytes(warps);
    if (smem <= kMaxDynSmem) break;
  }
  if (L > 8) return fail(s, TAMP_ERR_INVALID_ARG, "problem does not fit in shared memory");
  const int PT = 32 / L;
  const int tiles = (n + PT - 1) / PT;
  if (tiles > kStaticTiles)
    return fail(s, TAMP_ERR_INVALID_ARG,
                "batch of %d particles exceeds the static scratch limit of %d tiles (%d particles at %d lanes)", n,
                kStaticTiles, kStaticTiles * PT, L);
  ProbDesc d{};
  d.prob = pr->d_blob;
  d.prob_words = pr->opt_words;
  d.x_in = x; d.stride = n; d.P = n;
  d.out_cost = cost; d.out_terms = terms; d.out_flags = flags; d.out_grad = grad;
  d.n_steps = 0;
  d.gscale = 1.f; d.beta1 = pr->opt.beta1; d.beta2 = pr->opt.beta2; d.eps = pr->opt.eps;
  CUDA_TRY(s, cudaMemcpyAsync(scratch + kStaticDescOff, &d, sizeof d, cudaMemcpyHostToDevice, s->stream));
  CUDA_TRY(s, cudaMemsetAsync(scratch + kStaticCounterOff, 0, sizeof(int), s->stream));  // starts at zero
  LaunchArgs a{};
  a.scene = s->d_blob;
  a.scene_words = static_cast<int>(s->blob.size());
  a.probs = reinterpret_cast<const ProbDesc*>(scratch + kStaticDescOff);
  a.items = reinterpret_cast<const uint32_t*>(scratch + kStaticItemsOff);
  a.n_items = tiles;
  a.item_counter = reinterpret_cast<int*>(scratch + kStaticCounterOff);
  a.err = s->d_err;
  a.scratch_offset = static_cast<int>(smem - optimize_scratch_bytes(warps));
  a.feat = problem_feat(*pr);
  const int per_sm = std::max(1, optimize_blocks_per_sm(L, warps, smem));
  CUDA_TRY(s, launch_optimize(a, L, warps, std::min(tiles, s->sm_count * per_sm), smem, s->stream));
  return TAMP_OK;
}
