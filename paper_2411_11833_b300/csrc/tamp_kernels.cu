// Fused particle-optimisation kernels for sm_103a (B300).
//
// One CTA owns a tile of PT = 32 / L particles of one problem for the whole
// optimisation: the particles' values, Adam moments and gradient live in
// shared memory, every iteration (cost, hand-written adjoint, Adam, Eq. 3 flags)
// runs inside the CTA, and HBM is touched only to load the tile and to write it
// back.  Each configuration of the skeleton is evaluated in independent pieces
// (ranges of its links, with the held or placed box) that the warps pull from
// a per-pass counter for all PT particles; the L lanes of one (particle,
// configuration) pair split the collision environment (obstacles and
// environment-box spheres) between them and meet in a shuffle reduction.
//
// Per configuration (arXiv 2411.11833, Sec. V-A/V-B and the appendix):
//   forward kinematics of the serial arm (standard DH) into registers;
//   Kin: translation / geodesic rotation error between FK(q) and P(p) G(g);
//   CFreeHold: arm spheres and the held box's spheres (at FK(q) G(g)^-1)
//     against oriented cuboids (signed distance) and other boxes' spheres;
//   CFreePlace: the placed box's spheres at P(p) against the same environment;
//   joint limits, grasp bounds and footprint containment (bound distance);
// the adjoint is a reverse sweep over the chain: the links' frames are
// recovered from the tip (T_{l-1} = T_l A_l^-1) instead of being stored, and
// the per-sphere gradients are folded into a world wrench (F, M) whose
// projection on joint l's Plucker axis is dJ/dq_l = z.M + (o x z).F.
#include <cuda_runtime.h>

#include <cstdint>

#include "tamp_dev.cuh"

namespace tamp {

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// 1-D TMA bulk copy global -> shared, completion counted on an mbarrier.
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after `tries` polls (each poll may suspend briefly).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int tries) {
  for (int i = 0; i < tries; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    __nanosleep(64);
  }
  return false;
}

int optimize_warps(int K);

// The broad phase runs over chunks of QUEUE_CHUNK items per lane, so a warp's
// candidate queue never holds more than QUEUE_CAP entries.
constexpr int QUEUE_CHUNK = 16;
// pieces a configuration's evaluation is split into (work items of a pass)
constexpr int NPIECE = 2;
constexpr int QUEUE_CAP = 32 * QUEUE_CHUNK;
// A queue entry is 16 bits: owner lane << QUEUE_ITEM_BITS | item (items are
// the scene's cuboids, then the other boxes: fewer than MAX_OBS + MAX_BOX).
constexpr int QUEUE_ITEM_BITS = 11;
static_assert(MAX_OBS + MAX_BOX <= (1 << QUEUE_ITEM_BITS), "queue entry item field");
// shared memory of one warp's WarpScratch: accumulators, queue, counters
// (padded), then every lane's published batch: its NB spheres and their
// bounding sphere
constexpr int WARP_SCRATCH_BYTES = 32 * NB * 16 + QUEUE_CAP * 2 + 16 + 32 * (NB + 1) * 16;
static_assert(WARP_SCRATCH_BYTES % 16 == 0, "warp scratch alignment");

// ------------------------------------------------------------------ frame helpers
// A frame is R (row-major 3x3) and t.  Right-multiplications used by DH:
__device__ __forceinline__ void rz_right(float* R, float c, float s) {  // T <- T Rz(theta)
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float a = R[3 * i], b = R[3 * i + 1];
    R[3 * i] = fmaf(c, a, s * b);
    R[3 * i + 1] = fmaf(c, b, -s * a);
  }
}
__device__ __forceinline__ void rx_right(float* R, float c, float s) {  // T <- T Rx(alpha)
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float a = R[3 * i + 1], b = R[3 * i + 2];
    R[3 * i + 1] = fmaf(c, a, s * b);
    R[3 * i + 2] = fmaf(c, b, -s * a);
  }
}

__device__ __forceinline__ float tw(const uint32_t* terms, int t) { return __uint_as_float(terms[t * TERM_W + 1]); }

// ------------------------------------------------------------------ collision core
// An oriented cuboid: t' = R^T t, R row-major (columns = box axes), half extents.
struct Obb {
  float tx, ty, tz, r00, r01, r02, r10, r11, r12, r20, r21, r22, hx, hy, hz;
};
// Obstacle o of the structure-of-arrays table; past the end, a far-away box
// that nothing touches (every lane of the warp runs the same trip count).
__device__ __forceinline__ Obb load_obb(const float4* __restrict__ obs, int o, int O) {
  const bool ok = o < O;
  const float4* q = obs + (OBS_W / 4) * (ok ? o : 0);
  const float4 a = q[0], b4 = q[1], c = q[2], d = q[3];
  Obb b;
  b.tx = a.x + (ok ? 0.f : DUMMY_FAR); b.ty = a.y; b.tz = a.z;
  b.r00 = a.w; b.r01 = b4.x; b.r02 = b4.y;
  b.r10 = b4.z; b.r11 = b4.w; b.r12 = c.x;
  b.r20 = c.y; b.r21 = c.z; b.r22 = c.w;
  b.hx = d.x; b.hy = d.y; b.hz = d.z;
  return b;
}
// Point in the box frame: u = R^T c - t'.
__device__ __forceinline__ void obb_local(const Obb& b, float x, float y, float z, float& ux, float& uy, float& uz) {
  ux = fmaf(b.r00, x, fmaf(b.r10, y, fmaf(b.r20, z, -b.tx)));
  uy = fmaf(b.r01, x, fmaf(b.r11, y, fmaf(b.r21, z, -b.ty)));
  uz = fmaf(b.r02, x, fmaf(b.r12, y, fmaf(b.r22, z, -b.tz)));
}
// max_i(|u_i| - h_i): a sphere of radius r can only touch the box if this is < r.
__device__ __forceinline__ float obb_gap(const Obb& b, float x, float y, float z) {
  float ux, uy, uz;
  obb_local(b, x, y, z, ux, uy, uz);
  return fmaxf(fabsf(ux) - b.hx, fmaxf(fabsf(uy) - b.hy, fabsf(uz) - b.hz));
}
// Exact penetration max(0, r - sdf), sdf = ||max(q, 0)|| + min(max_i q_i, 0) with
// q = |u| - h, and its gradient with respect to the sphere centre (-R dsdf/du).
__device__ __forceinline__ float obb_pen(const Obb& b, float x, float y, float z, float r, float& gx, float& gy,
                                         float& gz) {
  float ux, uy, uz;
  obb_local(b, x, y, z, ux, uy, uz);
  const float qx = fabsf(ux) - b.hx, qy = fabsf(uy) - b.hy, qz = fabsf(uz) - b.hz;
  const float mx = fmaxf(qx, 0.f), my = fmaxf(qy, 0.f), mz = fmaxf(qz, 0.f);
  const float o2 = fmaf(mx, mx, fmaf(my, my, mz * mz));
  gx = gy = gz = 0.f;
  if (!(r > 0.f && o2 < r * r)) return 0.f;
  float dux = 0.f, duy = 0.f, duz = 0.f, sdf;
  if (o2 > 0.f) {
    const float d = sqrtf(o2);
    const float inv = 1.f / d;
    sdf = d;
    dux = copysignf(mx * inv, ux);
    duy = copysignf(my * inv, uy);
    duz = copysignf(mz * inv, uz);
  } else if (qx >= qy && qx >= qz) {
    sdf = qx;
    dux = copysignf(1.f, ux);
  } else if (qy >= qz) {
    sdf = qy;
    duy = copysignf(1.f, uy);
  } else {
    sdf = qz;
    duz = copysignf(1.f, uz);
  }
  gx = -fmaf(b.r00, dux, fmaf(b.r01, duy, b.r02 * duz));
  gy = -fmaf(b.r10, dux, fmaf(b.r11, duy, b.r12 * duz));
  gz = -fmaf(b.r20, dux, fmaf(b.r21, duy, b.r22 * duz));
  return r - sdf;
}

// Per-warp scratch of the exact phase in shared memory: the candidate queue
// (cuboid entries from the front, box entries from the back) and per-owner
// accumulators (gradient and penetration of each of its NB spheres).
struct WarpScratch {
  uint16_t* queue;   // QUEUE_CAP entries: owner lane << QUEUE_ITEM_BITS | item
  int* count;        // [2]: cuboid entries, box entries
  float4* acc;       // [32][NB]: (dpen/dc x, y, z; pen)
  float4* sph;       // [32][NB + 1]: each lane's batch (x, y, z, r) and its bounding sphere
};

// Penetration of the register batches of NB spheres held by the 32 lanes of a
// warp into the environment of their configurations: static cuboids and the
// spheres of every other box at its current pose.  Returns this lane's summed
// penetration depth (unweighted) and adds d(depth)/d(centre) into (gx, gy, gz);
// gradients towards boxes whose pose is a placement variable are added (times
// wenv) straight into the tile's gradient.
//
// Broad phase (per lane): a sphere (cb, Rb) bounding the lane's batch is tested
// once against every cuboid (max_i(|u_i| - h_i) < Rb, implied by any contact)
// and against the bounding sphere of every other box.  These tests never miss a
// contact; the few percent of items that pass are appended to the warp's queue.
// Exact phase (per warp): every lane takes one queued (owner, item) pair, pulls
// the owner's spheres by shuffle, computes the exact penetrations and gradients
// and adds them to the owner's accumulators -- all 32 lanes work whatever the
// owners.  Pairs the broad phase skips have zero penetration and gradient, so
// the result equals the all-pairs sum.  Lane `sub` of the L lanes of a
// (particle, configuration) takes items sub, sub + L, ...
template <int L, bool PR>
__device__ __forceinline__ float collide(const float (&cx)[NB], const float (&cy)[NB], const float (&cz)[NB],
                                         const float (&cr)[NB], float (&gx)[NB], float (&gy)[NB],
                                         float (&gz)[NB], float cbx, float cby, float cbz, float Rb,
                                         const float4* __restrict__ obs, const float4* __restrict__ obs2, int O,
                                         const int* __restrict__ env,
                                         int n_env, const float* __restrict__ boxr, const int* __restrict__ slots,
                                         const float4* __restrict__ bloc, const float4* __restrict__ binit,
                                         int NBS, const float4* __restrict__ place, float* G, int pl, int sub,
                                         int lane, float wenv, const WarpScratch& ws, unsigned& n_obb,
                                         unsigned& n_box) {
  constexpr int PT = 32 / L;
  const int n_items = O + n_env;  // cuboids, then the other boxes
  bool published = false;
  // the batch centre in both halves of a packed pair (two cuboids per test)
  const float2 cx2 = make_float2(cbx, cbx), cy2 = make_float2(cby, cby), cz2 = make_float2(cbz, cbz);
  for (int base = 0; base < n_items; base += QUEUE_CHUNK * L) {
    // ---- broad phase over this chunk of items: cuboids (PR: two at a time in
    // packed FP32 pairs, the same roundings as one at a time), then the other
    // boxes.  PR is the plain instantiation's choice: in the instantiations
    // with optional terms the pairs measured slower (more register pressure).
    const int end = min(base + QUEUE_CHUNK * L, n_items), cend = min(end, O);
    // the batch bound against the other box's bounding sphere and against the
    // oriented box holding its spheres (centre, yaw, sphere hull); a contact
    // needs both: |d| < Rb + r_box and ||max(|u| - hull, 0)|| < Rb
    auto box_test = [&](int i) {
      const int4 er = *reinterpret_cast<const int4*>(env + (i - O) * ENV_W);  // box, src, slot
      const float4* br = reinterpret_cast<const float4*>(boxr + er.x * BOX_W);
      const float4 b0 = br[0], b2 = br[2];  // (half extents, bound radius), (cos, sin, hull x, y)
      const float hull_z = br[3].x;
      float x, y, z, cy_, sy_;
      if (er.y < 0) {
        const float4 b1 = br[1];
        x = b1.x; y = b1.y; z = b1.z; cy_ = b2.x; sy_ = b2.y;
      } else {
        const float4 pp = place[er.z * PT + pl];
        x = pp.x; y = pp.y; z = __int_as_float(slots[er.z * SLOT_W + 2]); cy_ = pp.z; sy_ = pp.w;
      }
      const float dx = cbx - x, dy = cby - y, dz = cbz - z, R = Rb + b0.w;
      const float ux = fmaf(cy_, dx, sy_ * dy), uy = fmaf(-sy_, dx, cy_ * dy);
      const float qx = fmaxf(fabsf(ux) - b2.z, 0.f), qy = fmaxf(fabsf(uy) - b2.w, 0.f);
      const float qz = fmaxf(fabsf(dz) - hull_z, 0.f);
      if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < R * R && fmaf(qx, qx, fmaf(qy, qy, qz * qz)) < Rb * Rb) {
        const int q = atomicAdd(&ws.count[1], 1);
        ws.queue[QUEUE_CAP - 1 - q] = static_cast<uint16_t>(lane << QUEUE_ITEM_BITS | i);
      }
    };
    if constexpr (PR) {
      for (int i = base + 2 * sub; i < cend; i += 2 * L) {
        const float4* q = obs2 + (i >> 1) * (OBS2_W / 4);
        const float4 q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3], q4 = q[4], q5 = q[5], q6 = q[6], q7 = q[7];
        const float2 ux = __ffma2_rn(make_float2(q0.x, q0.y), cx2,
                                     __ffma2_rn(make_float2(q0.z, q0.w), cy2,
                                                __ffma2_rn(make_float2(q1.x, q1.y), cz2, make_float2(q1.z, q1.w))));
        const float2 uy = __ffma2_rn(make_float2(q2.x, q2.y), cx2,
                                     __ffma2_rn(make_float2(q2.z, q2.w), cy2,
                                                __ffma2_rn(make_float2(q3.x, q3.y), cz2, make_float2(q3.z, q3.w))));
        const float2 uz = __ffma2_rn(make_float2(q4.x, q4.y), cx2,
                                     __ffma2_rn(make_float2(q4.z, q4.w), cy2,
                                                __ffma2_rn(make_float2(q5.x, q5.y), cz2, make_float2(q5.z, q5.w))));
        // max_i(|u_i| - h_i) < Rb for each of the two (i + 1 = O: the far pad)
        if (fmaxf(fabsf(ux.x) - q6.x, fmaxf(fabsf(uy.x) - q6.z, fabsf(uz.x) - q7.x)) < Rb) {
          const int e = atomicAdd(&ws.count[0], 1);
          ws.queue[e] = static_cast<uint16_t>(lane << QUEUE_ITEM_BITS | i);
        }
        if (fmaxf(fabsf(ux.y) - q6.y, fmaxf(fabsf(uy.y) - q6.w, fabsf(uz.y) - q7.y)) < Rb) {
          const int e = atomicAdd(&ws.count[0], 1);
          ws.queue[e] = static_cast<uint16_t>(lane << QUEUE_ITEM_BITS | (i + 1));
        }
      }
      for (int i = max(base, O) + sub; i < end; i += L) box_test(i);
    } else {
      for (int i = base + sub; i < end; i += L) {
        if (i < O) {
          if (obb_gap(load_obb(obs, i, O), cbx, cby, cbz) < Rb) {
            const int e = atomicAdd(&ws.count[0], 1);
            ws.queue[e] = static_cast<uint16_t>(lane << QUEUE_ITEM_BITS | i);
          }
        } else {
          box_test(i);
        }
      }
    }
    __syncwarp();
    const int n_c = ws.count[0], n_b = ws.count[1];
    if (n_c + n_b == 0) continue;  // warp-uniform: nothing to resolve in this chunk
    if (!published) {
      // every lane publishes its batch once; the exact tasks read it from here
      float4* mine = ws.sph + lane * (NB + 1);
#pragma unroll
      for (int s = 0; s < NB; ++s) mine[s] = make_float4(cx[s], cy[s], cz[s], cr[s]);
      mine[NB] = make_float4(cbx, cby, cbz, Rb);
      published = true;
      __syncwarp();
    }

    // ---- exact phase, cuboids: one (queued pair, sphere) task per lane
    const int Tc = n_c * NB;
    for (int t0 = 0; t0 < Tc; t0 += 32) {
      const int t = t0 + lane;
      if (t < Tc) {
        const int ci = t / NB, s = t - ci * NB;
        const int ent = ws.queue[ci];
        const int owner = ent >> QUEUE_ITEM_BITS;
        if (s == 0) ++n_obb;
        const float4 sp = ws.sph[owner * (NB + 1) + s];
        if (sp.w > 0.f) {
          const Obb b = load_obb(obs, ent & ((1 << QUEUE_ITEM_BITS) - 1), O);
          float px_, py_, pz_;
          const float pen = obb_pen(b, sp.x, sp.y, sp.z, sp.w, px_, py_, pz_);
          if (pen > 0.f) {
            float4* a = &ws.acc[owner * NB + s];
            atomicAdd(&a->x, px_);
            atomicAdd(&a->y, py_);
            atomicAdd(&a->z, pz_);
            atomicAdd(&a->w, pen);
          }
        }
      }
    }

    // ---- exact phase, other boxes: one (queued pair, owner sphere) task per lane.
    // The sphere is first tested against the oriented box that holds every
    // sphere of the other box's model (any contact needs it within r of that
    // box); only then against the model's spheres:
    // pen = max(0, r_a + r_b - ||c_a - c_b||)
    const int Tb = n_b * NB;
    for (int t0 = 0; t0 < Tb; t0 += 32) {
      const int t = t0 + lane;
      if (t < Tb) {
        const int bi = t / NB, s = t - bi * NB;
        const int ent = ws.queue[QUEUE_CAP - 1 - bi];
        const int owner = ent >> QUEUE_ITEM_BITS;
        if (s == 0) ++n_box;
        const float4 sp = ws.sph[owner * (NB + 1) + s];
        const int opl = owner / L;  // the owner's particle in the tile
        const int4 er = *reinterpret_cast<const int4*>(env + ((ent & ((1 << QUEUE_ITEM_BITS) - 1)) - O) * ENV_W);
        const int j = er.x, src = er.y;
        const float4* br = reinterpret_cast<const float4*>(boxr + j * BOX_W);
        const float4 b2 = br[2];  // cos, sin, hull x, y
        const float hull_z = br[3].x;
        float bx, by, bz, cy_, sy_;
        if (src < 0) {
          const float4 b1 = br[1];
          bx = b1.x; by = b1.y; bz = b1.z; cy_ = b2.x; sy_ = b2.y;
        } else {
          const float4 pp = place[er.z * PT + opl];
          bx = pp.x; by = pp.y; bz = __int_as_float(slots[er.z * SLOT_W + 2]); cy_ = pp.z; sy_ = pp.w;
        }
        const float dx0 = sp.x - bx, dy0 = sp.y - by, dz0 = sp.z - bz;
        const float ux = fmaf(cy_, dx0, sy_ * dy0), uy = fmaf(-sy_, dx0, cy_ * dy0);
        const float qx = fmaxf(fabsf(ux) - b2.z, 0.f), qy = fmaxf(fabsf(uy) - b2.w, 0.f);
        const float qz = fmaxf(fabsf(dz0) - hull_z, 0.f);
        if (sp.w > 0.f && fmaf(qx, qx, fmaf(qy, qy, qz * qz)) < sp.w * sp.w) {
          float ax = 0.f, ay = 0.f, az = 0.f, pen = 0.f;
          float fx = 0.f, fy = 0.f, tq = 0.f;  // push on a moving box: force, torque about its centre
          for (int e = 0; e < NBS; ++e) {
            float4 c;
            if (src < 0) {
              c = binit[j * NBS + e];
            } else {
              const float4 l = bloc[j * NBS + e];
              c = make_float4(bx + fmaf(cy_, l.x, -sy_ * l.y), by + fmaf(sy_, l.x, cy_ * l.y), bz + l.z, l.w);
            }
            const float dx = sp.x - c.x, dy = sp.y - c.y, dz = sp.z - c.z;
            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float Rs = sp.w + c.w;
            if (c.w >= 0.f && d2 < Rs * Rs) {
              const float d = sqrtf(d2);
              pen += Rs - d;
              if (d > 0.f) {
                const float inv = 1.f / d;
                const float vx = dx * inv, vy = dy * inv, vz = dz * inv;
                ax -= vx;
                ay -= vy;
                az -= vz;
                fx += vx;
                fy += vy;
                tq = fmaf(c.x - bx, vy, fmaf(-(c.y - by), vx, tq));
              }
            }
          }
          if (pen > 0.f) {
            float4* a = &ws.acc[owner * NB + s];
            atomicAdd(&a->x, ax);
            atomicAdd(&a->y, ay);
            atomicAdd(&a->z, az);
            atomicAdd(&a->w, pen);
          }
          if (src >= 0 && (fx != 0.f || fy != 0.f || tq != 0.f)) {
            atomicAdd(&G[src * PT + opl], wenv * fx);
            atomicAdd(&G[(src + 1) * PT + opl], wenv * fy);
            atomicAdd(&G[(src + 2) * PT + opl], wenv * tq);
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) {
      ws.count[0] = 0;
      ws.count[1] = 0;
    }
    __syncwarp();  // the reset lands before any lane appends to the next chunk
  }
  // ---- each lane collects (and clears) its accumulators
  __syncwarp();
  float J = 0.f;
  if (published) {
#pragma unroll
    for (int s = 0; s < NB; ++s) {
      const float4 a = ws.acc[lane * NB + s];
      gx[s] += a.x;
      gy[s] += a.y;
      gz[s] += a.z;
      J += a.w;
      ws.acc[lane * NB + s] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
  }
  return J;
}

// Bound distance ||max(lo - v, v - hi, 0)|| and its gradient (appendix listing).
template <int N>
__device__ __forceinline__ float bound_dist(const float (&v)[N], const float (&lo)[N], const float (&hi)[N],
                                            float (&grad)[N]) {
  float e[N];
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    e[i] = fmaxf(fmaxf(lo[i] - v[i], v[i] - hi[i]), 0.f);
    s = fmaf(e[i], e[i], s);
  }
  const float d = sqrtf(s);
  const float inv = d > 0.f ? 1.f / d : 0.f;
#pragma unroll
  for (int i = 0; i < N; ++i) grad[i] = (v[i] > hi[i] ? e[i] : (v[i] < lo[i] ? -e[i] : 0.f)) * inv;
  return d;
}

// ------------------------------------------------------------------ one configuration
// A configuration is evaluated in two independent pieces so that warps can
// balance them dynamically:
//   head (piece 0)  Kin, the held box and links n .. m + 1, plus the scalar
//                   terms (joint limits, grasp bounds or containment)
//   tail (piece 1)  links m .. 1, the base spheres and the placed box
// Each piece sweeps from its top link down to joint 1: after each link the
// joint's torque dJ/dq_l = z.M + (o x z).F is taken from the wrench of the
// piece's own spheres so far, so the two pieces' torques add up to the
// configuration's.  Sphere batches are visited by one loop (a single inlined
// copy of the collision code keeps the kernel small):
//   phase 0  the held box, in the object frame FK(q) G(g)^-1 (head)
//   phase 1  links (tip to base); the frame steps back to T_{l-1} after each
//   phase 2  spheres fixed to the base (tail, cost only)
//   phase 3  the placed box at P(p) (tail of a Place: CFreePlace)
template <int L, bool EX, bool KT, bool PR>
__device__ void eval_config(const uint32_t* __restrict__ sc, const uint32_t* __restrict__ pb, int k, int piece,
                            const float* __restrict__ X, float* G, float* Tm, const int* __restrict__ slots,
                            const float4* __restrict__ place, const float2* __restrict__ trig,
                            const WarpScratch& ws, unsigned& n_obb, unsigned& n_box, int lane, int pl, int sub) {
  constexpr int PT = 32 / L;
  const int nj = sc[SH_NJ];
  const float* arm = reinterpret_cast<const float*>(sc + sc[SH_OFF_ARM]);
  const float4* sph = reinterpret_cast<const float4*>(sc + sc[SH_OFF_SPH]);
  const int O = sc[SH_O];
  const float4* obs = reinterpret_cast<const float4*>(sc + sc[SH_OFF_OBS]);
  const float4* obs2 = reinterpret_cast<const float4*>(sc + sc[SH_OFF_OBS2]);
  const float* boxr = reinterpret_cast<const float*>(sc + sc[SH_OFF_BOX]);
  const float4* bloc = reinterpret_cast<const float4*>(sc + sc[SH_OFF_BLOC]);
  const float4* binit = reinterpret_cast<const float4*>(sc + sc[SH_OFF_BINIT]);
  const float4* sphb = reinterpret_cast<const float4*>(sc + sc[SH_OFF_SPHB]);
  const float* surf = reinterpret_cast<const float*>(sc + sc[SH_OFF_SURF]);
  const int NBS = sc[SH_NBS];
  const int nbs_pad = (NBS + NB - 1) / NB * NB;

  const int* cf = reinterpret_cast<const int*>(pb + pb[PH_OFF_CFG] + k * CFG_W);
  const float* cff = reinterpret_cast<const float*>(cf);
  const int kind = cf[CF_KIND], b = cf[CF_BOX], qo = cf[CF_QOFF], go = cf[CF_GOFF], tsrc = cf[CF_TSRC];
  const int n_env = cf[CF_NENV];
  const int* env = reinterpret_cast<const int*>(pb + pb[PH_OFF_ENV]) + cf[CF_ENVOFF] * ENV_W;
  const uint32_t* terms = pb + pb[PH_OFF_TERMS];
  const float w_kp = tw(terms, cf[CF_T_KP]), w_kr = tw(terms, cf[CF_T_KR]);
  const float w_cf = tw(terms, cf[CF_T_CF]), w_jl = tw(terms, cf[CF_T_JL]), w_x = tw(terms, cf[CF_T_X]);
  const int cp_src = cf[CF_CP_SRC], cp_first = cf[CF_CP_FIRST], cp_count = cp_src >= 0 ? cf[CF_CP_COUNT] : 0;
  const float w_cp = cp_count > 0 ? tw(terms, cf[CF_CP_T]) : 0.f;
  const bool head = piece == 0, last = piece == NPIECE - 1;
  // a trajectory knot: no Kin, no grasp / containment term; the held box only on a MoveHold
  // (KT: the kernel is built for problems with knots; otherwise these are constants)
  const bool knot = KT && kind == CK_KNOT, hold = !KT || cf[CF_HOLD] != 0;
  // 6-DOF grasps (extended instantiation only): G(g) = Trans Rz(yaw) Ry(pitch) Rx(roll) Rx(pi)
  const bool g6 = EX && pb[PH_GRASP6] != 0;
  const int ntg = nj + 1 + (g6 ? 2 : 0);
  // links of each piece, so that sphere batches spread evenly: the head also
  // has the held box (2 batches), the tail the placed box (1)
  const int n_head = NPIECE == 2 ? nj / 2 : max(0, (nj + 3) / 3 - 2);       // links of the head
  const int n_tail = NPIECE == 2 ? nj - n_head : max(0, (nj + 3) / 3 - 1);  // links of the tail
  const int top = head ? nj : (last ? n_tail : nj - n_head);                  // this piece's top link
  const int lo = head ? nj - n_head + 1 : (last ? 1 : n_tail + 1);            // ... and bottom link
  // terms computed redundantly count on lane 0 only; Kin belongs to the head
  const float k0 = (sub == 0 && head && !knot) ? 1.f : 0.f;
#define XV(c) X[(c) * PT + pl]
  // (cos, sin) of this configuration's joint angles, then of its grasp yaw
  // (and roll, pitch): its table row, or for a knot, computed here for the
  // joints below this piece's top link and, on a MoveHold, the grasp angles
  const float2* tg = trig + (KT ? max(cf[CF_TG], 0) : k) * ntg * PT + pl;
  float2 kt[MAXJ + 3];
  if (knot) {
    for (int j = 0; j < top; ++j) {
      float sn, cs;
      sincosf(XV(qo + j) + arm[24 + j * ARM_JW + 4], &sn, &cs);
      kt[j] = make_float2(cs, sn);
    }
    if (head && hold)
      for (int j = 0; j < (g6 ? 3 : 1); ++j) {
        float sn, cs;
        sincosf(XV(go + 3 + j), &sn, &cs);
        kt[nj + j] = make_float2(cs, sn);
      }
  }
#define TG(j) (knot ? kt[j] : tg[(j) * PT])

  // ---------------- forward kinematics T_0 .. T_n (the tail stops at T_m)
  float R[9], t[3];
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = arm[i];
  t[0] = arm[9]; t[1] = arm[10]; t[2] = arm[11];
  const int jtop = top;
  for (int j = 0; j < jtop; ++j) {
    const float4 Jp = *reinterpret_cast<const float4*>(arm + 24 + j * ARM_JW);  // a, d, cos alpha, sin alpha
    const float2 cs = TG(j);
    rz_right(R, cs.x, cs.y);
    t[0] = fmaf(Jp.y, R[2], fmaf(Jp.x, R[0], t[0]));
    t[1] = fmaf(Jp.y, R[5], fmaf(Jp.x, R[3], t[1]));
    t[2] = fmaf(Jp.y, R[8], fmaf(Jp.x, R[6], t[2]));
    rx_right(R, Jp.z, Jp.w);
  }
  const float* tl = arm + 12;  // tool frame (R row-major, t)
  // end effector = T_n * tool
  float Re[9], te[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Re[3 * i + j] = fmaf(R[3 * i], tl[j], fmaf(R[3 * i + 1], tl[3 + j], R[3 * i + 2] * tl[6 + j]));
    te[i] = fmaf(R[3 * i], tl[9], fmaf(R[3 * i + 1], tl[10], fmaf(R[3 * i + 2], tl[11], t[i])));
  }

  // ---------------- Kin: target P(p) G(g) (head only)
  float px = 0.f, py = 0.f, cy = 1.f, sy = 0.f;  // target placement: position, yaw
  float gxv = 0.f, gyv = 0.f, gzv = 0.f;          // grasp position
  float sgr = 0.f, cgr = 1.f;  // grasp yaw: R_G = Rz(yaw) Rx(pi) = [[c, s, 0], [s, -c, 0], [0, 0, -1]] (symmetric)
  float F[3] = {0.f, 0.f, 0.f}, Mw[3] = {0.f, 0.f, 0.f}, gg[4] = {0.f, 0.f, 0.f, 0.f}, gp[3] = {0.f, 0.f, 0.f};
  float e_pos = 0.f, e_rot = 0.f;
  float rgx = 0.f, rgy = 0.f;
  float rg[9];                       // R_G with 6-DOF grasps (top-down: from cgr, sgr)
  float cth = 1.f, sth = 0.f;        // cos, sin of the grasp pitch
  float g_roll = 0.f, g_pitch = 0.f; // gradients of the grasp roll and pitch
  auto make_rg = [&]() {
    const float2 r = TG(nj + 1), t = TG(nj + 2);
    const float cph = r.x, sph = r.y;
    cth = t.x; sth = t.y;
    rg[0] = cgr * cth; rg[1] = fmaf(-cgr * sth, sph, sgr * cph); rg[2] = fmaf(-cgr * sth, cph, -sgr * sph);
    rg[3] = sgr * cth; rg[4] = fmaf(-sgr * sth, sph, -cgr * cph); rg[5] = fmaf(-sgr * sth, cph, cgr * sph);
    rg[6] = -sth; rg[7] = -cth * sph; rg[8] = -cth * cph;
  };
  if (head && !knot) {
    const float pz = cff[CF_TZ];
    if (tsrc < 0) {
      px = cff[CF_TX]; py = cff[CF_TY]; cy = cff[CF_TCOS]; sy = cff[CF_TSIN];
    } else {
      const float4 pp = place[cf[CF_T_SLOT] * PT + pl];
      px = pp.x; py = pp.y; cy = pp.z; sy = pp.w;
    }
    gxv = XV(go); gyv = XV(go + 1); gzv = XV(go + 2);
    const float2 gcs = TG(nj);
    cgr = gcs.x; sgr = gcs.y;
    rgx = fmaf(cy, gxv, -sy * gyv); rgy = fmaf(sy, gxv, cy * gyv);
    // yaw of the target frame: placement yaw + grasp yaw
    const float c2 = fmaf(cy, cgr, -sy * sgr), s2 = fmaf(sy, cgr, cy * sgr);
    const float ttx = px + rgx, tty = py + rgy, ttz = pz + gzv;
    float Mr[9];
    if (g6) {
      // M = Re^T R_tgt, R_tgt = Rz(placement yaw) R_G
      make_rg();
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float t0 = fmaf(cy, rg[j], -sy * rg[3 + j]), t1 = fmaf(sy, rg[j], cy * rg[3 + j]);
          Mr[3 * i + j] = fmaf(Re[i], t0, fmaf(Re[3 + i], t1, Re[6 + i] * rg[6 + j]));
        }
    } else {
      // M = Re^T R_tgt, R_tgt = [[c2, s2, 0], [s2, -c2, 0], [0, 0, -1]]
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float e0 = Re[i], e1 = Re[3 + i], e2 = Re[6 + i];
        Mr[3 * i] = fmaf(e0, c2, e1 * s2);
        Mr[3 * i + 1] = fmaf(e0, s2, -e1 * c2);
        Mr[3 * i + 2] = -e2;
      }
    }
    const float wx = Mr[7] - Mr[5], wy = Mr[2] - Mr[6], wz = Mr[3] - Mr[1];
    const float wn = sqrtf(fmaf(wx, wx, fmaf(wy, wy, wz * wz)));
    e_rot = atan2f(0.5f * wn, 0.5f * (Mr[0] + Mr[4] + Mr[8] - 1.f));
    const float dlx = te[0] - ttx, dly = te[1] - tty, dlz = te[2] - ttz;
    e_pos = sqrtf(fmaf(dlx, dlx, fmaf(dly, dly, dlz * dlz)));
    // world wrench on the end effector from Kin (lane 0 only)
    float fkx = 0.f, fky = 0.f, fkz = 0.f;
    if (e_pos > 0.f) {
      const float s = w_kp / e_pos;
      fkx = s * dlx; fky = s * dly; fkz = s * dlz;
    }
    float ubx = 0.f, uby = 0.f, ubz = 0.f;  // w_kr * R_EE * (unit axis of M)
    if (wn > 0.f) {
      const float s = w_kr / wn;
      const float ux = s * wx, uy = s * wy, uz = s * wz;
      ubx = fmaf(Re[0], ux, fmaf(Re[1], uy, Re[2] * uz));
      uby = fmaf(Re[3], ux, fmaf(Re[4], uy, Re[5] * uz));
      ubz = fmaf(Re[6], ux, fmaf(Re[7], uy, Re[8] * uz));
    }
    F[0] = k0 * fkx; F[1] = k0 * fky; F[2] = k0 * fkz;
    Mw[0] = k0 * (te[1] * fkz - te[2] * fky - ubx);
    Mw[1] = k0 * (te[2] * fkx - te[0] * fkz - uby);
    Mw[2] = k0 * (te[0] * fky - te[1] * fkx - ubz);
    // gradients of the target: dJ/dt_tgt = -f, dJ/domega_tgt = ub
    gg[0] = k0 * (-(cy * fkx + sy * fky));
    gg[1] = k0 * (-(-sy * fkx + cy * fky));
    gg[2] = k0 * (-fkz);
    gg[3] = k0 * ubz;
    if (g6) {
      // the target turns about R_P Rz(yaw) y (pitch) and R_P Rz(yaw) Ry(pitch) x (roll)
      g_pitch = k0 * fmaf(-s2, ubx, c2 * uby);
      g_roll = k0 * fmaf(c2 * cth, ubx, fmaf(s2 * cth, uby, -sth * ubz));
    }
    gp[0] = k0 * (-fkx);
    gp[1] = k0 * (-fky);
    gp[2] = k0 * (fkx * rgy - fky * rgx + ubz);
  } else if (head && hold) {  // a MoveHold knot: the held box's grasp
    gxv = XV(go); gyv = XV(go + 1); gzv = XV(go + 2);
    const float2 gcs = TG(nj);
    cgr = gcs.x; sgr = gcs.y;
    if (g6) make_rg();
  }
  float J_hold = 0.f, J_place = 0.f;
  float gpc[3] = {0.f, 0.f, 0.f};  // Kin target / containment -> this configuration's placement
  float gcp[3] = {0.f, 0.f, 0.f};  // CFreePlace part -> placement cp_src

  // ---------------- batches: held box, links n..1, base, placed box
  // Every batch is c = R l' + t with (R, t) the current link frame, except the
  // placed box (phase 3), which overwrites (R, t) with P(p) once the links are done.
  // A held-box sphere l (object frame) is first moved into frame n:
  // l' = tool (G(g)^-1 l) = t_tool + R_tool R_G (l - g).
  // a piece without links of its own below the end effector (the tail of a
  // very short arm) starts at the base spheres
  int phase = head ? 0 : (top >= 1 ? 1 : 2), l = top;
  int s0 = head ? 0 : sc[SH_LINK0 + top], s1 = head ? (hold ? nbs_pad : 0) : sc[SH_LINK0 + top + 1];
  if (!head && top < lo && !(last && top == 0)) s0 = s1 = 0;
  for (;;) {
    if (s0 >= s1) {
      if (phase == 0) {
        phase = 1;
        s0 = sc[SH_LINK0 + l]; s1 = sc[SH_LINK0 + l + 1];
        if (l < lo) s0 = s1 = 0;  // the head has no link of its own
      } else if (phase == 1) {
        // joint l: T_{l-1} = T_l Rx(-alpha) Tx(-a) Tz(-d) Rz(-theta); it turns the
        // links >= l about z_{l-1} through o_{l-1}: dJ/dq_l = z.M + (o x z).F
        const float4 Jp = *reinterpret_cast<const float4*>(arm + 24 + (l - 1) * ARM_JW);  // a, d, cos, sin alpha
        rx_right(R, Jp.z, -Jp.w);
        t[0] -= fmaf(Jp.x, R[0], Jp.y * R[2]);
        t[1] -= fmaf(Jp.x, R[3], Jp.y * R[5]);
        t[2] -= fmaf(Jp.x, R[6], Jp.y * R[8]);
        const float zx = R[2], zy = R[5], zz = R[8];
        const float ox = t[1] * zz - t[2] * zy, oy = t[2] * zx - t[0] * zz, oz = t[0] * zy - t[1] * zx;
        const float tq =
            fmaf(zx, Mw[0], fmaf(zy, Mw[1], fmaf(zz, Mw[2], fmaf(ox, F[0], fmaf(oy, F[1], oz * F[2])))));
        atomicAdd(&G[(qo + l - 1) * PT + pl], tq);
        const float2 cs = TG(l - 1);
        rz_right(R, cs.x, -cs.y);
        --l;
        if (l == 0) phase = 2;
        s0 = sc[SH_LINK0 + l]; s1 = sc[SH_LINK0 + l + 1];
        if (l < lo && !(last && l == 0)) s0 = s1 = 0;  // other pieces' links: torques only
      } else if (phase == 2 && cp_count > 0 && last) {
        phase = 3;
        s0 = cp_first; s1 = cp_first + (cp_count + NB - 1) / NB * NB;
        const float4 pp = place[cf[CF_CP_SLOT] * PT + pl];  // (x, y, cos yaw, sin yaw)
        R[0] = pp.z; R[1] = -pp.w; R[2] = 0.f;
        R[3] = pp.w; R[4] = pp.z; R[5] = 0.f;
        R[6] = 0.f; R[7] = 0.f; R[8] = 1.f;
        t[0] = pp.x; t[1] = pp.y; t[2] = cff[CF_PZ];
      } else {
        break;
      }
      continue;
    }
    float cx[NB], cyy[NB], cz[NB], cr[NB], gx[NB], gyy[NB], gz[NB];
#pragma unroll
    for (int s = 0; s < NB; ++s) {
      float4 p;
      if (phase == 0 || phase == 3) {
        const int lim = phase == 0 ? NBS : cp_first + cp_count;
        p = (s0 + s < lim) ? bloc[b * NBS + s0 + s] : make_float4(DUMMY_FAR, DUMMY_FAR, DUMMY_FAR, -1.f);
        if (phase == 0 && s0 + s < NBS) {
          const float vx = p.x - gxv, vy = p.y - gyv, vz = p.z - gzv;
          // R_G^T (l - g) (top-down R_G is symmetric)
          float wx = fmaf(cgr, vx, sgr * vy), wy = fmaf(sgr, vx, -cgr * vy), wz = -vz;
          if (g6) {
            wx = fmaf(rg[0], vx, fmaf(rg[3], vy, rg[6] * vz));
            wy = fmaf(rg[1], vx, fmaf(rg[4], vy, rg[7] * vz));
            wz = fmaf(rg[2], vx, fmaf(rg[5], vy, rg[8] * vz));
          }
          p.x = fmaf(tl[0], wx, fmaf(tl[1], wy, fmaf(tl[2], wz, tl[9])));
          p.y = fmaf(tl[3], wx, fmaf(tl[4], wy, fmaf(tl[5], wz, tl[10])));
          p.z = fmaf(tl[6], wx, fmaf(tl[7], wy, fmaf(tl[8], wz, tl[11])));
        }
      } else {
        p = sph[s0 + s];
      }
      cx[s] = fmaf(R[0], p.x, fmaf(R[1], p.y, fmaf(R[2], p.z, t[0])));
      cyy[s] = fmaf(R[3], p.x, fmaf(R[4], p.y, fmaf(R[5], p.z, t[1])));
      cz[s] = fmaf(R[6], p.x, fmaf(R[7], p.y, fmaf(R[8], p.z, t[2])));
      cr[s] = p.w;
      gx[s] = gyy[s] = gz[s] = 0.f;
    }
    // sphere bounding the batch: arm batches from the scene's per-batch table
    // (link frame); box batches from their spheres (a negative radius marks an
    // unused slot)
    float cbx, cby, cbz, Rb;
    if (phase == 1 || phase == 2) {
      const float4 bb = sphb[s0 / NB];
      cbx = fmaf(R[0], bb.x, fmaf(R[1], bb.y, fmaf(R[2], bb.z, t[0])));
      cby = fmaf(R[3], bb.x, fmaf(R[4], bb.y, fmaf(R[5], bb.z, t[1])));
      cbz = fmaf(R[6], bb.x, fmaf(R[7], bb.y, fmaf(R[8], bb.z, t[2])));
      Rb = bb.w;
    } else {
      float lox = 3.0e38f, loy = 3.0e38f, loz = 3.0e38f, hix = -3.0e38f, hiy = -3.0e38f, hiz = -3.0e38f;
#pragma unroll
      for (int s = 0; s < NB; ++s) {
        if (cr[s] >= 0.f) {
          lox = fminf(lox, cx[s]); hix = fmaxf(hix, cx[s]);
          loy = fminf(loy, cyy[s]); hiy = fmaxf(hiy, cyy[s]);
          loz = fminf(loz, cz[s]); hiz = fmaxf(hiz, cz[s]);
        }
      }
      cbx = 0.5f * (lox + hix); cby = 0.5f * (loy + hiy); cbz = 0.5f * (loz + hiz);
      Rb = -1.f;
#pragma unroll
      for (int s = 0; s < NB; ++s) {
        if (cr[s] >= 0.f) {
          const float dx = cx[s] - cbx, dy = cyy[s] - cby, dz = cz[s] - cbz;
          Rb = fmaxf(Rb, sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) + cr[s] + 1e-5f);
        }
      }
    }
    const float wenv = phase == 3 ? w_cp : w_cf;
    const float Jb = collide<L, PR>(cx, cyy, cz, cr, gx, gyy, gz, cbx, cby, cbz, Rb, obs, obs2, O, env, n_env, boxr, slots,
                                bloc, binit, NBS, place, G, pl, sub, lane, wenv, ws, n_obb, n_box);
    if (phase == 3) {
      J_place += Jb;
#pragma unroll
      for (int s = 0; s < NB; ++s) {
        const float fx = w_cp * gx[s], fy = w_cp * gyy[s];
        gcp[0] += fx;
        gcp[1] += fy;
        gcp[2] += (cx[s] - t[0]) * fy - (cyy[s] - t[1]) * fx;
      }
    } else {
      J_hold += Jb;
      if (phase <= 1) {
#pragma unroll
        for (int s = 0; s < NB; ++s) {
          const float fx = w_cf * gx[s], fy = w_cf * gyy[s], fz = w_cf * gz[s];
          F[0] += fx; F[1] += fy; F[2] += fz;
          Mw[0] += cyy[s] * fz - cz[s] * fy;
          Mw[1] += cz[s] * fx - cx[s] * fz;
          Mw[2] += cx[s] * fy - cyy[s] * fx;
        }
        if (phase == 0) {
          // c = t_EE + R_obj (l - g): the object-frame force G = R_obj^T f moves g
          // by -G and the grasp yaw by -(G x (l - g))_z; R_obj = R R_tool R_G
#pragma unroll
          for (int s = 0; s < NB; ++s) {
            if (s0 + s >= NBS) continue;
            const float fx = w_cf * gx[s], fy = w_cf * gyy[s], fz = w_cf * gz[s];
            const float ax = fmaf(R[0], fx, fmaf(R[3], fy, R[6] * fz));
            const float ay = fmaf(R[1], fx, fmaf(R[4], fy, R[7] * fz));
            const float az = fmaf(R[2], fx, fmaf(R[5], fy, R[8] * fz));
            const float bx = fmaf(tl[0], ax, fmaf(tl[3], ay, tl[6] * az));
            const float by = fmaf(tl[1], ax, fmaf(tl[4], ay, tl[7] * az));
            const float bz = fmaf(tl[2], ax, fmaf(tl[5], ay, tl[8] * az));
            float Gx = fmaf(cgr, bx, sgr * by), Gy = fmaf(sgr, bx, -cgr * by), Gz = -bz;
            if (g6) {
              Gx = fmaf(rg[0], bx, fmaf(rg[1], by, rg[2] * bz));
              Gy = fmaf(rg[3], bx, fmaf(rg[4], by, rg[5] * bz));
              Gz = fmaf(rg[6], bx, fmaf(rg[7], by, rg[8] * bz));
            }
            const float4 lp = bloc[b * NBS + s0 + s];
            const float vx = lp.x - gxv, vy = lp.y - gyv, vz = lp.z - gzv;
            gg[0] -= Gx; gg[1] -= Gy; gg[2] -= Gz;
            gg[3] -= Gy * vx - Gx * vy;
            if (g6) {
              // -(a x (l - g)) . G for the pitch axis a = Rz(yaw) y and the roll axis Rz(yaw) Ry(pitch) x
              const float ptx = cgr * vz, pty = sgr * vz, ptz = fmaf(-sgr, vy, -cgr * vx);  // (-s, c, 0) x v
              g_pitch -= fmaf(ptx, Gx, fmaf(pty, Gy, ptz * Gz));
              const float ax_ = cgr * cth, ay_ = sgr * cth, az_ = -sth;
              const float rx = fmaf(ay_, vz, -az_ * vy), ry = fmaf(az_, vx, -ax_ * vz), rz = fmaf(ax_, vy, -ay_ * vx);
              g_roll -= fmaf(rx, Gx, fmaf(ry, Gy, rz * Gz));
            }
          }
        }
      }
    }
    s0 += NB;
  }

  // ---------------- reduce over the L lanes of this (particle, configuration)
#pragma unroll
  for (int m = 1; m < L; m <<= 1) {
    J_hold += __shfl_xor_sync(0xffffffffu, J_hold, m);
    J_place += __shfl_xor_sync(0xffffffffu, J_place, m);
#pragma unroll
    for (int i = 0; i < 4; ++i) gg[i] += __shfl_xor_sync(0xffffffffu, gg[i], m);
    if (g6) {
      g_roll += __shfl_xor_sync(0xffffffffu, g_roll, m);
      g_pitch += __shfl_xor_sync(0xffffffffu, g_pitch, m);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) gpc[i] += __shfl_xor_sync(0xffffffffu, gpc[i], m);
#pragma unroll
    for (int i = 0; i < 3; ++i) gcp[i] += __shfl_xor_sync(0xffffffffu, gcp[i], m);
  }
  if (sub != 0) return;
  atomicAdd(&Tm[cf[CF_T_CF] * PT + pl], J_hold);
  if (!head) {
    if (!last) return;
    if (cp_count > 0) {
      atomicAdd(&Tm[cf[CF_CP_T] * PT + pl], J_place);
#pragma unroll
      for (int i = 0; i < 3; ++i) atomicAdd(&G[(cp_src + i) * PT + pl], gcp[i]);
    }
    return;
  }

  // ---------------- per-configuration scalar terms (lane 0)
  float jl = 0.f;
  {
    float e2 = 0.f;
    float ex[MAXJ];
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) {
      ex[j] = 0.f;
      if (j < nj) {
        const float* Jp = arm + 24 + j * ARM_JW;
        const float q = XV(qo + j);
        ex[j] = fmaxf(fmaxf(Jp[5] - q, q - Jp[6]), 0.f);
        e2 = fmaf(ex[j], ex[j], e2);
      }
    }
    jl = sqrtf(e2);
    const float inv = jl > 0.f ? w_jl / jl : 0.f;
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) {
      if (j < nj) {
        const float* Jp = arm + 24 + j * ARM_JW;
        const float q = XV(qo + j);
        const float gj = q > Jp[6] ? ex[j] * inv : (q < Jp[5] ? -ex[j] * inv : 0.f);
        if (gj != 0.f) atomicAdd(&G[(qo + j) * PT + pl], gj);
      }
    }
  }
  Tm[cf[CF_T_JL] * PT + pl] = jl;
  if (knot) {
    // a MoveHold knot's held-box collisions move the grasp
    if (hold) {
#pragma unroll
      for (int i = 0; i < 4; ++i) atomicAdd(&G[(go + i) * PT + pl], gg[i]);
      if (g6) {
        atomicAdd(&G[(go + 4) * PT + pl], g_roll);
        atomicAdd(&G[(go + 5) * PT + pl], g_pitch);
      }
    }
    return;
  }
  Tm[cf[CF_T_KP] * PT + pl] = e_pos;
  Tm[cf[CF_T_KR] * PT + pl] = e_rot;
  const float* br = boxr + b * BOX_W;
  if (kind == CK_PICK) {
    // Grasp(o, g): bound distance of g_xyz to [-hx, hx] x [-hy, hy] x [hz - 0.02, hz]
    const float v[3] = {gxv, gyv, gzv};
    const float lo[3] = {-br[0], -br[1], g6 ? -br[2] : br[2] - 0.02f};  // 6-DOF: the whole box
    const float hi[3] = {br[0], br[1], br[2]};
    float gr[3];
    const float d = bound_dist<3>(v, lo, hi, gr);
    Tm[cf[CF_T_X] * PT + pl] = d;
    gg[0] += w_x * gr[0]; gg[1] += w_x * gr[1]; gg[2] += w_x * gr[2];
  } else {
    // StablePlace containment: 4 footprint corners in the surface frame
    const float* sf = surf + cf[CF_SURF] * SURF_W;
    const float scx = sf[0], scy = sf[1], shx = sf[3], shy = sf[4], scs = sf[6], ssn = sf[7];
    float J = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float lx_ = (c & 1 ? 1.f : -1.f) * br[0], ly_ = (c & 2 ? 1.f : -1.f) * br[1];
      const float rx = fmaf(cy, lx_, -sy * ly_), ry = fmaf(sy, lx_, cy * ly_);
      const float wx_ = px + rx - scx, wy_ = py + ry - scy;
      const float v[2] = {fmaf(scs, wx_, ssn * wy_), fmaf(-ssn, wx_, scs * wy_)};
      const float lo[2] = {-shx, -shy}, hi[2] = {shx, shy};
      float gu[2];
      J += bound_dist<2>(v, lo, hi, gu);
      // d/dw = Rz(-yaw_s)^T d/du ; w depends on (px, py) directly and on yaw through r
      const float gwx = fmaf(scs, gu[0], -ssn * gu[1]), gwy = fmaf(ssn, gu[0], scs * gu[1]);
      gpc[0] += w_x * gwx;
      gpc[1] += w_x * gwy;
      gpc[2] += w_x * (rx * gwy - ry * gwx);
    }
    Tm[cf[CF_T_X] * PT + pl] = J;
  }
  // grasp gradient (shared by the Pick and the Place that hold the same grasp)
#pragma unroll
  for (int i = 0; i < 4; ++i) atomicAdd(&G[(go + i) * PT + pl], gg[i]);
  if (g6) {
    atomicAdd(&G[(go + 4) * PT + pl], g_roll);
    atomicAdd(&G[(go + 5) * PT + pl], g_pitch);
  }
  // placement gradient: Kin target if the target is a variable, plus CFreePlace/containment
  const int psrc = cf[CF_PSRC];
  if (tsrc >= 0) {
    gpc[0] += gp[0]; gpc[1] += gp[1]; gpc[2] += gp[2];
  }
  if (psrc >= 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) atomicAdd(&G[(psrc + i) * PT + pl], gpc[i]);
  }
#undef XV
#undef TG
}

// Goal MinimizeObjDist: sum over pairs of moved boxes of ||pos_i - pos_j||.
template <int L>
__device__ void eval_goal(const uint32_t* __restrict__ sc, const uint32_t* __restrict__ pb,
                          const float* __restrict__ X, float* G, float* Tm, int pl) {
  constexpr int PT = 32 / L;
  const int ng = pb[PH_NGOAL], gt = pb[PH_GOAL_T];
  if (gt < 0) return;
  const int* gl = reinterpret_cast<const int*>(pb + pb[PH_OFF_GOAL]);
  const float* boxr = reinterpret_cast<const float*>(sc + sc[SH_OFF_BOX]);
  const float w = tw(pb + pb[PH_OFF_TERMS], gt);
  float J = 0.f;
  for (int i = 0; i < ng; ++i) {
    const int si = gl[i * GOAL_W + 1];
    const float* bi = boxr + gl[i * GOAL_W] * BOX_W;
    const float xi = si >= 0 ? X[si * PT + pl] : bi[4];
    const float yi = si >= 0 ? X[(si + 1) * PT + pl] : bi[5];
    const float zi = si >= 0 ? __int_as_float(gl[i * GOAL_W + 2]) : bi[6];
    for (int j = i + 1; j < ng; ++j) {
      const int sj = gl[j * GOAL_W + 1];
      const float* bj = boxr + gl[j * GOAL_W] * BOX_W;
      const float dx = xi - (sj >= 0 ? X[sj * PT + pl] : bj[4]);
      const float dy = yi - (sj >= 0 ? X[(sj + 1) * PT + pl] : bj[5]);
      const float dz = zi - (sj >= 0 ? __int_as_float(gl[j * GOAL_W + 2]) : bj[6]);
      const float d = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
      J += d;
      if (d > 0.f) {
        const float s = w / d;
        if (si >= 0) {
          atomicAdd(&G[si * PT + pl], s * dx);
          atomicAdd(&G[(si + 1) * PT + pl], s * dy);
        }
        if (sj >= 0) {
          atomicAdd(&G[sj * PT + pl], -s * dx);
          atomicAdd(&G[(sj + 1) * PT + pl], -s * dy);
        }
      }
    }
  }
  Tm[gt * PT + pl] = J;
}

// TrajLength of every motion (Listing 1 MoveFree / MoveHold cost): the
// joint-space length sum_e ||w_{e+1} - w_e|| of the polyline start, knots, end,
// for one particle, with its gradient.
template <int L>
__device__ __noinline__ void eval_traj(const uint32_t* __restrict__ pb, const float* __restrict__ X, float* G, float* Tm, int nj,
                          int pl) {
  constexpr int PT = 32 / L;
  const int ns = pb[PH_NSEG];
  const uint32_t* seg = pb + pb[PH_OFF_SEG];
  const uint32_t* terms = pb + pb[PH_OFF_TERMS];
  for (int si = 0; si < ns; ++si) {
    const uint32_t* r = seg + si * SEG_W;
    const int qa = r[SG_QA], qb = r[SG_QB], qk = r[SG_QK], m = r[SG_M], t = r[SG_T];
    const float wt = tw(terms, t);
    float J = 0.f;
    for (int e = 0; e <= m; ++e) {
      const int o0 = e == 0 ? qa : qk + (e - 1) * nj;
      const int o1 = e == m ? qb : qk + e * nj;
      float d[MAXJ], d2 = 0.f;
#pragma unroll
      for (int j = 0; j < MAXJ; ++j) {
        d[j] = j < nj ? X[(o1 + j) * PT + pl] - X[(o0 + j) * PT + pl] : 0.f;
        d2 = fmaf(d[j], d[j], d2);
      }
      const float len = sqrtf(d2);
      J += len;
      if (len > 0.f) {
        const float inv = wt / len;
#pragma unroll
        for (int j = 0; j < MAXJ; ++j)
          if (j < nj) {
            atomicAdd(&G[(o1 + j) * PT + pl], inv * d[j]);
            atomicAdd(&G[(o0 + j) * PT + pl], -inv * d[j]);
          }
      }
    }
    Tm[t * PT + pl] = J;
  }
}

// One kinematic step: T <- T Rz(q_j + offset_j) Tz(d_j) Tx(a_j) Rx(alpha_j), with
// (cos, sin) of the joint angle from the per-iteration table.
__device__ __forceinline__ void fk_step(float (&R)[9], float (&t)[3], const float* arm, int j, float2 cs) {
  const float4 Jp = *reinterpret_cast<const float4*>(arm + 24 + j * ARM_JW);  // a, d, cos alpha, sin alpha
  rz_right(R, cs.x, cs.y);
  t[0] = fmaf(Jp.y, R[2], fmaf(Jp.x, R[0], t[0]));
  t[1] = fmaf(Jp.y, R[5], fmaf(Jp.x, R[3], t[1]));
  t[2] = fmaf(Jp.y, R[8], fmaf(Jp.x, R[6], t[2]));
  rx_right(R, Jp.z, Jp.w);
}

// SelfCollision of configuration k (the CFree constraints' "does not cause
// robot self-collisions"): for each lower link j, the kinematics walk up from
// T_j and test j's spheres against every higher link i of j's mask (link
// bounding spheres first), and against the held box once the walk reaches
// T_n.  A pair adds max(0, r_a + r_b - d) to the term; its gradient w.r.t. each
// sphere centre goes into that sphere's link wrench (force, moment about the
// origin) -- kept per lane in the warp's exact-phase scratch, idle during this
// item -- and the held box's also into the grasp.  A sweep from T_n down then
// turns the wrenches into joint torques: the two forces of a pair cancel below
// both links.  All lanes call this; lanes with sub != 0 only help restore the
// scratch.
template <int L, bool KT>
__device__ __noinline__ void eval_self(const uint32_t* __restrict__ sc, const uint32_t* __restrict__ pb, int k,
                                       const float* __restrict__ X, float* G, float* Tm,
                                       const float2* __restrict__ trig, const WarpScratch& ws, int lane, int pl,
                                       int sub) {
  constexpr int PT = 32 / L;
  const int nj = sc[SH_NJ];
  float* acc = reinterpret_cast<float*>(ws.acc);  // [6 nj][32]: per link 1..nj force, moment
  __syncwarp();
  if (sub == 0) {
    const float* arm = reinterpret_cast<const float*>(sc + sc[SH_OFF_ARM]);
    const float* tl = arm + 12;
    const float4* sph = reinterpret_cast<const float4*>(sc + sc[SH_OFF_SPH]);
    const float4* sphb = reinterpret_cast<const float4*>(sc + sc[SH_OFF_SPHB]);
    const float4* bloc = reinterpret_cast<const float4*>(sc + sc[SH_OFF_BLOC]);
    const uint32_t* smask = sc + sc[SH_OFF_SELF];
    const int NBS = sc[SH_NBS];
    const int* cf = reinterpret_cast<const int*>(pb + pb[PH_OFF_CFG] + k * CFG_W);
    const int t_self = cf[CF_T_SELF], qo = cf[CF_QOFF], go = cf[CF_GOFF], box = cf[CF_BOX];
    const bool hold = cf[CF_HOLD] != 0;
    const float w = tw(pb + pb[PH_OFF_TERMS], t_self);
    const bool g6 = pb[PH_GRASP6] != 0;
    const float2* tg = trig + (KT ? max(cf[CF_TG], 0) : k) * (nj + 1 + (g6 ? 2 : 0)) * PT + pl;
    // a knot has no table row: its angles are computed once here
    const bool knot = KT && cf[CF_KIND] == CK_KNOT;
    float2 kt[MAXJ + 3];
    if (knot) {
      const float* jr = arm + 24;
      for (int j = 0; j < nj; ++j) {
        float sn, cs;
        sincosf(X[(qo + j) * PT + pl] + jr[j * ARM_JW + 4], &sn, &cs);
        kt[j] = make_float2(cs, sn);
      }
      if (hold)
        for (int j = 0; j < (g6 ? 3 : 1); ++j) {
          float sn, cs;
          sincosf(X[(go + 3 + j) * PT + pl], &sn, &cs);
          kt[nj + j] = make_float2(cs, sn);
        }
    }
    auto TS = [&](int j) { return knot ? kt[j] : tg[j * PT]; };
    for (int i = 0; i < 6 * nj; ++i) acc[i * 32 + lane] = 0.f;
    float gxv = 0.f, gyv = 0.f, gzv = 0.f, cgr = 1.f, sgr = 0.f;
    // R_G (object frame -> gripper target), top-down unless 6-DOF; the pitch and roll axes
    float rg[9] = {1.f, 0.f, 0.f, 0.f, -1.f, 0.f, 0.f, 0.f, -1.f}, cth = 1.f, sth = 0.f;
    if (hold) {
      gxv = X[go * PT + pl]; gyv = X[(go + 1) * PT + pl]; gzv = X[(go + 2) * PT + pl];
      const float2 c = TS(nj);
      cgr = c.x; sgr = c.y;
      float cph = 1.f, sph = 0.f;
      if (g6) {
        const float2 r = TS(nj + 1), t = TS(nj + 2);
        cph = r.x; sph = r.y; cth = t.x; sth = t.y;
      }
      rg[0] = cgr * cth; rg[1] = fmaf(-cgr * sth, sph, sgr * cph); rg[2] = fmaf(-cgr * sth, cph, -sgr * sph);
      rg[3] = sgr * cth; rg[4] = fmaf(-sgr * sth, sph, -cgr * cph); rg[5] = fmaf(-sgr * sth, cph, cgr * sph);
      rg[6] = -sth; rg[7] = -cth * sph; rg[8] = -cth * cph;
    }
    float J = 0.f, gg[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    // adds w * dpen/dc (g) at centre c to the wrench of link l (l = 0: the base, no torque)
    auto add = [&](int l, float cx, float cy, float cz, float gx, float gy, float gz) {
      if (l == 0) return;
      float* a = acc + (l - 1) * 6 * 32 + lane;
      a[0] += gx; a[32] += gy; a[64] += gz;
      a[96] += cy * gz - cz * gy; a[128] += cz * gx - cx * gz; a[160] += cx * gy - cy * gx;
    };
    float Rj[9], tj[3];
#pragma unroll
    for (int i = 0; i < 9; ++i) Rj[i] = arm[i];
    tj[0] = arm[9]; tj[1] = arm[10]; tj[2] = arm[11];
    for (int j = 0; j <= nj; ++j) {
      if (j > 0) fk_step(Rj, tj, arm, j - 1, TS(j - 1));
      uint32_t m = 0;
      for (int i = j + 2; i <= nj; ++i)
        if ((smask[i] >> j) & 1u) m |= 1u << i;
      const bool hj = hold && ((smask[MAXJ + 1] >> j) & 1u);
      if (!m && !hj) continue;
      for (int s0 = sc[SH_LINK0 + j]; s0 < static_cast<int>(sc[SH_LINK0 + j + 1]); s0 += NB) {
        float cx[NB], cy[NB], cz[NB], cr[NB];
#pragma unroll
        for (int s = 0; s < NB; ++s) {
          const float4 p = sph[s0 + s];
          cx[s] = fmaf(Rj[0], p.x, fmaf(Rj[1], p.y, fmaf(Rj[2], p.z, tj[0])));
          cy[s] = fmaf(Rj[3], p.x, fmaf(Rj[4], p.y, fmaf(Rj[5], p.z, tj[1])));
          cz[s] = fmaf(Rj[6], p.x, fmaf(Rj[7], p.y, fmaf(Rj[8], p.z, tj[2])));
          cr[s] = p.w;
        }
        const float4 bj = sphb[s0 / NB];
        const float bjx = fmaf(Rj[0], bj.x, fmaf(Rj[1], bj.y, fmaf(Rj[2], bj.z, tj[0])));
        const float bjy = fmaf(Rj[3], bj.x, fmaf(Rj[4], bj.y, fmaf(Rj[5], bj.z, tj[1])));
        const float bjz = fmaf(Rj[6], bj.x, fmaf(Rj[7], bj.y, fmaf(Rj[8], bj.z, tj[2])));
        // one sphere (x, y, z, r) on link li against the batch of link j
        auto pair = [&](int li, float x, float y, float z, float r, float (&gh)[3]) {
          gh[0] = gh[1] = gh[2] = 0.f;
          if (!(r >= 0.f)) return;
          {  // the sphere against the bounding sphere of link j's batch first
            const float dx = x - bjx, dy = y - bjy, dz = z - bjz, R = r + bj.w;
            if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= R * R) return;
          }
#pragma unroll
          for (int t = 0; t < NB; ++t) {
            const float dx = x - cx[t], dy = y - cy[t], dz = z - cz[t];
            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float R = r + cr[t];
            if (cr[t] >= 0.f && d2 < R * R) {
              const float d = sqrtf(d2);
              J += R - d;
              if (d > 0.f) {
                const float s = w / d;  // w dpen/dc_i = -w u, w dpen/dc_j = +w u, u = (c_i - c_j) / d
                const float ux = s * dx, uy = s * dy, uz = s * dz;
                gh[0] -= ux; gh[1] -= uy; gh[2] -= uz;
                add(j, cx[t], cy[t], cz[t], ux, uy, uz);
              }
            }
          }
          if (gh[0] != 0.f || gh[1] != 0.f || gh[2] != 0.f) add(li, x, y, z, gh[0], gh[1], gh[2]);
        };
        float Ri[9], ti[3];
#pragma unroll
        for (int i = 0; i < 9; ++i) Ri[i] = Rj[i];
        ti[0] = tj[0]; ti[1] = tj[1]; ti[2] = tj[2];
        for (int i = j + 1; i <= nj; ++i) {
          fk_step(Ri, ti, arm, i - 1, TS(i - 1));
          if ((m >> i) & 1u) {
            for (int s1 = sc[SH_LINK0 + i]; s1 < static_cast<int>(sc[SH_LINK0 + i + 1]); s1 += NB) {
              const float4 bi = sphb[s1 / NB];
              const float bx = fmaf(Ri[0], bi.x, fmaf(Ri[1], bi.y, fmaf(Ri[2], bi.z, ti[0]))) - bjx;
              const float by = fmaf(Ri[3], bi.x, fmaf(Ri[4], bi.y, fmaf(Ri[5], bi.z, ti[1]))) - bjy;
              const float bz = fmaf(Ri[6], bi.x, fmaf(Ri[7], bi.y, fmaf(Ri[8], bi.z, ti[2]))) - bjz;
              const float Rb = bi.w + bj.w;
              if (fmaf(bx, bx, fmaf(by, by, bz * bz)) >= Rb * Rb) continue;  // the batches cannot touch
              for (int s = 0; s < NB; ++s) {
                const float4 p = sph[s1 + s];
                float gh[3];
                pair(i, fmaf(Ri[0], p.x, fmaf(Ri[1], p.y, fmaf(Ri[2], p.z, ti[0]))),
                     fmaf(Ri[3], p.x, fmaf(Ri[4], p.y, fmaf(Ri[5], p.z, ti[1]))),
                     fmaf(Ri[6], p.x, fmaf(Ri[7], p.y, fmaf(Ri[8], p.z, ti[2]))), p.w, gh);
              }
            }
          }
          if (i == nj && hj) {
            // the held box's spheres, rigid with frame n: c = T_n tool G(g)^-1 l; first its
            // bounding sphere (radius about the box centre) against link j's batch
            {
              const float vx = -gxv, vy = -gyv, vz = -gzv;
              const float wx = fmaf(rg[0], vx, fmaf(rg[3], vy, rg[6] * vz));
              const float wy = fmaf(rg[1], vx, fmaf(rg[4], vy, rg[7] * vz));
              const float wz = fmaf(rg[2], vx, fmaf(rg[5], vy, rg[8] * vz));
              const float px = fmaf(tl[0], wx, fmaf(tl[1], wy, fmaf(tl[2], wz, tl[9])));
              const float py = fmaf(tl[3], wx, fmaf(tl[4], wy, fmaf(tl[5], wz, tl[10])));
              const float pz = fmaf(tl[6], wx, fmaf(tl[7], wy, fmaf(tl[8], wz, tl[11])));
              const float dx = fmaf(Ri[0], px, fmaf(Ri[1], py, fmaf(Ri[2], pz, ti[0]))) - bjx;
              const float dy = fmaf(Ri[3], px, fmaf(Ri[4], py, fmaf(Ri[5], pz, ti[1]))) - bjy;
              const float dz = fmaf(Ri[6], px, fmaf(Ri[7], py, fmaf(Ri[8], pz, ti[2]))) - bjz;
              const float Rh = reinterpret_cast<const float*>(sc + sc[SH_OFF_BOX])[box * BOX_W + 3] + bj.w;
              if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= Rh * Rh) continue;  // i == nj: the walk ends here
            }
            for (int e = 0; e < NBS; ++e) {
              const float4 l = bloc[box * NBS + e];
              const float vx = l.x - gxv, vy = l.y - gyv, vz = l.z - gzv;
              const float wx = fmaf(rg[0], vx, fmaf(rg[3], vy, rg[6] * vz));
              const float wy = fmaf(rg[1], vx, fmaf(rg[4], vy, rg[7] * vz));
              const float wz = fmaf(rg[2], vx, fmaf(rg[5], vy, rg[8] * vz));
              const float px = fmaf(tl[0], wx, fmaf(tl[1], wy, fmaf(tl[2], wz, tl[9])));
              const float py = fmaf(tl[3], wx, fmaf(tl[4], wy, fmaf(tl[5], wz, tl[10])));
              const float pz = fmaf(tl[6], wx, fmaf(tl[7], wy, fmaf(tl[8], wz, tl[11])));
              float gh[3];
              pair(nj, fmaf(Ri[0], px, fmaf(Ri[1], py, fmaf(Ri[2], pz, ti[0]))),
                   fmaf(Ri[3], px, fmaf(Ri[4], py, fmaf(Ri[5], pz, ti[1]))),
                   fmaf(Ri[6], px, fmaf(Ri[7], py, fmaf(Ri[8], pz, ti[2]))), l.w, gh);
              // the grasp moves the sphere by -R_obj: g by -R_obj^T f, its yaw by -(R_obj^T f x (l - g))_z
              const float ax = fmaf(Ri[0], gh[0], fmaf(Ri[3], gh[1], Ri[6] * gh[2]));
              const float ay = fmaf(Ri[1], gh[0], fmaf(Ri[4], gh[1], Ri[7] * gh[2]));
              const float az = fmaf(Ri[2], gh[0], fmaf(Ri[5], gh[1], Ri[8] * gh[2]));
              const float bx = fmaf(tl[0], ax, fmaf(tl[3], ay, tl[6] * az));
              const float by = fmaf(tl[1], ax, fmaf(tl[4], ay, tl[7] * az));
              const float bz = fmaf(tl[2], ax, fmaf(tl[5], ay, tl[8] * az));
              const float Gx = fmaf(rg[0], bx, fmaf(rg[1], by, rg[2] * bz));
              const float Gy = fmaf(rg[3], bx, fmaf(rg[4], by, rg[5] * bz));
              const float Gz = fmaf(rg[6], bx, fmaf(rg[7], by, rg[8] * bz));
              gg[0] -= Gx; gg[1] -= Gy; gg[2] -= Gz;
              gg[3] -= Gy * vx - Gx * vy;
              if (g6) {  // -(a x (l - g)) . G for the pitch and roll axes
                gg[5] -= fmaf(cgr * vz, Gx, fmaf(sgr * vz, Gy, fmaf(-sgr, vy, -cgr * vx) * Gz));
                const float ax_ = cgr * cth, ay_ = sgr * cth, az_ = -sth;
                gg[4] -= fmaf(fmaf(ay_, vz, -az_ * vy), Gx, fmaf(fmaf(az_, vx, -ax_ * vz), Gy,
                                                                 fmaf(ax_, vy, -ay_ * vx) * Gz));
              }
            }
          }
        }
      }
    }
    Tm[t_self * PT + pl] = J;
    if (hold)
      for (int i = 0; i < (g6 ? 6 : 4); ++i) atomicAdd(&G[(go + i) * PT + pl], gg[i]);
    // torques: from T_n down, the wrench of links >= l at joint l
    float R[9], t[3];
#pragma unroll
    for (int i = 0; i < 9; ++i) R[i] = arm[i];
    t[0] = arm[9]; t[1] = arm[10]; t[2] = arm[11];
    for (int j = 0; j < nj; ++j) fk_step(R, t, arm, j, TS(j));
    float F[3] = {0.f, 0.f, 0.f}, M[3] = {0.f, 0.f, 0.f};
    for (int l = nj; l >= 1; --l) {
      const float* a = acc + (l - 1) * 6 * 32 + lane;
      F[0] += a[0]; F[1] += a[32]; F[2] += a[64];
      M[0] += a[96]; M[1] += a[128]; M[2] += a[160];
      const float4 Jp = *reinterpret_cast<const float4*>(arm + 24 + (l - 1) * ARM_JW);
      rx_right(R, Jp.z, -Jp.w);
      t[0] -= fmaf(Jp.x, R[0], Jp.y * R[2]);
      t[1] -= fmaf(Jp.x, R[3], Jp.y * R[5]);
      t[2] -= fmaf(Jp.x, R[6], Jp.y * R[8]);
      const float zx = R[2], zy = R[5], zz = R[8];
      const float ox = t[1] * zz - t[2] * zy, oy = t[2] * zx - t[0] * zz, oz = t[0] * zy - t[1] * zx;
      atomicAdd(&G[(qo + l - 1) * PT + pl],
                fmaf(zx, M[0], fmaf(zy, M[1], fmaf(zz, M[2], fmaf(ox, F[0], fmaf(oy, F[1], oz * F[2]))))));
      const float2 cs = TS(l - 1);
      rz_right(R, cs.x, -cs.y);
    }
  }
  // restore the scratch the exact phase expects: zero accumulators and counters
  __syncwarp();
  for (int i = lane; i < 32 * NB * 4; i += 32) acc[i] = 0.f;
  if (lane == 0) {
    ws.count[0] = 0;
    ws.count[1] = 0;
  }
  __syncwarp();
}

// ------------------------------------------------------------------ fused optimisation kernel
// One tile of PT particles of one problem: load it, run n_steps fused
// iterations (evaluation + adjoint, Eq. 3 check, Adam) and one final check,
// write it back.  All threads of the CTA call this together.
// FEAT: the optional terms the kernel is built for (a KernelFeat; 0: none,
// the configuration code of every skeleton without them).  REC: the launch
// keeps the problems' best-satisfying records (tamp_query_best); launches
// without them run none of that code.
template <int L, int FEAT, bool REC>
__device__ void run_tile(const ProbDesc& d, int tile, const uint32_t* s_sc, const uint32_t* s_pb, float* tile_mem,
                         const WarpScratch& ws, bool mv_global) {
  constexpr int PT = 32 / L;
  // EX: 6-DOF grasps; KT: knots (configurations of kind 2, TrajLength); SC: SelfCollision
  constexpr bool EX = FEAT == FEAT_EXT || FEAT == FEAT_KNOT6, KT = FEAT == FEAT_KNOT || FEAT == FEAT_KNOT6;
  constexpr bool SC = FEAT != 0;
  const int D = s_pb[PH_D], K = s_pb[PH_K], NT = s_pb[PH_NT];
  // the tile in shared memory: x, the Adam moments m and v (unless they are
  // used in place in global memory, for problems whose tile would not fit
  // otherwise), the gradient, the term values
  float* sx = tile_mem;
  float* sm = mv_global ? nullptr : sx + D * PT;
  float* sv = mv_global ? nullptr : sm + D * PT;
  float* sg = mv_global ? sx + D * PT : sv + D * PT;
  float* st = sg + D * PT;
  int* sflag = reinterpret_cast<int*>(st + NT * PT);
  // pose of every placed box of every particle at the current iterate: (x, y,
  // cos yaw, sin yaw), refreshed at the start of each iteration
  float4* splace = reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(sflag) + ((PT * 4 + 15) & ~15));
  const int NSLOT = s_pb[PH_NSLOT];
  // (cos, sin) of the joint angles and grasp angles of every Pick / Place
  // configuration at the current iterate (knots compute theirs where they use them)
  float2* strig = reinterpret_cast<float2*>(splace + NSLOT * PT);
  const int ntab = KT ? static_cast<int>(s_pb[PH_NTAB]) : K;
  const int* tab = reinterpret_cast<const int*>(s_pb + s_pb[PH_OFF_TAB]);
  const int nj = s_sc[SH_NJ], ntg = nj + 1 + ((EX && s_pb[PH_GRASP6] != 0) ? 2 : 0), NA = ntab * ntg;
  const float* arm = reinterpret_cast<const float*>(s_sc + s_sc[SH_OFF_ARM]);
  const uint32_t* cfg0 = s_pb + s_pb[PH_OFF_CFG];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int w = tid >> 5, lane = tid & 31;
  const int pl = lane / L, sub = lane % L;
  const int tile0 = tile * PT;
  const int t0 = d.t_dev ? *d.t_dev : d.t0;
  // best-satisfying record: the particles (bits) whose x_t beat their record at
  // the last check; warp 0 copies their staged x_t at the top of the next iteration
  __shared__ unsigned s_snap;

  for (int i = tid; i < D * PT; i += nthr) {
    const int c = i / PT, p = i % PT, gp = tile0 + p;
    float xv = 0.f, mv = 0.f, vv = 0.f;
    if (gp < d.P) {
      xv = d.x_in[c * d.stride + gp];
      if (d.load_mv && !mv_global) {
        mv = d.m[c * d.stride + gp];
        vv = d.v[c * d.stride + gp];
      }
      if (mv_global && !d.load_mv && d.m) {  // moments start at zero, in place
        d.m[c * d.stride + gp] = 0.f;
        d.v[c * d.stride + gp] = 0.f;
      }
    }
    sx[i] = xv; sg[i] = 0.f;
    if (!mv_global) {
      sm[i] = mv;
      sv[i] = vv;
    }
  }
  __syncthreads();  // the tile is loaded before the placement poses are read from it
  const uint32_t* terms = s_pb + s_pb[PH_OFF_TERMS];
  const float* lr = reinterpret_cast<const float*>(s_pb + s_pb[PH_OFF_LR]);
  const int* slots = reinterpret_cast<const int*>(s_pb + s_pb[PH_OFF_SLOT]);
  // work items of an evaluation pass: two pieces per configuration, later
  // configurations first (their environments hold more placed boxes), then the
  // goal cost; warps pull them from a counter so that they finish together
  __shared__ int s_next;
  const bool has_goal = s_pb[PH_GOAL_T] != 0xffffffffu, has_traj = KT && s_pb[PH_NSEG] != 0;
  // SelfCollision: one more item per configuration (after the pieces)
  const int n_self = (SC && static_cast<int>(s_pb[s_pb[PH_OFF_CFG] + CF_T_SELF]) >= 0) ? K : 0;
  const int n_work = NPIECE * K + n_self + (has_goal ? 1 : 0) + (has_traj ? 1 : 0);
  // Adam's bias corrections 1 / (1 - beta^t) of each iteration's step t, by one
  // thread, handed to the others through shared memory.  At one lane per
  // (particle, configuration): 1 - beta^t = -expm1(t log1p(beta - 1)), which
  // keeps FP32's relative accuracy (1.2e-7 against the FP64 value for t up to
  // 2e5) also where beta^t is close to 1, with no FP64 (slow on this part) and
  // no double carried across the pass (+0.9% on the packing workload).  With
  // more lanes the register allocation of the pass came out slower that way
  // (-1.4% on the stress scene at 2 lanes, A/B on one box), so there beta^t is
  // kept in FP64 and stepped by one multiplication per iteration.
  __shared__ float s_ib[2];
  const float lb1 = log1pf(d.beta1 - 1.f), lb2 = log1pf(d.beta2 - 1.f);
  double b1t = 0.0, b2t = 0.0;
  if (L > 1 && tid == 0) {
    b1t = pow(static_cast<double>(d.beta1), t0);
    b2t = pow(static_cast<double>(d.beta2), t0);
  }
  unsigned n_obb = 0, n_box = 0;  // broad-phase candidates resolved exactly (work accounting)
  // this thread's entries of the angle table: a = tid / PT + m (nthr / PT) (nthr is a multiple of PT),
  // particle tid % PT, row a / ntg, angle a % ntg
  const int tg_p = tid % PT, tg_a0 = tid / PT, tg_astep = nthr / PT;
  const int tg_r0 = tg_a0 / ntg, tg_j0 = tg_a0 - tg_r0 * ntg;
  const int tg_rstep = tg_astep / ntg, tg_jstep = tg_astep - tg_rstep * ntg;

  for (int it = 0;; ++it) {
    if (tid == 0) {
      s_next = 0;
      if constexpr (L == 1) {
        const float ts = static_cast<float>(t0 + it + 1);  // this iteration's step
        s_ib[0] = -1.f / expm1f(ts * lb1);
        s_ib[1] = -1.f / expm1f(ts * lb2);
      } else {
        b1t *= static_cast<double>(d.beta1);  // beta^(t0 + it + 1), for this iteration's step
        b2t *= static_cast<double>(d.beta2);
        s_ib[0] = static_cast<float>(1.0 / (1.0 - b1t));
        s_ib[1] = static_cast<float>(1.0 / (1.0 - b2t));
      }
    }
    if constexpr (REC) {
      // x_t is staged, as the tile's contiguous [D][PT] block, in the block of
      // this iteration's parity while the pass only reads it; warp 0 first copies
      // the last check's new records out of the other parity's block (staged at
      // the top of the last iteration, so complete and visible here).  The two
      // blocks of the problem are [ceil(P / 32) * 32 / PT tiles][D][PT] each.
      const long half = static_cast<long>(D) * ((d.P + 31) & ~31), toff = static_cast<long>(tile) * D * PT;
      if (w == 0 && it > 0) {
        const unsigned snap = s_snap;
        if (snap) {
          const float* prev = d.stage_x + ((it - 1) & 1) * half + toff;
          for (int i = lane; i < D * PT; i += 32) {
            const int c = i / PT, p = i - c * PT;
            if ((snap >> p) & 1u) d.best_x[static_cast<long>(c) * d.stride + tile0 + p] = prev[i];
          }
        }
      }
      const float4* src = reinterpret_cast<const float4*>(sx);
      float4* dst = reinterpret_cast<float4*>(d.stage_x + (it & 1) * half + toff);
      for (int j = tid; j < D * PT / 4; j += nthr) dst[j] = src[j];
    }
    for (int i = tid; i < NT * PT; i += nthr) st[i] = 0.f;  // collision terms are sums over pieces
    for (int i = tid; i < NSLOT * PT; i += nthr) {
      const int si = i / PT, p = i - si * PT;
      const int off = slots[si * SLOT_W + 1];
      float sn, cs;
      sincosf(sx[(off + 2) * PT + p], &sn, &cs);
      splace[i] = make_float4(sx[off * PT + p], sx[(off + 1) * PT + p], cs, sn);
    }
    // entry (row r, angle j) of particle tg_p; the row and angle step without a division
    for (int a = tg_a0, r = tg_r0, j = tg_j0; a < NA; a += tg_astep) {
      const int k = KT ? tab[r] : r;  // without knots every configuration has a row
      const int* cf = reinterpret_cast<const int*>(cfg0 + k * CFG_W);
      // joints, then the grasp yaw (and roll, pitch): components go + 3 (+ 4, 5)
      const float ang = j < nj ? sx[(cf[CF_QOFF] + j) * PT + tg_p] + arm[24 + j * ARM_JW + 4]
                               : sx[(cf[CF_GOFF] + 3 + (j - nj)) * PT + tg_p];
      float sn, cs;
      sincosf(ang, &sn, &cs);
      strig[a * PT + tg_p] = make_float2(cs, sn);
      r += tg_rstep;
      j += tg_jstep;
      if (j >= ntg) {
        j -= ntg;
        ++r;
      }
    }
    __syncthreads();
    for (;;) {
      int item = 0;
      if (lane == 0) item = atomicAdd(&s_next, 1);
      item = __shfl_sync(0xffffffffu, item, 0);
      if (item >= n_work) break;
      if (item < NPIECE * K) {
        eval_config<L, EX, KT, FEAT == 0>(s_sc, s_pb, K - 1 - item / NPIECE, item % NPIECE, sx, sg, st, slots, splace, strig, ws, n_obb,
                       n_box, lane, pl, sub);
      } else if (SC && item < NPIECE * K + n_self) {
        if constexpr (SC)
          eval_self<L, KT>(s_sc, s_pb, K - 1 - (item - NPIECE * K), sx, sg, st, strig, ws, lane, pl, sub);
      } else if (sub == 0) {
        if (has_goal && item == NPIECE * K + n_self)
          eval_goal<L>(s_sc, s_pb, sx, sg, st, pl);
        else if constexpr (KT)
          eval_traj<L>(s_pb, sx, sg, st, nj, pl);
      }
    }
    __syncthreads();
    // Eq. 3 at x_t
    if (w == 0) {
      int sat = 0;
      if (lane < PT) {
        sat = 1;
        for (int tt = 0; tt < NT; ++tt) {
          const uint32_t* tr = terms + tt * TERM_W;
          if (static_cast<int>(tr[3]) >= 0 && st[tt * PT + lane] > __uint_as_float(tr[2])) sat = 0;
        }
        sflag[lane] = sat;
        if (tile0 + lane >= d.P) sat = 0;
      }
      if (__any_sync(0xffffffffu, sat) && lane == 0 && d.first_iter) atomicMin(d.first_iter, t0 + it);
      if constexpr (REC) {
        // a satisfying particle whose Eq. 2 cost (summed as the query's cost) is
        // below its record takes the check's index and cost; its state is copied
        // straight from the tile at the launch's last check, otherwise from the
        // staging block at the top of the next iteration
        bool better = false;
        if (sat) {
          float c = 0.f;
          for (int tt = 0; tt < NT; ++tt) c = fmaf(__uint_as_float(terms[tt * TERM_W + 1]), st[tt * PT + lane], c);
          const int gp = tile0 + lane;
          if (c < d.best_cost[gp]) {
            d.best_cost[gp] = c;
            d.best_iter[gp] = t0 + it;
            better = true;
          }
        }
        const unsigned snap = __ballot_sync(0xffffffffu, better);
        if (it == d.n_steps) {
          if (snap)
            for (int i = lane; i < D * PT; i += 32) {
              const int c = i / PT, p = i - c * PT;
              if ((snap >> p) & 1u) d.best_x[static_cast<long>(c) * d.stride + tile0 + p] = sx[i];
            }
        } else if (lane == 0) {
          s_snap = snap;
        }
      }
    }
    if (it == d.n_steps) break;
    // Adam (Kingma & Ba) on the Eq. 4 gradient; the gradient buffer is cleared for the next pass
    const float ib1 = s_ib[0], ib2 = s_ib[1];
    for (int i = tid; i < D * PT; i += nthr) {
      const float g = sg[i] * d.gscale;
      float m0, v0;
      long gi = 0;
      if (mv_global) {
        const int c = i / PT, gp = tile0 + (i - c * PT);
        gi = static_cast<long>(c) * d.stride + gp;
        const bool in = gp < d.P;
        m0 = in ? d.m[gi] : 0.f;
        v0 = in ? d.v[gi] : 0.f;
      } else {
        m0 = sm[i];
        v0 = sv[i];
      }
      const float m = fmaf(d.beta1, m0, (1.f - d.beta1) * g);
      const float v = fmaf(d.beta2, v0, (1.f - d.beta2) * g * g);
      if (mv_global) {
        if (tile0 + (i % PT) < d.P) {
          d.m[gi] = m;
          d.v[gi] = v;
        }
      } else {
        sm[i] = m;
        sv[i] = v;
      }
      sx[i] -= lr[i / PT] * (m * ib1) / (sqrtf(v * ib2) + d.eps);
      sg[i] = 0.f;
    }
    __syncthreads();
  }
  __syncthreads();

  if (d.work) {
    unsigned long long no = n_obb, nb = n_box;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
      no += __shfl_xor_sync(0xffffffffu, no, m);
      nb += __shfl_xor_sync(0xffffffffu, nb, m);
    }
    if (lane == 0 && (no | nb)) {
      atomicAdd(&d.work[0], no);
      atomicAdd(&d.work[1], nb);
    }
  }

  // ---------------- outputs of the last check
  if (tid < PT && tile0 + tid < d.P) {
    const int gp = tile0 + tid;
    if (d.out_cost) {
      float c = 0.f;
      for (int tt = 0; tt < NT; ++tt) c = fmaf(__uint_as_float(terms[tt * TERM_W + 1]), st[tt * PT + tid], c);
      d.out_cost[gp] = c;
    }
    if (d.out_flags) d.out_flags[gp] = static_cast<uint8_t>(sflag[tid]);
  }
  if (d.out_terms)
    for (int i = tid; i < NT * PT; i += nthr) {
      const int tt = i / PT, p = i % PT;
      if (tile0 + p < d.P) d.out_terms[tt * d.stride + tile0 + p] = st[i];
    }
  if (d.out_counts)
    for (int tt = tid; tt < NT; tt += nthr) {
      const uint32_t* tr = terms + tt * TERM_W;
      const int ci = static_cast<int>(tr[3]);
      if (ci < 0) continue;
      const float tol = __uint_as_float(tr[2]);
      int cnt = 0;
      for (int p = 0; p < PT; ++p) cnt += (tile0 + p < d.P && st[tt * PT + p] <= tol) ? 1 : 0;
      if (cnt) atomicAdd(&d.out_counts[ci], cnt);
    }
  for (int i = tid; i < D * PT; i += nthr) {
    const int c = i / PT, p = i % PT, gp = tile0 + p;
    if (gp >= d.P) continue;
    if (d.out_grad) d.out_grad[c * d.stride + gp] = sg[i];
    if (d.x_out) d.x_out[c * d.stride + gp] = sx[i];
    if (d.m && !mv_global) d.m[c * d.stride + gp] = sm[i];
    if (d.v && !mv_global) d.v[c * d.stride + gp] = sv[i];
  }
}

// Persistent kernel: every CTA stages the scene tables once (TMA bulk copy),
// then takes (problem, tile) work items from a global counter -- longest
// skeletons first, as the host orders them -- staging a problem's tables
// whenever it moves to a new problem.  Many skeletons of uneven length and
// particle count thus share one launch and balance across the SMs.
template <int L, int FEAT, bool REC>
__global__ void __launch_bounds__(512, 1) optimize_kernel(LaunchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag, s_item;
  const int sw = (a.scene_words + 3) & ~3;
  uint32_t* s_sc = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* s_pb = s_sc + sw;
  const int tid = threadIdx.x;
  if (a.stop && *a.stop) return;  // a graph chunk after the stopping condition was met
  uint32_t phase = 0;
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(&bar, 1);
    fence_mbar_init();
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bar, static_cast<uint32_t>(sw * 4));
    tma_bulk_g2s(s_sc, a.scene, static_cast<uint32_t>(sw * 4), &bar);
    if (!mbar_wait_bounded(&bar, phase, 1 << 20)) {
      atomicOr(a.err, ERR_TMA_TIMEOUT);
      abort_flag = 1;
      mbar_wait_bounded(&bar, phase, 1 << 16);  // give the copy in flight a last chance to land
    }
  }
  phase ^= 1u;
  __syncthreads();
  if (abort_flag) return;

  const int w = tid >> 5, lane = tid & 31, W = blockDim.x >> 5;
  // exact-phase scratch of each warp at the end of the dynamic shared memory
  WarpScratch ws;
  {
    unsigned char* base = smem_raw + a.scratch_offset + static_cast<size_t>(w) * WARP_SCRATCH_BYTES;
    ws.acc = reinterpret_cast<float4*>(base);
    ws.queue = reinterpret_cast<uint16_t*>(base + 32 * NB * 16);
    ws.count = reinterpret_cast<int*>(base + 32 * NB * 16 + QUEUE_CAP * 2);
    ws.sph = reinterpret_cast<float4*>(base + 32 * NB * 16 + QUEUE_CAP * 2 + 16);
    for (int i = lane; i < 32 * NB; i += 32) ws.acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane == 0) { ws.count[0] = 0; ws.count[1] = 0; }
  }
  (void)W;
  int cur = -1;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(a.item_counter, 1);
    __syncthreads();
    const int idx = s_item;
    if (idx >= a.n_items) break;
    const uint32_t item = a.items[idx];
    const int p = static_cast<int>(item >> ITEM_TILE_BITS);
    const int tile = static_cast<int>(item & ((1u << ITEM_TILE_BITS) - 1));
    const ProbDesc& d = a.probs[p];
    const int pw = (d.prob_words + 3) & ~3;
    if (p != cur) {
      if (tid == 0) {
        fence_proxy_async_smem();  // earlier generic reads of the old tables before the async overwrite
        mbar_arrive_expect_tx(&bar, static_cast<uint32_t>(pw * 4));
        tma_bulk_g2s(s_pb, d.prob, static_cast<uint32_t>(pw * 4), &bar);
        if (!mbar_wait_bounded(&bar, phase, 1 << 20)) {
          atomicOr(a.err, ERR_TMA_TIMEOUT);
          abort_flag = 1;
          mbar_wait_bounded(&bar, phase, 1 << 16);
        }
      }
      phase ^= 1u;
      cur = p;
      __syncthreads();
      if (abort_flag) return;
    }
    run_tile<L, FEAT, REC>(d, tile, s_sc, s_pb, reinterpret_cast<float*>(s_pb + pw), ws, a.mv_global != 0);
    __syncthreads();  // everyone has read s_item and the tables before they change
  }
}

// ------------------------------------------------------------------ uniform sampler
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += W0;
      k.y += W1;
    }
    const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
    const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}
__device__ __forceinline__ float philox_u01(uint32_t i, uint32_t c, uint2 key) {
  const uint4 w = philox4x32_10(make_uint4(i, c, 0u, 0u), key);
  return static_cast<float>(w.x >> 8) * (1.0f / 16777216.0f);
}

__global__ void sample_uniform_kernel(const uint32_t* __restrict__ pb, const uint32_t* __restrict__ sc,
                                      float* __restrict__ x, float* __restrict__ m, float* __restrict__ v,
                                      int stride, int P, uint2 key) {
  const int c = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const uint32_t* rec = pb + pb[PH_OFF_SAMP] + c * SAMP_W;
  const int kind = static_cast<int>(rec[0]);
  const float lo = __uint_as_float(rec[1]), hi = __uint_as_float(rec[2]);
  float val;
  if (kind == SK_LINEAR) {
    val = fmaf(hi - lo, philox_u01(i, c, key), lo);
  } else {
    const float* sf = reinterpret_cast<const float*>(sc + sc[SH_OFF_SURF]) + rec[3] * SURF_W;
    const int cx = kind == SK_PLACE_X ? c : c - 1;
    const float su = fmaf(2.f * sf[3], philox_u01(i, cx, key), -sf[3]);
    const float sv = fmaf(2.f * sf[4], philox_u01(i, cx + 1, key), -sf[4]);
    val = kind == SK_PLACE_X ? sf[0] + fmaf(sf[6], su, -sf[7] * sv) : sf[1] + fmaf(sf[7], su, sf[6] * sv);
  }
  x[c * stride + i] = val;
  m[c * stride + i] = 0.f;
  v[c * stride + i] = 0.f;
}

// Learned proposals (Sec. V-A): overwrite the grasp / placement components of
// a uniformly sampled batch with draws from the network's per-row Gaussians.
// Slot k of row r draws t = mu + exp(clamp(s, -8, 3)) xi with xi a standard
// normal by Box-Muller from Philox at counter (i, 16 r + k, 1, 0); positions
// are clamped to the sampling bounds, yaws are atan2 of the (sin, cos) slots.
__device__ __forceinline__ float philox_normal(uint32_t i, uint32_t c, uint2 key) {
  const uint4 w = philox4x32_10(make_uint4(i, c, 1u, 0u), key);
  const float u1 = static_cast<float>((w.x >> 8) + 1u) * (1.0f / 16777216.0f);  // (0, 1]
  const float u2 = static_cast<float>(w.y >> 8) * (1.0f / 16777216.0f);         // [0, 1)
  return sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}

__global__ void sample_proposal_kernel(const uint32_t* __restrict__ rows, const float* __restrict__ out,
                                       float* __restrict__ x, int stride, int P, uint2 key) {
  const int r = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const uint32_t* rec = rows + r * PROW_W;
  const float* f = reinterpret_cast<const float*>(rec + 4);
  const float* o = out + r * 2 * PROP_NT;
  const int off = static_cast<int>(rec[1]);
  auto draw = [&](int k) {
    const float ls = fminf(fmaxf(o[PROP_NT + k], -8.f), 3.f);
    return fmaf(expf(ls), philox_normal(i, 16u * r + k, key), o[k]);
  };
  auto clamp1 = [](float t) { return fminf(fmaxf(t, -1.f), 1.f); };
  if (rec[0] == 0) {
    const float t0 = draw(0), t1 = draw(1), t2 = draw(2), t3 = draw(3), t4 = draw(4);
    x[off * stride + i] = f[0] * clamp1(t0);
    x[(off + 1) * stride + i] = f[1] * clamp1(t1);
    x[(off + 2) * stride + i] = f[2] - 0.02f + 0.01f * (clamp1(t2) + 1.f);
    x[(off + 3) * stride + i] = atan2f(t4, t3);
  } else {
    const float t5 = draw(5), t6 = draw(6), t7 = draw(7), t8 = draw(8);
    const float u = f[4] * clamp1(t5), v = f[5] * clamp1(t6);
    x[off * stride + i] = f[0] + fmaf(f[2], u, -f[3] * v);
    x[(off + 1) * stride + i] = f[1] + fmaf(f[3], u, f[2] * v);
    x[(off + 2) * stride + i] = atan2f(t8, t7);
  }
}

// Conditional configuration sampler (Sec. VI: joint positions solved by
// parallel inverse kinematics for the target poses implied by the sampled
// grasps and placements).  One thread per particle visits its configurations
// in skeleton order; each has one free yaw (a Pick's grasp yaw, a Place's
// placement yaw).  Damped least squares on r = [t* - t_EE ; log(R* R_EE^T)]
// over (q, y) with A = [J_q | -dr*/dy], step = A^T (A A^T + lam^2 I)^-1 r
// scaled to a largest entry <= dmax, q clamped to its limits.
__device__ __forceinline__ void rot_log(const float (&E)[9], float (&w)[3]) {
  const float vx = 0.5f * (E[7] - E[5]), vy = 0.5f * (E[2] - E[6]), vz = 0.5f * (E[3] - E[1]);
  const float s = sqrtf(vx * vx + vy * vy + vz * vz);
  const float c = 0.5f * (E[0] + E[4] + E[8] - 1.f);
  if (s > 1e-6f || c > 0.f) {
    const float f = s > 1e-6f ? atan2f(s, c) / s : 1.f;
    w[0] = f * vx; w[1] = f * vy; w[2] = f * vz;
    return;
  }
  // a half turn: (R + I) / 2 = axis axis^T
  const float d0 = 0.5f * (E[0] + 1.f), d1 = 0.5f * (E[4] + 1.f), d2 = 0.5f * (E[8] + 1.f);
  const int k = (d0 >= d1 && d0 >= d2) ? 0 : (d1 >= d2 ? 1 : 2);
  const float dk = fmaxf(k == 0 ? d0 : (k == 1 ? d1 : d2), 1e-30f);
  const float inv = 3.14159265358979f * rsqrtf(dk);
  // column k of (R + I) / 2
  w[0] = (k == 0 ? d0 : 0.5f * E[k]) * inv;
  w[1] = (k == 1 ? d1 : 0.5f * E[3 + k]) * inv;
  w[2] = (k == 2 ? d2 : 0.5f * E[6 + k]) * inv;
}

// The configurations of one box (its Picks and Places, in skeleton order) form
// a chain: a Place reads the grasp yaw its Pick chose, a later Pick the yaw its
// Place chose, and nothing reads another box's variables.  One thread per
// (particle, chain); chains[c * chain_w] is a chain's length, then its
// configuration indices.  Configurations whose joints lie below component
// `keep` belong to a prefix copied from another skeleton's batch (subgraph
// caching, Sec. VI) and keep their values; later ones read its grasps and yaws.
__global__ void __launch_bounds__(128) ik_configs_kernel(const uint32_t* __restrict__ pb,
                                                         const uint32_t* __restrict__ sc, float* __restrict__ x,
                                                         int stride, int P, int iters, float lam, float dmax,
                                                         const int* __restrict__ chains, int n_chains,
                                                         int chain_w, int keep) {
  const long g = static_cast<long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= static_cast<long>(P) * n_chains) return;
  const int i = static_cast<int>(g % P), chain = static_cast<int>(g / P);
  const int* ch = chains + chain * chain_w;
  const int nj = sc[SH_NJ];
  const float* arm = reinterpret_cast<const float*>(sc + sc[SH_OFF_ARM]);
  const float* tl = arm + 12;
  const float lam2 = lam * lam;
#define XG(c) x[(c) * stride + i]
  for (int ci = 0; ci < ch[0]; ++ci) {
    const int k = ch[1 + ci];
    const int* cf = reinterpret_cast<const int*>(pb + pb[PH_OFF_CFG] + k * CFG_W);
    const float* cff = reinterpret_cast<const float*>(cf);
    const int kind = cf[CF_KIND], qo = cf[CF_QOFF], go = cf[CF_GOFF], tsrc = cf[CF_TSRC];
    if (qo < keep) continue;  // a configuration of a kept prefix: its values stay as they are
    const bool place = kind == 1;
    float bx, by, bz, byaw;
    if (tsrc < 0) {
      bx = cff[CF_TX]; by = cff[CF_TY]; bz = cff[CF_TZ]; byaw = cff[CF_TYAW];
    } else {
      bx = XG(tsrc); by = XG(tsrc + 1); bz = cff[CF_TZ]; byaw = XG(tsrc + 2);
    }
    const float gx = XG(go), gy = XG(go + 1), gz = XG(go + 2);
    // 6-DOF grasps: roll and pitch stay as sampled
    const bool g6 = pb[PH_GRASP6] != 0;
    float cph = 1.f, sph = 0.f, cth = 1.f, sth = 0.f;
    if (g6) {
      sincosf(XG(go + 4), &sph, &cph);
      sincosf(XG(go + 5), &sth, &cth);
    }
    const int yo = place ? tsrc + 2 : go + 3;
    float y = XG(yo);
    float q[MAXJ];
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) q[j] = j < nj ? XG(qo + j) : 0.f;
    for (int it = 0; it < iters; ++it) {
      // target: position P_box g, orientation Rz(box yaw + grasp yaw) Rx(pi)
      const float pyaw = place ? y : byaw;
      const float phi = place ? y + XG(go + 3) : byaw + y;
      float sp, cp, sf, cfv;
      sincosf(pyaw, &sp, &cp);
      sincosf(phi, &sf, &cfv);
      const float tx = bx + fmaf(cp, gx, -sp * gy), ty = by + fmaf(sp, gx, cp * gy), tz = bz + gz;
      float Rt[9] = {cfv, sf, 0.f, sf, -cfv, 0.f, 0.f, 0.f, -1.f};
      if (g6) {
        // R* = Rz(box yaw) R_G, R_G = Rz(grasp yaw) Ry(pitch) Rx(roll) Rx(pi)
        float sgy, cgy;
        sincosf(place ? XG(go + 3) : y, &sgy, &cgy);
        const float rg[9] = {cgy * cth, fmaf(-cgy * sth, sph, sgy * cph), fmaf(-cgy * sth, cph, -sgy * sph),
                             sgy * cth, fmaf(-sgy * sth, sph, -cgy * cph), fmaf(-sgy * sth, cph, cgy * sph),
                             -sth, -cth * sph, -cth * cph};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          Rt[j] = fmaf(cp, rg[j], -sp * rg[3 + j]);
          Rt[3 + j] = fmaf(sp, rg[j], cp * rg[3 + j]);
          Rt[6 + j] = rg[6 + j];
        }
      }
      // forward kinematics, keeping each joint's axis and origin
      float R[9], t[3], oz[MAXJ][6];
#pragma unroll
      for (int a = 0; a < 9; ++a) R[a] = arm[a];
      t[0] = arm[9]; t[1] = arm[10]; t[2] = arm[11];
#pragma unroll
      for (int j = 0; j < MAXJ; ++j) {
        if (j < nj) {
          oz[j][0] = t[0]; oz[j][1] = t[1]; oz[j][2] = t[2];
          oz[j][3] = R[2]; oz[j][4] = R[5]; oz[j][5] = R[8];
          const float* Jp = arm + 24 + j * ARM_JW;
          float sj, cj;
          sincosf(q[j] + Jp[4], &sj, &cj);
          rz_right(R, cj, sj);
          t[0] = fmaf(Jp[1], R[2], fmaf(Jp[0], R[0], t[0]));
          t[1] = fmaf(Jp[1], R[5], fmaf(Jp[0], R[3], t[1]));
          t[2] = fmaf(Jp[1], R[8], fmaf(Jp[0], R[6], t[2]));
          rx_right(R, Jp[2], Jp[3]);
        }
      }
      float Re[9], pe[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b)
          Re[3 * a + b] = fmaf(R[3 * a], tl[b], fmaf(R[3 * a + 1], tl[3 + b], R[3 * a + 2] * tl[6 + b]));
        pe[a] = fmaf(R[3 * a], tl[9], fmaf(R[3 * a + 1], tl[10], fmaf(R[3 * a + 2], tl[11], t[a])));
      }
      // residual
      float E[9];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
          E[3 * a + b] = fmaf(Rt[3 * a], Re[3 * b], fmaf(Rt[3 * a + 1], Re[3 * b + 1], Rt[3 * a + 2] * Re[3 * b + 2]));
      float w[3];
      rot_log(E, w);
      const float r[6] = {tx - pe[0], ty - pe[1], tz - pe[2], w[0], w[1], w[2]};
      // A = [J_q | -dr*/dy]; the yaw column is [-(z x (t* - c_box)) ; -z] for a
      // Place (c_box the box centre) and [0 ; -z] for a Pick
      float A[6][MAXJ + 1];
#pragma unroll
      for (int j = 0; j < MAXJ; ++j) {
        const float dx = pe[0] - oz[j][0], dy = pe[1] - oz[j][1], dz = pe[2] - oz[j][2];
        const bool on = j < nj;
        A[0][j] = on ? oz[j][4] * dz - oz[j][5] * dy : 0.f;
        A[1][j] = on ? oz[j][5] * dx - oz[j][3] * dz : 0.f;
        A[2][j] = on ? oz[j][3] * dy - oz[j][4] * dx : 0.f;
        A[3][j] = on ? oz[j][3] : 0.f;
        A[4][j] = on ? oz[j][4] : 0.f;
        A[5][j] = on ? oz[j][5] : 0.f;
      }
      A[0][MAXJ] = place ? ty - by : 0.f;
      A[1][MAXJ] = place ? -(tx - bx) : 0.f;
      A[2][MAXJ] = 0.f;
      A[3][MAXJ] = 0.f; A[4][MAXJ] = 0.f; A[5][MAXJ] = -1.f;
      // M = A A^T + lam^2 I, Cholesky M = L L^T, solve M s = r
      float L[6][6];
#pragma unroll
      for (int a = 0; a < 6; ++a) {
#pragma unroll
        for (int b = 0; b <= a; ++b) {
          float m = a == b ? lam2 : 0.f;
#pragma unroll
          for (int c = 0; c <= MAXJ; ++c) m = fmaf(A[a][c], A[b][c], m);
#pragma unroll
          for (int c = 0; c < b; ++c) m = fmaf(-L[a][c], L[b][c], m);
          L[a][b] = a == b ? sqrtf(fmaxf(m, 1e-30f)) : m / L[b][b];
        }
      }
      float s[6];
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        float m = r[a];
#pragma unroll
        for (int c = 0; c < a; ++c) m = fmaf(-L[a][c], s[c], m);
        s[a] = m / L[a][a];
      }
#pragma unroll
      for (int a = 5; a >= 0; --a) {
        float m = s[a];
#pragma unroll
        for (int c = a + 1; c < 6; ++c) m = fmaf(-L[c][a], s[c], m);
        s[a] = m / L[a][a];
      }
      float st[MAXJ + 1], mx = 0.f;
#pragma unroll
      for (int c = 0; c <= MAXJ; ++c) {
        float m = 0.f;
#pragma unroll
        for (int a = 0; a < 6; ++a) m = fmaf(A[a][c], s[a], m);
        st[c] = m;
        mx = fmaxf(mx, fabsf(m));
      }
      const float sc_ = mx > dmax ? dmax / mx : 1.f;
#pragma unroll
      for (int j = 0; j < MAXJ; ++j) {
        if (j < nj) {
          const float* Jp = arm + 24 + j * ARM_JW;
          q[j] = fminf(fmaxf(fmaf(sc_, st[j], q[j]), Jp[5]), Jp[6]);
        }
      }
      y = fmaf(sc_, st[MAXJ], y);
    }
#pragma unroll
    for (int j = 0; j < MAXJ; ++j)
      if (j < nj) XG(qo + j) = q[j];
    XG(yo) = y;
  }
#undef XG
}

cudaError_t launch_ik(const uint32_t* pb, const uint32_t* sc, float* x, int stride, int P, int iters, float lam,
                      float dmax, const int* chains, int n_chains, int chain_w, int keep, cudaStream_t st) {
  if (P == 0 || iters <= 0 || n_chains == 0) return cudaSuccess;
  const long threads = static_cast<long>(P) * n_chains;
  ik_configs_kernel<<<static_cast<unsigned>((threads + 127) / 128), 128, 0, st>>>(pb, sc, x, stride, P, iters, lam,
                                                                                dmax, chains, n_chains, chain_w, keep);
  return cudaGetLastError();
}

// Knot initialisation (Sec. VIII: linear interpolation between a motion's start
// and end configurations): one thread per (particle, motion); knots of a
// motion inside a kept prefix (components below `keep`) stay as they are.
__global__ void knots_kernel(const uint32_t* __restrict__ pb, float* __restrict__ x, int stride, int P, int nj,
                             int keep) {
  const long g = static_cast<long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int ns = pb[PH_NSEG];
  if (g >= static_cast<long>(P) * ns) return;
  const int i = static_cast<int>(g % P);
  const uint32_t* r = pb + pb[PH_OFF_SEG] + static_cast<int>(g / P) * SEG_W;
  const int qa = r[SG_QA], qb = r[SG_QB], qk = r[SG_QK], m = r[SG_M];
  if (qk < keep) return;
  for (int j = 0; j < nj; ++j) {
    const float a = x[static_cast<long>(qa + j) * stride + i], b = x[static_cast<long>(qb + j) * stride + i];
    for (int k = 0; k < m; ++k)
      x[static_cast<long>(qk + k * nj + j) * stride + i] = fmaf(static_cast<float>(k + 1) / (m + 1), b - a, a);
  }
}

cudaError_t launch_knots(const uint32_t* pb, float* x, int stride, int P, int n_seg, int nj, int keep,
                         cudaStream_t st) {
  if (P == 0 || n_seg == 0) return cudaSuccess;
  const long threads = static_cast<long>(P) * n_seg;
  knots_kernel<<<static_cast<unsigned>((threads + 127) / 128), 128, 0, st>>>(pb, x, stride, P, nj, keep);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ FP32 peak probe
// Measurement utility (not part of the method): independent FFMA chains, 8 per
// thread, enough warps to fill every SM, so the FP32 pipes are the only limit.
// 2 FLOP per FFMA; the result is written so that nothing is optimised away.
__global__ void __launch_bounds__(256) ffma_probe_kernel(float* out, int iters, float a, float b) {
  float v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = threadIdx.x * 1e-3f + k;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = fmaf(v[k], a, b);
    }
  }
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) sum += v[k];
  if (sum == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = sum;  // practically never
}

cudaError_t launch_ffma_probe(float* out, int blocks, int iters, cudaStream_t st) {
  ffma_probe_kernel<<<blocks, 256, 0, st>>>(out, iters, 0.999999f, 1e-7f);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ chunk controller
// After each chunk of a chunked optimisation (a CUDA graph's, or
// tamp_optimize_steps stopping on the first satisfying particle): advance every
// problem's step count, and raise the stop flag when stopping on the first
// satisfying particle and some problem has one (the Eq. 3 check records its
// iteration).  When another chunk follows and runs, the problems' Eq. 5 counts
// are cleared for its final check; once stopped they keep the last check's.
__global__ void chunk_control_kernel(int* t_dev, const int* const* first_iters, int* const* counts,
                                     const int* n_counts, int n_problems, int steps, int stop_on_first, int* stop,
                                     int* chunks_run, int last) {
  __shared__ int s_next;
  if (threadIdx.x == 0) {
    s_next = 0;
    if (!*stop) {
      bool found = false;
      for (int p = 0; p < n_problems; ++p) {
        t_dev[p] += steps;
        found = found || *first_iters[p] != 0x7fffffff;
      }
      *chunks_run += 1;
      if (stop_on_first && found) *stop = 1;
      else s_next = !last;
    }
  }
  __syncthreads();
  if (!s_next) return;
  for (int p = 0; p < n_problems; ++p)
    for (int i = threadIdx.x; i < n_counts[p]; i += blockDim.x) counts[p][i] = 0;
}

cudaError_t launch_chunk_control(int* t_dev, const int* const* first_iters, int* const* counts, const int* n_counts,
                                 int n_problems, int steps, int stop_on_first, int* stop, int* chunks_run, int last,
                                 cudaStream_t st) {
  chunk_control_kernel<<<1, 128, 0, st>>>(t_dev, first_iters, counts, n_counts, n_problems, steps, stop_on_first,
                                          stop, chunks_run, last);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ launchers
// largest dynamic shared-memory size enabled so far for optimize_kernel<1,2,4,8>
// per feature set (0 .. N_FEAT - 1) and record flag
static size_t g_smem_enabled[2][N_FEAT][4] = {};
static int lane_slot(int L) { return L == 1 ? 0 : (L == 2 ? 1 : (L == 4 ? 2 : 3)); }

template <int L, int FEAT, bool REC>
static cudaError_t set_smem(size_t smem) {
  size_t& enabled = g_smem_enabled[REC ? 1 : 0][FEAT][lane_slot(L)];
  if (smem <= 48 * 1024 || smem <= enabled) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(optimize_kernel<L, FEAT, REC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e == cudaSuccess) enabled = smem;
  return e;
}

template <int L, int FEAT>
static cudaError_t launch_feat(const LaunchArgs& a, int warps, int grid, size_t smem, cudaStream_t st) {
  cudaError_t e = a.rec ? set_smem<L, FEAT, true>(smem) : set_smem<L, FEAT, false>(smem);
  if (e != cudaSuccess) return e;
  if (grid <= 0) return cudaSuccess;
  if (a.rec)
    optimize_kernel<L, FEAT, true><<<grid, warps * 32, smem, st>>>(a);
  else
    optimize_kernel<L, FEAT, false><<<grid, warps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <int L>
static cudaError_t launch_opt(const LaunchArgs& a, int warps, int grid, size_t smem, cudaStream_t st) {
  switch (a.feat) {
    case 0: return launch_feat<L, 0>(a, warps, grid, smem, st);
    case FEAT_SELF: return launch_feat<L, FEAT_SELF>(a, warps, grid, smem, st);
    case FEAT_EXT: return launch_feat<L, FEAT_EXT>(a, warps, grid, smem, st);
    case FEAT_KNOT: return launch_feat<L, FEAT_KNOT>(a, warps, grid, smem, st);
    case FEAT_KNOT6: return launch_feat<L, FEAT_KNOT6>(a, warps, grid, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

int optimize_blocks_per_sm(int L, int warps, size_t smem) {
  int n = 0;
  cudaError_t e = cudaSuccess;
  switch (L) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, optimize_kernel<1, 0, false>, warps * 32, smem); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, optimize_kernel<2, 0, false>, warps * 32, smem); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, optimize_kernel<4, 0, false>, warps * 32, smem); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, optimize_kernel<8, 0, false>, warps * 32, smem); break;
  }
  return e == cudaSuccess ? n : 1;
}

template <int L, bool REC>
static cudaError_t set_smem_feats(size_t smem) {
  cudaError_t e = set_smem<L, 0, REC>(smem);
  if (e == cudaSuccess) e = set_smem<L, FEAT_SELF, REC>(smem);
  if (e == cudaSuccess) e = set_smem<L, FEAT_EXT, REC>(smem);
  if (e == cudaSuccess) e = set_smem<L, FEAT_KNOT, REC>(smem);
  if (e == cudaSuccess) e = set_smem<L, FEAT_KNOT6, REC>(smem);
  return e;
}
template <int L>
static cudaError_t set_smem_all(size_t smem) {
  cudaError_t e = set_smem_feats<L, false>(smem);
  if (e == cudaSuccess) e = set_smem_feats<L, true>(smem);
  return e;
}

// Allow `smem` bytes of dynamic shared memory for optimize_kernel<L, *> (outside
// any stream capture).
cudaError_t optimize_set_smem(int L, size_t smem) {
  switch (L) {
    case 1: return set_smem_all<1>(smem);
    case 2: return set_smem_all<2>(smem);
    case 4: return set_smem_all<4>(smem);
    case 8: return set_smem_all<8>(smem);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_optimize(const LaunchArgs& a, int L, int warps, int grid, size_t smem, cudaStream_t st) {
  switch (L) {
    case 1: return launch_opt<1>(a, warps, grid, smem, st);
    case 2: return launch_opt<2>(a, warps, grid, smem, st);
    case 4: return launch_opt<4>(a, warps, grid, smem, st);
    case 8: return launch_opt<8>(a, warps, grid, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_sample(const uint32_t* pb, const uint32_t* sc, float* x, float* m, float* v, int stride, int P,
                          int D, uint64_t seed, cudaStream_t st) {
  if (P == 0 || D == 0) return cudaSuccess;
  dim3 grid((P + 255) / 256, D);
  const uint2 key = make_uint2(static_cast<uint32_t>(seed & 0xffffffffu), static_cast<uint32_t>(seed >> 32));
  sample_uniform_kernel<<<grid, 256, 0, st>>>(pb, sc, x, m, v, stride, P, key);
  return cudaGetLastError();
}

cudaError_t launch_sample_proposal(const uint32_t* rows, int R, const float* out, float* x, int stride, int P,
                                   uint64_t seed, cudaStream_t st) {
  if (P == 0 || R == 0) return cudaSuccess;
  dim3 grid((P + 255) / 256, R);
  const uint2 key = make_uint2(static_cast<uint32_t>(seed & 0xffffffffu), static_cast<uint32_t>(seed >> 32));
  sample_proposal_kernel<<<grid, 256, 0, st>>>(rows, out, x, stride, P, key);
  return cudaGetLastError();
}

// Dynamic shared memory: scene tables, the largest problem's tables and tile
// (x, m, v, gradient, terms, flags), then the warps' exact-phase scratch.
size_t optimize_tile_bytes(int prob_words, int D, int NT, int NSLOT, int NANG, int L, bool mv_global) {
  const int PT = 32 / L;
  const size_t pw = (prob_words + 3) & ~3;
  const size_t arrays = mv_global ? 2 : 4;  // x, g (and m, v unless they stay in global memory)
  return 4 * pw + 4 * (arrays * static_cast<size_t>(D) * PT + static_cast<size_t>(NT) * PT) +
         ((PT * 4 + 15) & ~15) + 16 * static_cast<size_t>(NSLOT) * PT + 8 * static_cast<size_t>(NANG) * PT;
}
size_t optimize_scratch_bytes(int warps) { return static_cast<size_t>(WARP_SCRATCH_BYTES) * warps; }

// Warps of the default launch shape: one per work item of an evaluation pass
// (two pieces per configuration), at most 16 (512 threads, 128 registers each).
int optimize_warps(int K) { return std::min(16, 2 * K); }

}  // namespace tamp
