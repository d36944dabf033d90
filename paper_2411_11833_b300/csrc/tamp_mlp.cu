// Proposal network kernels: BF16 tensor-core GEMMs on sm_103a (tcgen05 + TMEM)
// with FP32 accumulation, for inference and training.
//
// The network: 4 dense layers IN -> H -> H -> H -> OUT (48, 256, 256, 256, 32),
// exact GELU between layers, weights and inter-layer activations in BF16,
// accumulation in FP32; output k < 16 is the mean of target k, output 16 + k its
// log standard deviation, trained with the Gaussian negative log-likelihood.
//
// Every product is one tile GEMM D[128 x N] = A[128 x K] . B[N x K]^T: the CTA's
// threads stage A and B into shared memory in the canonical K-major layout
// without swizzle (8 x 16-byte core matrices: 128 B apart along K, 256 B apart
// per group of 8 rows, K in chunks of 16), one thread issues K/16
// tcgen05.mma instructions into a tensor-memory accumulator and commits them to
// an mbarrier, and every thread reads back its own row with tcgen05.ld.  A
// transposed operand is just staged transposed, so the backward pass (dA = dZ W,
// dW = dZ^T A) uses the same instruction forms as the forward pass.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "tamp.h"

namespace mlpk {

constexpr int IN = 48, H = 256, OUT = 32, NTGT = 16;
constexpr int ROWS = 128;    // samples per CTA tile = MMA M
// 16 warps: warp w reads the TMEM lanes (tile rows) 32 (w % 4) .. + 31 and the
// column group w / 4 of the accumulator in the epilogues
constexpr int THREADS = 512;
constexpr int NGRP = THREADS / 128;
constexpr int TMEM_COLS = 256;
constexpr size_t SMEM_A = 128 * 256 * 2;   // largest A operand (128 x 256 bf16)
constexpr size_t SMEM_B = 256 * 256 * 2;   // largest B operand (256 x 256 bf16)
constexpr size_t SMEM_BYTES = SMEM_A + SMEM_B;
__host__ __device__ constexpr int kdim(int l) { return l == 0 ? IN : H; }  // inputs of layer l
__host__ __device__ constexpr int ndim(int l) { return l == 3 ? OUT : H; } // outputs of layer l
enum { ERR_WAIT = 1 };

__host__ __device__ constexpr size_t w_off(int l) {
  return l == 0 ? 0 : (l == 1 ? (size_t)H * IN + H : (l == 2 ? (size_t)H * IN + H + H * H + H : (size_t)H * IN + H + 2 * ((size_t)H * H + H)));
}
__host__ __device__ constexpr size_t b_off(int l) { return w_off(l) + (size_t)ndim(l) * kdim(l); }
constexpr size_t N_PARAMS = w_off(3) + (size_t)OUT * H + OUT;
// BF16 weights pre-packed in the canonical K-major layout of the GEMM operands:
// per layer the forward operand W [N][K] and the transposed operand W^T [K][N]
// (the backward pass's dA = dZ W), each one contiguous block that one bulk copy
// moves into shared memory
__host__ __device__ constexpr size_t pk_bytes(int l) { return (size_t)ndim(l) * kdim(l) * 2; }
__host__ __device__ constexpr size_t pk_off(int l) {
  return l == 0 ? 0 : pk_off(l - 1) + pk_bytes(l - 1);
}
constexpr size_t PK_BYTES = pk_off(4);

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// 1-D bulk copy global -> shared; completion counted on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < (1 << 22); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    __nanosleep(32);
  }
  return false;
}
// Programmatic dependent launch, for the kernels of a training step, which
// are launched with programmatic stream serialisation: pdl_wait blocks until
// the grids this one depends on have completed and their writes are visible
// (a no-op for a grid launched without the attribute); pdl_release lets the
// next grid in the stream be scheduled, where it runs its own set-up up to
// its pdl_wait.  No kernel reads another grid's output before its pdl_wait.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// tensor memory: allocated and freed by one whole warp
__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(TMEM_COLS)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TMEM_COLS) : "memory");
}
// shared-memory matrix descriptor: K-major, no swizzle, LBO 128 B (next core
// matrix along K), SBO 256 B (next group of 8 rows), descriptor version 1
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) | (static_cast<uint64_t>(128 >> 4) << 16) |
         (static_cast<uint64_t>(256 >> 4) << 32) | (1ull << 46);
}
// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t u[32];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]), "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(u[i]);
}

// the same load without the wait: several may be in flight before one tcgen05.wait::ld
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&u)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]), "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
               : "r"(taddr)
               : "memory");
}

// ------------------------------------------------------------------ tile GEMM
// byte offset of element (r, k) of an R-row operand in the staged layout
__host__ __device__ __forceinline__ uint32_t blk_off(int r, int k, int R) {
  return static_cast<uint32_t>((k >> 4) * (R * 32) + (r >> 3) * 256 + ((k >> 3) & 1) * 128 + (r & 7) * 16 +
                               (k & 7) * 2);
}
__device__ __forceinline__ float ld_f(const float* p) { return *p; }
__device__ __forceinline__ float ld_f(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// Stage an R x K operand (element (r, k) = src[r * rs + k * ks], zero outside
// rows < Rv and columns < Kv) as BF16 in the K-major layout.
template <typename T>
__device__ void stage(unsigned char* dst, int R, int K, const T* src, long rs, long ks, int Rv, int Kv) {
  for (int i = threadIdx.x; i < R * K; i += blockDim.x) {
    const int r = i / K, k = i % K;
    float v = 0.f;
    if (r < Rv && k < Kv) v = ld_f(src + r * rs + k * ks);
    *reinterpret_cast<__nv_bfloat16*>(dst + blk_off(r, k, R)) = __float2bfloat16_rn(v);
  }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
// GELU'(Z_l) is written by the training forward and read by the dZ chain,
// both with thread (warp w, lane i) on row 32 (w % 4) + i of a 128-row tile
// and the 32-column chunks of column group w / 4.  It is kept in the layout
// they share: per tile, warp, chunk and 16-byte piece q of a row's chunk, the
// 32 lanes' pieces side by side -- each store and load of a warp moves 512
// contiguous bytes (by rows, each would touch 32 rows).  64 KB per tile.
__device__ __forceinline__ uint4* g_pieces(__half* G, int tile, int warp, int chunk, int lane) {
  return reinterpret_cast<uint4*>(G) + static_cast<long>(((tile * (THREADS / 32) + warp) * 2 + chunk) * 4) * 32 + lane;
}
__device__ __forceinline__ uint32_t pack_f16x2(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
// the two FP16 halves of a word as floats (exact): low half first
__device__ __forceinline__ float2 unpack_f16x2(uint32_t w) {
  return __half22float2(*reinterpret_cast<const __half2*>(&w));
}

// Issue D[128 x N] = A[128 x K] . B[N x K]^T (one thread) and commit it.
__device__ __forceinline__ void issue_gemm(uint32_t tmem, const unsigned char* A, const unsigned char* B, int N, int K,
                                           uint64_t* bar) {
  tc_fence_after();
  const uint32_t a0 = smem_u32(A), b0 = smem_u32(B), id = instr_desc(ROWS, N);
  for (int c = 0; c < K / 16; ++c)
    umma_bf16(tmem, smem_desc(a0 + c * ROWS * 32), smem_desc(b0 + c * N * 32), id, c > 0 ? 1u : 0u);
  umma_commit(bar);
}

// D[128 x N] = A[128 x K] . B[N x K]^T into tensor memory; every thread calls
// it; on return the accumulator is complete (or *err has ERR_WAIT set).
__device__ bool gemm_tile(uint32_t tmem, const unsigned char* A, const unsigned char* B, int N, int K,
                          uint64_t* bar, uint32_t& phase, int* err) {
  fence_proxy_async();  // the staged operands, written by every thread, to the tensor core
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) issue_gemm(tmem, A, B, N, K, bar);
  const bool ok = mbar_wait_bounded(bar, phase);
  phase ^= 1u;
  if (!ok) atomicOr(err, ERR_WAIT);
  tc_fence_after();
  return __syncthreads_and(ok) != 0;
}

// TMEM address of column `col` in this warp's quarter of the lanes
__device__ __forceinline__ uint32_t lane_addr(uint32_t tmem, int col) {
  return tmem + (static_cast<uint32_t>(32 * ((threadIdx.x >> 5) & 3)) << 16) + static_cast<uint32_t>(col);
}
// Phi(z), the standard normal CDF, for the exact GELU z Phi(z) and its
// derivative Phi(z) + z phi(z), on the FP32 pipe only (no special-function
// unit for Phi): Phi(z) - 1/2 = z p(z^2), where p -- (Phi(z) - 1/2) / z is a
// smooth even function -- is a degree-8 polynomial, fitted to Phi by least
// squares in the Chebyshev basis of t = z^2 / Zc^2 - 1 on |z| <= Zc = 2.9
// sqrt 2 (4.1012; 1 - Phi(Zc) = 2.1e-5), rewritten in powers of s = z^2 (its
// terms stay below 10 in magnitude on |z| <= Zc, so FP32 Horner keeps the
// fit's error) and evaluated by Horner's rule in s.  Beyond Zc the polynomial
// keeps growing (1/2 + z p(z^2) passes 1 at z = 4.15 and never comes back; it
// is odd in z), so the last step, 1/2 + z p, saturates to [0, 1] instead of
// clamping z: Phi = 1 or 0 there, also where p overflows to infinity.
// Measured in FP32 against the double-precision Phi: |error| <= 2.1e-5; GELU's
// absolute error <= 8e-6 on |z| <= 2, 4.2e-5 on |z| <= 4, 9e-5 everywhere, its
// derivative's <= 2.1e-5 -- against a BF16 rounding of 2^-9 relative (1e-3 at
// an activation of 0.5) in the activations the kernels store.  With z as the
// variable the 1 / sqrt 2 of erf(z / sqrt 2) and GELU's 1/2 fold into the
// coefficients: a pair of values takes 9 paired instructions and 2 saturating
// FMAs.
// coefficients of s^8 .. s^0
__device__ constexpr float kPhiFit[9] = {
    7.3491581e-11f, -6.5462733e-09f, 2.5961910e-07f, -6.1287783e-06f, 9.7603224e-05f,
    -1.1281440e-03f, 9.8639885e-03f, -6.6396549e-02f, 3.9891848e-01f};
__device__ __forceinline__ float fma_sat(float a, float b, float c) {  // a b + c, saturated to [0, 1]
  float d;
  asm("fma.rn.ftz.sat.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
// two at a time: the polynomial on the paired FP32 instructions (FFMA2 / FMUL2;
// the same roundings as one at a time, half the instructions)
__device__ __forceinline__ float2 phi_fit2(float2 z) {
  const float2 s = __fmul2_rn(z, z);
  float2 p = make_float2(kPhiFit[0], kPhiFit[0]);
#pragma unroll
  for (int k = 1; k < 9; ++k) p = __ffma2_rn(p, s, make_float2(kPhiFit[k], kPhiFit[k]));
  return make_float2(fma_sat(z.x, p.x, 0.5f), fma_sat(z.y, p.y, 0.5f));
}
// GELU(z) = z Phi(z) and its derivative Phi(z) + z phi(z), phi(z) = exp(-z^2 / 2) / sqrt(2 pi), for two values
__device__ __forceinline__ float2 gelu2(float2 z) { return __fmul2_rn(z, phi_fit2(z)); }
__device__ __forceinline__ float2 gelu_grad2(float2 z) {
  const float2 pdf = make_float2(0.39894228040143268f * __expf(-0.5f * z.x * z.x),
                                 0.39894228040143268f * __expf(-0.5f * z.y * z.y));
  return __ffma2_rn(z, pdf, phi_fit2(z));
}

// ------------------------------------------------------------------ training: forward, NLL, dZ chain
struct TrainArgs {
  const float* x; int B;              // inputs [B][IN]
  const float* y;                     // [B][NTGT] targets
  const float* mask;                  // [B][NTGT]
  const unsigned char* Wp;            // packed BF16 forward operands (pk_off)
  const unsigned char* WpT;           // packed W^T operands (pk_off)
  const float* b[4];
  // GELU'(Z_l) (FP16: GELU' lies in [-0.17, 1.13], where FP16 rounds 8 times
  // finer than BF16; in the g_pieces layout) -- the backward pass uses the
  // pre-activations only through it -- and the BF16 operands of the weight
  // gradients x, A_l and dZ_l in the f8 layout (ldR rows)
  __half* G[3]; uint4* X8; uint4* A8[3]; uint4* dZ8[4]; int ldR;
  float* loss;                        // the NLL's mean over rows, zeroed here and accumulated
  float* grad;                        // the gradient accumulator [N_PARAMS], zeroed here for dW
  int* err;
};

// One CTA per 128 rows: the forward through the 4 layers, the Gaussian NLL
// and its gradient dZ_3 at the outputs, then the dZ chain back to dZ_0
// (dA_{l-1} = dZ_l W_l on the tensor core, dZ_{l-1} = dA_{l-1} * GELU'(Z_{l-1})).
// Each product's packed weights (W_l forward, W_l^T backward) arrive by one
// bulk copy, issued as soon as the previous product has finished reading the
// operand buffer, so it overlaps that layer's epilogue; activations and dZ_l
// stay in shared memory as the next product's A operand.  A 256-wide product
// runs in two column halves with their own barriers, so that the epilogue of
// the first half overlaps the product of the second.
__global__ void __launch_bounds__(THREADS, 1) mlp_train_kernel(TrainArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* opA = smem;
  unsigned char* opB = smem + SMEM_A;
  __shared__ __align__(8) uint64_t bar_mma[2], bar_w;  // the product's two column halves; the weights
  __shared__ uint32_t tslot;
  __shared__ __align__(16) float s_bias[3 * H + OUT];  // every layer's bias, read by the epilogues
  __shared__ float s_loss[4];                          // the output layer's warps' NLL sums
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31, grp = warp >> 2;
  const int row = 32 * (warp & 3) + lane, row0 = blockIdx.x * ROWS, r = row0 + row;
  const int Rv = min(ROWS, a.B - row0);
  bool w_pending = false;  // thread 0: a weight copy is in flight
  if (t == 0) {
    mbar_init(&bar_mma[0]);
    mbar_init(&bar_mma[1]);
    mbar_init(&bar_w);
    fence_proxy_async();
  }
  if (warp == 0) tmem_alloc(&tslot);
  pdl_wait();  // the weights of the last update, the inputs
  pdl_release();
  if (t == 0) {
    mbar_expect_tx(&bar_w, static_cast<uint32_t>(pk_bytes(0)));
    bulk_g2s(opB, a.Wp + pk_off(0), static_cast<uint32_t>(pk_bytes(0)), &bar_w);
    w_pending = true;
    if (a.loss && blockIdx.x == 0) *a.loss = 0.f;
  }
  if (a.grad)  // the dW kernel adds every split's share into it
    for (int i = blockIdx.x * THREADS + t; i < static_cast<int>(N_PARAMS / 4); i += gridDim.x * THREADS)
      reinterpret_cast<float4*>(a.grad)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = t; i < 3 * H + OUT; i += THREADS) s_bias[i] = i < 3 * H ? a.b[i / H][i % H] : a.b[3][i - 3 * H];
  // inputs: 8 columns (one 16-byte chunk of the layout) per step
  for (int c = t; c < ROWS * (IN / 8); c += THREADS) {
    const int rr = c / (IN / 8), kk = (c % (IN / 8)) * 8;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = rr < Rv ? a.x[static_cast<long>(row0 + rr) * IN + kk + e] : 0.f;
    const uint4 pk =
        make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
    *reinterpret_cast<uint4*>(opA + blk_off(rr, kk, ROWS)) = pk;
    if (a.X8) a.X8[static_cast<long>(kk >> 3) * a.ldR + row0 + rr] = pk;  // rows past B: zeros
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  uint32_t ph_mma = 0, ph_w = 0;
  int copy_par = -1;  // thread 256: the barrier phase parity of the last weight copy it issued
  bool alive = true;  // no wait has given up
  static_assert(H / NGRP == 64, "a thread's columns of dA: two 32-column chunks");
  for (int l = 0; l < 4; ++l) {
    const int K = kdim(l), N = ndim(l);
    bool fail = false;
    if (t == 0) {
      const bool okw = mbar_wait_bounded(&bar_w, ph_w);
      w_pending = !okw;
      if (okw && N == H) {
        // two column halves, each committed to its own barrier: the epilogue
        // warps of columns 0 .. 127 start while the tensor core computes 128 .. 255
        tc_fence_after();
        const uint32_t a0 = smem_u32(opA), b0 = smem_u32(opB), id = instr_desc(ROWS, H / 2);
        for (int h = 0; h < 2; ++h) {
          for (int c = 0; c < K / 16; ++c)
            umma_bf16(tmem + h * (H / 2), smem_desc(a0 + c * ROWS * 32), smem_desc(b0 + h * (H / 16) * 256 + c * H * 32),
                      id, c > 0 ? 1u : 0u);
          umma_commit(&bar_mma[h]);
        }
      } else if (okw) {
        issue_gemm(tmem, opA, opB, N, K, &bar_mma[0]);
        umma_commit(&bar_mma[1]);
      } else {
        atomicOr(a.err, ERR_WAIT);
        fail = true;
      }
    }
    ph_w ^= 1u;
    const bool okm = mbar_wait_bounded(&bar_mma[grp >> 1], ph_mma);  // this group's column half
    ph_mma ^= 1u;
    if (!okm) {
      atomicOr(a.err, ERR_WAIT);
      fail = true;
    }
    tc_fence_after();
    if (t == 256 && okm) {
      // the second half's commit covers every product of the layer: opB is free
      // for the next layer's weights (after the output layer: W_3^T, the first
      // operand of the backward pass)
      const unsigned char* src = l < 3 ? a.Wp + pk_off(l + 1) : a.WpT + pk_off(3);
      const uint32_t bytes = static_cast<uint32_t>(l < 3 ? pk_bytes(l + 1) : pk_bytes(3));
      mbar_expect_tx(&bar_w, bytes);
      bulk_g2s(opB, src, bytes, &bar_w);
      copy_par = (l + 1) & 1;
    }
    // epilogue: this warp's rows, its group's columns (the 32-wide last layer:
    // group 0 only)
    const int per = N >= 128 ? N / NGRP : N;
    if (!fail && (N >= 128 || grp == 0)) {
      for (int c0 = grp * per; c0 < grp * per + per; c0 += 32) {
        float v[32];
        tmem_ld32(lane_addr(tmem, c0), v);
        const float* bias = s_bias + l * H + c0;
        if (l < 3) {
          uint32_t hp[16], gp[16];
#pragma unroll
          for (int j = 0; j < 32; j += 2) {
            const float2 z = __fadd2_rn(make_float2(v[j], v[j + 1]), make_float2(bias[j], bias[j + 1]));
            const float2 g = gelu2(z);
            hp[j / 2] = pack_bf16x2(g.x, g.y);
            if (a.G[l]) {  // GELU'(z) for the backward pass, sharing gelu2's Phi(z)
              const float2 d = gelu_grad2(z);
              gp[j / 2] = pack_f16x2(d.x, d.y);
            }
          }
#pragma unroll
          for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint4*>(opA + blk_off(row, c0 + 8 * q, ROWS)) =
                make_uint4(hp[4 * q], hp[4 * q + 1], hp[4 * q + 2], hp[4 * q + 3]);
          if (a.G[l]) {
            uint4* gd = g_pieces(a.G[l], blockIdx.x, warp, (c0 - grp * per) >> 5, lane);
            uint4* ad = a.A8[l] + static_cast<long>(c0 >> 3) * a.ldR + r;  // f8: the warp's 32 rows side by side
            const bool in = r < a.B;  // rows past B: zeros in A8 (the weight-gradient copies read whole chunks)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (in) gd[32 * q] = make_uint4(gp[4 * q], gp[4 * q + 1], gp[4 * q + 2], gp[4 * q + 3]);
              ad[static_cast<long>(q) * a.ldR] =
                  in ? make_uint4(hp[4 * q], hp[4 * q + 1], hp[4 * q + 2], hp[4 * q + 3]) : make_uint4(0u, 0u, 0u, 0u);
            }
          }
        } else {
          // the outputs (mu_k, s_k = log sigma_k) and from them dZ_3 = dL/d(outputs) of
          // the Gaussian NLL, the mean over the B rows of sum over masked k of
          // (y_k - mu_k)^2 exp(-2 s_k) / 2 + s_k:
          // dL/dmu_k = -m (y_k - mu_k) exp(-2 s_k) / B, dL/ds_k = m (1 - (y_k - mu_k)^2 exp(-2 s_k)) / B.
          // It is the A operand (K = 32) of the first backward product, and goes to
          // dZ8[3] for the weight gradients; this warp's rows' NLL terms are summed.
          const float inv = 1.f / static_cast<float>(a.B);
          float dz[OUT], lsum = 0.f;
#pragma unroll
          for (int k = 0; k < NTGT; ++k) {
            dz[k] = 0.f;
            dz[NTGT + k] = 0.f;
            if (r < a.B) {
              const float mu = v[k] + bias[k], sg = v[NTGT + k] + bias[NTGT + k];
              const float m = a.mask[static_cast<long>(r) * NTGT + k], d = a.y[static_cast<long>(r) * NTGT + k] - mu;
              const float ex = expf(-2.f * sg);
              dz[k] = m * (-d * ex) * inv;
              dz[NTGT + k] = m * (1.f - d * d * ex) * inv;
              lsum += m * (0.5f * d * d * ex + sg);
            }
          }
#pragma unroll
          for (int q = 0; q < OUT / 8; ++q) {
            const uint4 pk = make_uint4(pack_bf16x2(dz[8 * q], dz[8 * q + 1]), pack_bf16x2(dz[8 * q + 2], dz[8 * q + 3]),
                                        pack_bf16x2(dz[8 * q + 4], dz[8 * q + 5]),
                                        pack_bf16x2(dz[8 * q + 6], dz[8 * q + 7]));
            *reinterpret_cast<uint4*>(opA + blk_off(row, 8 * q, ROWS)) = pk;
            a.dZ8[3][static_cast<long>(q) * a.ldR + r] = pk;  // rows past B: zeros
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
          if (lane == 0) s_loss[warp] = lsum;
        }
      }
    }
    fence_proxy_async();  // the activations, written by every thread, to the tensor core
    tc_fence_before();
    const int any_fail = __syncthreads_or(fail);  // every row's activations staged; accumulator free
    tc_fence_after();
    if (any_fail) {
      alive = false;
      break;
    }
  }
  // the mean NLL: the output layer's warps' sums (complete after the last forward barrier)
  if (t == 0 && alive) atomicAdd(a.loss, (s_loss[0] + s_loss[1] + s_loss[2] + s_loss[3]) / static_cast<float>(a.B));
  // ---- the dZ chain, from dZ_3 in opA and W_3^T arriving in opB
  for (int l = 3; alive && l >= 1; --l) {
    const int K = kdim(l), N = ndim(l);
    // this layer's GELU'(Z_{l-1}) pieces, loaded while the product runs (the
    // global loads' latency off the path from the product to the epilogue)
    uint4 gpre[2][4];
    if (r < a.B) {
#pragma unroll
      for (int ch = 0; ch < 2; ++ch) {
        const uint4* gs = g_pieces(a.G[l - 1], blockIdx.x, warp, ch, lane);
#pragma unroll
        for (int q = 0; q < 4; ++q) gpre[ch][q] = gs[32 * q];
      }
    }
    bool fail = false;
    if (t == 0) {
      const bool okw = mbar_wait_bounded(&bar_w, ph_w);
      w_pending = !okw;
      if (okw) {
        // dA_{l-1} [128 x K] = dZ_l [128 x N] . W_l in two column halves, each
        // committed to its own barrier (the first half's epilogue overlaps the
        // second half's product)
        tc_fence_after();
        const uint32_t a0 = smem_u32(opA), b0 = smem_u32(opB), id = instr_desc(ROWS, K / 2);
        for (int h = 0; h < 2; ++h) {
          for (int c = 0; c < N / 16; ++c)
            umma_bf16(tmem + h * (K / 2), smem_desc(a0 + c * ROWS * 32), smem_desc(b0 + h * (K / 16) * 256 + c * K * 32),
                      id, c > 0 ? 1u : 0u);
          umma_commit(&bar_mma[h]);
        }
      } else {
        atomicOr(a.err, ERR_WAIT);
        fail = true;
      }
    }
    ph_w ^= 1u;
    const bool okm = mbar_wait_bounded(&bar_mma[grp >> 1], ph_mma);  // this group's column half
    ph_mma ^= 1u;
    if (!okm) {
      atomicOr(a.err, ERR_WAIT);
      fail = true;
    }
    tc_fence_after();
    if (t == 256 && l > 1 && okm) {  // every product of the layer is done with opB: the next weights
      mbar_expect_tx(&bar_w, static_cast<uint32_t>(pk_bytes(l - 1)));
      bulk_g2s(opB, a.WpT + pk_off(l - 1), static_cast<uint32_t>(pk_bytes(l - 1)), &bar_w);
      copy_par = l & 1;  // the copy of W_{l-1}^T completes the barrier's phase 8 - l
    }
    uint4* dz8 = a.dZ8[l - 1];
#pragma unroll
    for (int ch = 0; ch < 2 && !fail; ++ch) {
      const int c0 = grp * 64 + 32 * ch;
      float v[32];
      tmem_ld32(lane_addr(tmem, c0), v);
      uint32_t hp[16];
      if (r < a.B) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint4 g = gpre[ch][q];
          const uint32_t gw[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const float2 d = __fmul2_rn(make_float2(v[8 * q + 2 * h], v[8 * q + 2 * h + 1]), unpack_f16x2(gw[h]));
            hp[4 * q + h] = pack_bf16x2(d.x, d.y);
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) hp[q] = 0u;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(opA + blk_off(row, c0 + 8 * q, ROWS)) =
            make_uint4(hp[4 * q], hp[4 * q + 1], hp[4 * q + 2], hp[4 * q + 3]);
      {
        uint4* dd = dz8 + static_cast<long>(c0 >> 3) * a.ldR + r;  // f8: the warp's 32 rows side by side (zeros past B)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          dd[static_cast<long>(q) * a.ldR] = make_uint4(hp[4 * q], hp[4 * q + 1], hp[4 * q + 2], hp[4 * q + 3]);
      }
    }
    fence_proxy_async();
    tc_fence_before();
    const int any_fail = __syncthreads_or(fail);
    tc_fence_after();
    if (any_fail) {
      alive = false;
      break;
    }
  }
  // no copy may land after the CTA ends
  if (t == 0 && w_pending) mbar_wait_bounded(&bar_w, ph_w);
  if (t == 256 && copy_par >= 0) mbar_wait_bounded(&bar_w, static_cast<uint32_t>(copy_par));
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem);
}

// ------------------------------------------------------------------ forward, two tiles in turn
// Inference forward over many rows: each CTA takes pairs of 128-row tiles and
// runs them half a layer apart, so that the tensor core computes one tile's
// layer while the 16 epilogue warps turn the other tile's accumulator into
// its next activations:
//   MMA(t0, L0) | epi(t0, L0) + MMA(t1, L0) | epi(t1, L0) + MMA(t0, L1) | ...
// Each tile keeps its activations in its own 64 KB operand buffer and its
// accumulator in its own 256 tensor-memory columns.  The weights stream in
// K-chunks of 64 (at most 32 KB, one bulk copy each) through a 2-stage ring,
// once per (tile, layer), in the order the MMAs use them.  A tile's inputs,
// the first layer's operand, sit in a 12 KB buffer of their own, which a
// staging warp fills with the tile's inputs of the next pair once the first
// layer's MMA of this pair has read it: the global loads' latency stays off
// the path between the output layer and the next pair's first layer.  Roles:
// warps 0-15 epilogue (warp w: TMEM lane quarter w % 4, column group w / 4),
// warp 16 the copies, warp 17 the MMAs, warp 18 the input staging (the first
// pair's inputs are staged by the epilogue warps at the start).  Every wait is
// bounded; a wait that gives up sets the error word and every role stops at
// its next wait.
constexpr int PP_EPI_WARPS = 16;
static_assert(H / 4 == 64, "an epilogue warp's column group is two 32-column accumulator loads");
constexpr int PP_THREADS = (PP_EPI_WARPS + 3) * 32;
constexpr int PP_KCHUNK = 64;                               // K per weight chunk (4 MMAs of K = 16)
constexpr size_t PP_STAGE = 256 * PP_KCHUNK * 2;            // largest chunk: N = 256
constexpr size_t PP_SMEM_IN = ROWS * IN * 2;                // a tile's inputs as the first layer's operand
// two activation tiles, the weight ring, two input tiles
constexpr size_t PP_SMEM = 2 * SMEM_A + 2 * PP_STAGE + 2 * PP_SMEM_IN;
// chunks of layer l: 48 inputs -> one chunk of 3 K-blocks, 256 -> four of 4
__host__ __device__ constexpr int pp_chunks(int l) { return (kdim(l) + PP_KCHUNK - 1) / PP_KCHUNK; }
__host__ __device__ constexpr int pp_kblocks(int l, int c) {
  return (kdim(l) - c * PP_KCHUNK) >= PP_KCHUNK ? PP_KCHUNK / 16 : (kdim(l) - c * PP_KCHUNK) / 16;
}

__device__ __forceinline__ void tmem_alloc512(uint32_t* slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(slot)) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc512(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(taddr) : "memory");
}
__device__ __forceinline__ void mbar_init_cnt(uint64_t* bar, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive_one(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

struct PpArgs {
  const float* x; int B;              // inputs [B][IN]
  const unsigned char* Wp;            // packed BF16 forward operands (pk_off)
  const float* b[4];
  float* out;                         // [B][OUT]
  int* err;
};

// Stage the inputs of rows row0 .. row0 + 127 as a BF16 operand (zeros past B):
// 768 groups of 8, group c at row c / 6, columns 8 (c % 6) .. + 7, taken by
// `n` threads (thread t: groups t, t + n, ...) `G` groups at a time, so that
// 8 G loads are in flight per thread.
constexpr int PP_IN_GROUPS = ROWS * (IN / 8);
template <int G>
__device__ __forceinline__ void pp_stage_input(unsigned char* S, const float* x, int B, int row0, int t, int n) {
  for (int c0 = t; c0 < PP_IN_GROUPS; c0 += G * n) {
    float v[G][8];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int c = c0 + g * n, rr = c / (IN / 8), kk = (c % (IN / 8)) * 8;
      const bool in = c < PP_IN_GROUPS && row0 + rr < B;
#pragma unroll
      for (int e = 0; e < 8; ++e) v[g][e] = in ? x[static_cast<long>(row0 + rr) * IN + kk + e] : 0.f;
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int c = c0 + g * n, rr = c / (IN / 8), kk = (c % (IN / 8)) * 8;
      if (c < PP_IN_GROUPS)
        *reinterpret_cast<uint4*>(S + blk_off(rr, kk, ROWS)) =
            make_uint4(pack_bf16x2(v[g][0], v[g][1]), pack_bf16x2(v[g][2], v[g][3]), pack_bf16x2(v[g][4], v[g][5]),
                       pack_bf16x2(v[g][6], v[g][7]));
    }
  }
}

__global__ void __launch_bounds__(PP_THREADS, 1) mlp_forward_pp_kernel(PpArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* ring = smem + 2 * SMEM_A;
  unsigned char* sin = ring + 2 * PP_STAGE;  // the two tiles' inputs: the first layer's A operands
  // in_ready: a tile's inputs of the next pair staged; l0_done: its first-layer MMA has read them
  __shared__ __align__(8) uint64_t w_full[2], w_empty[2], acc_full[2], a_ready[2], in_ready[2], l0_done[2];
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  __shared__ __align__(16) float s_bias[3 * H + OUT];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int n_tiles = (a.B + ROWS - 1) / ROWS, n_pairs = (n_tiles + 1) / 2;
  if (t == 0) {
    abort_flag = 0;
    for (int i = 0; i < 2; ++i) {
      mbar_init_cnt(&w_full[i], 1);
      mbar_init_cnt(&w_empty[i], 1);
      mbar_init_cnt(&acc_full[i], 1);
      mbar_init_cnt(&a_ready[i], PP_EPI_WARPS);
      mbar_init_cnt(&in_ready[i], 1);
      mbar_init_cnt(&l0_done[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc512(&tslot);
  pdl_wait();  // the inputs, the weights of the last update
  pdl_release();
  for (int i = t; i < 3 * H + OUT; i += PP_THREADS) s_bias[i] = i < 3 * H ? a.b[i / H][i % H] : a.b[3][i - 3 * H];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  int my_pairs = 0;
  for (int p = blockIdx.x; p < n_pairs; p += gridDim.x) ++my_pairs;
  auto give_up = [&]() {
    atomicOr(a.err, ERR_WAIT);
    abort_flag = 1;
  };

  if (warp == PP_EPI_WARPS) {
    // ---- copies: every (pair, layer, tile) job's weight chunks, in MMA order
    if (lane == 0) {
      int q = 0;
      for (int i = 0; i < my_pairs; ++i)
        for (int l = 0; l < 4; ++l)
          for (int tt = 0; tt < 2; ++tt)
            for (int c = 0; c < pp_chunks(l); ++c) {
              const int s = q & 1;
              if (q >= 2 && (abort_flag || !mbar_wait_bounded(&w_empty[s], static_cast<uint32_t>((q >> 1) - 1) & 1u))) {
                give_up();
                goto copies_done;
              }
              const uint32_t bytes = static_cast<uint32_t>(pp_kblocks(l, c) * ndim(l) * 32);
              mbar_expect_tx(&w_full[s], bytes);
              bulk_g2s(ring + s * PP_STAGE, a.Wp + pk_off(l) + static_cast<size_t>(c) * (PP_KCHUNK / 16) * ndim(l) * 32,
                       bytes, &w_full[s]);
              ++q;
            }
    copies_done:
      // no copy may land after the CTA ends
      for (int qq = max(0, q - 2); qq < q; ++qq) mbar_wait_bounded(&w_full[qq & 1], static_cast<uint32_t>(qq >> 1) & 1u);
    }
  } else if (warp == PP_EPI_WARPS + 1) {
    // ---- MMAs: job (tile tt, layer l) once tile tt's activations for layer l are staged
    if (lane == 0) {
      int q = 0, j0 = 0, j1 = 0;
      for (int i = 0; i < my_pairs; ++i)
        for (int l = 0; l < 4; ++l)
          for (int tt = 0; tt < 2; ++tt) {
            const int j = tt ? j1 : j0;
            if (abort_flag || !mbar_wait_bounded(&a_ready[tt], static_cast<uint32_t>(j) & 1u) ||
                (l == 0 && i > 0 && !mbar_wait_bounded(&in_ready[tt], static_cast<uint32_t>(i - 1) & 1u))) {
              give_up();
              goto mma_done;
            }
            tc_fence_after();
            const uint32_t acc = tmem + static_cast<uint32_t>(tt * 256);
            const uint32_t id = instr_desc(ROWS, ndim(l));
            const uint32_t A0 = smem_u32(l == 0 ? sin + tt * PP_SMEM_IN : smem + tt * SMEM_A);
            for (int c = 0; c < pp_chunks(l); ++c) {
              const int s = q & 1;
              if (!mbar_wait_bounded(&w_full[s], static_cast<uint32_t>(q >> 1) & 1u)) {
                give_up();
                goto mma_done;
              }
              const uint32_t b0 = smem_u32(ring + s * PP_STAGE);
              for (int kb = 0; kb < pp_kblocks(l, c); ++kb)
                umma_bf16(acc, smem_desc(A0 + (c * (PP_KCHUNK / 16) + kb) * ROWS * 32),
                          smem_desc(b0 + kb * ndim(l) * 32), id, (c > 0 || kb > 0) ? 1u : 0u);
              umma_commit(&w_empty[s]);
              ++q;
            }
            umma_commit(&acc_full[tt]);
            if (l == 0) umma_commit(&l0_done[tt]);  // the tile's input buffer may take the next pair's
            if (tt) ++j1; else ++j0;
          }
    mma_done:;
    }
  } else if (warp == PP_EPI_WARPS + 2) {
    // ---- input staging: each later pair's inputs, tile by tile, once the tile's
    // first-layer MMA of the pair before has read its buffer
    for (int i = 1; i < my_pairs; ++i) {
      const int pair = blockIdx.x + i * gridDim.x;
      for (int tt = 0; tt < 2; ++tt) {
        if (abort_flag || !mbar_wait_bounded(&l0_done[tt], static_cast<uint32_t>(i - 1) & 1u)) {
          give_up();
          goto staging_done;
        }
        pp_stage_input<4>(sin + tt * PP_SMEM_IN, a.x, a.B, (2 * pair + tt) * ROWS, lane, 32);
        fence_proxy_async();  // the operand, written by this warp, to the tensor core
        __syncwarp();
        if (lane == 0) mbar_arrive_one(&in_ready[tt]);
      }
    }
  staging_done:;
  } else {
    // ---- epilogues: warp w reads TMEM lanes 32 (w % 4) .. + 31, column group w / 4
    const int grp = warp >> 2, row = 32 * (warp & 3) + lane;
    int j0 = 0, j1 = 0;
    if (my_pairs > 0) {  // the first pair's inputs (the staging warp takes the later pairs')
      pp_stage_input<1>(sin, a.x, a.B, 2 * blockIdx.x * ROWS, t, PP_EPI_WARPS * 32);
      pp_stage_input<1>(sin + PP_SMEM_IN, a.x, a.B, (2 * blockIdx.x + 1) * ROWS, t, PP_EPI_WARPS * 32);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) {
      mbar_arrive_one(&a_ready[0]);
      mbar_arrive_one(&a_ready[1]);
    }
    for (int i = 0; i < my_pairs; ++i) {
      const int pair = blockIdx.x + i * gridDim.x;
      for (int l = 0; l < 4; ++l)
        for (int tt = 0; tt < 2; ++tt) {
          const int j = tt ? j1 : j0;
          if (abort_flag || !mbar_wait_bounded(&acc_full[tt], static_cast<uint32_t>(j) & 1u)) {
            give_up();
            goto epi_done;
          }
          tc_fence_after();
          unsigned char* A = smem + tt * SMEM_A;
          const uint32_t acc = tmem + static_cast<uint32_t>(tt * 256);
          const int r = (2 * pair + tt) * ROWS + row;
          if (l < 3) {
            // the warp's 64 columns: both accumulator loads in flight before one wait
            uint32_t u0[32], u1[32];
            const int cb = grp * (H / 4);
            tmem_ld32_nowait(lane_addr(acc, cb), u0);
            tmem_ld32_nowait(lane_addr(acc, cb + 32), u1);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
              const int c0 = cb + 32 * h2;
              const float* bias = s_bias + l * H + c0;
              uint32_t hp[16];
#pragma unroll
              for (int e = 0; e < 32; e += 2) {
                const float vx = __uint_as_float(h2 ? u1[e] : u0[e]), vy = __uint_as_float(h2 ? u1[e + 1] : u0[e + 1]);
                const float2 g = gelu2(__fadd2_rn(make_float2(vx, vy), make_float2(bias[e], bias[e + 1])));
                hp[e / 2] = pack_bf16x2(g.x, g.y);
              }
#pragma unroll
              for (int qd = 0; qd < 4; ++qd)
                *reinterpret_cast<uint4*>(A + blk_off(row, c0 + 8 * qd, ROWS)) =
                    make_uint4(hp[4 * qd], hp[4 * qd + 1], hp[4 * qd + 2], hp[4 * qd + 3]);
            }
          } else {
            if (grp == 0) {
              float v[32];
              tmem_ld32(lane_addr(acc, 0), v);
              if (r < a.B) {
                const float* bias = s_bias + 3 * H;
                float4* od = reinterpret_cast<float4*>(a.out + static_cast<long>(r) * OUT);
#pragma unroll
                for (int qd = 0; qd < 8; ++qd)
                  od[qd] = make_float4(v[4 * qd] + bias[4 * qd], v[4 * qd + 1] + bias[4 * qd + 1],
                                       v[4 * qd + 2] + bias[4 * qd + 2], v[4 * qd + 3] + bias[4 * qd + 3]);
              }
            }
          }
          fence_proxy_async();  // the activations, written by every thread, to the tensor core
          tc_fence_before();    // ... after this warp's reads of the accumulator
          __syncwarp();
          if (lane == 0) mbar_arrive_one(&a_ready[tt]);
          if (tt) ++j1; else ++j0;
        }
    }
  epi_done:;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc512(tmem);
}

// ------------------------------------------------------------------ backward: weight gradients
// The weight gradients dW_l = dZ_l^T A_{l-1} (and db_l = column sums of dZ_l):
// per CTA one layer, 128 of its outputs and a split of the batch rows, which
// are the GEMM's K.  The operands -- x, A_l, dZ_l -- arrive in the f8 layout
// the forward and the dZ chain write: per group of 8 features, every row's 8
// BF16 values (16 bytes) one after the other, so that a chunk's 64 rows of a
// group are 1 KB in one piece.  TMA tensor copies (cp.async.bulk.tensor, 3-D:
// 128-byte core matrices x feature groups x 8-row blocks) bring each 64-row
// chunk of both operands into a ring of DW_STAGES shared-memory stages, a K
// group's core matrices side by side (so that the tensor core's reads of
// neighbouring feature groups fall on different banks): the MN-major operand
// layout without swizzle, core matrices of 8 rows (K) x 16 bytes, the next
// feature group 128 bytes on, the next 8 rows G x 128 bytes on (G: the
// operand's feature groups); a K step of 16 rows moves 2 G x 128 bytes.  One thread
// issues the MMAs of the chunks that have landed; the 128 threads of the
// epilogue warps add their output's chunk values for db before releasing a
// stage.  Batch rows past B are zeros, written by the producers.
constexpr int DW_STAGES = 3;
constexpr int DW_CHUNK = 64;                              // batch rows per stage (4 MMAs of K = 16)
constexpr int DW_THREADS = 160;                           // 4 epilogue warps (TMEM lane quarters) + 1 issuing warp
constexpr size_t DW_STAGE_A = 128 * DW_CHUNK * 2, DW_STAGE_B = 128 * DW_CHUNK * 2;  // B: at most 128 features
constexpr size_t DW_STAGE = DW_STAGE_A + DW_STAGE_B;
// + alignment of the ring to 1 KB, + the all-ones operand of the bias gradients (16 x 64 BF16)
constexpr size_t DW_ONES = 16 * DW_CHUNK * 2;
constexpr size_t DW_SMEM = DW_STAGES * DW_STAGE + 1024 + DW_ONES;
constexpr int DW_MAX_SPLITS = 32;
// CTAs of one row split: the 256-wide layers 1 and 2 as (128 outputs) x (128
// inputs) blocks, 4 each; layers 0 (48 inputs) and 3 (32 outputs, swapped) as
// 128-row blocks of the whole product, 2 each -- blocks of similar work, two
// CTAs per SM (99 KB of shared memory, 256 tensor-memory columns each)
constexpr int DW_BLOCKS = 12;

// tensor maps (f8 layout): A operands (16 feature groups: 128 features) dZ_0,
// dZ_1, dZ_2, A_2; B operands (every feature group) x, A_0, A_1, dZ_3
struct DwMaps {
  CUtensorMap map[8];
};
struct DwArgs {
  int B, rows_per_split;
  float* grad;                        // [N_PARAMS]: every split adds its share of dW and db (zeroed by the forward)
  int* err;
};

__device__ __forceinline__ void mbar_init_n(uint64_t* bar, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// 3-D tensor copy global -> shared, completion counted on the mbarrier
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
// MN-major without swizzle, as the stages hold the operands: core matrices of
// 8 rows (K) x 16 bytes (8 features), the feature groups' core matrices of a
// K group side by side (128 B apart: stride offset), K groups G x 128 B apart
// (leading offset; G = the operand's feature groups), descriptor version 1,
// layout type 0
__device__ __forceinline__ uint64_t smem_desc_f8(uint32_t saddr, uint32_t kgroup_bytes) {
  return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) | (static_cast<uint64_t>(kgroup_bytes >> 4) << 16) |
         (static_cast<uint64_t>(128 >> 4) << 32) | (1ull << 46);
}
constexpr uint32_t IDESC_MN = (1u << 15) | (1u << 16);  // kind::f16: both operands MN-major

__global__ void __launch_bounds__(DW_THREADS, 2) mlp_backward_dw_kernel(const __grid_constant__ DwMaps tm, DwArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[DW_STAGES], empty[DW_STAGES];
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  const int t = threadIdx.x, warp = t >> 5;
  // block: layers 1, 2 -> (layer, output half, input half); layers 0, 3 -> (layer, half)
  const int bx = blockIdx.x;
  const int l = bx < 8 ? 1 + (bx >> 2) : (bx < 10 ? 0 : 3);
  const int half = bx < 8 ? (bx >> 1) & 1 : bx & 1, nh = bx < 8 ? bx & 1 : 0;
  const bool swapped = l == 3;  // 32 outputs: M runs over the inputs, D = dW^T
  const int K = kdim(l), N = ndim(l);
  const int NB_ = swapped ? N : (K == H ? H / 2 : K);  // the GEMM's N' (rows of the B operand)
  const CUtensorMap* mA = &tm.map[swapped ? 3 : l];
  const CUtensorMap* mB = &tm.map[4 + l];
  const bool sum_a = !swapped && nh == 0, sum_b = swapped && half == 0;  // db: each output's column once
  const int r_begin = blockIdx.y * a.rows_per_split, r_end = min(a.B, r_begin + a.rows_per_split);
  const int n_chunks = r_end > r_begin ? (r_end - r_begin + DW_CHUNK - 1) / DW_CHUNK : 0;
  const uint32_t stage_tx = static_cast<uint32_t>((128 + NB_) * DW_CHUNK * 2);
  if (t == 0) {
    abort_flag = 0;
    for (int st = 0; st < DW_STAGES; ++st) {
      mbar_init_n(&full[st], 1);
      // the MMAs' commit (and, for the 32-output layer, the 128 threads summing db)
      mbar_init_n(&empty[st], swapped ? 1 + 128 : 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tslot);  // dW: columns 0 .. N' - 1 (at most 128); db: 128 .. 143
  unsigned char* ring = smem + ((1024u - (smem_u32(smem) & 1023u)) & 1023u);  // 1 KB aligned
  // db_l[n] = sum over rows of dZ_l[row][n] = (dZ_l^T . 1)[n]: a second product of
  // the same A operand with a 16-column block of ones (the f8 layout of 16
  // features x 64 rows), accumulated in tensor memory next to dW
  unsigned char* ones = ring + DW_STAGES * DW_STAGE;
  if (t < 128) reinterpret_cast<uint4*>(ones)[t] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
  fence_proxy_async();
  pdl_wait();  // the operands written by the forward and the dZ chain
  pdl_release();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  auto stage_a = [&](int st) { return ring + st * DW_STAGE; };
  auto stage_b = [&](int st) { return ring + st * DW_STAGE + DW_STAGE_A; };

  if (t == 128) {
    // copies and MMAs: chunk c lives in stage c % DW_STAGES; its stage is refilled
    // with chunk c + DW_STAGES once the MMAs of c and its db sums are done
    auto load = [&](int c) {
      const int st = c % DW_STAGES, y0 = r_begin + c * DW_CHUNK;
      mbar_expect_tx(&full[st], stage_tx);
      tma_load_3d(stage_a(st), mA, 0, half * 16, y0 / 8, &full[st]);
      tma_load_3d(stage_b(st), mB, 0, nh * 16, y0 / 8, &full[st]);
    };
    const uint32_t id = instr_desc(ROWS, NB_) | IDESC_MN, id_db = instr_desc(ROWS, 16) | IDESC_MN;
    const uint32_t o0 = smem_u32(ones);
    int issued = 0;
    for (; issued < n_chunks && issued < DW_STAGES; ++issued) load(issued);
    for (int c = 0; c < n_chunks; ++c) {
      const int st = c % DW_STAGES;
      const uint32_t par = static_cast<uint32_t>(c / DW_STAGES) & 1u;
      if (!mbar_wait_bounded(&full[st], par)) {
        atomicOr(a.err, ERR_WAIT);
        abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(stage_a(st)), b0 = smem_u32(stage_b(st));
      for (int kk = 0; kk < DW_CHUNK / 16; ++kk)
        umma_bf16(tmem, smem_desc_f8(a0 + kk * 2 * 16 * 128, 16 * 128),
                  smem_desc_f8(b0 + kk * 2 * (NB_ / 8) * 128, (NB_ / 8) * 128), id, (c > 0 || kk > 0) ? 1u : 0u);
      if (sum_a)
        for (int kk = 0; kk < DW_CHUNK / 16; ++kk)
          umma_bf16(tmem + 128, smem_desc_f8(a0 + kk * 2 * 16 * 128, 16 * 128), smem_desc_f8(o0 + kk * 2 * 256, 256),
                    id_db, (c > 0 || kk > 0) ? 1u : 0u);
      umma_commit(&empty[st]);
      if (issued < n_chunks) {
        if (!mbar_wait_bounded(&empty[st], par)) {
          atomicOr(a.err, ERR_WAIT);
          abort_flag = 1;
          break;
        }
        load(issued++);
      }
    }
    // no copy may land after the CTA ends: wait for every chunk issued
    for (int c = max(0, issued - DW_STAGES); c < issued; ++c)
      mbar_wait_bounded(&full[c % DW_STAGES], static_cast<uint32_t>(c / DW_STAGES) & 1u);
  } else if (t < 128 && swapped) {
    // db of the 32-output layer (its outputs are the B operand): this thread's
    // output summed over the chunk's rows, then the stage released
    const int row = t;
    const bool mine = sum_b && row < NB_;
    float cs = 0.f;
    for (int c = 0; c < n_chunks; ++c) {
      const int st = c % DW_STAGES;
      const uint32_t par = static_cast<uint32_t>(c / DW_STAGES) & 1u;
      if (!mbar_wait_bounded(&full[st], par)) {
        atomicOr(a.err, ERR_WAIT);
        abort_flag = 1;
        break;
      }
      if (mine) {
        // output `row`: element row % 8 of the 16-byte rows of its feature group's
        // core matrices, one per K group (G x 128 B apart)
        const int G = NB_ / 8;
        const unsigned char* base = stage_b(st) + (row >> 3) * 128 + (row & 7) * 2;
#pragma unroll
        for (int kg = 0; kg < DW_CHUNK / 8; ++kg)
#pragma unroll
          for (int ri = 0; ri < 8; ++ri)
            cs += __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(base + kg * G * 128 + ri * 16));
      }
      mbar_arrive(&empty[st]);
    }
    if (mine && n_chunks > 0) atomicAdd(a.grad + b_off(l) + row, cs);
  }
  __syncthreads();
  // every MMA has completed once the last chunk's stage was released
  bool ok = abort_flag == 0;
  if (ok && n_chunks > 0 && t < 128) {
    const int c = n_chunks - 1;
    if (!mbar_wait_bounded(&empty[c % DW_STAGES], static_cast<uint32_t>(c / DW_STAGES) & 1u)) {
      atomicOr(a.err, ERR_WAIT);
      ok = false;
    }
  }
  tc_fence_after();
  ok = __syncthreads_and(ok) != 0;
  // this split's share of dW (and db), added into the gradient
  if (ok && t < 128 && n_chunks > 0) {
    float* gW = a.grad + w_off(l);
    const int row = t;
    for (int c0 = 0; c0 < NB_; c0 += 32) {
      float v[32];
      tmem_ld32(lane_addr(tmem, c0), v);
      if (swapped) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (c0 + j < NB_) atomicAdd(gW + static_cast<long>(c0 + j) * K + half * 128 + row, v[j]);
      } else {
        float4* dst = reinterpret_cast<float4*>(gW + static_cast<long>(half * 128 + row) * K + nh * 128 + c0);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (c0 + 4 * q < NB_) atomicAdd(dst + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
      }
    }
    if (sum_a) {  // db of this block's outputs, from the ones product
      float v[32];
      tmem_ld32(lane_addr(tmem, 128), v);
      atomicAdd(a.grad + b_off(l) + half * 128 + row, v[0]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem);
}

// ------------------------------------------------------------------ Adam on the FP32 master weights
// Element i of the parameter vector: its layer and (row, column) if it is a
// weight, so that the BF16 copy can be written straight into both packed
// operand layouts.
__device__ __forceinline__ void store_packed(int i, float w, unsigned char* Wp, unsigned char* WpT) {
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const int off = static_cast<int>(w_off(l)), K = kdim(l), N = ndim(l);
    if (i >= off && i < off + N * K) {
      const int n = (i - off) / K, k = (i - off) % K;
      const __nv_bfloat16 h = __float2bfloat16_rn(w);
      *reinterpret_cast<__nv_bfloat16*>(Wp + pk_off(l) + blk_off(n, k, N)) = h;
      *reinterpret_cast<__nv_bfloat16*>(WpT + pk_off(l) + blk_off(k, n, K)) = h;
    }
  }
}

// the gradient as the dW kernel has summed it over the row splits
__global__ void mlp_adam_kernel(float* p, const float* __restrict__ grad, float* m, float* v, unsigned char* Wp,
                                unsigned char* WpT, int n, float lr, float b1, float b2, float eps, float ib1,
                                float ib2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_wait();  // the gradient
  pdl_release();
  if (i >= n) return;
  const float gi = grad[i];
  const float mi = fmaf(b1, m[i], (1.f - b1) * gi), vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
  m[i] = mi;
  v[i] = vi;
  const float w = p[i] - lr * (mi * ib1) / (sqrtf(vi * ib2) + eps);
  p[i] = w;
  store_packed(i, w, Wp, WpT);
}

__global__ void pack_kernel(const float* p, unsigned char* Wp, unsigned char* WpT, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) store_packed(i, p[i], Wp, WpT);
}

}  // namespace mlpk

using namespace mlpk;

struct tamp_mlp {
  int device = 0;
  cudaStream_t stream = nullptr;
  int max_batch = 0;
  float* params = nullptr;     // FP32 master
  unsigned char* wp = nullptr;  // BF16 weights packed as forward GEMM operands (pk_off)
  unsigned char* wpt = nullptr; // ... and as transposed operands for the backward pass
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  __half* G = nullptr;           // [3][g_rows][H]: GELU'(Z_l) of the last training forward (FP16, g_pieces layout)
  // weight-gradient operands in the f8 layout ([features / 8][g_rows] x 16 bytes)
  uint4* X8 = nullptr;           // x: IN / 8 groups
  uint4* A8 = nullptr;           // A_0 .. A_2: 3 x H / 8 groups
  uint4* dZ8 = nullptr;          // dZ_0 .. dZ_2 (3 x H / 8 groups), then dZ_3 (OUT / 8)
  float* out = nullptr;        // [max_batch][OUT]
  mlpk::DwMaps dw_maps;        // tensor maps of the weight-gradient operands for batches of dw_maps_B rows
  int dw_maps_B = -1;
  float* loss = nullptr;
  int* err = nullptr;
  long step = 0;
  std::string last_error;
};

namespace {
// rows of each layer's GELU'(Z) block: whole 128-row tiles
size_t g_rows(const tamp_mlp* n) { return (static_cast<size_t>(n->max_batch) + ROWS - 1) / ROWS * ROWS; }
tamp_status mfail(tamp_mlp* n, tamp_status st, const std::string& msg) {
  if (n) n->last_error = msg;
  return st;
}
#define MLP_TRY(n, call)                                                                          \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return mfail((n), e_ == cudaErrorMemoryAllocation ? TAMP_ERR_OOM : TAMP_ERR_CUDA,          \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                          \
  } while (0)

struct Dev {
  int prev = -1;
  explicit Dev(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~Dev() {
    int c;
    cudaGetDevice(&c);
    if (prev >= 0 && c != prev) cudaSetDevice(prev);
  }
};

cudaError_t enable_smem(int device) {
  static unsigned long long done = 0;  // one bit per device ordinal < 64
  const unsigned long long bit = device < 64 ? 1ull << device : 0;
  if (done & bit) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(SMEM_BYTES));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_backward_dw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(DW_SMEM));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_forward_pp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(PP_SMEM));
  if (e == cudaSuccess) done |= bit;
  return e;
}


// cuTensorMapEncodeTiled from the driver, through the runtime (no link-time
// dependency on the driver library)
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_tiled() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

// The weight-gradient operands in the f8 layout as 3-D tensors: 8 rows of a
// feature group (one 128-byte core matrix) x feature groups x blocks of 8 rows
// (g_rows / 8), with boxes of 128 bytes x 16 groups (A operands: 128
// features) or every group (B operands) x 8 blocks (a 64-row chunk): in shared
// memory a K group's core matrices lie side by side.  No swizzle.  Rows past
// B hold zeros, written by the producers for every row of their tiles.
tamp_status make_dw_maps(tamp_mlp* n, int B) {
  if (n->dw_maps_B == B) return TAMP_OK;
  EncodeTiled enc = encode_tiled();
  if (!enc) return mfail(n, TAMP_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const size_t lr = g_rows(n), g = static_cast<size_t>(H / 8) * lr;  // uint4 per 256-feature array
  struct Spec { const void* base; int groups, box; };
  const Spec spec[8] = {
      {n->dZ8, H / 8, 16}, {n->dZ8 + g, H / 8, 16}, {n->dZ8 + 2 * g, H / 8, 16}, {n->A8 + 2 * g, H / 8, 16},
      {n->X8, IN / 8, IN / 8}, {n->A8, H / 8, 16}, {n->A8 + g, H / 8, 16}, {n->dZ8 + 3 * g, OUT / 8, OUT / 8}};
  for (int i = 0; i < 8; ++i) {
    const cuuint64_t dims[3] = {64, static_cast<cuuint64_t>(spec[i].groups), static_cast<cuuint64_t>(lr / 8)};
    const cuuint64_t strides[2] = {static_cast<cuuint64_t>(lr * 16), 128};
    const cuuint32_t box[3] = {64, static_cast<cuuint32_t>(spec[i].box), static_cast<cuuint32_t>(DW_CHUNK / 8)};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = enc(&n->dw_maps.map[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(spec[i].base),
                           dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return mfail(n, TAMP_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(r) + ")");
  }
  n->dw_maps_B = B;
  return TAMP_OK;
}

// a kernel launched with programmatic stream serialisation (the training
// step's kernels, the inference forward): it may be scheduled while the
// previous kernel of the stream finishes, and waits for it (pdl_wait) before
// reading its outputs
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// Inference forward: pairs of 128-row tiles, about one CTA per SM, each taking
// pairs until none is left.
cudaError_t launch_forward_pp(tamp_mlp* n, const float* x, int B, float* out, cudaStream_t st) {
  PpArgs a{};
  a.x = x; a.B = B; a.out = out; a.err = n->err; a.Wp = n->wp;
  for (int l = 0; l < 4; ++l) a.b[l] = n->params + b_off(l);
  int sm = 148;
  cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, n->device);
  const int pairs = ((B + ROWS - 1) / ROWS + 1) / 2;
  return launch_pdl(mlp_forward_pp_kernel, dim3(std::min(pairs, sm)), dim3(PP_THREADS), PP_SMEM, st, a);
}

tamp_status check_err(tamp_mlp* n) {
  int e = 0;
  MLP_TRY(n, cudaMemcpyAsync(&e, n->err, 4, cudaMemcpyDeviceToHost, n->stream));
  MLP_TRY(n, cudaStreamSynchronize(n->stream));
  if (e) return mfail(n, TAMP_ERR_TIMEOUT, "a tensor-core completion wait timed out on the device");
  return TAMP_OK;
}


// forward (training form) + loss + backward: the gradient in n->grad (every
// row split's share added by the dW kernel into the buffer the forward zeroed)
tamp_status gradient(tamp_mlp* n, const float* x, const float* y, const float* mask, int B) {
  MLP_TRY(n, enable_smem(n->device));
  const int tiles = (B + ROWS - 1) / ROWS;
  TrainArgs ta{};
  ta.x = x; ta.B = B; ta.y = y; ta.mask = mask; ta.err = n->err;
  ta.Wp = n->wp; ta.WpT = n->wpt;
  for (int l = 0; l < 4; ++l) ta.b[l] = n->params + b_off(l);
  ta.ldR = static_cast<int>(g_rows(n));
  ta.X8 = n->X8;
  for (int l = 0; l < 3; ++l) {
    ta.G[l] = n->G + static_cast<size_t>(l) * g_rows(n) * H;
    ta.A8[l] = n->A8 + static_cast<size_t>(l) * (H / 8) * g_rows(n);
  }
  for (int l = 0; l < 4; ++l) ta.dZ8[l] = n->dZ8 + static_cast<size_t>(l) * (H / 8) * g_rows(n);
  ta.loss = n->loss;  // zeroed by the kernel, summed over its tiles
  ta.grad = n->grad;  // zeroed by the kernel, summed by the dW kernel
  MLP_TRY(n, launch_pdl(mlp_train_kernel, dim3(tiles), dim3(THREADS), SMEM_BYTES, n->stream, ta));
  // weight gradients: DW_BLOCKS blocks x row splits
  const tamp_status ms = make_dw_maps(n, B);
  if (ms != TAMP_OK) return ms;
  DwArgs w{};
  int sm = 148;
  cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, n->device);
  // row splits: about two CTAs per SM over the DW_BLOCKS blocks of each split
  const int splits = std::max(1, std::min({DW_MAX_SPLITS, 2 * sm / DW_BLOCKS, (B + DW_CHUNK - 1) / DW_CHUNK}));
  w.B = B; w.grad = n->grad; w.err = n->err;
  w.rows_per_split = ((B + splits - 1) / splits + DW_CHUNK - 1) / DW_CHUNK * DW_CHUNK;
  MLP_TRY(n, launch_pdl(mlp_backward_dw_kernel, dim3(DW_BLOCKS, splits), dim3(DW_THREADS), DW_SMEM, n->stream,
                        n->dw_maps, w));
  return TAMP_OK;
}
}  // namespace

extern "C" {

tamp_status tamp_mlp_create(int device, void* stream, int max_batch, tamp_mlp** out) {
  if (!out || max_batch <= 0 || max_batch > (1 << 22)) return TAMP_ERR_INVALID_ARG;
  *out = nullptr;
  tamp_mlp* n = new tamp_mlp();
  n->device = device;
  n->stream = static_cast<cudaStream_t>(stream);
  n->max_batch = max_batch;
  Dev g(device);
  const size_t mb = static_cast<size_t>(max_batch);
  cudaError_t e = cudaMalloc(&n->params, N_PARAMS * 4);
  if (e == cudaSuccess) e = cudaMalloc(&n->wp, PK_BYTES);
  if (e == cudaSuccess) e = cudaMalloc(&n->wpt, PK_BYTES);
  if (e == cudaSuccess) e = cudaMalloc(&n->grad, N_PARAMS * 4);
  if (e == cudaSuccess) e = cudaMalloc(&n->m, N_PARAMS * 4);
  if (e == cudaSuccess) e = cudaMalloc(&n->v, N_PARAMS * 4);
  const size_t lr = g_rows(n);
  if (e == cudaSuccess) e = cudaMalloc(&n->G, 3 * g_rows(n) * H * 2);
  if (e == cudaSuccess) e = cudaMalloc(&n->X8, IN * lr * 2);
  if (e == cudaSuccess) e = cudaMalloc(&n->A8, 3 * H * lr * 2);
  if (e == cudaSuccess) e = cudaMalloc(&n->dZ8, (3 * H + OUT) * lr * 2);
  if (e == cudaSuccess) e = cudaMalloc(&n->out, mb * OUT * 4);
  if (e == cudaSuccess) e = cudaMalloc(&n->loss, 4);
  if (e == cudaSuccess) e = cudaMalloc(&n->err, 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->params, 0, N_PARAMS * 4, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->wp, 0, PK_BYTES, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->wpt, 0, PK_BYTES, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, N_PARAMS * 4, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, N_PARAMS * 4, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->err, 0, 4, n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) {
    tamp_mlp_destroy(n);
    return e == cudaErrorMemoryAllocation ? TAMP_ERR_OOM : TAMP_ERR_CUDA;
  }
  *out = n;
  return TAMP_OK;
}

tamp_status tamp_mlp_destroy(tamp_mlp* n) {
  if (!n) return TAMP_ERR_INVALID_ARG;
  Dev g(n->device);
  cudaStreamSynchronize(n->stream);
  cudaFree(n->params); cudaFree(n->wp); cudaFree(n->wpt); cudaFree(n->grad); cudaFree(n->m); cudaFree(n->v);
  cudaFree(n->G); cudaFree(n->X8); cudaFree(n->A8); cudaFree(n->dZ8); cudaFree(n->out);
  cudaFree(n->loss); cudaFree(n->err);
  delete n;
  return TAMP_OK;
}

int tamp_mlp_param_count(void) { return static_cast<int>(N_PARAMS); }

tamp_status tamp_mlp_set_params(tamp_mlp* n, const float* host, int count) {
  if (!n) return TAMP_ERR_INVALID_ARG;
  if (!host || count != static_cast<int>(N_PARAMS)) return mfail(n, TAMP_ERR_INVALID_ARG, "parameter count");
  Dev g(n->device);
  MLP_TRY(n, cudaMemcpyAsync(n->params, host, N_PARAMS * 4, cudaMemcpyHostToDevice, n->stream));
  pack_kernel<<<static_cast<int>((N_PARAMS + 255) / 256), 256, 0, n->stream>>>(n->params, n->wp, n->wpt,
                                                                              static_cast<int>(N_PARAMS));
  MLP_TRY(n, cudaGetLastError());
  MLP_TRY(n, cudaMemsetAsync(n->m, 0, N_PARAMS * 4, n->stream));
  MLP_TRY(n, cudaMemsetAsync(n->v, 0, N_PARAMS * 4, n->stream));
  n->step = 0;
  MLP_TRY(n, cudaStreamSynchronize(n->stream));
  return TAMP_OK;
}

tamp_status tamp_mlp_get_params(tamp_mlp* n, float* host, int count) {
  if (!n) return TAMP_ERR_INVALID_ARG;
  if (!host || count != static_cast<int>(N_PARAMS)) return mfail(n, TAMP_ERR_INVALID_ARG, "parameter count");
  Dev g(n->device);
  MLP_TRY(n, cudaMemcpyAsync(host, n->params, N_PARAMS * 4, cudaMemcpyDeviceToHost, n->stream));
  MLP_TRY(n, cudaStreamSynchronize(n->stream));
  return TAMP_OK;
}

tamp_status tamp_mlp_forward(tamp_mlp* n, const float* x_dev, int B, float* out_dev) {
  if (!n) return TAMP_ERR_INVALID_ARG;
  if (!x_dev || !out_dev || B <= 0) return mfail(n, TAMP_ERR_INVALID_ARG, "bad forward arguments");
  Dev g(n->device);
  MLP_TRY(n, enable_smem(n->device));
  MLP_TRY(n, launch_forward_pp(n, x_dev, B, out_dev, n->stream));
  return TAMP_OK;
}

tamp_status tamp_mlp_gradient(tamp_mlp* n, const float* x, const float* y, const float* mask, int B,
                              float* grad_dev, float* loss) {
  if (!n) return TAMP_ERR_INVALID_ARG;
  if (!x || !y || !mask || B <= 0 || B > n->max_batch) return mfail(n, TAMP_ERR_INVALID_ARG, "bad batch");
  Dev g(n->device);
  tamp_status st = gradient(n, x, y, mask, B);
  if (st != TAMP_OK) return st;
  if (grad_dev) MLP_TRY(n, cudaMemcpyAsync(grad_dev, n->grad, N_PARAMS * 4, cudaMemcpyDeviceToDevice, n->stream));
  if (loss) MLP_TRY(n, cudaMemcpyAsync(loss, n->loss, 4, cudaMemcpyDeviceToHost, n->stream));
  return check_err(n);
}

tamp_status tamp_mlp_train_step(tamp_mlp* n, const float* x, const float* y, const float* mask, int B, float lr,
                                float* loss) {
  if (!n) return TAMP_ERR_INVALID_ARG;
  if (!x || !y || !mask || B <= 0 || B > n->max_batch || !(lr >= 0.f)) return mfail(n, TAMP_ERR_INVALID_ARG, "bad batch");
  Dev g(n->device);
  tamp_status st = gradient(n, x, y, mask, B);
  if (st != TAMP_OK) return st;
  ++n->step;
  const double b1 = 0.9, b2 = 0.999;
  const float ib1 = static_cast<float>(1.0 / (1.0 - std::pow(b1, static_cast<double>(n->step))));
  const float ib2 = static_cast<float>(1.0 / (1.0 - std::pow(b2, static_cast<double>(n->step))));
  MLP_TRY(n, launch_pdl(mlp_adam_kernel, dim3(static_cast<int>((N_PARAMS + 255) / 256)), dim3(256), 0, n->stream,
                        n->params, n->grad, n->m, n->v, n->wp, n->wpt, static_cast<int>(N_PARAMS), lr, 0.9f, 0.999f,
                        1e-8f, ib1, ib2));
  if (loss) {
    MLP_TRY(n, cudaMemcpyAsync(loss, n->loss, 4, cudaMemcpyDeviceToHost, n->stream));
    return check_err(n);
  }
  return TAMP_OK;
}

const char* tamp_mlp_last_error(const tamp_mlp* n) { return n ? n->last_error.c_str() : "null network"; }

}  // extern "C"

// The proposal sampler's forward pass, on the scene's stream after any work
// queued on the network's own stream (training) has finished.
tamp_status mlp_forward_on_stream(tamp_mlp* n, const float* x_dev, int B, float* out_dev, cudaStream_t st,
                                  int device) {
  if (!n || !x_dev || !out_dev || B <= 0) return TAMP_ERR_INVALID_ARG;
  if (n->device != device) return mfail(n, TAMP_ERR_INVALID_ARG, "network and scene are on different devices");
  MLP_TRY(n, cudaStreamSynchronize(n->stream));
  MLP_TRY(n, enable_smem(n->device));
  MLP_TRY(n, launch_forward_pp(n, x_dev, B, out_dev, st));
  return TAMP_OK;
}
