// rgeo_mlp.cu -- tensor-core kernels of the learned exponential map (sm_103a).
//
// The surrogate maps (position, unit direction, arc length) to the endpoint and
// tangent residuals of a geodesic segment (Eq. 3.5: exp_p(s v)); it is a
// 7 -> 256 -> 256 -> 256 -> 7 MLP with ReLU.  Its 256 x 256 layers -- forward and
// both backward products -- run on the 5th-generation tensor cores:
//   * tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulation) issued by one thread,
//   * accumulators in tensor memory (TMEM), read back with tcgen05.ld,
//   * operands in shared memory in the canonical K-major layout without swizzle
//     (8-row x 16-byte core matrices): staged with cp.async by the training GEMM,
//     bulk-copied (cp.async.bulk) by the persistent inference kernel,
//   * completion signalled through mbarriers by tcgen05.commit.
// Inference runs all four layers in one persistent, warp-specialised kernel
// (k_mlp_infer_ws).  Every wait is bounded: a wait that runs out records kErrTimeout
// in the error word and the kernel returns after releasing its tensor memory.
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "rgeo.h"
#include "rgeo_internal.h"

namespace rgeo {
namespace {

constexpr int kTileM = 128;     // rows of A (and of C) per CTA
constexpr int kTileK = 64;      // K elements per shared-memory stage (4 MMAs of K = 16)
constexpr int kMaxTileN = 256;  // columns of C per CTA (TMEM columns)
constexpr long long kSpinLimit = 1ll << 22;

__device__ unsigned int g_mlp_error;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (K-major, no swizzle): start address, leading
// byte offset (between the two core matrices of one K = 16 step), stride byte
// offset (between 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  return d;  // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Bounded wait for the phase with the given parity; false when the limit (polls of the
// barrier) ran out.  The waits that drain a kernel's own copies and MMAs before it
// releases tensor memory keep the fixed limit; the waits of the work itself take the
// launch's polls (rgeo_tuning.wait_limit), which a test may set to give up at once.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit = kSpinLimit) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Copy rows [row0, row0 + rows) x K columns [k0, k0 + 64) of a row-major bf16
// matrix (leading dimension ld elements) into the canonical layout: core matrix
// (row group g, K chunk c) of 8 rows x 8 elements at byte offset (g * 8 + c) * 128;
// within it, row r at r * 16.  Hence LBO = 128 (next K chunk), SBO = 1024 (next
// row group).  Rows at or beyond nrows are filled with zeros.
__device__ __forceinline__ void stage_tile(uint8_t *dst, const __nv_bfloat16 *src, int ld, int row0, int rows,
                                           int nrows, int k0) {
  const int chunks = rows * (kTileK / 8);  // 16-byte chunks
  for (int q = threadIdx.x; q < chunks; q += blockDim.x) {
    const int r = q >> 3, c = q & 7;
    uint8_t *d = dst + ((r >> 3) * 8 + c) * 128 + (r & 7) * 16;
    if (row0 + r < nrows) {
      cp_async16(d, src + (size_t)(row0 + r) * ld + k0 + c * 8);
    } else {
      *reinterpret_cast<uint4 *>(d) = make_uint4(0u, 0u, 0u, 0u);
    }
  }
}

// C[M x N] = A[M x K] B[N x K]^T (+ bias), with an epilogue:
//   mode 0: C fp32 row-major (ldc), plus bias
//   mode 1: relu(C + bias) as bf16 row-major (ldc) and, when ct != null, its transpose
//           (N x M, leading dimension ldt) as bf16
//   mode 2: atomicAdd of C into fp32 row-major (split-K: blockIdx.y picks a K range)
// Requirements (checked by the launcher): K % 64 == 0, N % 16 == 0, 16 <= N <= 256.
__global__ void __launch_bounds__(128) k_gemm_bf16(const __nv_bfloat16 *__restrict__ A,
                                                   const __nv_bfloat16 *__restrict__ B, int M, int N, int K,
                                                   int k_per_split, const float *__restrict__ bias, int mode,
                                                   void *C, int ldc, __nv_bfloat16 *ct, int ldt, long long polls) {
  extern __shared__ __align__(1024) uint8_t gsm[];
  uint8_t *sA[2] = {gsm, gsm + kTileM * kTileK * 2};
  uint8_t *sB[2] = {gsm + 2 * kTileM * kTileK * 2, gsm + 2 * kTileM * kTileK * 2 + kMaxTileN * kTileK * 2};
  __shared__ uint64_t bar_stage[2];
  __shared__ uint64_t bar_done;
  __shared__ uint32_t tmem_base_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5;
  const int m0 = blockIdx.x * kTileM;
  const int kbeg = blockIdx.y * k_per_split;
  const int kend = min(K, kbeg + k_per_split);
  const int nstages = (kend - kbeg) / kTileK;
  const int ncols = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));

  if (threadIdx.x == 0) {
    mbar_init(&bar_stage[0], 1);
    mbar_init(&bar_stage[1], 1);
    mbar_init(&bar_done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_slot;
  const uint32_t idesc = idesc_bf16(kTileM, N);

  // prologue: stage 0
  if (nstages > 0) {
    stage_tile(sA[0], A, K, m0, kTileM, M, kbeg);
    stage_tile(sB[0], B, K, 0, N, N, kbeg);
    cp_async_commit();
  }
  uint32_t phase[2] = {0u, 0u};
  for (int s = 0; s < nstages; ++s) {
    const int buf = s & 1;
    cp_async_wait_all();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // make the staged data visible to the tensor core
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA[buf]), b0 = smem_u32(sB[buf]);
      for (int kk = 0; kk < kTileK / 16; ++kk) {
        const uint64_t ad = smem_desc(a0 + kk * 256, 128, 1024);
        const uint64_t bd = smem_desc(b0 + kk * 256, 128, 1024);
        const uint32_t acc = (s > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bar_stage[buf]))
                   : "memory");
    }
    // stage s + 1 into the other buffer once the MMAs that read it (stage s - 1) are done
    if (s + 1 < nstages) {
      const int nb = buf ^ 1;
      if (s >= 1) {
        if (!mbar_wait(&bar_stage[nb], phase[nb], polls)) abort_flag = 1;
        phase[nb] ^= 1u;
      }
      __syncthreads();
      if (abort_flag) break;
      stage_tile(sA[nb], A, K, m0, kTileM, M, kbeg + (s + 1) * kTileK);
      stage_tile(sB[nb], B, K, 0, N, N, kbeg + (s + 1) * kTileK);
      cp_async_commit();
    }
  }
  cp_async_wait_all();
  // All MMAs issued (also after an abort): one more commit tracks every one of them,
  // so the tensor memory is released only once none is in flight.
  if (threadIdx.x == 0 && nstages > 0) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&bar_done))
                 : "memory");
  }
  __syncthreads();
  bool ok = !abort_flag;
  if (nstages > 0 && !mbar_wait(&bar_done, 0u)) ok = false;
  if (!ok) atomicOr(&g_mlp_error, kErrTimeout);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // epilogue: warp w owns rows 32 w .. 32 w + 31 (TMEM lanes); 32 columns per load
  const int row = m0 + warp * 32 + (threadIdx.x & 31);
  if (ok && nstages > 0) {
    for (int c0 = 0; c0 < N; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
            "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
            "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
        const int nn = min(32, N - c0);
        if (mode == 0) {
          float *crow = reinterpret_cast<float *>(C) + (size_t)row * ldc + c0;
          for (int j = 0; j < nn; ++j) crow[j] = __uint_as_float(v[j]) + (bias ? bias[c0 + j] : 0.f);
        } else if (mode == 1) {
          __nv_bfloat16 *crow = reinterpret_cast<__nv_bfloat16 *>(C) + (size_t)row * ldc + c0;
          for (int j = 0; j < nn; ++j) {
            const float y = fmaxf(__uint_as_float(v[j]) + (bias ? bias[c0 + j] : 0.f), 0.f);
            const __nv_bfloat16 yb = __float2bfloat16_rn(y);
            crow[j] = yb;
            if (ct) ct[(size_t)(c0 + j) * ldt + row] = yb;
          }
        } else {
          float *crow = reinterpret_cast<float *>(C) + (size_t)row * ldc + c0;
          for (int j = 0; j < nn; ++j) atomicAdd(crow + j, __uint_as_float(v[j]));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}


// ------------------------------------------------------------------ the MLP
// Parameters (FP32 master copy, flat): W1 [256 x 7], b1 [256], W2 [256 x 256], b2,
// W3 [256 x 256], b3, W4 [7 x 256], b4 [7]; every W is row-major out x in.
constexpr int kIn = 7, kOut = 7, kWid = 256;
constexpr int oW1 = 0, ob1 = oW1 + kWid * kIn, oW2 = ob1 + kWid, ob2 = oW2 + kWid * kWid, oW3 = ob2 + kWid,
              ob3 = oW3 + kWid * kWid, oW4 = ob3 + kWid, ob4 = oW4 + kOut * kWid, kParams = ob4 + kOut;

// Layer 1 in FP32 (K = 7 is too small for the tensor cores): H1 = relu(X W1^T + b1),
// written as bf16 rows and (when H1t is set) as the transposed bf16 copy used by the
// weight gradient.
__global__ void k_layer_in(const float *__restrict__ X, int B, const float *__restrict__ P,
                           __nv_bfloat16 *H1, __nv_bfloat16 *H1t) {
  const int b = blockIdx.x;
  const int j = threadIdx.x;  // 256 threads: one output unit each
  __shared__ float xs[kIn];
  if (j < kIn) xs[j] = X[(size_t)b * kIn + j];
  __syncthreads();
  float z = P[ob1 + j];
  for (int k = 0; k < kIn; ++k) z = fmaf(P[oW1 + j * kIn + k], xs[k], z);
  const __nv_bfloat16 h = __float2bfloat16_rn(fmaxf(z, 0.f));
  H1[(size_t)b * kWid + j] = h;
  if (H1t) H1t[(size_t)j * B + b] = h;
}

// Layer 4 in FP32 (N = 7): Y = H3 W4^T + b4.  One warp per row.
__global__ void k_layer_out(const __nv_bfloat16 *__restrict__ H3, int B, const float *__restrict__ P, float *Y) {
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= B) return;
  float acc[kOut];
  for (int o = 0; o < kOut; ++o) acc[o] = 0.f;
  for (int k = lane; k < kWid; k += 32) {
    const float h = __bfloat162float(H3[(size_t)b * kWid + k]);
    for (int o = 0; o < kOut; ++o) acc[o] = fmaf(P[oW4 + o * kWid + k], h, acc[o]);
  }
  for (int o = 0; o < kOut; ++o)
    for (int off = 16; off > 0; off >>= 1) acc[o] += __shfl_down_sync(0xffffffffu, acc[o], off);
  if (lane == 0)
    for (int o = 0; o < kOut; ++o) Y[(size_t)b * kOut + o] = acc[o] + P[ob4 + o];
}

// Loss and its gradient.  Outputs 0..5 regress the scaled residuals T (mean squared
// error); output 6 regresses e = log(sum_i (Y_i - T_i)^2 + 1e-6), the log squared
// error of the same sample (a target that is not differentiated), weighted by lam.
__global__ void k_loss_grad(const float *__restrict__ Y, const float *__restrict__ T, int B, float lam, float *dY,
                            float *loss) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (b < B) {
    float se = 0.f;
    for (int o = 0; o < 6; ++o) {
      const float d = Y[(size_t)b * kOut + o] - T[(size_t)b * 6 + o];
      se = fmaf(d, d, se);
      dY[(size_t)b * kOut + o] = 2.f * d / (6.f * B);
    }
    const float e = logf(se + 1e-6f);
    const float d6 = Y[(size_t)b * kOut + 6] - e;
    dY[(size_t)b * kOut + 6] = 2.f * lam * d6 / B;
    l = se / (6.f * B) + lam * d6 * d6 / B;
  }
  for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l);
}

// Gradient of layer 4 and the error into layer 3:
//   dW4[o, k] += sum_b dY[b, o] H3[b, k], db4[o] += sum_b dY[b, o]  (atomics per block)
//   dZ3[b, k] = (sum_o dY[b, o] W4[o, k]) [H3[b, k] > 0], as bf16 rows and transposed.
__global__ void k_back_out(const float *__restrict__ dY, const __nv_bfloat16 *__restrict__ H3, int B,
                           const float *__restrict__ P, float *G, __nv_bfloat16 *dZ3, __nv_bfloat16 *dZ3t) {
  const int k = threadIdx.x;  // 256 threads: one hidden unit each
  const int b0 = blockIdx.x * 32, b1 = min(B, b0 + 32);
  float gw[kOut];
  for (int o = 0; o < kOut; ++o) gw[o] = 0.f;
  float w4[kOut];
  for (int o = 0; o < kOut; ++o) w4[o] = P[oW4 + o * kWid + k];
  for (int b = b0; b < b1; ++b) {
    const float h = __bfloat162float(H3[(size_t)b * kWid + k]);
    float dh = 0.f;
    for (int o = 0; o < kOut; ++o) {
      const float dy = dY[(size_t)b * kOut + o];
      gw[o] = fmaf(dy, h, gw[o]);
      dh = fmaf(dy, w4[o], dh);
    }
    const __nv_bfloat16 dz = __float2bfloat16_rn(h > 0.f ? dh : 0.f);
    dZ3[(size_t)b * kWid + k] = dz;
    dZ3t[(size_t)k * B + b] = dz;
  }
  for (int o = 0; o < kOut; ++o) atomicAdd(&G[oW4 + o * kWid + k], gw[o]);
  if (k < kOut) {
    float s = 0.f;
    for (int b = b0; b < b1; ++b) s += dY[(size_t)b * kOut + k];
    atomicAdd(&G[ob4 + k], s);
  }
}

// dZ = dH [H > 0] for a hidden layer: bf16 rows + transposed copy (layers 2, 3), or
// FP32 rows (layer 1).  Also the bias gradient db[k] += sum_b dZ[b, k].
__global__ void k_relu_back(const float *__restrict__ dH, const __nv_bfloat16 *__restrict__ H, int B, float *db,
                            __nv_bfloat16 *dZ, __nv_bfloat16 *dZt, float *dZf) {
  const int k = threadIdx.x;
  const int b0 = blockIdx.x * 32, b1 = min(B, b0 + 32);
  float s = 0.f;
  for (int b = b0; b < b1; ++b) {
    const float g = __bfloat162float(H[(size_t)b * kWid + k]) > 0.f ? dH[(size_t)b * kWid + k] : 0.f;
    s += g;
    if (dZ) {
      const __nv_bfloat16 gb = __float2bfloat16_rn(g);
      dZ[(size_t)b * kWid + k] = gb;
      dZt[(size_t)k * B + b] = gb;
    }
    if (dZf) dZf[(size_t)b * kWid + k] = g;
  }
  atomicAdd(&db[k], s);
}

// Bias gradient of a layer whose dZ exists only in bf16 (layer 3): db[k] += sum_b dZ[b, k].
__global__ void k_bias_back(const __nv_bfloat16 *__restrict__ dZ, int B, float *db) {
  const int k = threadIdx.x;
  const int b0 = blockIdx.x * 32, b1 = min(B, b0 + 32);
  float s = 0.f;
  for (int b = b0; b < b1; ++b) s += __bfloat162float(dZ[(size_t)b * kWid + k]);
  atomicAdd(&db[k], s);
}

// Layer-1 weight gradient: dW1[j, i] += sum_b dZ1[b, j] X[b, i].
__global__ void k_back_in(const float *__restrict__ dZ1, const float *__restrict__ X, int B, float *G) {
  const int j = threadIdx.x;
  const int b0 = blockIdx.x * 32, b1 = min(B, b0 + 32);
  float g[kIn];
  for (int i = 0; i < kIn; ++i) g[i] = 0.f;
  for (int b = b0; b < b1; ++b) {
    const float dz = dZ1[(size_t)b * kWid + j];
    for (int i = 0; i < kIn; ++i) g[i] = fmaf(dz, X[(size_t)b * kIn + i], g[i]);
  }
  for (int i = 0; i < kIn; ++i) atomicAdd(&G[oW1 + j * kIn + i], g[i]);
}

// Adam (Kingma and Ba 2015) on the FP32 master parameters; then the bf16 copies of
// W2 and W3 (row-major, and transposed for the backward products).
__global__ void k_adam(float *P, const float *G, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_refresh_bf16(const float *P, __nv_bfloat16 *W2b, __nv_bfloat16 *W3b, __nv_bfloat16 *W2t,
                               __nv_bfloat16 *W3t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kWid * kWid) return;
  const int r = i / kWid, c = i % kWid;
  const __nv_bfloat16 a = __float2bfloat16_rn(P[oW2 + i]), b = __float2bfloat16_rn(P[oW3 + i]);
  W2b[i] = a;
  W3b[i] = b;
  W2t[c * kWid + r] = a;
  W3t[c * kWid + r] = b;
}

// Counter-based uniform in [0, 1) from (seed, i): SplitMix64 (Steele, Lea, Flood 2014) output of
// the state seed + (i + 1) * golden, top 24 bits.
__device__ __forceinline__ float u01(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)(z >> 40) * (1.f / 16777216.f);
}

// Batch sampling for training: row i of the batch takes segment floor(u n) of the training
// set, u from the counter-based generator at (seed, step * batch + i).
__global__ void k_gather_batch(const float *__restrict__ X, const float *__restrict__ T, long long n, int B,
                               unsigned long long seed, long long step, float *Xb, float *Tb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const float u = u01(seed, (unsigned long long)(step * B + i));
  long long j = (long long)(u * (float)n);
  if (j >= n) j = n - 1;
  for (int c = 0; c < kIn; ++c) Xb[(size_t)i * kIn + c] = X[(size_t)j * kIn + c];
  for (int c = 0; c < 6; ++c) Tb[(size_t)i * 6 + c] = T[(size_t)j * 6 + c];
}

// He-uniform initialisation of the weights, zero biases.
__global__ void k_init(float *P, unsigned long long seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kParams) return;
  float fan = 0.f;
  if (i < ob1) fan = kIn;
  else if (i >= oW2 && i < ob2) fan = kWid;
  else if (i >= oW3 && i < ob3) fan = kWid;
  else if (i >= oW4 && i < ob4) fan = kWid;
  P[i] = fan > 0.f ? (2.f * u01(seed, i) - 1.f) * sqrtf(6.f / fan) : 0.f;
}


// ------------------------------------ persistent, warp-specialised fused inference
// All four layers on the tensor core; the CUDA cores only build the layer-1 operand and
// run the epilogues (ReLU, BF16 rounding, the final sum).  One CTA per SM walks the tiles
// blockIdx.x + i * gridDim.x; tile i uses slot s = i % 2 (shared-memory operand H[s],
// TMEM accumulator s, columns 256 s .. 256 s + 255), so two tiles are in flight.
//
// Layers 1 and 4 take FP32 operands.  To keep their products at FP32 accuracy on the BF16
// tensor core, each FP32 value a is split into a_hi = bf16(a) and a_lo = bf16(a - a_hi)
// (16 significant bits together), and every cross term is kept:
//   layer 1 (K = 32): A row = [x_hi 1 | x_hi 1 | x_lo 0 | x_lo 0],
//                     B row = [w_hi b_hi | w_lo b_lo | w_hi 0 | w_lo 0]  (b1 folded in);
//   layer 4 (N = 16): columns 0..6 take W4_hi, columns 8..14 take W4_lo, and the epilogue
//                     adds the two halves and b4.  Its A operand is H3 rounded to BF16, as
//                     in the training forward.
// Layers 2 and 3 are the BF16 products of the training forward; their biases enter as one
// more K = 16 step: the activations carry a constant block [1 1 0 ... 0] after their 256
// columns, and the matching "bias chunk" of B holds [b_hi b_lo 0 ... 0].  Every epilogue is
// then ReLU and BF16 rounding only.
//
// Roles:
//   warp 0 (producer): lane 0 bulk-copies the resident layer-1 and layer-4 operands once,
//     then streams the 16 KB K-chunks of W2 and W3 into a ring of kWsRing slots, one pass
//     over both per pair of tiles;
//   warp 1 (MMA): lane 0 takes the tiles in pairs (2 j in slot 0, 2 j + 1 in slot 1):
//     layer 1 of each, then layers 2 and 3 chunk by chunk with each chunk's MMAs issued for
//     both tiles before the chunk is released, then layer 4 of each; it commits every
//     finished layer to acc_full[s];
//   warps 2..9 and 10..17 (worker groups 0 and 1): group g owns slot g (tiles g, g + 2, ...):
//     it writes the layer-1 operand from X, then after each of the first three layers reads
//     the accumulator, adds the bias, applies ReLU and writes the next layer's BF16 operand
//     into H[g]; after layer 4 it writes Y.
// Sharing each chunk between the two tiles halves the weight traffic from L2, which bounds
// the rate at which the ring can be refilled.
constexpr int kChunkK = 32;                       // K columns per streamed weight chunk
constexpr int kWChunkBytes = kWid * kChunkK * 2;  // 16 KB
constexpr int kWsGroupThreads = 256;
constexpr int kWsThreads = 64 + 2 * kWsGroupThreads;
constexpr int kWsRing = 4;
constexpr int kK1 = 32;                              // layer-1 K (split inputs and bias)
constexpr int kN4 = 16;                              // layer-4 N (split W4)
constexpr int kB1Bytes = kWid * kK1 * 2;             // 16 KB
constexpr int kB4Bytes = kN4 * kWid * 2;             // 8 KB
constexpr int kBiasChunkBytes = kWid * 16 * 2;       // 8 KB: the bias step of layers 2 and 3
constexpr int kPackedElems = 2 * kWid * kWid + (kB1Bytes + kB4Bytes + 2 * kBiasChunkBytes) / 2;
// activations of one tile: 16 row groups of 34 core matrices (256 columns + the bias block)
constexpr int kHGroupBytes = (kWid / 8 + 2) * 128;  // 4352
constexpr int kHsBytes = (kTileM / 8) * kHGroupBytes;  // 68 KB
// shared memory: H[2] | weight ring | B1 | B4 | b4 (8)
constexpr int kWsSmem = 2 * kHsBytes + kWsRing * kWChunkBytes + kB1Bytes + kB4Bytes + 8 * 4;
constexpr long long kWsSpin = 1ll << 21;
static_assert(kWsSmem <= 227 * 1024, "shared memory of the persistent inference kernel");

__device__ __forceinline__ void split_bf16(float a, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
  hi = __float2bfloat16_rn(a);
  lo = __float2bfloat16_rn(a - __bfloat162float(hi));
}

// Wp = [W2 chunks 0..7 | W3 chunks 0..7 | B1 | B4 | bias chunk of W2 | bias chunk of W3], every
// piece in the canonical K-major layout its MMAs read (8-row x 16-byte core matrices):
//   chunk c of W2 / W3 (K columns 32 c .. 32 c + 31): core (n / 8, k / 8) at (4 (n / 8) + k / 8) * 128;
//   B1 (256 x 32): the same layout as a chunk;
//   B4 (16 x 256): core (n / 8, k / 8) at (32 (n / 8) + k / 8) * 128;
//   bias chunk (256 x 16, row n = [b_hi b_lo 0 ... 0]): core (n / 8, k / 8) at (2 (n / 8) + k / 8) * 128.
__global__ void k_pack_chunks(const float *__restrict__ P, const __nv_bfloat16 *__restrict__ W2b,
                              const __nv_bfloat16 *__restrict__ W3b, __nv_bfloat16 *__restrict__ Wp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 2 * kWid * kWid) {
    const int l = i / (kWid * kWid), r = i % (kWid * kWid);
    const int nn = r / kWid, k = r % kWid, c = k / kChunkK, kk = k % kChunkK;
    const int byte = ((nn >> 3) * 4 + (kk >> 3)) * 128 + (nn & 7) * 16 + (kk & 7) * 2;
    Wp[(size_t)(l * 8 + c) * (kWChunkBytes / 2) + byte / 2] = (l == 0 ? W2b : W3b)[r];
  } else if (i < 2 * kWid * kWid + kWid * kK1) {
    const int r = i - 2 * kWid * kWid, nn = r / kK1, k = r % kK1, blk = k >> 3, kk = k & 7;
    // blocks: 0 [w_hi b_hi], 1 [w_lo b_lo], 2 [w_hi 0], 3 [w_lo 0]
    const float a = kk < kIn ? P[oW1 + nn * kIn + kk] : (blk < 2 ? P[ob1 + nn] : 0.f);
    __nv_bfloat16 hi, lo;
    split_bf16(a, hi, lo);
    const int byte = ((nn >> 3) * 4 + blk) * 128 + (nn & 7) * 16 + kk * 2;
    Wp[(size_t)2 * kWid * kWid + byte / 2] = (blk & 1) ? lo : hi;
  } else if (i < 2 * kWid * kWid + kWid * kK1 + kN4 * kWid) {
    const int r = i - 2 * kWid * kWid - kWid * kK1, nn = r / kWid, k = r % kWid, o = nn & 7;
    __nv_bfloat16 hi, lo;
    split_bf16(o < kOut ? P[oW4 + o * kWid + k] : 0.f, hi, lo);
    const int byte = ((nn >> 3) * 32 + (k >> 3)) * 128 + (nn & 7) * 16 + (k & 7) * 2;
    Wp[(size_t)2 * kWid * kWid + kWid * kK1 + byte / 2] = nn < 8 ? hi : lo;
  } else if (i < kPackedElems) {
    const int r = i - 2 * kWid * kWid - kWid * kK1 - kN4 * kWid, l = r / (kWid * 16), nn = (r / 16) % kWid,
              k = r % 16;
    __nv_bfloat16 hi, lo;
    split_bf16(P[(l == 0 ? ob2 : ob3) + nn], hi, lo);
    const __nv_bfloat16 v = k == 0 ? hi : (k == 1 ? lo : __float2bfloat16_rn(0.f));
    const int byte = ((nn >> 3) * 2 + (k >> 3)) * 128 + (nn & 7) * 16 + (k & 7) * 2;
    Wp[(size_t)2 * kWid * kWid + kWid * kK1 + kN4 * kWid + (size_t)l * (kBiasChunkBytes / 2) + byte / 2] = v;
  }
}

// max(a, 0), max(b, 0) rounded to BF16 and packed (a in the low half), in one conversion
__device__ __forceinline__ uint32_t pack_bf16_relu(float a, float b) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
  return d;
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t acc, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
        "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
        "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// Bounded wait that also gives up once another role has raised the abort flag; a wait
// that runs out raises it.
__device__ __forceinline__ bool ws_wait(uint64_t *bar, uint32_t parity, volatile int *abort, long long limit) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 255 && *abort) return false;
  }
  *abort = 1;
  return false;
}
// OR of pred over the 256 threads of named barrier id (1 or 2).
__device__ __forceinline__ bool group_any(int id, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred q, p;\n setp.ne.u32 q, %2, 0;\n bar.red.or.pred p, %1, %3, q;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"(id), "r"((uint32_t)pred), "n"(kWsGroupThreads)
      : "memory");
  return r != 0;
}

__global__ void __launch_bounds__(kWsThreads, 1)
    k_mlp_infer_ws(const float *__restrict__ X, long long n, const float *__restrict__ P,
                   const __nv_bfloat16 *__restrict__ Wp, float *__restrict__ Y, long long polls) {
  extern __shared__ __align__(1024) uint8_t wsm[];
  uint8_t *ring = wsm + 2 * kHsBytes;
  uint8_t *B1 = ring + kWsRing * kWChunkBytes;
  uint8_t *B4 = B1 + kB1Bytes;
  float *b4s = reinterpret_cast<float *>(B4 + kB4Bytes);  // [8]
  __shared__ uint64_t chunk_full[kWsRing], chunk_empty[kWsRing], h_full[2], acc_full[2], const_full, drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  volatile int *abortp = &abort_flag;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const long long ntiles = (n + kTileM - 1) / kTileM;
  const long long T = ntiles > (long long)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long npairs = (T + 1) / 2;

  if (t == 0) {
    for (int r = 0; r < kWsRing; ++r) {
      mbar_init(&chunk_full[r], 1);
      mbar_init(&chunk_empty[r], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&h_full[s], kWsGroupThreads / 32);  // one arrival per worker warp
      mbar_init(&acc_full[s], 1);
    }
    mbar_init(&const_full, 1);
    mbar_init(&drain, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(2 * kWid)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // the constant bias block of both slots' activations: core matrices 32 ([1 1 0 ... 0]) and 33 (0)
  for (int i = t; i < 2 * kTileM; i += blockDim.x) {
    const int s = i / kTileM, r = i % kTileM;
    uint8_t *q = wsm + s * kHsBytes + (r >> 3) * kHGroupBytes + (kWid / 8) * 128 + (r & 7) * 16;
    *reinterpret_cast<uint4 *>(q) = make_uint4(0x3F803F80u, 0u, 0u, 0u);  // BF16 1.0, 1.0
    *reinterpret_cast<uint4 *>(q + 128) = make_uint4(0u, 0u, 0u, 0u);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (t < 8) b4s[t] = t < kOut ? P[ob4 + t] : 0.f;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ---- producer
    if (lane == 0) {
      mbar_expect_tx(&const_full, kB1Bytes + kB4Bytes);
      bulk_copy(B1, Wp + 2 * kWid * kWid, kB1Bytes, &const_full);
      bulk_copy(B4, Wp + 2 * kWid * kWid + kB1Bytes / 2, kB4Bytes, &const_full);
    }
    long long chunk = 0;
    bool ok = true;
    // one pass over W2 and W3 per pair of tiles: each chunk serves both tiles
    for (long long j = 0; j < npairs && ok; ++j) {
      for (int l = 0; l < 2 && ok; ++l) {
        for (int c = 0; c <= kWid / kChunkK && ok; ++c, ++chunk) {  // 8 chunks, then the bias chunk
          const int r = (int)(chunk % kWsRing);
          if (lane == 0) {
            if (chunk >= kWsRing) ok = ws_wait(&chunk_empty[r], (uint32_t)((chunk / kWsRing - 1) & 1), abortp, polls);
            if (ok) {
              const bool bias = c == kWid / kChunkK;
              const uint32_t bytes = bias ? kBiasChunkBytes : kWChunkBytes;
              const __nv_bfloat16 *src =
                  bias ? Wp + 2 * kWid * kWid + (kB1Bytes + kB4Bytes) / 2 + (size_t)l * (kBiasChunkBytes / 2)
                       : Wp + (size_t)(l * 8 + c) * (kWChunkBytes / 2);
              mbar_expect_tx(&chunk_full[r], bytes);
              bulk_copy(ring + r * kWChunkBytes, src, bytes, &chunk_full[r]);
            }
          }
          ok = __shfl_sync(0xffffffffu, ok, 0);
          if (!ok) --chunk;  // this chunk was not issued
        }
      }
    }
    // every copy issued has landed before the CTA may leave (immediate when all were consumed)
    if (lane == 0) {
      mbar_wait(&const_full, 0u);
      for (long long c = chunk - 1; c >= 0 && c >= chunk - kWsRing; --c)
        mbar_wait(&chunk_full[c % kWsRing], (uint32_t)((c / kWsRing) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer.  Per pair of tiles (a = 2 j in slot 0, b = 2 j + 1 in slot 1):
    // L1(a), L1(b); L2 and L3 chunk by chunk, each chunk's MMAs for a then b; L4(a), L4(b).
    const uint32_t idesc_n256 = idesc_bf16(kTileM, kWid), idesc_n16 = idesc_bf16(kTileM, kN4);
    // descriptors of the operand bases; an offset of o bytes adds o / 16 to the address field
    const uint64_t dH[2] = {smem_desc(smem_u32(wsm), 128, kHGroupBytes),
                            smem_desc(smem_u32(wsm + kHsBytes), 128, kHGroupBytes)};
    const uint64_t dRingBias = smem_desc(smem_u32(ring), 128, 256);  // bias chunk: 2 core matrices per row group
    const uint64_t dRing = smem_desc(smem_u32(ring), 128, 512);
    const uint64_t dB1 = smem_desc(smem_u32(B1), 128, 512), dB4 = smem_desc(smem_u32(B4), 128, 4096);
    long long chunk = 0;
    uint32_t hwait[2] = {0u, 0u};  // completions of h_full[s] waited for
    bool ok = true;
    if (lane == 0) ok = ws_wait(&const_full, 0u, abortp, polls);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    for (long long j = 0; j < npairs && ok; ++j) {
      const int ns = 2 * j + 1 < T ? 2 : 1;
      if (lane == 0) {
        auto wait_operand = [&](int s) {
          ok = ok && ws_wait(&h_full[s], hwait[s] & 1u, abortp, polls);
          ++hwait[s];
        };
        for (int s = 0; s < ns; ++s) {  // layer 1: K = 32 (split inputs, folded bias)
          wait_operand(s);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t acc = tmem + (uint32_t)(s * kWid);
          mma_bf16(acc, dH[s], dB1, idesc_n256, 0u);
          mma_bf16(acc, dH[s] + 16, dB1 + 16, idesc_n256, 1u);
          mma_commit(&acc_full[s]);
        }
        for (int l = 0; l < 2 && ok; ++l) {  // layers 2 and 3: 8 chunks of K = 32
          for (int s = 0; s < ns; ++s) wait_operand(s);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          for (int c = 0; c <= kWid / kChunkK; ++c, ++chunk) {
            const int r = (int)(chunk % kWsRing);
            ok = ws_wait(&chunk_full[r], (uint32_t)((chunk / kWsRing) & 1), abortp, polls);
            if (!ok) break;
            if (c < kWid / kChunkK) {
              const uint64_t dB = dRing + (uint64_t)(r * (kWChunkBytes >> 4));
              for (int s = 0; s < ns; ++s) {
                const uint32_t acc = tmem + (uint32_t)(s * kWid);
                const uint64_t dA = dH[s] + (uint64_t)(c * 32);
                mma_bf16(acc, dA, dB, idesc_n256, c > 0 ? 1u : 0u);
                mma_bf16(acc, dA + 16, dB + 16, idesc_n256, 1u);
              }
            } else {  // the bias step: K columns 256..271 of the activations
              const uint64_t dB = dRingBias + (uint64_t)(r * (kWChunkBytes >> 4));
              for (int s = 0; s < ns; ++s) {
                mma_bf16(tmem + (uint32_t)(s * kWid), dH[s] + (uint64_t)((kWid / 8) * 8), dB, idesc_n256, 1u);
                mma_commit(&acc_full[s]);
              }
            }
            mma_commit(&chunk_empty[r]);
          }
        }
        for (int s = 0; s < ns && ok; ++s) {  // layer 4: N = 16 (split W4)
          wait_operand(s);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t acc = tmem + (uint32_t)(s * kWid);
#pragma unroll
          for (int k = 0; k < kWid / 16; ++k)
            mma_bf16(acc, dH[s] + (uint64_t)(k * 16), dB4 + (uint64_t)(k * 16), idesc_n16, k > 0 ? 1u : 0u);
          mma_commit(&acc_full[s]);
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
    }
    // all MMAs issued have completed before the tensor memory is released
    if (lane == 0) {
      mma_commit(&drain);
      if (!mbar_wait(&drain, 0u)) *abortp = 1;
    }
    __syncwarp();
  } else {
    // ---- worker group g: 256 threads, slot g, tiles g, g + 2, ...
    const int g = (warp - 2) >> 3, bar_id = 1 + g;
    const int wt = t - 64 - g * kWsGroupThreads;
    const int wq = warp & 3, half = ((warp - 2) >> 2) & 1, row = wq * 32 + lane;
    uint8_t *sH = wsm + g * kHsBytes;
    const uint32_t acc = tmem + (uint32_t)(g * kWid) + ((uint32_t)(wq * 32) << 16);
    uint32_t await_n = 0u;
    bool bad = false;
    // This thread's part of H[g] is written (and its accumulator reads are done): make the
    // writes visible to the tensor core, then one arrival per warp.
    auto operand_ready = [&]() {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&h_full[g]);
    };
    // X rows of tile i into L2 ahead of use (one 128-byte line per thread)
    auto prefetch_x = [&](long long i) {
      const long long row0 = ((long long)blockIdx.x + i * gridDim.x) * kTileM;
      const long long b0 = row0 * kIn * 4, b1 = (row0 + kTileM < n ? row0 + kTileM : n) * kIn * 4;
      const long long b = (b0 & ~127ll) + (long long)wt * 128;
      if (wt < (kTileM * kIn * 4) / 128 + 1 && b < b1)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char *>(X) + b));
    };
    // the layer-1 operand of tile i: thread wt writes K blocks 2 (wt / 128) and 2 (wt / 128) + 1
    // of row wt % 128 (blocks 0, 1: [x_hi 1]; blocks 2, 3: [x_lo 0])
    auto operand1 = [&](long long i) {
      const long long row0 = ((long long)blockIdx.x + i * gridDim.x) * kTileM;
      const int r = wt & (kTileM - 1), hh = wt >> 7;
      const long long gr = row0 + r;
      uint32_t w[4];
      float xv[8];
      for (int k = 0; k < kIn; ++k) xv[k] = gr < n ? __ldg(X + gr * kIn + k) : 0.f;
      xv[7] = hh == 0 ? 1.f : 0.f;
      for (int k = 0; k < 8; k += 2) {
        __nv_bfloat16 h0, l0, h1, l1;
        split_bf16(xv[k], h0, l0);
        split_bf16(xv[k + 1], h1, l1);
        const __nv_bfloat162 p = hh == 0 ? __halves2bfloat162(h0, h1) : __halves2bfloat162(l0, l1);
        w[k >> 1] = *reinterpret_cast<const uint32_t *>(&p);
      }
      const uint4 q = make_uint4(w[0], w[1], w[2], w[3]);
      uint8_t *base = sH + (r >> 3) * kHGroupBytes + (r & 7) * 16 + hh * 256;
      *reinterpret_cast<uint4 *>(base) = q;
      *reinterpret_cast<uint4 *>(base + 128) = q;
      operand_ready();
    };
    if (g < T) {
      prefetch_x(g);
      operand1(g);
    }
    for (long long i = g; i < T; i += 2) {
      const long long row0 = ((long long)blockIdx.x + i * gridDim.x) * kTileM;
      if (i + 2 < T) prefetch_x(i + 2);
      for (int layer = 0; layer < 4 && !bad; ++layer) {
        if (!ws_wait(&acc_full[g], await_n & 1u, abortp, polls)) {
          bad = true;
          break;
        }
        ++await_n;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (layer < 3) {
          // ReLU and BF16 (the bias is in the accumulator) into the next layer's operand; this
          // half's 128 columns, two 32-column loads in flight
#pragma unroll 1
          for (int k2 = 0; k2 < 2; ++k2) {
            uint32_t v[2][32];
            tmem_ld32_nowait(acc + (uint32_t)(half * 128 + k2 * 64), v[0]);
            tmem_ld32_nowait(acc + (uint32_t)(half * 128 + k2 * 64 + 32), v[1]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int c0 = half * 128 + k2 * 64 + u * 32;
              uint8_t *dst = sH + (row >> 3) * kHGroupBytes + (c0 >> 3) * 128 + (row & 7) * 16;
#pragma unroll
              for (int q = 0; q < 4; ++q)
                *reinterpret_cast<uint4 *>(dst + q * 128) =
                    make_uint4(pack_bf16_relu(__uint_as_float(v[u][8 * q]), __uint_as_float(v[u][8 * q + 1])),
                               pack_bf16_relu(__uint_as_float(v[u][8 * q + 2]), __uint_as_float(v[u][8 * q + 3])),
                               pack_bf16_relu(__uint_as_float(v[u][8 * q + 4]), __uint_as_float(v[u][8 * q + 5])),
                               pack_bf16_relu(__uint_as_float(v[u][8 * q + 6]), __uint_as_float(v[u][8 * q + 7])));
            }
          }
          operand_ready();
        } else if (half == 0) {
          // layer 4: hi + lo columns, plus b4
          uint32_t v[16];
          tmem_ld16(acc, v);
          if (row0 + row < n) {
            float *yr = Y + (row0 + row) * kOut;
#pragma unroll
            for (int o = 0; o < kOut; ++o) yr[o] = (__uint_as_float(v[o]) + __uint_as_float(v[8 + o])) + b4s[o];
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      // every thread of the group takes the same branch from here on
      if (group_any(bar_id, bad)) {
        bad = true;
        break;
      }
      if (i + 2 < T) operand1(i + 2);
    }
    if (bad) *abortp = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (t == 0 && *abortp) atomicOr(&g_mlp_error, kErrTimeout);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kWid) : "memory");
}
}  // namespace

// Polls of the work's own barrier waits for a launch: the kernel's default, or the
// process-wide tuning (rgeo_tuning.wait_limit: n > 0 polls, -1 none).
long long wait_polls(long long dflt) {
  const int w = tuning().wait_limit;
  return w == 0 ? dflt : (w < 0 ? 0ll : (long long)w);
}

cudaError_t launch_gemm_bf16(const void *A, const void *B, int M, int N, int K, int splits, const float *bias,
                             int mode, void *C, int ldc, void *ct, int ldt, cudaStream_t st) {
  if (M <= 0 || N < 16 || N > kMaxTileN || N % 16 != 0 || K <= 0 || K % kTileK != 0 || splits < 1)
    return cudaErrorInvalidValue;
  if (splits > 1 && mode != 2) return cudaErrorInvalidValue;
  // cp.async moves 16-byte chunks: both operands must start on a 16-byte boundary
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15u) return cudaErrorInvalidValue;
  if (reinterpret_cast<uintptr_t>(C) & (mode == 1 ? 1u : 3u)) return cudaErrorInvalidValue;
  if (mode == 1 && ct && (reinterpret_cast<uintptr_t>(ct) & 1u)) return cudaErrorInvalidValue;
  const int kchunk = ((K / kTileK + splits - 1) / splits) * kTileK;
  const size_t smem = (size_t)2 * (kTileM + kMaxTileN) * kTileK * 2;  // 96 KB
  cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((M + kTileM - 1) / kTileM), (unsigned)((K + kchunk - 1) / kchunk));
  k_gemm_bf16<<<grid, 128, smem, st>>>(reinterpret_cast<const __nv_bfloat16 *>(A),
                                        reinterpret_cast<const __nv_bfloat16 *>(B), M, N, K, kchunk, bias, mode, C,
                                        ldc, reinterpret_cast<__nv_bfloat16 *>(ct), ldt, wait_polls(kSpinLimit));
  return cudaGetLastError();
}

// Persistent form: one CTA per SM (at most one per tile); Wp holds W2 and W3 as packed
// by k_pack_chunks and must start on a 16-byte boundary (bulk copies).
cudaError_t launch_mlp_infer_ws(const float *X, long long n, const float *P, const __nv_bfloat16 *Wp, float *Y,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (reinterpret_cast<uintptr_t>(Wp) & 15u) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_infer_ws, cudaFuncAttributeMaxDynamicSharedMemorySize, kWsSmem);
  if (e != cudaSuccess) return e;
  const long long tiles = (n + kTileM - 1) / kTileM;
  const unsigned grid = (unsigned)(tiles < sms ? tiles : sms);
  k_mlp_infer_ws<<<grid, kWsThreads, kWsSmem, st>>>(X, n, P, Wp, Y, wait_polls(kWsSpin));
  return cudaGetLastError();
}

cudaError_t launch_gather_batch(const float *X, const float *T, long long n, int B, unsigned long long seed,
                                long long step, float *Xb, float *Tb, cudaStream_t st) {
  k_gather_batch<<<(B + 255) / 256, 256, 0, st>>>(X, T, n, B, seed, step, Xb, Tb);
  return cudaGetLastError();
}

cudaError_t read_and_clear_mlp_error(unsigned *word) {
  cudaError_t e = cudaMemcpyFromSymbol(word, g_mlp_error, sizeof(unsigned));
  if (e != cudaSuccess) return e;
  const unsigned zero = 0;
  return cudaMemcpyToSymbol(g_mlp_error, &zero, sizeof(unsigned));
}

}  // namespace rgeo

namespace rgeo {
namespace {

struct ExpmapDev {
  int bmax;
  long long step;
  float *P, *G, *m, *v;
  __nv_bfloat16 *W2b, *W3b, *W2t, *W3t;
  __nv_bfloat16 *Wp;  // the operands of the persistent inference kernel, packed by k_pack_chunks
  __nv_bfloat16 *H1, *H2, *H3, *H1t, *H2t, *H3t, *dZ, *dZt;
  float *Y, *dY, *dH, *dZ1, *loss;
};

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
  return cudaMalloc((void **)p, n * sizeof(T));
}

void free_all(ExpmapDev &d) {
  void *ptrs[] = {d.P, d.G, d.m, d.v, d.W2b, d.W3b, d.W2t, d.W3t, d.Wp, d.H1, d.H2, d.H3, d.H1t, d.H2t, d.H3t,
                  d.dZ, d.dZt, d.Y, d.dY, d.dH, d.dZ1, d.loss};
  for (void *q : ptrs) cudaFree(q);
}

// Training forward pass over B rows: keeps H1..H3 and their transposes for back-propagation.
cudaError_t forward(const ExpmapDev &d, const float *X, int B, float *Y, cudaStream_t st) {
  k_layer_in<<<B, kWid, 0, st>>>(X, B, d.P, d.H1, d.H1t);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_gemm_bf16(d.H1, d.W2b, B, kWid, kWid, 1, d.P + ob2, 1, d.H2, kWid, d.H2t, B, st);
  if (e != cudaSuccess) return e;
  e = launch_gemm_bf16(d.H2, d.W3b, B, kWid, kWid, 1, d.P + ob3, 1, d.H3, kWid, d.H3t, B, st);
  if (e != cudaSuccess) return e;
  k_layer_out<<<(B + 7) / 8, 256, 0, st>>>(d.H3, B, d.P, Y);
  return cudaGetLastError();
}

// Gradients of the loss w.r.t. every parameter into d.G (zeroed first); loss into d.loss.
cudaError_t gradients(ExpmapDev &d, const float *X, const float *T, int B, float lam, cudaStream_t st) {
  cudaError_t e = forward(d, X, B, d.Y, st);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(d.G, 0, sizeof(float) * kParams, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(d.loss, 0, sizeof(float), st)) != cudaSuccess) return e;
  k_loss_grad<<<(B + 255) / 256, 256, 0, st>>>(d.Y, T, B, lam, d.dY, d.loss);
  const unsigned rb = (unsigned)((B + 31) / 32);
  k_back_out<<<rb, kWid, 0, st>>>(d.dY, d.H3, B, d.P, d.G, d.dZ, d.dZt);
  k_bias_back<<<rb, kWid, 0, st>>>(d.dZ, B, d.G + ob3);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int splits = B >= 2048 ? 16 : 1;
  // dW3 = dZ3^T H2, dH2 = dZ3 W3
  e = launch_gemm_bf16(d.dZt, d.H2t, kWid, kWid, B, splits, nullptr, 2, d.G + oW3, kWid, nullptr, 0, st);
  if (e != cudaSuccess) return e;
  e = launch_gemm_bf16(d.dZ, d.W3t, B, kWid, kWid, 1, nullptr, 0, d.dH, kWid, nullptr, 0, st);
  if (e != cudaSuccess) return e;
  k_relu_back<<<rb, kWid, 0, st>>>(d.dH, d.H2, B, d.G + ob2, d.dZ, d.dZt, nullptr);
  // dW2 = dZ2^T H1, dH1 = dZ2 W2
  e = launch_gemm_bf16(d.dZt, d.H1t, kWid, kWid, B, splits, nullptr, 2, d.G + oW2, kWid, nullptr, 0, st);
  if (e != cudaSuccess) return e;
  e = launch_gemm_bf16(d.dZ, d.W2t, B, kWid, kWid, 1, nullptr, 0, d.dH, kWid, nullptr, 0, st);
  if (e != cudaSuccess) return e;
  k_relu_back<<<rb, kWid, 0, st>>>(d.dH, d.H1, B, d.G + ob1, nullptr, nullptr, d.dZ1);
  k_back_in<<<rb, kWid, 0, st>>>(d.dZ1, X, B, d.G);
  return cudaGetLastError();
}

cudaError_t refresh(ExpmapDev &d, cudaStream_t st) {
  k_refresh_bf16<<<(kWid * kWid + 255) / 256, 256, 0, st>>>(d.P, d.W2b, d.W3b, d.W2t, d.W3t);
  k_pack_chunks<<<(kPackedElems + 255) / 256, 256, 0, st>>>(d.P, d.W2b, d.W3b, d.Wp);
  return cudaGetLastError();
}

constexpr float kErrWeight = 0.1f;
constexpr char kMagic[8] = {'R', 'G', 'E', 'O', 'X', 'M', 'P', '1'};

rgeo_status mlp_fail(rgeo_status s, const char *msg) {
  set_last_error(msg);
  return s;
}

rgeo_status mlp_cuda(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return RGEO_OK;
  static thread_local char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  return mlp_fail(e == cudaErrorMemoryAllocation ? RGEO_ENOMEM : RGEO_ECUDA, buf);
}

}  // namespace
}  // namespace rgeo

struct rgeo_expmap {
  rgeo::ExpmapDev d;
};

namespace rgeo {
// Inference over n rows: the persistent fused kernel (no host sync).
cudaError_t expmap_infer(const rgeo_expmap *x, const float *X, long long n, float *Y, cudaStream_t st) {
  return launch_mlp_infer_ws(X, n, x->d.P, x->d.Wp, Y, st);
}
}  // namespace rgeo

extern "C" {

int64_t rgeo_expmap_param_count(void) { return rgeo::kParams; }

rgeo_status rgeo_expmap_create(int32_t max_batch, uint64_t seed, rgeo_expmap **out) {
  using namespace rgeo;
  set_last_error("");
  if (!out) return mlp_fail(RGEO_EINVAL, "rgeo_expmap_create: out is NULL");
  *out = nullptr;
  if (max_batch < 128 || max_batch % 128 != 0 || max_batch > (1 << 20))
    return mlp_fail(RGEO_EINVAL, "rgeo_expmap_create: max_batch must be a multiple of 128 in [128, 2^20]");
  rgeo_expmap *x = new rgeo_expmap();
  std::memset(&x->d, 0, sizeof(x->d));
  ExpmapDev &d = x->d;
  d.bmax = max_batch;
  const size_t B = (size_t)max_batch, HW = B * kWid;
  cudaError_t e = dalloc(&d.P, kParams);
  if (e == cudaSuccess) e = dalloc(&d.G, kParams);
  if (e == cudaSuccess) e = dalloc(&d.m, kParams);
  if (e == cudaSuccess) e = dalloc(&d.v, kParams);
  if (e == cudaSuccess) e = dalloc(&d.W2b, (size_t)kWid * kWid);
  if (e == cudaSuccess) e = dalloc(&d.W3b, (size_t)kWid * kWid);
  if (e == cudaSuccess) e = dalloc(&d.W2t, (size_t)kWid * kWid);
  if (e == cudaSuccess) e = dalloc(&d.W3t, (size_t)kWid * kWid);
  if (e == cudaSuccess) e = dalloc(&d.Wp, (size_t)kPackedElems);
  __nv_bfloat16 **bufs[] = {&d.H1, &d.H2, &d.H3, &d.H1t, &d.H2t, &d.H3t, &d.dZ, &d.dZt};
  for (auto b : bufs)
    if (e == cudaSuccess) e = dalloc(b, HW);
  if (e == cudaSuccess) e = dalloc(&d.Y, B * kOut);
  if (e == cudaSuccess) e = dalloc(&d.dY, B * kOut);
  if (e == cudaSuccess) e = dalloc(&d.dH, HW);
  if (e == cudaSuccess) e = dalloc(&d.dZ1, HW);
  if (e == cudaSuccess) e = dalloc(&d.loss, 1);
  if (e == cudaSuccess) {
    k_init<<<(kParams + 255) / 256, 256>>>(d.P, (unsigned long long)seed);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemset(d.m, 0, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMemset(d.v, 0, sizeof(float) * kParams);
  if (e == cudaSuccess) e = refresh(d, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_all(d);
    delete x;
    return mlp_cuda(e, "rgeo_expmap_create");
  }
  *out = x;
  return RGEO_OK;
}

void rgeo_expmap_destroy(rgeo_expmap *x) {
  if (!x) return;
  rgeo::free_all(x->d);
  delete x;
}

rgeo_status rgeo_expmap_forward(const rgeo_expmap *x, const float *inputs, int64_t n, float *outputs,
                                void *cuda_stream) {
  using namespace rgeo;
  set_last_error("");
  if (!x || (n > 0 && (!inputs || !outputs)) || n < 0) return mlp_fail(RGEO_EINVAL, "rgeo_expmap_forward: bad argument");
  return mlp_cuda(expmap_infer(x, inputs, n, outputs, (cudaStream_t)cuda_stream), "rgeo_expmap_forward");
}

rgeo_status rgeo_expmap_gradients(rgeo_expmap *x, const float *inputs, const float *targets, int32_t batch,
                                  float *grads, float *loss, void *cuda_stream) {
  using namespace rgeo;
  set_last_error("");
  if (!x || !inputs || !targets) return mlp_fail(RGEO_EINVAL, "rgeo_expmap_gradients: NULL argument");
  if (batch < 128 || batch % 128 != 0 || batch > x->d.bmax)
    return mlp_fail(RGEO_EINVAL, "rgeo_expmap_gradients: batch must be a multiple of 128, at most max_batch");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  rgeo_status s = mlp_cuda(gradients(x->d, inputs, targets, batch, kErrWeight, st), "rgeo_expmap_gradients");
  if (s != RGEO_OK) return s;
  if (grads) s = mlp_cuda(cudaMemcpyAsync(grads, x->d.G, sizeof(float) * kParams, cudaMemcpyDeviceToDevice, st),
                          "rgeo_expmap_gradients: copy");
  if (s == RGEO_OK && loss)
    s = mlp_cuda(cudaMemcpyAsync(loss, x->d.loss, sizeof(float), cudaMemcpyDeviceToDevice, st), "rgeo_expmap_gradients");
  return s;
}

rgeo_status rgeo_expmap_train_step(rgeo_expmap *x, const float *inputs, const float *targets, int32_t batch,
                                   float lr, float *loss, void *cuda_stream) {
  using namespace rgeo;
  rgeo_status s = rgeo_expmap_gradients(x, inputs, targets, batch, nullptr, loss, cuda_stream);
  if (s != RGEO_OK) return s;
  if (!(lr > 0.f)) return mlp_fail(RGEO_EINVAL, "rgeo_expmap_train_step: lr must be > 0");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  x->d.step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)x->d.step), c2 = 1.f - powf(b2, (float)x->d.step);
  k_adam<<<(kParams + 255) / 256, 256, 0, st>>>(x->d.P, x->d.G, x->d.m, x->d.v, kParams, lr, b1, b2, 1e-8f, c1, c2);
  s = mlp_cuda(cudaGetLastError(), "rgeo_expmap_train_step: adam");
  if (s == RGEO_OK) s = mlp_cuda(refresh(x->d, st), "rgeo_expmap_train_step: refresh");
  return s;
}

rgeo_status rgeo_expmap_get_params(const rgeo_expmap *x, float *host, int64_t n) {
  using namespace rgeo;
  set_last_error("");
  if (!x || !host || n != kParams) return mlp_fail(RGEO_EINVAL, "rgeo_expmap_get_params: bad argument");
  return mlp_cuda(cudaMemcpy(host, x->d.P, sizeof(float) * kParams, cudaMemcpyDeviceToHost), "rgeo_expmap_get_params");
}

rgeo_status rgeo_expmap_set_params(rgeo_expmap *x, const float *host, int64_t n) {
  using namespace rgeo;
  set_last_error("");
  if (!x || !host || n != kParams) return mlp_fail(RGEO_EINVAL, "rgeo_expmap_set_params: bad argument");
  rgeo_status s = mlp_cuda(cudaMemcpy(x->d.P, host, sizeof(float) * kParams, cudaMemcpyHostToDevice), "set_params");
  if (s == RGEO_OK) s = mlp_cuda(refresh(x->d, 0), "rgeo_expmap_set_params: refresh");
  if (s == RGEO_OK) s = mlp_cuda(cudaDeviceSynchronize(), "rgeo_expmap_set_params");
  return s;
}

// Checkpoint: magic, parameter count, step, then parameters and both Adam moments.
rgeo_status rgeo_expmap_save(const rgeo_expmap *x, const char *path) {
  using namespace rgeo;
  set_last_error("");
  if (!x || !path) return mlp_fail(RGEO_EINVAL, "rgeo_expmap_save: NULL argument");
  std::vector<float> buf(3 * (size_t)kParams);
  rgeo_status s = mlp_cuda(cudaMemcpy(buf.data(), x->d.P, sizeof(float) * kParams, cudaMemcpyDeviceToHost), "save");
  if (s == RGEO_OK) s = mlp_cuda(cudaMemcpy(buf.data() + kParams, x->d.m, sizeof(float) * kParams, cudaMemcpyDeviceToHost), "save");
  if (s == RGEO_OK) s = mlp_cuda(cudaMemcpy(buf.data() + 2 * kParams, x->d.v, sizeof(float) * kParams, cudaMemcpyDeviceToHost), "save");
  if (s != RGEO_OK) return s;
  FILE *f = fopen(path, "wb");
  if (!f) return mlp_fail(RGEO_EINVAL, "rgeo_expmap_save: cannot open file");
  const int64_t hdr[2] = {(int64_t)kParams, (int64_t)x->d.step};
  bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
            fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? RGEO_OK : mlp_fail(RGEO_EINVAL, "rgeo_expmap_save: write failed");
}

rgeo_status rgeo_expmap_load(rgeo_expmap *x, const char *path) {
  using namespace rgeo;
  set_last_error("");
  if (!x || !path) return mlp_fail(RGEO_EINVAL, "rgeo_expmap_load: NULL argument");
  FILE *f = fopen(path, "rb");
  if (!f) return mlp_fail(RGEO_EINVAL, "rgeo_expmap_load: cannot open file");
  char magic[8];
  int64_t hdr[2];
  std::vector<float> buf(3 * (size_t)kParams);
  bool ok = fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 && fread(hdr, sizeof(hdr), 1, f) == 1 &&
            hdr[0] == kParams && fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  fclose(f);
  if (!ok) return mlp_fail(RGEO_EINVAL, "rgeo_expmap_load: not a checkpoint of this network");
  x->d.step = hdr[1];
  rgeo_status s = mlp_cuda(cudaMemcpy(x->d.P, buf.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice), "load");
  if (s == RGEO_OK) s = mlp_cuda(cudaMemcpy(x->d.m, buf.data() + kParams, sizeof(float) * kParams, cudaMemcpyHostToDevice), "load");
  if (s == RGEO_OK) s = mlp_cuda(cudaMemcpy(x->d.v, buf.data() + 2 * kParams, sizeof(float) * kParams, cudaMemcpyHostToDevice), "load");
  if (s == RGEO_OK) s = mlp_cuda(refresh(x->d, 0), "load");
  if (s == RGEO_OK) s = mlp_cuda(cudaDeviceSynchronize(), "rgeo_expmap_load");
  return s;
}

rgeo_status rgeo_gemm_bf16(const void *A, const void *B, int32_t M, int32_t N, int32_t K, int32_t splits,
                           const float *bias, int32_t mode, void *C, int32_t ldc, void *ct, int32_t ldt,
                           void *cuda_stream) {
  using namespace rgeo;
  set_last_error("");
  if (!A || !B || !C || mode < 0 || mode > 2) return mlp_fail(RGEO_EINVAL, "rgeo_gemm_bf16: bad argument");
  cudaError_t e = launch_gemm_bf16(A, B, M, N, K, splits, bias, mode, C, ldc, ct, ldt, (cudaStream_t)cuda_stream);
  if (e == cudaErrorInvalidValue)
    return mlp_fail(RGEO_EINVAL,
                    "rgeo_gemm_bf16: need M >= 1, 16 <= N <= 256, N % 16 == 0, K % 64 == 0, A and B 16-byte aligned");
  return mlp_cuda(e, "rgeo_gemm_bf16");
}

}  // extern "C"
