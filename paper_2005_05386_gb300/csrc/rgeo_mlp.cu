// rgeo_mlp.cu -- tensor-core kernels of the learned exponential map (sm_103a).
//
// The surrogate maps (position, unit direction, arc length) to the endpoint and
// tangent residuals of a geodesic segment (Eq. 3.5: exp_p(s v)); it is a
// 7 -> 256 -> 256 -> 256 -> 7 MLP with ReLU.  Its 256 x 256 layers -- forward and
// both backward products -- run on the 5th-generation tensor cores:
//   * tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulation) issued by one thread,
//   * accumulators in tensor memory (TMEM), read back with tcgen05.ld,
//   * operands in shared memory in the canonical K-major layout without swizzle
//     (8-row x 16-byte core matrices): staged with cp.async by the GEMM and the
//     training kernel, bulk-copied (cp.async.bulk) by the persistent inference kernel,
//   * completion signalled through mbarriers by tcgen05.commit.
// Inference runs all four layers in one persistent, warp-specialised kernel
// (k_mlp_infer_ws); a training step is one persistent kernel over the batch's 128-row
// tiles (k_train_tile) and one kernel that sums its partial gradients and takes the Adam
// step (k_reduce_adam).  Every wait is bounded: a wait that runs out records kErrTimeout
// in the error word and the kernel returns after releasing its tensor memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
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

// The BF16 copies of W2 and W3 (row-major, and transposed for the backward products).
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

// ------------------------------------------------------------ fused training step
// One training step's forward and backward pass in one persistent kernel: CTA c takes the
// 128-row tiles c, c + grid, ... of the batch.  Per tile, the six products of the 256-wide
// layers run on the tensor core (Z2 = H1 W2^T, Z3 = H2 W3^T, the tile's dW3 = dZ3^T H2,
// dH2 = dZ3 W3, its dW2 = dZ2^T H1 and dH1 = dZ2 W2), each into TMEM (the two 128-row halves
// of a weight gradient side by side: 512 columns).  Their epilogues run the rest on the CUDA
// cores, one tile row per thread: layer 1 before them, then layer 4, the loss and dY, the
// ReLU masks, and the gradients of the biases and of the 7-wide layers, whose sums over the
// tile's rows are taken across the warp's lanes by a fixed shuffle tree and across its four
// row quarters in order.  Each epilogue writes the next product's activation operand straight
// into shared memory in the canonical layout (the rows H1, H2, dZ3, dZ2 in sAct; dZ3^T and
// dZ2^T in sTr), so only the weights and the transposed activations H2^T and H1^T that the
// weight gradients take are staged, by cp.async from L2.  Each CTA sums its tiles' gradients in
// tile order into its own slot of part (kPartStride floats: the parameters in the order of P,
// then the loss); k_reduce_adam sums the slots in CTA order, so a step's gradient does not
// depend on timing.  The roundings are those of the training arithmetic: H1, H2, H3, dZ3 and
// dZ2 are BF16 operands, everything else FP32.
constexpr int kTrThreads = 256;
constexpr int kTrAct = kTileM * kWid * 2;          // 64 KB: 128 rows x K = 256 (core matrices, SBO 4096 B)
constexpr int kTrTr = kWid * kTileM * 2;           // 64 KB: M = 256 x K = 128 (two 128-row halves, SBO 2048 B)
constexpr int kTrKStep = 32;                         // K columns per staged step of B
constexpr int kTrNBuf = 4;                           // B stages in the ring: three loads in flight
constexpr int kTrStageB = kMaxTileN * kTrKStep * 2;  // 16 KB: 256 x 32 (SBO 512 B)
constexpr int kTrFloats = kOut * kWid + 2 * kWid + 3 * kTileM * 8;
constexpr int kTrSmem = kTrAct + kTrTr + kTrNBuf * kTrStageB + kTrFloats * 4;  // 213 KB: one CTA per SM
constexpr int kPartStride = (kParams + 1 + 3) & ~3;                      // floats per slot, 16-byte aligned
constexpr int kRedQty = 8;  // column sums reduced at once (in the stage buffers, free in an epilogue)
static_assert(kTrSmem <= 227 * 1024, "shared memory of the training kernel (one CTA per SM: it takes all of TMEM)");
static_assert(kRedQty * 4 * kWid * 4 <= 2 * kTrStageB, "column-sum buffer in stage buffers 0 and 1");
static_assert(oW2 % 4 == 0 && oW3 % 4 == 0, "vector access to the weight-gradient slots");

struct TrainArgs {
  const float *X, *T;
  int B;
  float lam;
  const float *P;
  const __nv_bfloat16 *W2b, *W3b, *W2t, *W3t;
  float *part;
  __nv_bfloat16 *H1, *H2, *H1t, *H2t;
  long long polls;
};

__device__ __forceinline__ uint4 pack8_bf16(const __nv_bfloat16 (&h)[8]) {
  uint32_t w[4];
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 p = __halves2bfloat162(h[2 * i], h[2 * i + 1]);
    w[i] = *reinterpret_cast<const uint32_t *>(&p);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}
// element j (0 or 1) of a packed BF16 pair as FP32, and as BF16
__device__ __forceinline__ float bf16_of(uint32_t pair, int j) {
  return __uint_as_float(j ? (pair & 0xFFFF0000u) : (pair << 16));
}
__device__ __forceinline__ __nv_bfloat16 bf16_at(uint32_t pair, int j) {
  return __ushort_as_bfloat16((unsigned short)(j ? (pair >> 16) : (pair & 0xFFFFu)));
}

// Byte offset of element (m, k) of a K-major canonical operand whose row groups are sbo bytes
// apart: core matrix (m / 8, k / 8) of 8 rows x 16 bytes, row m % 8 at 16 (m % 8).
__device__ __forceinline__ uint32_t canon_off(int m, int k, uint32_t sbo) {
  return (uint32_t)(m >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(m & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// For every j, the sum of v[j] over the warp's 32 lanes; lane l returns the sum for j = l.  A
// fixed tree (halves exchanged at distance 16, 8, 4, 2, 1), so the result does not depend on
// timing.  v is clobbered.
__device__ __forceinline__ float lane_sums(float (&v)[32]) {
  const unsigned lane = threadIdx.x & 31u;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const bool up = (lane & (unsigned)w) != 0u;
#pragma unroll
    for (int j = 0; j < w; ++j) {
      const float send = up ? v[j] : v[j + w];
      const float keep = up ? v[j + w] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  return v[0];
}

// K columns k0 .. k0 + 31 of rows row0 .. row0 + rows - 1 of the row-major BF16 src (leading
// dimension ld) into the canonical K-major layout of one B stage: core matrix (row group g, K
// chunk c) at (4 g + c) * 128, row r at 16 (r % 8) within it (LBO 128, SBO 512).
__device__ __forceinline__ void stage_b32(uint8_t *dst, const __nv_bfloat16 *src, int ld, int row0, int rows, int k0) {
  for (int q = threadIdx.x; q < rows * 4; q += blockDim.x) {
    const int r = q >> 2, c = q & 3;
    cp_async16(dst + ((r >> 3) * 4 + c) * 128 + (r & 7) * 16, src + (size_t)(row0 + r) * ld + k0 + c * 8);
  }
}

// One K step of a product's B (rows brow0 .. brow0 + N - 1, K columns bk0 .. bk0 + 31) into sB as
// one cp.async group; issued by all threads, also ahead of the product while the previous
// product's epilogue runs.
__device__ __forceinline__ void prefetch_b(uint8_t *sB, const __nv_bfloat16 *B, int ldb, int brow0, int bk0, int N) {
  stage_b32(sB, B, ldb, brow0, N, bk0);
  cp_async_commit();
}

// Waits until at most n (0, 1 or 2) of this thread's most recent cp.async groups are pending.
__device__ __forceinline__ void cp_async_wait_upto(int n) {
  if (n >= 2)
    asm volatile("cp.async.wait_group 2;" ::: "memory");
  else if (n == 1)
    asm volatile("cp.async.wait_group 1;" ::: "memory");
  else
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// All threads of the CTA: TMEM columns acc.. (128 lanes x N) = A x B[brow0 + 0..N-1][bk0 + 0..K-1]^T,
// A the 128 x K canonical operand in shared memory at a_base (row groups a_sbo bytes apart), B
// row-major BF16 (leading dimension ldb) staged in 32-wide K steps through the ring sB of
// kTrNBuf buffers, step s in sB[(fb + s) % kTrNBuf] and signalled on that buffer's bar, whose
// phases ph tracks (K a multiple of 32): up to three steps load while the MMAs of an earlier one
// run.  With pre, step 0 is already in flight (prefetch_b into sB[fb]).  With a_off2 > 0, a
// second 128-row A at a_base + a_off2 is multiplied by the same staged B into columns acc2..
// (the two halves of a weight gradient).  Returns with every MMA complete, or false once a wait
// ran out (abort raised; the caller leaves, and the kernel's drain waits for what is in flight).
__device__ bool tile_gemm(uint32_t a_base, uint32_t a_sbo, uint8_t *const *sB, const __nv_bfloat16 *B, int ldb,
                          int brow0, int bk0, int N, int K, uint32_t acc, uint64_t *bar, uint32_t (&ph)[kTrNBuf],
                          volatile int *abort, long long polls, int fb, bool pre, uint32_t a_off2 = 0u,
                          uint32_t acc2 = 0u) {
  const int nst = K / kTrKStep;
  const int ahead = nst < kTrNBuf - 1 ? nst : kTrNBuf - 1;  // steps loaded ahead of the MMAs
  const uint32_t idesc = idesc_bf16(kTileM, N);
  for (int i = pre ? 1 : 0; i < ahead; ++i) prefetch_b(sB[(fb + i) % kTrNBuf], B, ldb, brow0, bk0 + i * kTrKStep, N);
  for (int s = 0; s < nst; ++s) {
    const int buf = (fb + s) % kTrNBuf;
    const int committed = s + ahead < nst ? s + ahead : nst;  // steps 0 .. committed - 1 are in flight or landed
    cp_async_wait_upto(committed - s - 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // also orders the epilogue's operand writes
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t b0 = smem_u32(sB[buf]);
      for (int kk = 0; kk < kTrKStep / 16; ++kk) {
        const uint32_t ao = (uint32_t)(s * 512 + kk * 256), accum = (s > 0 || kk > 0) ? 1u : 0u;
        const uint64_t bd = smem_desc(b0 + kk * 256, 128, 512);
        mma_bf16(acc, smem_desc(a_base + ao, 128, a_sbo), bd, idesc, accum);
        if (a_off2) mma_bf16(acc2, smem_desc(a_base + a_off2 + ao, 128, a_sbo), bd, idesc, accum);
      }
      mma_commit(&bar[buf]);
    }
    const int nxt = s + ahead;  // the step loaded now, into the buffer of step s - 1
    if (nxt < nst) {
      if (s >= 1) {  // the MMAs of step s - 1 read that buffer
        const int pb = (fb + s - 1) % kTrNBuf;
        if (!mbar_wait(&bar[pb], ph[pb], polls)) *abort = 1;
        ph[pb] ^= 1u;
      }
      __syncthreads();
      if (*abort) return false;
      prefetch_b(sB[(fb + nxt) % kTrNBuf], B, ldb, brow0, bk0 + nxt * kTrKStep, N);
    }
  }
  // the steps whose MMAs have not been waited for: the in-loop waits took steps 0 .. nst - ahead - 2
  for (int s = nst - ahead - 1 > 0 ? nst - ahead - 1 : 0; s < nst; ++s) {
    const int b = (fb + s) % kTrNBuf;
    if (!mbar_wait(&bar[b], ph[b], polls)) *abort = 1;
    ph[b] ^= 1u;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return !*abort;
}

// 32 consecutive BF16 columns c0.. of tile row `row` (packed pairs pk) into the canonical
// row operand sAct (four 16-byte stores) and, when sTr is set, as column `row` of the
// canonical transposed operand sTr (one element per column).
__device__ __forceinline__ void put_operand32(uint8_t *sAct, uint8_t *sTr, int row, int c0, const uint32_t (&pk)[16]) {
  for (int u = 0; u < 4; ++u)
    *reinterpret_cast<uint4 *>(sAct + canon_off(row, c0 + 8 * u, 4096)) =
        make_uint4(pk[4 * u], pk[4 * u + 1], pk[4 * u + 2], pk[4 * u + 3]);
  if (sTr)
    for (int j = 0; j < 32; ++j)
      *reinterpret_cast<__nv_bfloat16 *>(sTr + canon_off(c0 + j, row, 2048)) = bf16_at(pk[j >> 1], j & 1);
}

// Writes 32 consecutive BF16 columns c0.. of one row: row-major (dst + c0) and transposed
// (column c at dstT + c * ld).
__device__ __forceinline__ void store_row32(__nv_bfloat16 *dst, __nv_bfloat16 *dstT, size_t ld, int c0,
                                            const uint32_t (&pk)[16]) {
  uint4 *d = reinterpret_cast<uint4 *>(dst + c0);
  for (int u = 0; u < 4; ++u) d[u] = make_uint4(pk[4 * u], pk[4 * u + 1], pk[4 * u + 2], pk[4 * u + 3]);
  for (int j = 0; j < 32; ++j) dstT[(size_t)(c0 + j) * ld] = bf16_at(pk[j >> 1], j & 1);
}

// The tile's dW (two 128-row halves in TMEM columns 0..255 and 256..511) into the slot's W
// (added to what the CTA's earlier tiles left there).
__device__ __forceinline__ void add_weight_grad(uint32_t tl, int half, int row, float *Wslot, bool first) {
  for (int mh = 0; mh < 2; ++mh)
    for (int c0 = half * 128; c0 < half * 128 + 128; c0 += 32) {
      uint32_t v[32];
      tmem_ld32_nowait(tl + (uint32_t)(mh * kWid + c0), v);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float4 *g = reinterpret_cast<float4 *>(Wslot + (size_t)(mh * kTileM + row) * kWid + c0);
      for (int u = 0; u < 8; ++u) {
        float4 s = make_float4(__uint_as_float(v[4 * u]), __uint_as_float(v[4 * u + 1]),
                               __uint_as_float(v[4 * u + 2]), __uint_as_float(v[4 * u + 3]));
        if (!first) {
          const float4 o = g[u];
          s = make_float4(o.x + s.x, o.y + s.y, o.z + s.z, o.w + s.w);
        }
        g[u] = s;
      }
    }
}

__global__ void __launch_bounds__(kTrThreads, 1) k_train_tile(const TrainArgs a) {
  extern __shared__ __align__(1024) uint8_t tsm[];
  uint8_t *sAct = tsm, *sTr = tsm + kTrAct;
  uint8_t *const sB[kTrNBuf] = {sTr + kTrTr, sTr + kTrTr + kTrStageB, sTr + kTrTr + 2 * kTrStageB,
                                sTr + kTrTr + 3 * kTrStageB};
  // [kRedQty][4 row quarters][256 columns] in an epilogue, over stage buffers 0 and 1 (an epilogue
  // that uses it prefetches the next product's first step into buffer 2)
  float *red = reinterpret_cast<float *>(sB[0]);
  float *w4s = reinterpret_cast<float *>(sB[kTrNBuf - 1] + kTrStageB);  // [7][256]
  float *b2s = w4s + kOut * kWid, *b3s = b2s + kWid;
  float *xs = b3s + kWid, *dys = xs + kTileM * 8, *part4 = dys + kTileM * 8;  // [128][8] each
  const uint32_t aAct = smem_u32(sAct), aTr = smem_u32(sTr);
  __shared__ uint64_t bar[kTrNBuf], drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ float loss_w[kTrThreads / 32];
  volatile int *abortp = &abort_flag;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  // epilogues: warp w reads TMEM lanes 32 (w % 4) .. (its row quarter q) and the column half w / 4
  const int q = warp & 3, half = warp >> 2, row = q * 32 + lane;
  const int Bn = a.B, ntiles = Bn / kTileM;
  if (t == 0) {
    for (int b = 0; b < kTrNBuf; ++b) mbar_init(&bar[b], 1);
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
  for (int i = t; i < kOut * kWid; i += kTrThreads) w4s[i] = a.P[oW4 + i];
  b2s[t] = a.P[ob2 + t];
  b3s[t] = a.P[ob3 + t];
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
  uint32_t ph[kTrNBuf] = {0u, 0u, 0u, 0u};
  float *slot = a.part + (size_t)blockIdx.x * kPartStride;
  // this thread's share of the small gradients, summed over the CTA's tiles: column t of
  // layers 1 (dW1 row, db1), 2 (db2), 3 (db3) and 4 (dW4 column; db4 for t < 7)
  float gw1[kIn], gw4[kOut], gb1 = 0.f, gb2 = 0.f, gb3 = 0.f, gb4 = 0.f, lsum = 0.f;
  for (int i = 0; i < kIn; ++i) gw1[i] = 0.f;
  for (int o = 0; o < kOut; ++o) gw4[o] = 0.f;
  // column t's sum of quantity k over the four row quarters of red, in order
  auto red_sum = [&](int k) {
    float s = 0.f;
    for (int qq = 0; qq < 4; ++qq) s += red[(k * 4 + qq) * kWid + t];
    return s;
  };
  bool first = true;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, first = false) {
    const int m0 = tile * kTileM;
    for (int i = t; i < kTileM * 8; i += kTrThreads) {
      const int r = i >> 3, k = i & 7;
      xs[i] = k < kIn ? a.X[(size_t)(m0 + r) * kIn + k] : 0.f;
    }
    __syncthreads();
    // ---- layer 1 (FP32, K = 7): H1 = relu(X W1^T + b1) into sAct, and as BF16 rows and
    // transposed rows in L2 (the ReLU mask of dH1, the operand of dW2); unit j = t
    {
      float w1[kIn];
      for (int k = 0; k < kIn; ++k) w1[k] = a.P[oW1 + t * kIn + k];
      const float b1 = a.P[ob1 + t];
      for (int r0 = 0; r0 < kTileM; r0 += 8) {
        __nv_bfloat16 hv[8];
        for (int u = 0; u < 8; ++u) {
          float z = b1;
          for (int k = 0; k < kIn; ++k) z = fmaf(w1[k], xs[(r0 + u) * 8 + k], z);
          hv[u] = __float2bfloat16_rn(fmaxf(z, 0.f));
          a.H1[(size_t)(m0 + r0 + u) * kWid + t] = hv[u];
          *reinterpret_cast<__nv_bfloat16 *>(sAct + canon_off(r0 + u, t, 4096)) = hv[u];
        }
        *reinterpret_cast<uint4 *>(a.H1t + (size_t)t * Bn + m0 + r0) = pack8_bf16(hv);
      }
    }
    // ---- Z2 = H1 W2^T; H2 = relu(Z2 + b2) into sAct, and as BF16 rows and transposed in L2
    // (step 0 of W2 was prefetched into buffer 2 during the previous tile's last epilogue)
    if (!tile_gemm(aAct, 4096, sB, a.W2b, kWid, 0, 0, kWid, kWid, tmem, bar, ph, abortp, a.polls, 2, !first))
      break;
    prefetch_b(sB[0], a.W3b, kWid, 0, 0, kWid);
    for (int c0 = half * 128; c0 < half * 128 + 128; c0 += 32) {
      uint32_t v[32], pk[16];
      tmem_ld32_nowait(tl + (uint32_t)c0, v);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      for (int j = 0; j < 16; ++j)
        pk[j] = pack_bf16_relu(__uint_as_float(v[2 * j]) + b2s[c0 + 2 * j],
                               __uint_as_float(v[2 * j + 1]) + b2s[c0 + 2 * j + 1]);
      put_operand32(sAct, nullptr, row, c0, pk);
      store_row32(a.H2 + (size_t)(m0 + row) * kWid, a.H2t + m0 + row, Bn, c0, pk);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    // ---- Z3 = H2 W3^T; H3 = relu(Z3 + b3) (BF16); layer 4 (FP32) from the BF16 H3
    if (!tile_gemm(aAct, 4096, sB, a.W3b, kWid, 0, 0, kWid, kWid, tmem, bar, ph, abortp, a.polls, 0, true))
      break;
    prefetch_b(sB[2], a.H2t, Bn, 0, m0, kWid);  // the epilogue's column sums use buffers 0 and 1
    {
      float y[kOut];
      for (int o = 0; o < kOut; ++o) y[o] = 0.f;
      for (int c0 = half * 128; c0 < half * 128 + 128; c0 += 32) {
        uint32_t v[32];
        tmem_ld32_nowait(tl + (uint32_t)c0, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        for (int j = 0; j < 32; j += 2) {
          const uint32_t pk = pack_bf16_relu(__uint_as_float(v[j]) + b3s[c0 + j],
                                             __uint_as_float(v[j + 1]) + b3s[c0 + j + 1]);
          for (int u = 0; u < 2; ++u)
            for (int o = 0; o < kOut; ++o) y[o] = fmaf(w4s[o * kWid + c0 + j + u], bf16_of(pk, u), y[o]);
        }
      }
      if (half == 1)
        for (int o = 0; o < kOut; ++o) part4[row * 8 + o] = y[o];
      __syncthreads();
      // the loss and its gradient dY (outputs 0..5: mean squared error against T; output 6: the
      // log squared error of the same row, weighted by lam), by the column-half-0 thread of each row
      if (half == 0) {
        float Y[kOut];
        for (int o = 0; o < kOut; ++o) Y[o] = (y[o] + part4[row * 8 + o]) + a.P[ob4 + o];
        const float *Tr = a.T + (size_t)(m0 + row) * 6;
        float se = 0.f;
        for (int o = 0; o < 6; ++o) {
          const float d = Y[o] - Tr[o];
          se = fmaf(d, d, se);
          dys[row * 8 + o] = 2.f * d / (6.f * Bn);
        }
        const float e = logf(se + 1e-6f);
        const float d6 = Y[6] - e;
        dys[row * 8 + 6] = 2.f * a.lam * d6 / Bn;
        lsum += se / (6.f * Bn) + a.lam * d6 * d6 / Bn;
      }
      __syncthreads();
    }
    // ---- layer 4 backward from the same accumulator: dZ3 = bf16(dH3 [H3 > 0]) with dH3 = dY W4, into
    // sAct (rows) and sTr (transposed); the tile's dW4 = dY^T H3 and db3 = sum of dZ3 as column sums
    {
      float dy[kOut];
      for (int o = 0; o < kOut; ++o) dy[o] = dys[row * 8 + o];
      for (int c0 = half * 128; c0 < half * 128 + 128; c0 += 32) {
        uint32_t v[32], pz[16];
        tmem_ld32_nowait(tl + (uint32_t)c0, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float h[32], z[32], w[32];
        for (int j = 0; j < 32; j += 2) {
          const uint32_t pk = pack_bf16_relu(__uint_as_float(v[j]) + b3s[c0 + j],
                                             __uint_as_float(v[j + 1]) + b3s[c0 + j + 1]);
          h[j] = bf16_of(pk, 0);
          h[j + 1] = bf16_of(pk, 1);
        }
        for (int j = 0; j < 32; j += 2) {
          __nv_bfloat16 zb[2];
          for (int u = 0; u < 2; ++u) {
            float dh = 0.f;
            for (int o = 0; o < kOut; ++o) dh = fmaf(dy[o], w4s[o * kWid + c0 + j + u], dh);
            zb[u] = __float2bfloat16_rn(h[j + u] > 0.f ? dh : 0.f);
            z[j + u] = __bfloat162float(zb[u]);
          }
          const __nv_bfloat162 p2 = __halves2bfloat162(zb[0], zb[1]);
          pz[j >> 1] = *reinterpret_cast<const uint32_t *>(&p2);
        }
        put_operand32(sAct, sTr, row, c0, pz);
        for (int o = 0; o < kOut; ++o) {
          for (int j = 0; j < 32; ++j) w[j] = dy[o] * h[j];
          red[(o * 4 + q) * kWid + c0 + lane] = lane_sums(w);
        }
        red[(7 * 4 + q) * kWid + c0 + lane] = lane_sums(z);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      for (int o = 0; o < kOut; ++o) gw4[o] += red_sum(o);
      gb3 += red_sum(7);
      if (t < kOut)
        for (int r = 0; r < kTileM; ++r) gb4 += dys[r * 8 + t];
      __syncthreads();
    }
    // ---- the tile's dW3 = dZ3^T H2 (K = its 128 rows; both 128-row halves of dW3 per staged H2^T
    // stage), added into the CTA's slot
    if (!tile_gemm(aTr, 2048, sB, a.H2t, Bn, 0, m0, kWid, kTileM, tmem, bar, ph, abortp, a.polls, 2, true,
                   16u * 2048u, tmem + kWid))
      break;
    prefetch_b(sB[0], a.W3t, kWid, 0, 0, kWid);
    add_weight_grad(tl, half, row, slot + oW3, first);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    // ---- dH2 = dZ3 W3; dZ2 = bf16(dH2 [H2 > 0]) into sAct and sTr; db2 = column sums of the FP32 values
    if (!tile_gemm(aAct, 4096, sB, a.W3t, kWid, 0, 0, kWid, kWid, tmem, bar, ph, abortp, a.polls, 0, true))
      break;
    prefetch_b(sB[2], a.H1t, Bn, 0, m0, kWid);  // the epilogue's column sums use buffers 0 and 1
    for (int c0 = half * 128; c0 < half * 128 + 128; c0 += 32) {
      uint32_t v[32], pz[16];
      tmem_ld32_nowait(tl + (uint32_t)c0, v);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const uint4 *hr = reinterpret_cast<const uint4 *>(a.H2 + (size_t)(m0 + row) * kWid + c0);
      float g[32];
      for (int u = 0; u < 4; ++u) {
        const uint4 hb = hr[u];
        const uint32_t hw[4] = {hb.x, hb.y, hb.z, hb.w};
        for (int j = 0; j < 8; ++j)
          g[8 * u + j] = bf16_of(hw[j >> 1], j & 1) > 0.f ? __uint_as_float(v[8 * u + j]) : 0.f;
      }
      for (int j = 0; j < 32; j += 2) {
        const __nv_bfloat162 p2 = __halves2bfloat162(__float2bfloat16_rn(g[j]), __float2bfloat16_rn(g[j + 1]));
        pz[j >> 1] = *reinterpret_cast<const uint32_t *>(&p2);
      }
      put_operand32(sAct, sTr, row, c0, pz);
      red[q * kWid + c0 + lane] = lane_sums(g);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    gb2 += red_sum(0);
    // (the next product's first stage overwrites red: tile_gemm synchronises before it stages)
    __syncthreads();
    // ---- the tile's dW2 = dZ2^T H1, as dW3
    if (!tile_gemm(aTr, 2048, sB, a.H1t, Bn, 0, m0, kWid, kTileM, tmem, bar, ph, abortp, a.polls, 2, true,
                   16u * 2048u, tmem + kWid))
      break;
    prefetch_b(sB[0], a.W2t, kWid, 0, 0, kWid);
    add_weight_grad(tl, half, row, slot + oW2, first);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    // ---- dH1 = dZ2 W2; dZ1 = dH1 [H1 > 0] (FP32); db1 and dW1 = dZ1^T X as column sums
    if (!tile_gemm(aAct, 4096, sB, a.W2t, kWid, 0, 0, kWid, kWid, tmem, bar, ph, abortp, a.polls, 0, true))
      break;
    if (tile + (int)gridDim.x < ntiles) prefetch_b(sB[2], a.W2b, kWid, 0, 0, kWid);  // the next tile's Z2
    {
      float xr[kIn];
      for (int i = 0; i < kIn; ++i) xr[i] = xs[row * 8 + i];
      for (int c0 = half * 128; c0 < half * 128 + 128; c0 += 32) {
        uint32_t v[32];
        tmem_ld32_nowait(tl + (uint32_t)c0, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const uint4 *hr = reinterpret_cast<const uint4 *>(a.H1 + (size_t)(m0 + row) * kWid + c0);
        float g[32], w[32];
        for (int u = 0; u < 4; ++u) {
          const uint4 hb = hr[u];
          const uint32_t hw[4] = {hb.x, hb.y, hb.z, hb.w};
          for (int j = 0; j < 8; ++j)
            g[8 * u + j] = bf16_of(hw[j >> 1], j & 1) > 0.f ? __uint_as_float(v[8 * u + j]) : 0.f;
        }
        for (int i = 0; i < kIn; ++i) {
          for (int j = 0; j < 32; ++j) w[j] = g[j] * xr[i];
          red[((1 + i) * 4 + q) * kWid + c0 + lane] = lane_sums(w);
        }
        red[q * kWid + c0 + lane] = lane_sums(g);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      gb1 += red_sum(0);
      for (int i = 0; i < kIn; ++i) gw1[i] += red_sum(1 + i);
      __syncthreads();
    }
  }
  if (!*abortp && blockIdx.x < ntiles) {
    // the CTA's small gradients and loss into its slot
    for (int i = 0; i < kIn; ++i) slot[oW1 + t * kIn + i] = gw1[i];
    slot[ob1 + t] = gb1;
    slot[ob2 + t] = gb2;
    slot[ob3 + t] = gb3;
    for (int o = 0; o < kOut; ++o) slot[oW4 + o * kWid + t] = gw4[o];
    if (t < kOut) slot[ob4 + t] = gb4;
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, off);
    if (lane == 0) loss_w[warp] = lsum;
    __syncthreads();
    if (t == 0) {
      float s = 0.f;
      for (int w = 0; w < kTrThreads / 32; ++w) s += loss_w[w];
      slot[kParams] = s;
    }
  }
  // every MMA issued has completed before the tensor memory is released
  cp_async_wait_all();
  if (t == 0) mma_commit(&drain);
  if (!mbar_wait(&drain, 0u)) *abortp = 1;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (t == 0 && *abortp) atomicOr(&g_mlp_error, kErrTimeout);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kWid) : "memory");
}

// The step's gradient and loss: each parameter's slots summed in CTA order (so the result does
// not depend on timing), into G and *loss when set.  With lr > 0, an Adam step (Kingma and Ba
// 2015) on the FP32 master parameters, and the BF16 copies of W2 and W3 (row-major and
// transposed) that the next step's products read.  Nothing is written while the error word
// is set: the slots of a training kernel that gave up are incomplete.
__global__ void k_reduce_adam(const float *__restrict__ part, int nparts, float *G, float *loss, float *P, float *m,
                              float *v, float lr, float b1, float b2, float eps, float c1, float c2,
                              __nv_bfloat16 *W2b, __nv_bfloat16 *W3b, __nv_bfloat16 *W2t, __nv_bfloat16 *W3t) {
  if (*(volatile unsigned *)&g_mlp_error) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && loss) {
    float s = 0.f;
    for (int c = 0; c < nparts; ++c) s += part[(size_t)c * kPartStride + kParams];
    *loss = s;
  }
  if (i >= kParams) return;
  float g = 0.f;
  for (int c = 0; c < nparts; ++c) g += part[(size_t)c * kPartStride + i];
  if (G) G[i] = g;
  if (!(lr > 0.f)) return;
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float p = P[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  P[i] = p;
  if (i >= oW2 && i < ob2) {
    const int e = i - oW2, r = e / kWid, c = e % kWid;
    const __nv_bfloat16 w = __float2bfloat16_rn(p);
    W2b[e] = w;
    W2t[c * kWid + r] = w;
  } else if (i >= oW3 && i < ob3) {
    const int e = i - oW3, r = e / kWid, c = e % kWid;
    const __nv_bfloat16 w = __float2bfloat16_rn(p);
    W3b[e] = w;
    W3t[c * kWid + r] = w;
  }
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
  int sms;     // CTAs of the training kernel at most (one per SM)
  long long step;
  float *P, *m, *v;
  __nv_bfloat16 *W2b, *W3b, *W2t, *W3t;
  __nv_bfloat16 *Wp;  // the operands of the persistent inference kernel, packed by k_pack_chunks
  bool wp_stale;      // P has changed since Wp was packed
  __nv_bfloat16 *H1, *H2, *H1t, *H2t;  // scratch rows of the training step (row-major and transposed)
  float *part;  // the training CTAs' gradient slots, kPartStride floats each
};

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
  return cudaMalloc((void **)p, n * sizeof(T));
}

void free_all(ExpmapDev &d) {
  void *ptrs[] = {d.P, d.m, d.v, d.W2b, d.W3b, d.W2t, d.W3t, d.Wp, d.H1, d.H2, d.H1t, d.H2t, d.part};
  for (void *q : ptrs) cudaFree(q);
}

// Forward and backward pass over B rows (B a multiple of 128): the CTAs' gradient slots; the
// grid (one CTA per SM, at most one per tile) depends only on B and the device, so the
// slots' sum is the same on every call.
cudaError_t train_pass(ExpmapDev &d, const float *X, const float *T, int B, float lam, cudaStream_t st,
                       int *nparts) {
  const int tiles = B / kTileM, grid = tiles < d.sms ? tiles : d.sms;
  cudaError_t e = cudaFuncSetAttribute(k_train_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrSmem);
  if (e != cudaSuccess) return e;
  TrainArgs a;
  a.X = X;
  a.T = T;
  a.B = B;
  a.lam = lam;
  a.P = d.P;
  a.W2b = d.W2b;
  a.W3b = d.W3b;
  a.W2t = d.W2t;
  a.W3t = d.W3t;
  a.part = d.part;
  a.H1 = d.H1;
  a.H2 = d.H2;
  a.H1t = d.H1t;
  a.H2t = d.H2t;
  a.polls = wait_polls(kSpinLimit);
  k_train_tile<<<grid, kTrThreads, kTrSmem, st>>>(a);
  *nparts = grid;
  return cudaGetLastError();
}

// The slots' sum into G and loss (device pointers, each may be null); with lr > 0 also the
// Adam step of step count d.step and the refreshed BF16 weight copies.
cudaError_t reduce_adam(ExpmapDev &d, int nparts, float *G, float *loss, float lr, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = lr > 0.f ? 1.f - powf(b1, (float)d.step) : 1.f, c2 = lr > 0.f ? 1.f - powf(b2, (float)d.step) : 1.f;
  k_reduce_adam<<<(kParams + 255) / 256, 256, 0, st>>>(d.part, nparts, G, loss, d.P, d.m, d.v, lr, b1, b2, 1e-8f,
                                                      c1, c2, d.W2b, d.W3b, d.W2t, d.W3t);
  if (lr > 0.f) d.wp_stale = true;
  return cudaGetLastError();
}

cudaError_t refresh(ExpmapDev &d, cudaStream_t st) {
  k_refresh_bf16<<<(kWid * kWid + 255) / 256, 256, 0, st>>>(d.P, d.W2b, d.W3b, d.W2t, d.W3t);
  k_pack_chunks<<<(kPackedElems + 255) / 256, 256, 0, st>>>(d.P, d.W2b, d.W3b, d.Wp);
  d.wp_stale = false;
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
// The packed operands are brought up to date first when training steps have changed P since
// (stream-ordered, like the steps themselves).
cudaError_t expmap_infer(const rgeo_expmap *x, const float *X, long long n, float *Y, cudaStream_t st) {
  ExpmapDev &d = const_cast<rgeo_expmap *>(x)->d;
  if (d.wp_stale) {
    k_pack_chunks<<<(kPackedElems + 255) / 256, 256, 0, st>>>(d.P, d.W2b, d.W3b, d.Wp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    d.wp_stale = false;
  }
  return launch_mlp_infer_ws(X, n, d.P, d.Wp, Y, st);
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
  if (e == cudaSuccess) e = dalloc(&d.m, kParams);
  if (e == cudaSuccess) e = dalloc(&d.v, kParams);
  if (e == cudaSuccess) e = dalloc(&d.W2b, (size_t)kWid * kWid);
  if (e == cudaSuccess) e = dalloc(&d.W3b, (size_t)kWid * kWid);
  if (e == cudaSuccess) e = dalloc(&d.W2t, (size_t)kWid * kWid);
  if (e == cudaSuccess) e = dalloc(&d.W3t, (size_t)kWid * kWid);
  if (e == cudaSuccess) e = dalloc(&d.Wp, (size_t)kPackedElems);
  __nv_bfloat16 **bufs[] = {&d.H1, &d.H2, &d.H1t, &d.H2t};
  for (auto b : bufs)
    if (e == cudaSuccess) e = dalloc(b, HW);
  int dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    const int slots = std::min(max_batch / kTileM, d.sms);
    e = dalloc(&d.part, (size_t)slots * kPartStride);
  }
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
  int nparts = 0;
  rgeo_status s = mlp_cuda(train_pass(x->d, inputs, targets, batch, kErrWeight, st, &nparts), "rgeo_expmap_gradients");
  if (s == RGEO_OK) s = mlp_cuda(reduce_adam(x->d, nparts, grads, loss, 0.f, st), "rgeo_expmap_gradients: sum");
  return s;
}

rgeo_status rgeo_expmap_train_step(rgeo_expmap *x, const float *inputs, const float *targets, int32_t batch,
                                   float lr, float *loss, void *cuda_stream) {
  using namespace rgeo;
  set_last_error("");
  if (!x || !inputs || !targets) return mlp_fail(RGEO_EINVAL, "rgeo_expmap_train_step: NULL argument");
  if (batch < 128 || batch % 128 != 0 || batch > x->d.bmax)
    return mlp_fail(RGEO_EINVAL, "rgeo_expmap_train_step: batch must be a multiple of 128, at most max_batch");
  if (!(lr > 0.f) || !std::isfinite(lr)) return mlp_fail(RGEO_EINVAL, "rgeo_expmap_train_step: lr must be > 0");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int nparts = 0;
  rgeo_status s = mlp_cuda(train_pass(x->d, inputs, targets, batch, kErrWeight, st, &nparts), "rgeo_expmap_train_step");
  if (s != RGEO_OK) return s;
  x->d.step += 1;
  return mlp_cuda(reduce_adam(x->d, nparts, nullptr, loss, lr, st), "rgeo_expmap_train_step: adam");
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
