// rgeo_internal.h -- device data layouts and launch interfaces shared by the
// translation units of librgeo (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "rgeo.h"

namespace rgeo {

// Bump table, isotropic form: two float4 per bump,
//   A_k = (-cx, -cy, -cz, R2)   R2 = (cutoff sigma)^2, +inf untruncated, -1 inert (a = 0)
//   B_k = (qn2, la, qs, q)      q = 1 / sigma^2, qn2 = -q log2(e) / 2, la = log2 |a|, qs = -q sign(a)
// at float4 2k and 2k + 1.  The table holds Ke + 1 bumps, Ke = K rounded up to even:
// bumps K .. Ke are inert, so that the dense sums can take bumps (2i, 2i + 1) two at a
// time and bump Ke (the pad) can fill the second half of a paired evaluation.  With
// d = x - c, r2 = |d|^2 and w = 2^(r2 qn2 + la) = |a| exp(-q r2 / 2):
//   grad f        += (w qs) d
//   -v^T Hess f v += (w qs) (q (d.v)^2 - |v|^2)
// Anisotropic bumps use three float4 per bump:
//   b0 = (cx, cy, cz, Rball2)  Rball2 = (cutoff * max_i sigma_i)^2 (support ball for the flat skip)
//   b1 = (qx, qy, qz, sgn)     q_i = 1 / sigma_i^2, sgn = sign(a)
//   b2 = (la, c2, 0, 0)        c2 = cutoff^2 (+inf when untruncated, -1 when inert)
constexpr int kIsoBumpStride = 2;  // float4 per isotropic bump
constexpr int kAnisoStride = 3;    // float4 per anisotropic bump
// Ke: the isotropic bump count rounded up to even (the pad bump's index)
__host__ __device__ inline int iso_pad_index(int K) { return (K + 1) & ~1; }
// float4 count of a packed table of K bumps
__host__ __device__ inline int packed_float4s(int K, int aniso) {
  return aniso ? kAnisoStride * K : (K > 0 ? kIsoBumpStride * (iso_pad_index(K) + 1) : 0);
}
#ifdef __CUDACC__
// Writes isotropic bump k of the table from its centre, amplitude and spread (a = 0:
// inert).  Shared by the metric's packer and the allocation-free entry point.
__device__ __forceinline__ void pack_iso_bump(float4 *table, int k, float cx, float cy, float cz, float a,
                                              float sigma, float cutoff) {
  const float inf = __int_as_float(0x7f800000);
  const bool inert = a == 0.f;
  const float q = 1.f / (sigma * sigma);
  float R2 = cutoff > 0.f ? (cutoff * sigma) * (cutoff * sigma) : inf;
  if (inert) R2 = -1.f;
  const float sgn = a > 0.f ? 1.f : (a < 0.f ? -1.f : 0.f);
  table[kIsoBumpStride * k] = make_float4(-cx, -cy, -cz, R2);
  table[kIsoBumpStride * k + 1] =
      make_float4(-0.5f * q * 1.4426950408889634f, inert ? -inf : log2f(fabsf(a)), -q * sgn, q);
}
#endif
// Pixel of item `sub` (0..31) of frame tile `tile`: tiles of 2^lw x 2^(5 - lw) pixels in
// row-major order over a W x H frame, tiles_x of them per row.  False for the part of an
// edge tile outside the frame.  Shared by the kernels and the host partition helper.
__host__ __device__ inline bool tile_pixel(int W, int H, int tiles_x, int lw, unsigned tile, unsigned sub,
                                           int &pix) {
  const unsigned tw = 1u << lw, th = 32u >> lw;
  const int px = (int)((tile % (unsigned)tiles_x) * tw + (sub & (tw - 1u)));
  const int py = (int)((tile / (unsigned)tiles_x) * th + (sub >> lw));
  if (px >= W || py >= H) return false;
  pix = py * W + px;
  return true;
}
// Cull-grid bit masks: bit k of a cell's words marks bump k.
__host__ __device__ inline int cull_words_for(int K) { return (K + 31) / 32; }
// Per-warp list of the bump pairs a warp evaluates for one right-hand side (the culled
// sums): int2 entries, x = float4 index of an even bump, y = of an odd bump.
constexpr int kListPairs = 64;
// Local maps (metric kind 2), five float4 each:
//   (c.x, c.y, c.z, a), (v.x, v.y, v.z, qn2), (B row 0, q), (B row 1, has_field), (B row 2, 0)
// with q = 1 / sigma^2 and qn2 = -q log2(e) / 2, so that f = a * 2^(qn2 |p - c|^2).
constexpr int kLocalStride = 5;
// float4s of a metric's device table by kind (0 graph, 1 twist, 2 local maps).
__host__ __device__ inline int table_float4s(int kind, int K, int aniso) {
  return kind == 2 ? kLocalStride * K : (kind == 1 ? 0 : packed_float4s(K, aniso));
}

struct MetricDev {
  int kind;            // 0 graph, 1 twist
  int K;               // bumps (inert ones included)
  int aniso;           // 1: anisotropic layout
  int skippable;       // graph, truncated, A == 0: flat space outside the supports
  float4 *bumps;       // packed table (device)
  float *raw;          // raw centres/amplitudes/sigmas (device) [K*7], in the caller's bump order
  int32_t *perm;       // (device) bump of table slot k, or null: slot k is bump k
  float b[3];
  float A[9];
  int has_affine, has_quad;
  float cutoff;
  float twist_k;
  // bump-support cull grid (isotropic, truncated): G^3 cells, `words` uint32 of bump bits per cell
  int cull_G, cull_words;
  uint32_t *cull_masks;  // [G^3 * words]
  float4 *cull_hdr;      // (gmin.xyz, 1 / cell)
  float cull_reach;      // the masks' reach margin beyond kCullInflate: cull_reach_for(K)
  // bound on |x''| over the whole space for a g-unit tangent: (sum_k |a_k| / sigma_k^2 +
  // ||A||_F) / 2 (Eq. 5.4 with |grad f| / (1 + |grad f|^2) <= 1/2, ||Hess f_k|| <= |a_k| q_k)
  float accel_max;
  // sinusoidal motion of the centres: [K*3 c0 | K*3 A | K f | K phi] and the time t
  float *motion;
  float *time;
};

// Cull grid: inflation of every support radius (absolute).  kCullInflate covers float32
// rounding of the cell look-up.  A metric that may take step lists (at most kStepListBumps
// bumps) adds its reach margin kStepReach: the cell of a step's start then lists every bump
// whose support can meet any RK4 stage point of the steps whose stage points stay within
// kStepReach of it (step lists, below).  Larger metrics add none, so that their per-RHS
// lists stay as short as the supports allow.
constexpr float kCullInflate = 1e-3f;
constexpr float kStepReach = 0.04f;
constexpr int kStepListBumps = 512;
__host__ __device__ constexpr float cull_reach_for(int K) { return K <= kStepListBumps ? kStepReach : 0.f; }

// BVH node: two float4.  n0 = (lo.xyz, int first_or_left), n1 = (hi.xyz, int count);
// count > 0: leaf over primitives [first, first + count); count == 0: children at
// left, left + 1.  Primitives in BVH order, three float4 each, the first carrying
// the object id in .w: id < S is sphere id, (c.xyz, id), (r, 0, 0, 0), unused;
// otherwise triangle id - S, (v0.xyz, id), (v1.xyz, 0), (v2.xyz, 0).
struct SceneDev {
  int S, T, n_nodes;
  float4 *spheres;   // [S]
  float *albedo;     // [(S+1)*3]
  float4 *nodes;     // [2 * n_nodes]
  float4 *prims;     // [3 * (S + T)]
  float *grid;       // [gx * gy * gz] lower bounds of the distance to the scene
  int gdim[3];
  float gmin[3];
  float ginv;        // 1 / cell size
  float smin[3], smax[3];  // scene bounding box
  int has_grid;
  float fog, fog_rgb[3];     // hit colour c -> c T + fog_rgb (1 - T), T = exp(-fog * arc length)
};

struct TraceParams {
  // metric
  const float4 *bumps;
  int K, kind, aniso, skippable;
  const uint32_t *cull_masks;  // null: dense sums over all bumps
  const float4 *cull_hdr;
  int cull_G, cull_words;
  int step_lists;              // culled sums from step lists (the step's reach <= the masks' reach margin)
  int list_steps;              // steps one list serves (their reach together <= the margin)
  int bundle;                  // segment tests in bundles of several chords (one query each)
  float b[3];
  float A[9];
  int has_affine, has_quad;
  float twist_k;
  // scene
  const float4 *spheres;
  int S;
  const float *albedo;
  const float4 *nodes;  // null: no BVH, spheres tested one by one from shared memory
  const float4 *prims;
  int T;
  const float *grid;
  int gdim[3];
  float gmin[3];
  float ginv;
  float smin[3], smax[3];
  int has_grid, safe_skip;
  float fog, fog_rgb[3];
  // camera
  float cam_pos[3], cam_fwd[3], cam_up[3];
  float vfov_deg;
  int W, H, tiles_x;
  int tile_lw;          // refill tiles of 2^tile_lw x 2^(5 - tile_lw) pixels (32 items each)
  uint32_t tile0;       // first frame tile of this launch
  uint32_t tile_step;   // launch tile i is frame tile tile0 + i tile_step
  uint32_t n_items;     // items of this launch (32 per launch tile)
  // integration
  float h;
  int max_steps, integrator, shading, energy;
  // outputs
  int32_t *id;
  float *hit;
  int32_t *steps;
  uchar4 *rgba;
  double *drift;
  unsigned long long *bump_evals;  // optional work counter: bump terms of the rays' own cells
  unsigned long long *bump_slots;  // optional work counter: bump terms the lanes evaluated
  float *hit_nrm;                  // optional [3][N]: unit normal of each hit, facing the incoming segment
  uint32_t *counter;
  // launch shape
  int rays_per_thread;  // 1, or 2 (isotropic graph metric only)
  int refill_lanes;     // 0: a warp takes new rays once all of its rays have finished; 1: each lane as its ray finishes
};

// State of the surrogate tracer: per-ray SoA over the N = W * H pixels, the queue of
// rays waiting for a surrogate jump, and the network's inputs and outputs per slot.
struct WaveArgs {
  float *st;            // [15][N]: xh[3], xl[3], vh[3], vl[3], dleft, e0m1, arc
  int32_t *steps;       // [N] equivalent RK4 steps taken
  int32_t *cool;        // [N] RK4 steps to take before the next jump attempt
  const int32_t *list_in;  // rays advanced this round (round > 0)
  int first;            // round 0: rays start at the camera
  int32_t *queue;       // [N] pixels queued for a jump, by slot
  uint32_t *n_queue;    // queue length
  int32_t *jump_k;      // [N] jump length in steps, by slot
  float *X;             // [N][7] network inputs, by slot
  const float *Y;       // [N][7] network outputs, by slot
  unsigned long long *stats;  // [2]: accepted, rejected jumps
  float box, s_max, log_tau2;
  float accel_bound;    // > 0: jumps only where the far-field bound holds; outputs scaled by it
  int k_min, cool_check;
  long long N;
};

// Riemannian illumination by one point light (rgeo_trace_lit): the light geodesics'
// step, budget and Gauss-Newton parameters, and the optional lit flags.
struct LightParams {
  float L[3];
  float h;
  int max_steps, iters;
  float tol, delta;
  int32_t *lit;    // optional [N]
  int list_steps;  // steps a lane's culled-sum list serves at step h (0: a cell per right-hand side)
  int per_lane;    // 1: each lane walks its own cell's list (no lockstep marches)
  int32_t *hits;       // [N] the hit list of the lockstep form (k_hit_list)
  uint32_t *n_hits;    // its length
  uint32_t *hit_next;  // the next unclaimed entry
};

// Instance table of a batch passed by value in the kernel's parameter space (CUDA
// allows 32 KB of parameters; 64 x 392 B = 24.5 KB fits).
constexpr int kMaxParamInstances = 64;
struct BatchTable {
  TraceParams inst[kMaxParamInstances];
};

// Process-wide launch tuning (set by rgeo_set_tuning, read at every trace).
struct Tuning {
  int rays_per_thread = 1;  // measured faster on GB300 at 64 bumps (occupancy beats shared traffic)
  int batch_params = 0;     // 0: parameter space when n <= kMaxParamInstances; 1: shared-memory copies
  int wait_limit = 0;       // tensor-core kernels' work waits: 0 default, n > 0 polls, -1 none (give up at once)
  int ctas_per_sm = 0;      // persistent trace grids: 0 as many as fit, else at most this many per SM
  int tile_lw = 2;          // refill tile width log2: 2 (4 x 8, default), 3 (8 x 4), 4 (16 x 2)
  int batch_order = 0;      // batch instances: 0 by decreasing cost, 1 as given
  int sum_lists = 0;        // culled sums: 0 one list per RK4 step where it applies, 1 one per right-hand side
  int refill = 0;           // 0: a warp takes new rays in generations of 32; 1: each lane as soon as it is free
};
Tuning &tuning();

// Sets the message rgeo_last_error() returns on this host thread.
void set_last_error(const char *msg);

// Host-side scene acceleration structures (rgeo_scene_build.cpp).
struct HostBVH {
  std::vector<float4> nodes;  // 2 per node
  std::vector<float4> prims;  // 3 per primitive (spheres, then triangles), BVH order
  int depth = 0;
};
bool build_bvh(const float *spheres, int n_spheres, const float *verts, int n_verts, const int32_t *tris,
               int n_tris, HostBVH &out, int max_depth);

struct HostGrid {
  std::vector<float> dist;
  int dim[3] = {0, 0, 0};
  float gmin[3] = {0, 0, 0};
  float cell = 1.0f;
  float smin[3] = {0, 0, 0}, smax[3] = {0, 0, 0};
};
void build_safe_grid(const float *spheres, int S, const float *verts, const int32_t *tris, int T,
                     int res, HostGrid &out);

constexpr int kMaxBvhDepth = 48;
constexpr int kTraversalStack = 64;

// Device error word bits (sticky, per device).
constexpr unsigned kErrStackOverflow = 1u;
constexpr unsigned kErrTimeout = 2u;

// Kernel launchers (rgeo_trace.cu).
cudaError_t launch_pack_bumps(const float *raw, int K, float cutoff, int aniso, const int32_t *perm, float4 *out,
                              cudaStream_t st);
cudaError_t launch_trace(const TraceParams &p, cudaStream_t st);
// Illumination pass over the hits of a finished trace p (p.hit_nrm filled by it).
cudaError_t launch_illuminate(const TraceParams &p, const LightParams &l, cudaStream_t st);
cudaError_t launch_set_centers(const float *c, int K, int aniso, const int32_t *perm, float4 *bumps, cudaStream_t st);
cudaError_t launch_build_cull(const float4 *bumps, int K, int G, int words, float reach, float4 *hdr, uint32_t *masks,
                              cudaStream_t st);
cudaError_t launch_batch(const TraceParams *dev_inst, const TraceParams *host_inst, int n, int kind, int aniso,
                         int integrator,
                         int max_table_f4, long long total_items, cudaStream_t st);
cudaError_t launch_advance_motion(const float *motion, int K, int aniso, const int32_t *perm, float *raw,
                                  float4 *bumps, float *t, float dt, cudaStream_t st);
cudaError_t launch_set_time(float *t, float value, cudaStream_t st);
cudaError_t launch_segments(const TraceParams &p, long long n, unsigned long long seed, float box, float s_max,
                            float accel_bound, float *X, float *T, cudaStream_t st);
// Surrogate tracer: one round of RK4 until each ray finishes or queues a jump, and
// the application of the network's jumps to the queued rays.
cudaError_t launch_wave_trace(const TraceParams &p, const WaveArgs &w, cudaStream_t st);
cudaError_t launch_wave_apply(const WaveArgs &w, unsigned n, float h, cudaStream_t st);
// rgeo_mlp.cu
cudaError_t launch_gemm_bf16(const void *A, const void *B, int M, int N, int K, int splits, const float *bias,
                             int mode, void *C, int ldc, void *ct, int ldt, cudaStream_t st);
cudaError_t read_and_clear_mlp_error(unsigned *word);
// Training batch of B rows sampled (counter-based) from n segments (stream-ordered).
cudaError_t launch_gather_batch(const float *X, const float *T, long long n, int B, unsigned long long seed,
                                long long step, float *Xb, float *Tb, cudaStream_t st);
// Surrogate forward pass over n rows of 7 inputs into n rows of 7 outputs (stream-ordered).
cudaError_t expmap_infer(const rgeo_expmap *x, const float *X, long long n, float *Y, cudaStream_t st);
cudaError_t read_and_clear_device_error(unsigned *word, cudaStream_t st);  // all three parts
cudaError_t read_and_clear_trace_error_1(unsigned *word, cudaStream_t st);
cudaError_t read_and_clear_trace_error_2(unsigned *word, cudaStream_t st);
cudaError_t read_and_clear_trace_error_3(unsigned *word, cudaStream_t st);
cudaError_t run_ffma_probe(int mode, float *tflops, float *ms);

}  // namespace rgeo
