// rgeo_trace.cu -- the geodesic ray-tracing kernels (sm_103a).
//
// One thread per ray, persistent blocks, rays handed out per warp from a global
// counter.  Each loop iteration advances a ray by one integration step of the
// geodesic flow (Eq. 3.3) and tests the new polygon segment against the scene
// (Section 4.1).  A lane whose ray terminates writes its pixel and takes the next
// ray in the same iteration, so warps stay full until the queue drains.
//
// Graph metric (Eq. 5.2) of f = b.x + 1/2 x^T A x + sum of Gaussian bumps (Eq. 6.1):
// Eq. 5.3 gives the acceleration of Eq. 5.4,
//     x'' = -(v^T Hess f v) / (1 + |grad f|^2) grad f,
// so per step only grad f and the scalar v^T Hess f v are summed over the bumps
// (Section 6, "Summing functions"); the full Hessian is never formed.
// Twist metric (Eq. 5.6, Section 5.2): Theorem 5.1 gives x'' = -J^-1 (v^T H(x_s) v)_s
// (Eq. 5.8) with J and the Hessians of the twist in closed form.
#include <cfloat>
#include <cstdint>
#include <cstring>

#include "rgeo_internal.h"

// This file is compiled three times (RGEO_TRACE_PART = 1, 2, 3), each time emitting one group
// of launchers and the kernels they instantiate, so that the parts compile in parallel:
//   1  single traces (k_trace and its variants) and the metric's table and grid kernels
//   2  batches (k_trace_batch)
//   3  the surrogate tracer, training segments and Riemannian illumination
#ifndef RGEO_TRACE_PART
#error "compile rgeo_trace.cu with -DRGEO_TRACE_PART=1, 2 or 3"
#endif
#define RGEO_PART(n) (RGEO_TRACE_PART == (n))
#define RGEO_PART_NAME_(base, n) base##n
#define RGEO_PART_NAME(base, n) RGEO_PART_NAME_(base, n)

namespace rgeo {

namespace {

__device__ unsigned int g_rgeo_error;  // sticky per-device error word of this part's kernels

constexpr int MK_GRAPH_ISO = 0;
constexpr int MK_GRAPH_ANISO = 1;
constexpr int MK_TWIST = 2;
constexpr int MK_LOCAL = 3;
constexpr int MK_GRAPH_SL = 4;  // isotropic graph metric whose culled sums take one list per RK4 step
__host__ __device__ constexpr bool is_iso(int mk) { return mk == MK_GRAPH_ISO || mk == MK_GRAPH_SL; }
constexpr float kLog2e = 1.4426950408889634f;
constexpr int kSegTries = 4096;  // candidates per training segment under a far-field bound

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct F3 {
  float x, y, z;
};
__device__ __forceinline__ F3 f3(float x, float y, float z) { return F3{x, y, z}; }
__device__ __forceinline__ F3 operator+(F3 a, F3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ F3 operator-(F3 a, F3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ F3 operator*(float s, F3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(F3 a, F3 b) { return fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)); }
__device__ __forceinline__ F3 cross(F3 a, F3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ F3 normalize(F3 a) { return rsqrtf(dot(a, a)) * a; }
__device__ __forceinline__ F3 axpy(float s, F3 a, F3 b) {  // s a + b
  return f3(fmaf(s, a.x, b.x), fmaf(s, a.y, b.y), fmaf(s, a.z, b.z));
}
__device__ __forceinline__ float comp(F3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

// (hi, lo) += d with an error-free TwoSum, kept out of FMA contraction.
__device__ __forceinline__ void comp_add(float &hi, float &lo, float d) {
  float y = __fadd_rn(d, lo);
  float t = __fadd_rn(hi, y);
  float bp = __fsub_rn(t, hi);
  float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(y, bp));
  hi = t;
  lo = e;
}

// ---------------------------------------------------------------- metrics

// grad f and -(v^T Hess f v) for the quadratic and affine part of f.
__device__ __forceinline__ void poly_terms(const TraceParams &P, F3 x, F3 v, float &gx, float &gy,
                                           float &gz, float &sn) {
  if (P.has_affine) {
    gx += P.b[0];
    gy += P.b[1];
    gz += P.b[2];
  }
  if (P.has_quad) {
    const float *A = P.A;
    F3 Ax = f3(A[0] * x.x + A[1] * x.y + A[2] * x.z, A[3] * x.x + A[4] * x.y + A[5] * x.z,
               A[6] * x.x + A[7] * x.y + A[8] * x.z);
    F3 Av = f3(A[0] * v.x + A[1] * v.y + A[2] * v.z, A[3] * v.x + A[4] * v.y + A[5] * v.z,
               A[6] * v.x + A[7] * v.y + A[8] * v.z);
    gx += Ax.x;
    gy += Ax.y;
    gz += Ax.z;
    sn -= dot(v, Av);
  }
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Per-lane work counters: evals, the bump terms of the cells of the lane's own rays (the
// counter bump_evals); slots, the bump terms the lane evaluated, every pair of its warp's
// lists included (bump_slots).  flush adds the warp's sums to the requested counters.
struct WorkCount {
  unsigned long long evals = 0ull;
  unsigned slots = 0u;  // per lane: well below 2^32 at every frame size here
  __device__ __forceinline__ void flush(const TraceParams &P) {
    if (P.bump_evals) {
      unsigned long long e = evals;
      for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
      if ((threadIdx.x & 31u) == 0) atomicAdd(P.bump_evals, e);
    }
    if (P.bump_slots) {
      unsigned long long e = slots;  // summed in 64 bits
      for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
      if ((threadIdx.x & 31u) == 0) atomicAdd(P.bump_slots, e);
    }
    evals = 0ull;
    slots = 0u;
  }
};

// Position and velocity of one ray, and its paired accumulators: the .x halves sum the
// even-numbered bumps, the .y halves the odd-numbered ones, each in increasing order.
struct PairAcc {
  float x, y, z;
  float2 VX, VY, VZ, NVV;
  float2 gx, gy, gz, sn;
  bool in;
};

__device__ __forceinline__ void pair_acc_init(PairAcc &a, F3 x, F3 v) {
  const float vv = dot(v, v);
  a.x = x.x; a.y = x.y; a.z = x.z;
  a.VX = f2(v.x, v.x); a.VY = f2(v.y, v.y); a.VZ = f2(v.z, v.z); a.NVV = f2(-vv, -vv);
  a.gx = a.gy = a.gz = a.sn = f2(0.f, 0.f);
  a.in = false;
}

// Adds the bumps whose table entries start at float4 i0 (an even-numbered bump, or the
// pad) and i1 (an odd-numbered bump, or the pad): grad f and -v^T Hess f v of Eq. 6.1,
// one paired-FP32 half each.  A bump whose truncated support misses x adds exactly zero.
template <bool INSIDE>
__device__ __forceinline__ void pair_eval(PairAcc &a, const float4 *__restrict__ sb, int i0, int i1) {
  const float4 A0 = sb[i0], B0 = sb[i0 + 1], A1 = sb[i1], B1 = sb[i1 + 1];
  const float2 dx = f2(a.x + A0.x, a.x + A1.x);
  const float2 dy = f2(a.y + A0.y, a.y + A1.y);
  const float2 dz = f2(a.z + A0.z, a.z + A1.z);
  float2 r2 = __fmul2_rn(dx, dx);
  r2 = __ffma2_rn(dy, dy, r2);
  r2 = __ffma2_rn(dz, dz, r2);
  const float w0 = ex2_approx(fmaf(r2.x, B0.x, B0.y)), w1 = ex2_approx(fmaf(r2.y, B1.x, B1.y));
  const bool in0 = r2.x < A0.w, in1 = r2.y < A1.w;
  if (INSIDE) a.in |= in0 | in1;
  const float2 g = f2(in0 ? w0 * B0.z : 0.f, in1 ? w1 * B1.z : 0.f);  // -a q e
  a.gx = __ffma2_rn(g, dx, a.gx);
  a.gy = __ffma2_rn(g, dy, a.gy);
  a.gz = __ffma2_rn(g, dz, a.gz);
  float2 dv = __fmul2_rn(dx, a.VX);
  dv = __ffma2_rn(dy, a.VY, dv);
  dv = __ffma2_rn(dz, a.VZ, dv);
  const float2 t = __ffma2_rn(f2(dv.x * B0.w, dv.y * B1.w), dv, a.NVV);  // q (d.v)^2 - |v|^2
  a.sn = __ffma2_rn(g, t, a.sn);                                          // -v^T Hess f v
}

// Eq. 5.4 from the accumulated sums (plus the affine and quadratic part of f).
__device__ __forceinline__ F3 pair_acc_finish(const TraceParams &P, const PairAcc &a, F3 x, F3 v) {
  float sgx = a.gx.x + a.gx.y, sgy = a.gy.x + a.gy.y, sgz = a.gz.x + a.gz.y, ssn = a.sn.x + a.sn.y;
  poly_terms(P, x, v, sgx, sgy, sgz, ssn);
  // the denominator 1 + |grad f|^2 is >= 1, so the fast division is accurate to 2 ulp
  const float coef = __fdividef(ssn, fmaf(sgz, sgz, fmaf(sgy, sgy, fmaf(sgx, sgx, 1.f))));
  return f3(coef * sgx, coef * sgy, coef * sgz);
}

// Adds packed pair i of a step list (layout in WarpLists): the same sums as pair_eval on
// the pair's two bumps, with every operation on both halves at once.
template <bool INSIDE>
__device__ __forceinline__ void pair_eval_packed(PairAcc &a, const float4 *__restrict__ pk, int i) {
  const float4 p0 = pk[4 * i], p1 = pk[4 * i + 1], p2 = pk[4 * i + 2], p3 = pk[4 * i + 3];
  const float2 dx = __fadd2_rn(f2(a.x, a.x), f2(p0.x, p0.y));
  const float2 dy = __fadd2_rn(f2(a.y, a.y), f2(p0.z, p0.w));
  const float2 dz = __fadd2_rn(f2(a.z, a.z), f2(p1.x, p1.y));
  float2 r2 = __fmul2_rn(dx, dx);
  r2 = __ffma2_rn(dy, dy, r2);
  r2 = __ffma2_rn(dz, dz, r2);
  const float2 arg = __ffma2_rn(r2, f2(p2.x, p2.y), f2(p2.z, p2.w));
  float w0 = ex2_approx(arg.x), w1 = ex2_approx(arg.y);
  const bool in0 = r2.x < p1.z, in1 = r2.y < p1.w;
  if (INSIDE) a.in |= in0 | in1;
  w0 = in0 ? w0 : 0.f;
  w1 = in1 ? w1 : 0.f;
  const float2 g = __fmul2_rn(f2(w0, w1), f2(p3.x, p3.y));  // -a q e
  a.gx = __ffma2_rn(g, dx, a.gx);
  a.gy = __ffma2_rn(g, dy, a.gy);
  a.gz = __ffma2_rn(g, dz, a.gz);
  float2 dv = __fmul2_rn(dx, a.VX);
  dv = __ffma2_rn(dy, a.VY, dv);
  dv = __ffma2_rn(dz, a.VZ, dv);
  const float2 t = __ffma2_rn(__fmul2_rn(dv, f2(p3.z, p3.w)), dv, a.NVV);  // q (d.v)^2 - |v|^2
  a.sn = __ffma2_rn(g, t, a.sn);                                           // -v^T Hess f v
}

// Eq. 5.4 over all isotropic bumps in shared memory, bumps 2i and 2i + 1 together (the
// table layout is described in rgeo_internal.h).  With INSIDE, also reports whether x
// lies in some truncated support (the flat-skip test).
template <bool INSIDE>
__device__ __forceinline__ F3 accel_graph_iso(const TraceParams &P, const float4 *__restrict__ sb, int K, F3 x,
                                              F3 v, bool &inside) {
  PairAcc a;
  pair_acc_init(a, x, v);
  const int n4 = kIsoBumpStride * iso_pad_index(K);
#pragma unroll 2
  for (int i = 0; i < n4; i += 2 * kIsoBumpStride) pair_eval<INSIDE>(a, sb, i, i + kIsoBumpStride);
  if (INSIDE) inside = a.in;
  return pair_acc_finish(P, a, x, v);
}

// The warp's bump lists in shared memory (culled sums).  idx holds index pairs: x the
// float4 index of an even-numbered bump, y of an odd-numbered one (the pad bump fills a
// missing partner), so that every lane's sums take its own bumps in the order of the dense
// sums (the .x halves the even ones, the .y halves the odd ones, each in increasing
// order) and the result is the same whatever else the warp evaluates.  pk, when present,
// holds the pairs of a step list packed for pair_eval_packed, four float4 per pair:
//   (-cx_e, -cx_o, -cy_e, -cy_o), (-cz_e, -cz_o, R2_e, R2_o), (qn2_e, qn2_o, la_e, la_o),
//   (qs_e, qs_o, q_e, q_o)
// for the even bump e and the odd bump o of the pair.  np (the same on every lane) is the
// number of packed pairs of the current step, or -1 when each right-hand side looks up
// its own cells; own (per lane) counts the bumps of the lane's own cell in the step list;
// age (the same on every lane) counts the steps the list has served since it was built.
struct WarpLists {
  int2 *idx;   // [kListPairs]
  float4 *pk;  // [4 * kListPairs], or null: no step lists
  int np;
  unsigned own;
  int age;
};

// Lists the union of the participating lanes' cell masks, even-numbered bumps in idx[.].x
// and odd-numbered ones in idx[.].y, starting at column counts ne and no; called by all 32
// lanes with the same word.  Returns the lane's own bump count of the word.
__device__ __forceinline__ unsigned list_word(int2 *idx, unsigned m, int wi, int &ne, int &no) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned below = (1u << lane) - 1u;
  const unsigned u = __reduce_or_sync(0xffffffffu, m);
  const unsigned ue = u & 0x55555555u, uo = u & 0xaaaaaaaau;
  if ((u >> lane) & 1u) {
    const int k4 = kIsoBumpStride * ((wi << 5) + (int)lane);
    if (lane & 1u) idx[no + __popc(uo & below)].y = k4;
    else idx[ne + __popc(ue & below)].x = k4;
  }
  ne += __popc(ue);
  no += __popc(uo);
  return (unsigned)__popc(m);
}

// Gives the shorter column of idx[0 .. max(ne, no)) the pad bump; returns the pair count.
__device__ __forceinline__ int list_pad(int2 *idx, int ne, int no, int pad) {
  const int nmin = min(ne, no), nmax = max(ne, no);
  for (int i = nmin + (int)(threadIdx.x & 31u); i < nmax; i += 32) {
    if (ne < no) idx[i].x = pad;
    else idx[i].y = pad;
  }
  return nmax;
}

// Cell-grid index of x, or -1 outside the grid.
__device__ __forceinline__ long long cull_cell(const TraceParams &P, float4 ghdr, F3 x) {
  const int G = P.cull_G;
  const float fx = (x.x - ghdr.x) * ghdr.w, fy = (x.y - ghdr.y) * ghdr.w, fz = (x.z - ghdr.z) * ghdr.w;
  if (!(fx >= 0.f && fy >= 0.f && fz >= 0.f && fx < (float)G && fy < (float)G && fz < (float)G)) return -1;
  return ((long long)(int)fz * G + (int)fy) * G + (int)fx;
}

// The step list (all 32 lanes together): the union of the cells of the participating
// lanes' positions x, listed and packed into the warp's pk.  The cull grid's supports are
// inflated by the metric's reach margin, which bounds the distance from x to every RK4 stage
// point of the next P.list_steps steps (the launcher checks that), so the list holds every
// bump that can be nonzero at any of their stages.  A union beyond the list's capacity leaves np = -1
// (the dense sums).
__device__ __forceinline__ void step_list(const TraceParams &P, const float4 *__restrict__ sb, WarpLists &wl,
                                          float4 ghdr, bool part, F3 x) {
  const long long cell = part ? cull_cell(P, ghdr, x) : -1;
  const uint32_t *cm = P.cull_masks + (cell >= 0 ? cell * P.cull_words : 0);
  int ne = 0, no = 0;
  unsigned own = 0;
  bool full = false;
  unsigned mnext = cell >= 0 ? __ldg(cm) : 0u;
  __syncwarp();  // the previous lists have been read by every lane
  for (int wi = 0; wi < P.cull_words; ++wi) {
    const unsigned m = mnext;
    if (wi + 1 < P.cull_words) mnext = cell >= 0 ? __ldg(cm + wi + 1) : 0u;
    own += list_word(wl.idx, m, wi, ne, no);
    if (max(ne, no) > kListPairs - 16) {  // a further word could overflow a column
      full = wi + 1 < P.cull_words;
      if (full) break;
    }
  }
  wl.own = own;
  wl.age = 0;
  if (full) {
    wl.np = -1;
    return;
  }
  const int np = list_pad(wl.idx, ne, no, kIsoBumpStride * iso_pad_index(P.K));
  __syncwarp();
  for (int t = (int)(threadIdx.x & 31u); t < 4 * np; t += 32) {
    const int2 e = wl.idx[t >> 2];
    const int half = (t >> 1) & 1;  // float4 0, 1 from A, 2, 3 from B
    const float4 a = sb[e.x + half], b = sb[e.y + half];
    wl.pk[t] = (t & 1) == 0 ? make_float4(a.x, b.x, a.y, b.y) : make_float4(a.z, b.z, a.w, b.w);
  }
  __syncwarp();
  wl.np = np;
}

// Keeps the warp's step list while it still covers every lane (it has served fewer than
// P.list_steps steps and no lane took a new ray, fresh), else lists afresh at the lanes' x.
__device__ __forceinline__ void step_list_refresh(const TraceParams &P, const float4 *__restrict__ sb,
                                                  WarpLists &wl, float4 ghdr, bool part, bool fresh, F3 x) {
  if (!P.step_lists) {
    wl.np = -1;
    return;
  }
  if (wl.np >= 0 && wl.age < P.list_steps && !__any_sync(0xffffffffu, fresh)) return;
  step_list(P, sb, wl, ghdr, part, x);
}

// Eq. 5.4 over the packed pairs of the warp's step list (every lane together or not: no
// collective).  UNROLL takes four pairs per iteration: 1.7 % faster for the dense sums over
// the block's packed table, slower for the short step lists (1.7 %) and the illumination (11 %).
template <bool INSIDE, bool UNROLL = false>
__device__ __forceinline__ F3 accel_step_list(const TraceParams &P, const WarpLists &wl, F3 x, F3 v, bool &inside) {
  PairAcc a;
  pair_acc_init(a, x, v);
  if constexpr (UNROLL) {
#pragma unroll 4
    for (int i = 0; i < wl.np; ++i) pair_eval_packed<INSIDE>(a, wl.pk, i);
  } else {
    for (int i = 0; i < wl.np; ++i) pair_eval_packed<INSIDE>(a, wl.pk, i);
  }
  if (INSIDE) inside = a.in;
  return pair_acc_finish(P, a, x, v);
}

// Culled form with a list per right-hand side, called by all 32 lanes of a warp together:
// each participating lane looks up the cull-grid cell of x, the warp lists the union of
// the cells' masks and evaluates it in lockstep.  Bumps outside the union have supports
// that miss every participating lane's cell, so they add exactly zero there.  A long union
// is evaluated in parts as the list fills.  evals counts the bumps of the lane's own cell.
template <bool INSIDE>
__device__ __forceinline__ F3 accel_graph_iso_culled(const TraceParams &P, const float4 *__restrict__ sb,
                                                     int2 *lst, float4 ghdr, bool part, F3 x, F3 v,
                                                     bool &inside, WorkCount &wc) {
  PairAcc a;
  pair_acc_init(a, x, v);
  const int words = P.cull_words;
  const int pad = kIsoBumpStride * iso_pad_index(P.K);
  const long long cell = part ? cull_cell(P, ghdr, x) : -1;
  const uint32_t *cm = P.cull_masks + (cell >= 0 ? cell * words : 0);
  int ne = 0, no = 0;  // entries in the even and odd columns of the list (the same on every lane)
  // word wi + 1 of the cell's mask is loaded while word wi is listed
  unsigned mnext = cell >= 0 ? __ldg(cm) : 0u;
  __syncwarp();  // the previous list has been read by every lane
  for (int wi = 0; wi < words; ++wi) {
    const unsigned m = mnext;
    if (wi + 1 < words) mnext = cell >= 0 ? __ldg(cm + wi + 1) : 0u;
    wc.evals += list_word(lst, m, wi, ne, no);  // the bumps of this lane's own cell
    if (max(ne, no) > kListPairs - 16 || wi + 1 == words) {  // full (a word adds up to 16 a column) or done
      const int np = list_pad(lst, ne, no, pad);
      wc.slots += 2u * (unsigned)np;
      __syncwarp();
      for (int i = 0; i < np; ++i) {
        const int2 e = lst[i];
        pair_eval<INSIDE>(a, sb, e.x, e.y);
      }
      __syncwarp();
      ne = no = 0;
    }
  }
  if (INSIDE) inside = a.in;
  return pair_acc_finish(P, a, x, v);
}

// One bump of the isotropic table: centre, R2 and the exponent/scale constants.
struct IsoBump {
  F3 c;
  float R2, qn2, la, qs, q;
};
__device__ __forceinline__ IsoBump iso_bump(const float4 *sb, int k) {
  const float4 A = sb[kIsoBumpStride * k], B = sb[kIsoBumpStride * k + 1];
  IsoBump b;
  b.c = f3(-A.x, -A.y, -A.z);
  b.R2 = A.w; b.qn2 = B.x; b.la = B.y; b.qs = B.z; b.q = B.w;
  return b;
}

// Far-field certificate: an upper bound on |x''| (Eq. 5.4) along every path of
// Euclidean length <= s from x, for a g-unit tangent (|v| <= 1 because g >= I).
// |x''| = |v^T Hess f v| t / (1 + t^2) with t = |grad f|, and t / (1 + t^2) <=
// min(t, 1/2).  Per bump of Eq. 6.1 at distance r, |grad f_k| = |a| q r e^{-q r^2/2}
// and ||Hess f_k|| <= |a| q (1 + q r^2) e^{-q r^2/2}; both are non-increasing in r
// once q r^2 >= 1, so they are taken at r^2 = max(rho^2, 1/q) with rho = max(0,
// |x - c| - s), the nearest the path can come.  A bump whose truncated support the
// path cannot reach adds nothing.  Isotropic bumps without polynomial part only.
__device__ float far_field_bound(const float4 *sb, int K, F3 x, float s) {
  float Hb = 0.f, Gb = 0.f;
  for (int k = 0; k < K; ++k) {
    const IsoBump b = iso_bump(sb, k);
    if (b.R2 < 0.f) continue;  // inert (a = 0)
    const F3 d = x - b.c;
    const float rho = fmaxf(sqrtf(dot(d, d)) - s, 0.f);
    if (rho * rho >= b.R2) continue;
    const float u = fmaxf(b.q * rho * rho, 1.f);
    const float e = b.q * exp2f(fmaf(-0.5f * kLog2e, u, b.la));  // |a| q e^{-u/2}
    Gb = fmaf(e, sqrtf(u / b.q), Gb);
    Hb = fmaf(e, 1.f + u, Hb);
  }
  return Hb * fminf(Gb, 0.5f) * 1.0001f;  // slack for float32 rounding
}

template <bool INSIDE>
__device__ __forceinline__ F3 accel_graph_aniso(const TraceParams &P, const float4 *__restrict__ sb,
                                                int K, F3 x, F3 v, bool &inside) {
  float gx = 0.f, gy = 0.f, gz = 0.f, sn = 0.f;
  bool in = false;
  for (int k = 0; k < K; ++k) {
    const float4 b0 = sb[3 * k], b1 = sb[3 * k + 1], b2 = sb[3 * k + 2];
    const float dx = x.x - b0.x, dy = x.y - b0.y, dz = x.z - b0.z;
    const float u = fmaf(b1.z * dz, dz, fmaf(b1.y * dy, dy, b1.x * dx * dx));
    float w = ex2_approx(fmaf(u, -0.5f * kLog2e, b2.x));
    const bool p = u < b2.y;
    if (INSIDE) in |= fmaf(dz, dz, fmaf(dy, dy, dx * dx)) < b0.w;
    w = p ? w : 0.f;
    const float e = b1.w * w;  // a exp(-u/2)
    gx = fmaf(-e * b1.x, dx, gx);
    gy = fmaf(-e * b1.y, dy, gy);
    gz = fmaf(-e * b1.z, dz, gz);
    const float qdv = fmaf(b1.z * dz, v.z, fmaf(b1.y * dy, v.y, b1.x * dx * v.x));
    const float qvv = fmaf(b1.z * v.z, v.z, fmaf(b1.y * v.y, v.y, b1.x * v.x * v.x));
    sn = fmaf(-e, fmaf(qdv, qdv, -qvv), sn);
  }
  poly_terms(P, x, v, gx, gy, gz, sn);
  const float coef = sn / fmaf(gz, gz, fmaf(gy, gy, fmaf(gx, gx, 1.f)));
  if (INSIDE) inside = in;
  return f3(coef * gx, coef * gy, coef * gz);
}

// Eq. 5.8 for the twist: x'' = -J^-1 (v^T H_1 v, v^T H_2 v, 0).
__device__ __forceinline__ F3 accel_twist(float k, F3 x, F3 v) {
  float s, c;
  sincosf(k * x.z, &s, &c);
  const float X = c * x.x - s * x.y, Y = s * x.x + c * x.y;
  const float kvz = k * v.z;
  const float q1 = -2.f * kvz * (s * v.x + c * v.y) - kvz * kvz * X;
  const float q2 = 2.f * kvz * (c * v.x - s * v.y) - kvz * kvz * Y;
  return f3(-(c * q1 + s * q2), -(c * q2 - s * q1), 0.f);
}

// Per-launch context of the bump sums: the cull-grid header and the lanes that
// take part in the current call (for the warp-wide mask reduction).
// ------------------------------------------------------- local maps
// One local map of Section 6 ("Using diffeomorphism"): Phi(p) = p + f(p) V(p), f the
// Gaussian of Eq. 6.1 (isotropic, untruncated), V(p) = v + B (p - c).  local_push moves
// the 2-jet of a curve through it -- y <- Phi(y), u <- J u, w <- J w + D^2 Phi[u, u] (the
// Hessian of a composition, Eq. 6.3, taken along u) -- and the Jacobian product M <- J M
// (the chain rule of Section 6, "Composing diffeomorphisms"), with
//   J z = z + V (grad f . z) + f B z,  D^2 Phi[u, u] = V (u^T Hess f u) + 2 (grad f . u) B u,
//   grad f = -q f d,  u^T Hess f u = q f (q (d . u)^2 - |u|^2),  d = y - c.
struct Jet {
  F3 y, u, w;
  float M[9];  // row-major: M[3 s + j] = d_j (x_s)
};

__device__ __forceinline__ void local_push(const float4 *__restrict__ sb, int k, Jet &j, bool second) {
  const float4 t0 = sb[kLocalStride * k], t1 = sb[kLocalStride * k + 1], t2 = sb[kLocalStride * k + 2],
               t3 = sb[kLocalStride * k + 3], t4 = sb[kLocalStride * k + 4];
  const F3 d = j.y - f3(t0.x, t0.y, t0.z);
  const float f = t0.w * ex2_approx(t1.w * dot(d, d));
  const float q = t2.w;
  const float mqf = -q * f;
  const F3 gr = mqf * d;
  const bool field = t3.w != 0.f;
  const F3 B0 = f3(t2.x, t2.y, t2.z), B1 = f3(t3.x, t3.y, t3.z), B2 = f3(t4.x, t4.y, t4.z);
  F3 V = f3(t1.x, t1.y, t1.z);
  if (field) V = V + f3(dot(B0, d), dot(B1, d), dot(B2, d));
  for (int c = 0; c < 3; ++c) {
    const F3 col = f3(j.M[c], j.M[3 + c], j.M[6 + c]);
    F3 nc = axpy(dot(gr, col), V, col);
    if (field) nc = axpy(f, f3(dot(B0, col), dot(B1, col), dot(B2, col)), nc);
    j.M[c] = nc.x;
    j.M[3 + c] = nc.y;
    j.M[6 + c] = nc.z;
  }
  if (second) {
    const float du = dot(d, j.u);
    const float hq = q * f * fmaf(q * du, du, -dot(j.u, j.u));  // u^T Hess f u
    const float gu = mqf * du;                                  // grad f . u
    F3 w = axpy(dot(gr, j.w) + hq, V, j.w);
    F3 u = axpy(gu, V, j.u);
    if (field) {
      const F3 Bu = f3(dot(B0, j.u), dot(B1, j.u), dot(B2, j.u));
      const F3 Bw = f3(dot(B0, j.w), dot(B1, j.w), dot(B2, j.w));
      w = axpy(2.f * gu, Bu, axpy(f, Bw, w));
      u = axpy(f, Bu, u);
    }
    j.w = w;
    j.u = u;
  }
  j.y = axpy(f, V, j.y);
}

// Jacobian of the composition Phi = Phi_1 o ... o Phi_K at x (map K - 1 acts first).
__device__ __forceinline__ void local_jacobian(const float4 *sb, int K, F3 x, Jet &j) {
  j.y = x;
  j.u = j.w = f3(0.f, 0.f, 0.f);
  for (int i = 0; i < 9; ++i) j.M[i] = (i % 4 == 0) ? 1.f : 0.f;
  for (int k = K - 1; k >= 0; --k) local_push(sb, k, j, false);
}

// x'' = -J^-1 D^2 Phi[v, v]: Theorem 5.1 (Gamma^m_ij v_i v_j = sum_s [J^-1]_ms v^T H(x_s) v)
// for the composition, with J^-1 w from the adjugate (columns r1 x r2, r2 x r0, r0 x r1 of
// the rows r_s of J, over det J).
__device__ __forceinline__ F3 accel_local(const float4 *sb, int K, F3 x, F3 v) {
  Jet j;
  j.y = x;
  j.u = v;
  j.w = f3(0.f, 0.f, 0.f);
  for (int i = 0; i < 9; ++i) j.M[i] = (i % 4 == 0) ? 1.f : 0.f;
  for (int k = K - 1; k >= 0; --k) local_push(sb, k, j, true);
  const F3 r0 = f3(j.M[0], j.M[1], j.M[2]), r1 = f3(j.M[3], j.M[4], j.M[5]), r2 = f3(j.M[6], j.M[7], j.M[8]);
  const F3 c0 = cross(r1, r2), c1 = cross(r2, r0), c2 = cross(r0, r1);
  const float inv = -1.f / dot(r0, c0);
  return inv * axpy(j.w.x, c0, axpy(j.w.y, c1, j.w.z * c2));
}

// |J v|^2 in FP64 for the drift diagnostic (Eq. 5.6: g = J^T J).
__device__ double local_energy(const float4 *sb, int K, F3 x, F3 v) {
  double y[3] = {x.x, x.y, x.z}, M[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  for (int k = K - 1; k >= 0; --k) {
    const float4 t0 = sb[kLocalStride * k], t1 = sb[kLocalStride * k + 1], t2 = sb[kLocalStride * k + 2],
                 t3 = sb[kLocalStride * k + 3], t4 = sb[kLocalStride * k + 4];
    const double d[3] = {y[0] - t0.x, y[1] - t0.y, y[2] - t0.z};
    const double q = t2.w, f = t0.w * exp(-0.5 * q * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
    const double B[9] = {t2.x, t2.y, t2.z, t3.x, t3.y, t3.z, t4.x, t4.y, t4.z};
    double V[3], gr[3], N[9];
    for (int s = 0; s < 3; ++s) {
      V[s] = (double)(s == 0 ? t1.x : (s == 1 ? t1.y : t1.z)) + B[3 * s] * d[0] + B[3 * s + 1] * d[1] +
             B[3 * s + 2] * d[2];
      gr[s] = -q * f * d[s];
    }
    for (int s = 0; s < 3; ++s)
      for (int c = 0; c < 3; ++c) {
        double acc = M[3 * s + c] + V[s] * (gr[0] * M[c] + gr[1] * M[3 + c] + gr[2] * M[6 + c]);
        acc += f * (B[3 * s] * M[c] + B[3 * s + 1] * M[3 + c] + B[3 * s + 2] * M[6 + c]);
        N[3 * s + c] = acc;
      }
    for (int i = 0; i < 9; ++i) M[i] = N[i];
    for (int s = 0; s < 3; ++s) y[s] += f * V[s];
  }
  double e = 0.0;
  for (int s = 0; s < 3; ++s) {
    const double r = M[3 * s] * v.x + M[3 * s + 1] * v.y + M[3 * s + 2] * v.z;
    e += r * r;
  }
  return e;
}

// Context of one right-hand-side evaluation.  For the isotropic graph metric (kConverged)
// every lane of the warp calls together, and part says whether this lane's sums are
// wanted; the other kinds are called by the lanes that hold a ray only.
struct SumCtx {
  float4 ghdr;                // cull-grid header (culled sums)
  WarpLists *wl;              // the warp's lists in shared memory (culled sums)
  bool part;                  // this lane's ray needs the sums
  WorkCount *evals;           // per-lane work counters
};

template <int MK>
struct Converged {
  static constexpr bool value = is_iso(MK);
};

template <int MK, bool INSIDE>
__device__ __forceinline__ F3 accel(const TraceParams &P, const float4 *sb, const SumCtx &cx, F3 x, F3 v,
                                    bool &inside) {
  if (MK == MK_GRAPH_SL) {  // the warp's step list; the dense sums where there is none
    if (cx.wl->np >= 0) {
      if (cx.part) cx.evals->evals += cx.wl->own;
      cx.evals->slots += 2u * (unsigned)cx.wl->np;
      return accel_step_list<INSIDE>(P, *cx.wl, x, v, inside);
    }
    if (cx.part) cx.evals->evals += (unsigned)P.K;
    cx.evals->slots += (unsigned)iso_pad_index(P.K);
    return accel_graph_iso<INSIDE>(P, sb, P.K, x, v, inside);
  }
  if (MK == MK_GRAPH_ISO) {
    if (P.cull_masks)
      return accel_graph_iso_culled<INSIDE>(P, sb, cx.wl->idx, cx.ghdr, cx.part, x, v, inside, *cx.evals);
    if (cx.part) cx.evals->evals += (unsigned)P.K;
    cx.evals->slots += (unsigned)iso_pad_index(P.K);
    // the block's packed table (k_trace) or the table itself: the same sums in the same order
    if (cx.wl->pk) return accel_step_list<INSIDE, true>(P, *cx.wl, x, v, inside);
    return accel_graph_iso<INSIDE>(P, sb, P.K, x, v, inside);
  }
  if (MK == MK_GRAPH_ANISO) {
    cx.evals->evals += (unsigned)P.K;
    cx.evals->slots += (unsigned)P.K;
    return accel_graph_aniso<INSIDE>(P, sb, P.K, x, v, inside);
  }
  if (MK == MK_LOCAL) return accel_local(sb, P.K, x, v);
  return accel_twist(P.twist_k, x, v);
}

// grad f at x (graph metrics), for the g-unit initial tangent and the drift diagnostic.
template <int MK>
__device__ F3 grad_f(const TraceParams &P, const float4 *sb, F3 x) {
  float gx = 0.f, gy = 0.f, gz = 0.f, sn = 0.f;
  for (int k = 0; k < P.K; ++k) {
    float4 b0, b1, b2;
    float dx, dy, dz, u;
    if (is_iso(MK)) {
      const IsoBump b = iso_bump(sb, k);
      dx = x.x - b.c.x; dy = x.y - b.c.y; dz = x.z - b.c.z;
      u = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      const float w = u < b.R2 ? ex2_approx(fmaf(u, b.qn2, b.la)) : 0.f;
      gx = fmaf(w * b.qs, dx, gx);
      gy = fmaf(w * b.qs, dy, gy);
      gz = fmaf(w * b.qs, dz, gz);
    } else {
      b0 = sb[3 * k];
      b1 = sb[3 * k + 1];
      b2 = sb[3 * k + 2];
      dx = x.x - b0.x; dy = x.y - b0.y; dz = x.z - b0.z;
      u = fmaf(b1.z * dz, dz, fmaf(b1.y * dy, dy, b1.x * dx * dx));
      const float e = u < b2.y ? b1.w * ex2_approx(fmaf(u, -0.5f * kLog2e, b2.x)) : 0.f;
      gx = fmaf(-e * b1.x, dx, gx);
      gy = fmaf(-e * b1.y, dy, gy);
      gz = fmaf(-e * b1.z, dz, gz);
    }
  }
  poly_terms(P, x, f3(0.f, 0.f, 0.f), gx, gy, gz, sn);
  return f3(gx, gy, gz);
}

// g_x(v, v) in FP64 (Eq. 3.1 with Eq. 5.2 or Eq. 5.6); used only by the drift diagnostic.
template <int MK>
__device__ double energy(const TraceParams &P, const float4 *sb, F3 x, F3 v) {
  if (MK == MK_LOCAL) return local_energy(sb, P.K, x, v);
  if (MK == MK_TWIST) {
    const float k = P.twist_k;
    float s, c;
    sincosf(k * x.z, &s, &c);
    const double X = (double)c * x.x - (double)s * x.y, Y = (double)s * x.x + (double)c * x.y;
    const double j0 = (double)c * v.x - (double)s * v.y - k * Y * v.z;
    const double j1 = (double)s * v.x + (double)c * v.y + k * X * v.z;
    return j0 * j0 + j1 * j1 + (double)v.z * v.z;
  }
  const F3 g = grad_f<MK>(P, sb, x);
  const double gv = (double)g.x * v.x + (double)g.y * v.y + (double)g.z * v.z;
  return (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z + gv * gv;
}

// ---------------------------------------------------------- intersection

struct HitRec {
  float s;
  int id;   // sphere index or S + original triangle index
  int tq;   // triangle slot in BVH order (for the normal), -1 for spheres
};

// Segment O + s D, s in [0, smax), against a sphere; a segment that starts
// inside or on the sphere hits it at s = 0.  The discriminant is formed from the
// perpendicular offset of the centre, which keeps it accurate for short segments.
__device__ __forceinline__ bool hit_sphere(F3 O, F3 D, float dd, float4 sp, float &s) {
  const F3 oc = f3(O.x - sp.x, O.y - sp.y, O.z - sp.z);
  const float r2 = sp.w * sp.w;
  const float cc = dot(oc, oc) - r2;
  if (cc <= 0.f) {
    s = 0.f;
    return true;
  }
  const float b = dot(oc, D);
  if (b >= 0.f) return false;
  const float ba = b / dd;
  const F3 l = f3(fmaf(-ba, D.x, oc.x), fmaf(-ba, D.y, oc.y), fmaf(-ba, D.z, oc.z));
  const float disc = r2 - dot(l, l);
  if (disc < 0.f) return false;
  const float q = sqrtf(dd * disc) - b;  // > 0
  s = cc / q;
  return true;
}

// Ray-space frame of the watertight triangle test (Woop, Benthin and Wald, JCGT 2013).
struct WFrame {
  int kx, ky, kz;
  float Sx, Sy, Sz;
};

__device__ __forceinline__ WFrame make_frame(F3 D) {
  const float ax = fabsf(D.x), ay = fabsf(D.y), az = fabsf(D.z);
  int kz = 0;
  if (ay > ax) kz = 1;
  if (az > fmaxf(ax, ay)) kz = 2;
  int kx = kz == 2 ? 0 : kz + 1, ky = kx == 2 ? 0 : kx + 1;
  const float dz = comp(D, kz);
  if (dz < 0.f) {
    int t = kx;
    kx = ky;
    ky = t;
  }
  WFrame f;
  f.kx = kx;
  f.ky = ky;
  f.kz = kz;
  f.Sx = comp(D, kx) / dz;
  f.Sy = comp(D, ky) / dz;
  f.Sz = 1.f / dz;
  return f;
}

// Watertight segment-triangle test: returns the segment parameter in [0, smax) or -1.
// The 2D edge functions are formed without FMA contraction so that a shared edge
// yields exactly opposite values in its two triangles.
__device__ __forceinline__ float hit_triangle(const WFrame &f, F3 O, float smax, float4 a4, float4 b4,
                                              float4 c4) {
  const F3 A = f3(a4.x - O.x, a4.y - O.y, a4.z - O.z);
  const F3 B = f3(b4.x - O.x, b4.y - O.y, b4.z - O.z);
  const F3 C = f3(c4.x - O.x, c4.y - O.y, c4.z - O.z);
  const float Akz = comp(A, f.kz), Bkz = comp(B, f.kz), Ckz = comp(C, f.kz);
  const float Ax = comp(A, f.kx) - f.Sx * Akz, Ay = comp(A, f.ky) - f.Sy * Akz;
  const float Bx = comp(B, f.kx) - f.Sx * Bkz, By = comp(B, f.ky) - f.Sy * Bkz;
  const float Cx = comp(C, f.kx) - f.Sx * Ckz, Cy = comp(C, f.ky) - f.Sy * Ckz;
  const float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
  const float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
  const float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
  if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return -1.f;
  const float det = U + V + W;
  if (det == 0.f) return -1.f;
  const float T = U * (f.Sz * Akz) + V * (f.Sz * Bkz) + W * (f.Sz * Ckz);
  const float s = __fdiv_rn(T, det);
  return (s >= 0.f && s < smax) ? s : -1.f;
}

// Earliest hit of O + s D, s in [0, smax), against the scene.  With a BVH, spheres
// and triangles are found through it; without one (scenes passed as bare sphere
// arrays), every sphere in shared memory is tested.  Ties: smaller s, then lower
// id (spheres come before triangles).
__device__ bool scene_hit(const TraceParams &P, const float4 *ss, F3 O, F3 D, float smax,
                          HitRec &hr) {
  hr.id = -1;
  hr.tq = -1;
  hr.s = smax;
  const float dd = dot(D, D);
  if (P.nodes == nullptr) {
    for (int k = 0; k < P.S; ++k) {
      float s;
      if (hit_sphere(O, D, dd, ss[k], s) && s < smax && (hr.id < 0 || s < hr.s)) {
        hr.s = s;
        hr.id = k;
      }
    }
    return hr.id >= 0;
  }
  const WFrame fr = make_frame(D);
  const F3 inv = f3(1.f / (D.x != 0.f ? D.x : 1e-30f), 1.f / (D.y != 0.f ? D.y : 1e-30f),
                    1.f / (D.z != 0.f ? D.z : 1e-30f));
  int stack[kTraversalStack];
  int sp = 0;
  int node = 0;
  for (;;) {
    const float4 n0 = __ldg(&P.nodes[2 * node]);
    const float4 n1 = __ldg(&P.nodes[2 * node + 1]);
    const float lim = hr.id >= 0 ? hr.s : smax;
    const float tx0 = (n0.x - O.x) * inv.x, tx1 = (n1.x - O.x) * inv.x;
    const float ty0 = (n0.y - O.y) * inv.y, ty1 = (n1.y - O.y) * inv.y;
    const float tz0 = (n0.z - O.z) * inv.z, tz1 = (n1.z - O.z) * inv.z;
    const float tmin = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.f));
    const float tmax = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), lim));
    if (tmin <= tmax) {
      const int first = __float_as_int(n0.w);
      const int cnt = __float_as_int(n1.w);
      if (cnt > 0) {
        for (int q = first; q < first + cnt; ++q) {
          const float4 a4 = __ldg(&P.prims[3 * q]);
          const float4 b4 = __ldg(&P.prims[3 * q + 1]);
          const int id = __float_as_int(a4.w);
          float s;
          bool got;
          if (id < P.S) {
            got = hit_sphere(O, D, dd, make_float4(a4.x, a4.y, a4.z, b4.x), s) && s < smax;
          } else {
            const float4 c4 = __ldg(&P.prims[3 * q + 2]);
            s = hit_triangle(fr, O, smax, a4, b4, c4);
            got = s >= 0.f;
          }
          if (got && (hr.id < 0 || s < hr.s || (s == hr.s && id < hr.id))) {
            hr.s = s;
            hr.id = id;
            hr.tq = id < P.S ? -1 : q;
          }
        }
      } else {
        if (sp >= kTraversalStack) {
          atomicOr(&g_rgeo_error, kErrStackOverflow);
          break;
        }
        stack[sp++] = first + 1;
        node = first;
        continue;
      }
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  return hr.id >= 0;
}

// Earliest hit of the polygon's chords [p_j, p_j+1], j = 0 .. n - 1 (n <= NB), in one
// query (Section 4.1: many segments per intersection query): the BVH is walked once with
// the bounding box of all the chords, and every primitive of a leaf it reaches is tested
// against each chord up to the best hit so far.  Each chord-primitive test is the one
// scene_hit makes, so the result -- the first chord with a hit, its earliest s and then
// lowest id -- is the one the chords tested one by one give.  pts[i * stride] holds p_i.
template <int NB>
__device__ bool scene_hit_bundle(const TraceParams &P, const float4 *ss, const float4 *pts, int stride, int n,
                                 HitRec &hr, int &jbest) {
  F3 p[NB + 1];
#pragma unroll
  for (int i = 0; i <= NB; ++i) {
    const float4 q = pts[(i <= n ? i : n) * stride];
    p[i] = f3(q.x, q.y, q.z);
  }
  F3 lo = p[0], hi = p[0];
#pragma unroll
  for (int i = 1; i <= NB; ++i) {
    lo = f3(fminf(lo.x, p[i].x), fminf(lo.y, p[i].y), fminf(lo.z, p[i].z));
    hi = f3(fmaxf(hi.x, p[i].x), fmaxf(hi.y, p[i].y), fmaxf(hi.z, p[i].z));
  }
  hr.id = -1;
  hr.tq = -1;
  hr.s = 1.f;
  jbest = NB;
  // chord j against one primitive (sphere: sp; triangle: a4, b4, c4 at BVH slot q)
  auto consider = [&](int j, int id, int q, float s) {
    if (j < jbest || (j == jbest && (s < hr.s || (s == hr.s && id < hr.id)))) {
      jbest = j;
      hr.s = s;
      hr.id = id;
      hr.tq = q;
    }
  };
  if (P.nodes == nullptr) {
    for (int k = 0; k < P.S; ++k) {
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (j >= n || j > jbest) break;
        const F3 D = p[j + 1] - p[j];
        float s;
        if (hit_sphere(p[j], D, dot(D, D), ss[k], s) && s < 1.f) consider(j, k, -1, s);
      }
    }
    return hr.id >= 0;
  }
  int stack[kTraversalStack];
  int sp = 0;
  int node = 0;
  for (;;) {
    const float4 n0 = __ldg(&P.nodes[2 * node]);
    const float4 n1 = __ldg(&P.nodes[2 * node + 1]);
    if (n0.x <= hi.x && n0.y <= hi.y && n0.z <= hi.z && lo.x <= n1.x && lo.y <= n1.y && lo.z <= n1.z) {
      const int first = __float_as_int(n0.w);
      const int cnt = __float_as_int(n1.w);
      if (cnt > 0) {
        for (int q = first; q < first + cnt; ++q) {
          const float4 a4 = __ldg(&P.prims[3 * q]);
          const float4 b4 = __ldg(&P.prims[3 * q + 1]);
          const int id = __float_as_int(a4.w);
          const float4 c4 = id < P.S ? a4 : __ldg(&P.prims[3 * q + 2]);
#pragma unroll
          for (int j = 0; j < NB; ++j) {
            if (j >= n || j > jbest) break;
            const F3 D = p[j + 1] - p[j];
            if (id < P.S) {
              float s;
              if (hit_sphere(p[j], D, dot(D, D), make_float4(a4.x, a4.y, a4.z, b4.x), s) && s < 1.f)
                consider(j, id, -1, s);
            } else {
              const float s = hit_triangle(make_frame(D), p[j], 1.f, a4, b4, c4);
              if (s >= 0.f) consider(j, id, q, s);
            }
          }
        }
      } else {
        if (sp >= kTraversalStack) {
          atomicOr(&g_rgeo_error, kErrStackOverflow);
          break;
        }
        stack[sp++] = first + 1;
        node = first;
        continue;
      }
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  return hr.id >= 0;
}

// Lower bound of the distance from x to the scene.
__device__ __forceinline__ float safe_distance(const TraceParams &P, F3 x) {
  const float fx = (x.x - P.gmin[0]) * P.ginv, fy = (x.y - P.gmin[1]) * P.ginv,
              fz = (x.z - P.gmin[2]) * P.ginv;
  if (fx >= 0.f && fy >= 0.f && fz >= 0.f && fx < (float)P.gdim[0] && fy < (float)P.gdim[1] &&
      fz < (float)P.gdim[2]) {
    const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
    return __ldg(&P.grid[((size_t)iz * P.gdim[1] + iy) * P.gdim[0] + ix]);
  }
  const float ex = fmaxf(fmaxf(P.smin[0] - x.x, x.x - P.smax[0]), 0.f);
  const float ey = fmaxf(fmaxf(P.smin[1] - x.y, x.y - P.smax[1]), 0.f);
  const float ez = fmaxf(fmaxf(P.smin[2] - x.z, x.z - P.smax[2]), 0.f);
  return fmaxf(sqrtf(ex * ex + ey * ey + ez * ez) * (1.f - 1e-5f) - 1e-4f, 0.f);
}

// Smallest t >= 0 at which x + t v enters a support ball (flat skip), +inf if none.
template <int MK>
__device__ float support_entry(const float4 *sb, int K, F3 x, F3 v) {
  const float A = dot(v, v);
  float best = __int_as_float(0x7f800000);
  for (int k = 0; k < K; ++k) {
    F3 c;
    float R2;
    if (is_iso(MK)) {
      const IsoBump b = iso_bump(sb, k);
      c = b.c;
      R2 = b.R2;
    } else {
      const float4 b0 = sb[kAnisoStride * k];
      c = f3(b0.x, b0.y, b0.z);
      R2 = b0.w;
    }
    if (R2 < 0.f) continue;
    const F3 o = f3(x.x - c.x, x.y - c.y, x.z - c.z);
    const float B = dot(o, v);
    if (B >= 0.f) continue;
    const float C = dot(o, o) - R2;
    const float disc = B * B - A * C;
    if (disc < 0.f) continue;
    const float t = fmaxf((-B - sqrtf(disc)) / A, 0.f);
    best = fminf(best, t);
  }
  return best;
}

// ---------------------------------------------------------------- shading

__device__ __forceinline__ unsigned char to_u8(float c) {
  c = fminf(fmaxf(c, 0.f), 1.f);
  return (unsigned char)floorf(255.f * c + 0.5f);
}

__device__ uchar4 shade(const TraceParams &P, const float4 *ss, const HitRec &hr, F3 Ph, F3 D, float arc) {
  float r, g, b;
  if (P.shading == 1) {
    r = 0.5f + Ph.x * 0.125f;
    g = 0.5f + Ph.y * 0.125f;
    b = 0.5f + Ph.z * 0.125f;
  } else {
    F3 n;
    int obj;
    if (hr.id < P.S) {
      const float4 sp = P.nodes ? __ldg(&P.spheres[hr.id]) : ss[hr.id];
      n = f3(Ph.x - sp.x, Ph.y - sp.y, Ph.z - sp.z);
      obj = hr.id;
    } else {
      const float4 a4 = P.prims[3 * hr.tq], b4 = P.prims[3 * hr.tq + 1], c4 = P.prims[3 * hr.tq + 2];
      n = cross(f3(b4.x - a4.x, b4.y - a4.y, b4.z - a4.z), f3(c4.x - a4.x, c4.y - a4.y, c4.z - a4.z));
      if (dot(n, D) > 0.f) n = -1.f * n;
      obj = P.S;
    }
    n = normalize(n);
    const F3 dv = normalize(D);
    const float inten = 0.1f + 0.9f * fmaxf(0.f, -dot(n, dv));
    r = P.albedo[3 * obj] * inten;
    g = P.albedo[3 * obj + 1] * inten;
    b = P.albedo[3 * obj + 2] * inten;
  }
  if (P.fog > 0.f) {  // the grid figures' fog: c T + fog_rgb (1 - T), T = exp(-density * arc length)
    const float T = expf(-P.fog * arc), U = 1.f - T;
    r = fmaf(r, T, P.fog_rgb[0] * U);
    g = fmaf(g, T, P.fog_rgb[1] * U);
    b = fmaf(b, T, P.fog_rgb[2] * U);
  }
  return make_uchar4(to_u8(r), to_u8(g), to_u8(b), 255);
}

// Unit normal of the hit surface, facing the segment D that reached it (sphere: radial;
// triangle: geometric), for the illumination pass.
__device__ F3 hit_normal(const TraceParams &P, const float4 *ss, const HitRec &hr, F3 Ph, F3 D) {
  F3 n;
  if (hr.id < P.S) {
    const float4 sp = P.nodes ? __ldg(&P.spheres[hr.id]) : ss[hr.id];
    n = f3(Ph.x - sp.x, Ph.y - sp.y, Ph.z - sp.z);
  } else {
    const float4 a4 = P.prims[3 * hr.tq], b4 = P.prims[3 * hr.tq + 1], c4 = P.prims[3 * hr.tq + 2];
    n = cross(f3(b4.x - a4.x, b4.y - a4.y, b4.z - a4.z), f3(c4.x - a4.x, c4.y - a4.y, c4.z - a4.z));
  }
  if (dot(n, D) > 0.f) n = -1.f * n;
  return normalize(n);
}

// ----------------------------------------------------------------- kernel

struct Ray {
  float xh[3], xl[3], vh[3], vl[3];
  int steps;
  int pix;
  float dleft;
  float e0m1;
  float arc;  // arc length travelled: h per step, the parameter length of straight advances
  int nb;     // chords of the open bundle (segment tests deferred to one query), 0: none
};

__device__ __forceinline__ F3 xhi(const Ray &r) { return f3(r.xh[0], r.xh[1], r.xh[2]); }
__device__ __forceinline__ F3 vhi(const Ray &r) { return f3(r.vh[0], r.vh[1], r.vh[2]); }
// Pixel of queue item `item` of this launch: launch tile item / 32 is frame tile
// tile0 + (item / 32) tile_step (tile_pixel gives the layout).  False for the part of an
// edge tile that lies outside the frame.
__device__ __forceinline__ bool item_pixel(const TraceParams &P, unsigned item, int &pix) {
  return tile_pixel(P.W, P.H, P.tiles_x, P.tile_lw, P.tile0 + (item >> 5) * P.tile_step, item & 31u, pix);
}

// A lane without a ray keeps finite state (it still joins the warp's bump sums).
__device__ __forceinline__ void ray_clear(Ray &r) {
  for (int c = 0; c < 3; c++) r.xh[c] = r.xl[c] = r.vh[c] = r.vl[c] = 0.f;
  r.steps = 0;
  r.pix = 0;
  r.dleft = r.e0m1 = r.arc = 0.f;
  r.nb = 0;
}

template <int MK>
__device__ void init_ray(const TraceParams &P, const float4 *sb, int pix, Ray &r) {
  const int i = pix % P.W, j = pix / P.W;
  const F3 Fw = normalize(f3(P.cam_fwd[0], P.cam_fwd[1], P.cam_fwd[2]));
  const F3 R = normalize(cross(f3(P.cam_up[0], P.cam_up[1], P.cam_up[2]), Fw));
  const F3 U = cross(Fw, R);
  const float th = tanf(P.vfov_deg * 0.00872664625997164788f);  // pi / 360
  const float u = (2.f * (i + 0.5f) / P.W - 1.f) * th * ((float)P.W / (float)P.H);
  const float w = (1.f - 2.f * (j + 0.5f) / P.H) * th;
  const F3 d = normalize(axpy(w, U, axpy(u, R, Fw)));
  const F3 x = f3(P.cam_pos[0], P.cam_pos[1], P.cam_pos[2]);
  float gdd;  // g_x(d, d)
  if (MK == MK_TWIST) {
    float s, c;
    sincosf(P.twist_k * x.z, &s, &c);
    const float X = c * x.x - s * x.y, Y = s * x.x + c * x.y;
    const float j0 = c * d.x - s * d.y - P.twist_k * Y * d.z;
    const float j1 = s * d.x + c * d.y + P.twist_k * X * d.z;
    gdd = j0 * j0 + j1 * j1 + d.z * d.z;
  } else if (MK == MK_LOCAL) {
    Jet jt;
    local_jacobian(sb, P.K, x, jt);
    const F3 jd = f3(dot(f3(jt.M[0], jt.M[1], jt.M[2]), d), dot(f3(jt.M[3], jt.M[4], jt.M[5]), d),
                     dot(f3(jt.M[6], jt.M[7], jt.M[8]), d));
    gdd = dot(jd, jd);
  } else {
    const F3 g = grad_f<MK>(P, sb, x);
    const float gd = dot(g, d);
    gdd = fmaf(gd, gd, dot(d, d));
  }
  const F3 v = rsqrtf(gdd) * d;
  for (int c = 0; c < 3; c++) {
    r.xh[c] = comp(x, c);
    r.xl[c] = 0.f;
    r.vh[c] = comp(v, c);
    r.vl[c] = 0.f;
  }
  r.steps = 0;
  r.pix = pix;
  r.dleft = 0.f;
  r.e0m1 = 0.f;
  r.arc = 0.f;
  r.nb = 0;
  if (P.energy) r.e0m1 = (float)(energy<MK>(P, sb, x, v) - 1.0);
}

template <int MK>
__device__ void finish_ray(const TraceParams &P, const float4 *sb, const float4 *ss, const Ray &r,
                           int id, const HitRec &hr, F3 Ph, F3 D, float arc = 0.f) {
  const int p = r.pix;
  const size_t N = (size_t)P.W * P.H;
  P.id[p] = id;
  P.steps[p] = r.steps;
  const F3 o = id >= 0 ? Ph : xhi(r);
  P.hit[p] = o.x;
  P.hit[N + p] = o.y;
  P.hit[2 * N + p] = o.z;
  P.rgba[p] = id >= 0 ? shade(P, ss, hr, Ph, D, arc) : make_uchar4(0, 0, 0, 0);
  if (P.hit_nrm && id >= 0) {
    const F3 n = hit_normal(P, ss, hr, Ph, D);
    P.hit_nrm[p] = n.x;
    P.hit_nrm[N + p] = n.y;
    P.hit_nrm[2 * N + p] = n.z;
  }
  if (P.energy) {
    const double e = energy<MK>(P, sb, xhi(r), vhi(r));
    P.drift[p] = e / (1.0 + (double)r.e0m1) - 1.0;
  }
}

// The rare paths of a ray (its start and end, the search for the next support ball of a flat
// advance), called out of line with OOL: k_trace does so for the isotropic graph metric, whose
// hot loop's code and registers then stay small (4 % faster at 1080p / 64 bumps); the other
// kinds and kernels take them inline (3 % faster for the twist metric).
template <int MK>
__device__ __noinline__ void init_ray_ool(const TraceParams &P, const float4 *sb, int pix, Ray &r) {
  init_ray<MK>(P, sb, pix, r);
}
template <int MK>
__device__ __noinline__ void finish_ray_ool(const TraceParams &P, const float4 *sb, const float4 *ss, const Ray &r,
                                            int id, const HitRec &hr, F3 Ph, F3 D, float arc) {
  finish_ray<MK>(P, sb, ss, r, id, hr, Ph, D, arc);
}
template <int MK>
__device__ __noinline__ float support_entry_ool(const float4 *sb, int K, F3 x, F3 v) {
  return support_entry<MK>(sb, K, x, v);
}
template <int MK, bool OOL>
__device__ __forceinline__ void start_ray(const TraceParams &P, const float4 *sb, int pix, Ray &r) {
  if constexpr (OOL) init_ray_ool<MK>(P, sb, pix, r);
  else init_ray<MK>(P, sb, pix, r);
}
template <int MK, bool OOL>
__device__ __forceinline__ void end_ray(const TraceParams &P, const float4 *sb, const float4 *ss, const Ray &r,
                                        int id, const HitRec &hr, F3 Ph, F3 D, float arc = 0.f) {
  if constexpr (OOL) finish_ray_ool<MK>(P, sb, ss, r, id, hr, Ph, D, arc);
  else finish_ray<MK>(P, sb, ss, r, id, hr, Ph, D, arc);
}
template <int MK, bool OOL>
__device__ __forceinline__ float next_support(const float4 *sb, int K, F3 x, F3 v) {
  if constexpr (OOL) return support_entry_ool<MK>(sb, K, x, v);
  else return support_entry<MK>(sb, K, x, v);
}

// Stage the bump table and the spheres in shared memory; returns the bump part size.
template <int MK>
__device__ __forceinline__ int stage_shared(const TraceParams &P, float4 *smem) {
  const int nb4 = MK == MK_TWIST ? 0 : (MK == MK_LOCAL ? kLocalStride * P.K : packed_float4s(P.K, MK == MK_GRAPH_ANISO));
  for (int i = threadIdx.x; i < nb4; i += blockDim.x) smem[i] = P.bumps[i];
  if (P.nodes == nullptr)  // spheres are tested one by one only when there is no BVH
    for (int i = threadIdx.x; i < P.S; i += blockDim.x) smem[nb4 + i] = P.spheres[i];
  __syncthreads();
  return nb4;
}

// Warp-synchronous refill: every lane calls this; lanes whose slot is empty take
// the next queue items (one atomic per warp).  Items walk 32-pixel tiles so that
// a warp's rays start close together.
template <int MK>
__device__ __forceinline__ void refill(const TraceParams &P, const float4 *sb, bool &active,
                                       bool &drained, Ray &r) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned need = __ballot_sync(0xffffffffu, !active && !drained);
  if (!need) return;
  const int leader = __ffs(need) - 1;
  unsigned base = 0;
  if ((int)lane == leader) base = atomicAdd(P.counter, (unsigned)__popc(need));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (base + (unsigned)__popc(need) >= P.n_items) drained = true;
  if (!active && ((need >> lane) & 1u)) {
    const unsigned item = base + (unsigned)__popc(need & ((1u << lane) - 1u));
    int pix;
    if (item < P.n_items && item_pixel(P, item, pix)) {
      init_ray<MK>(P, sb, pix, r);
      active = true;
    }
  }
}

// Warp-synchronous refill from a warp-private chunk of 32 consecutive items (one 32-pixel
// tile, 4 x 8 by default) taken from the queue one chunk at a time: the rays a warp starts come from the same
// tile, so its lanes stay closer together and the union of their cull cells stays smaller.
// By default (P.refill_lanes == 0) the warp takes rays in generations: only once every ray
// it holds has finished, so that the 32 rays of a tile march side by side from the camera
// (most of them run to the step budget together) instead of a fresh ray starting next to
// rays far along their paths, which widens the warp's bump lists.  cnext / cend (the chunk's
// next and end item) are the same on every lane.
template <int MK, bool OOL = false>
__device__ __forceinline__ void refill_tile(const TraceParams &P, const float4 *sb, bool &active, bool &drained,
                                            Ray &r, unsigned &cnext, unsigned &cend) {
  const unsigned lane = threadIdx.x & 31u;
  if (!P.refill_lanes && __any_sync(0xffffffffu, active)) return;
  for (int pass = 0; pass < 2; ++pass) {
    const unsigned need = __ballot_sync(0xffffffffu, !active && !drained);
    if (!need) return;
    if (cnext >= cend) {
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(P.counter, 32u);
      base = __shfl_sync(0xffffffffu, base, 0);
      cnext = base;
      cend = base + 32u;
      if (base >= P.n_items) {
        drained = true;
        return;
      }
    }
    const unsigned take = min((unsigned)__popc(need), cend - cnext);
    const unsigned rank = (unsigned)__popc(need & ((1u << lane) - 1u));
    if (((need >> lane) & 1u) && rank < take) {
      const unsigned item = cnext + rank;
      int pix;
      if (item < P.n_items && item_pixel(P, item, pix)) {
        start_ray<MK, OOL>(P, sb, pix, r);
        active = true;
      }
    }
    cnext += take;
  }
}

// Tests the open bundle of r (its chords' end points and arc lengths in the thread's slots
// bs[i * blockDim.x], i = 0 .. r.nb) in one query; on a hit the ray finishes as the chord
// that hit would have finished it tested alone (its step count, hit point and arc length).
// Returns true on a hit.  The bundle is closed either way.
template <int MK, int NB, bool OOL = false>
__device__ __noinline__ bool bundle_flush(const TraceParams &P, const float4 *sb, const float4 *ss, Ray &r,
                                          const float4 *bs) {
  HitRec hr;
  int j;
  const int stride = (int)blockDim.x;
  const bool hit = scene_hit_bundle<NB>(P, ss, bs, stride, r.nb, hr, j);
  if (hit) {
    const float4 a = bs[j * stride], b = bs[(j + 1) * stride];
    const F3 A = f3(a.x, a.y, a.z), D = f3(b.x - a.x, b.y - a.y, b.z - a.z);
    r.steps -= r.nb - 1 - j;
    end_ray<MK, OOL>(P, sb, ss, r, hr.id, hr, axpy(hr.s, D, A), D, fmaf(hr.s - 1.f, P.h, b.w));
  }
  r.nb = 0;
  r.dleft = 0.f;
  return hit;
}

// Before a step: closed-form advance through flat space when x lies outside every
// truncated support (exact: Hess f = 0 there, Eq. 5.4), then the step budget.  An open
// bundle of chords (NB > 1) is tested first, since the flat advance and the budget end
// come after its chords.  a1 is the stage-1 acceleration at x; it is recomputed if x
// moves.  Returns false when the ray finished (its pixel is written) or the lane holds no
// ray (cx.part false; such lanes call only when CONV, to join the warp's sums; with CONV
// every lane of the warp calls together).
template <int MK, bool CONV = Converged<MK>::value, int NB = 1, bool OOL = false>
__device__ __forceinline__ bool pre_step(const TraceParams &P, const float4 *sb, const float4 *ss,
                                         const SumCtx &cx, Ray &r, F3 &a1, bool inside,
                                         const float4 *bs = nullptr) {
  F3 x = xhi(r);
  const F3 v = vhi(r);
  bool moved = false, finished = false;
  const bool flat = MK != MK_TWIST && MK != MK_LOCAL && P.skippable && !inside;
  if (NB > 1 && cx.part && r.nb > 0 && (flat || r.steps >= P.max_steps))
    finished = bundle_flush<MK, NB, OOL>(P, sb, ss, r, bs);
  if (cx.part && !finished && flat) {
    const float t = next_support<MK, OOL>(sb, P.K, x, v);
    HitRec hr;
    if (scene_hit(P, ss, x, v, t, hr)) {
      end_ray<MK, OOL>(P, sb, ss, r, hr.id, hr, axpy(hr.s, v, x), v, r.arc + hr.s);
      finished = true;
    } else if (isinf(t)) {
      end_ray<MK, OOL>(P, sb, ss, r, RGEO_ID_MISS, hr, x, v);
      finished = true;
    } else {
      for (int c = 0; c < 3; c++) comp_add(r.xh[c], r.xl[c], t * comp(v, c));
      r.arc += t;  // a straight advance of parameter length t is also its g-length (v is g-unit)
      r.dleft = 0.f;
      x = xhi(r);
      moved = true;
    }
  }
  if (CONV) {
    if (__any_sync(0xffffffffu, moved)) {
      // a step list must cover the moved lanes' new positions: list again for every lane that goes on
      if (MK == MK_GRAPH_SL && cx.wl->np >= 0) step_list(P, sb, *cx.wl, cx.ghdr, cx.part && !finished, x);
      bool dummy;
      const F3 am = accel<MK, false>(P, sb, SumCtx{cx.ghdr, cx.wl, moved, cx.evals}, x, v, dummy);
      if (moved) a1 = am;
    }
  } else if (moved) {
    bool dummy;
    a1 = accel<MK, false>(P, sb, cx, x, v, dummy);
  }
  if (!cx.part || finished) return false;
  if (r.steps >= P.max_steps) {
    HitRec hr;
    hr.id = -1;
    end_ray<MK, OOL>(P, sb, ss, r, RGEO_ID_BUDGET, hr, x, v);
    return false;
  }
  return true;
}

// After a step: compensated update of (x, v), then the new polygon segment
// [x_i, x_{i+1}] against the scene (Section 4.1), skipped exactly while the polygon
// cannot have left a ball that holds no scene point.  With NB > 1 a segment that needs a
// test opens a bundle instead; the next NB - 1 chords join it, and the bundle is tested
// in one query (Section 4.1, many segments per query) once it holds NB chords (or before
// a flat advance or the budget end, in pre_step).  Returns false on a hit.
template <int MK, int NB = 1, bool OOL = false>
__device__ __forceinline__ bool post_step(const TraceParams &P, const float4 *sb, const float4 *ss,
                                          Ray &r, F3 dx, F3 dvel, float4 *bs = nullptr) {
  const F3 x = xhi(r);
  for (int c = 0; c < 3; c++) {
    comp_add(r.xh[c], r.xl[c], comp(dx, c));
    comp_add(r.vh[c], r.vl[c], comp(dvel, c));
  }
  r.steps++;
  r.arc += P.h;
  const F3 xn = xhi(r);
  const F3 D = xn - x;
  const int stride = (int)blockDim.x;
  if (NB > 1 && r.nb > 0) {  // an open bundle: this chord joins it
    bs[(r.nb + 1) * stride] = make_float4(xn.x, xn.y, xn.z, r.arc);
    if (++r.nb == NB) return !bundle_flush<MK, NB, OOL>(P, sb, ss, r, bs);
    return true;
  }
  if (P.safe_skip) {
    const float L = sqrtf(dot(D, D)) * (1.f + 1e-6f);
    if (L < r.dleft) {
      r.dleft -= L;
      return true;
    }
    const float d0 = safe_distance(P, x);
    if (L < d0) {
      r.dleft = d0 - L;
      return true;
    }
    r.dleft = 0.f;
  }
  if (NB > 1) {  // open a bundle with this chord
    bs[0] = make_float4(x.x, x.y, x.z, 0.f);
    bs[stride] = make_float4(xn.x, xn.y, xn.z, r.arc);
    r.nb = 1;
    return true;
  }
  HitRec hr;
  if (scene_hit(P, ss, x, D, 1.f, hr)) {
    end_ray<MK, OOL>(P, sb, ss, r, hr.id, hr, axpy(hr.s, D, x), D, fmaf(hr.s - 1.f, P.h, r.arc));
    return false;
  }
  return true;
}

// RK4 (or Euler, Eq. 4.1) increments of one step from (x, v) with stage-1 value a1.
template <int MK, int INTEG>
__device__ __forceinline__ void step_increments(const TraceParams &P, const float4 *sb, const SumCtx &cx, F3 x,
                                                F3 v, F3 a1, F3 &dx, F3 &dvel) {
  const float h = P.h;
  if (INTEG == 0) {
    bool dummy;
    const float h2 = 0.5f * h;
    const F3 v2 = axpy(h2, a1, v);
    const F3 a2 = accel<MK, false>(P, sb, cx, axpy(h2, v, x), v2, dummy);
    const F3 v3 = axpy(h2, a2, v);
    const F3 a3 = accel<MK, false>(P, sb, cx, axpy(h2, v2, x), v3, dummy);
    const F3 v4 = axpy(h, a3, v);
    const F3 a4 = accel<MK, false>(P, sb, cx, axpy(h, v3, x), v4, dummy);
    const float h6 = h * (1.f / 6.f);
    dx = h6 * (v + 2.f * (v2 + v3) + v4);
    dvel = h6 * (a1 + 2.f * (a2 + a3) + a4);
  } else {
    dx = h * v;
    dvel = h * a1;
  }
}

// The warp's lists in shared memory, after the bump table and the spheres: the index
// pairs, then (with step lists) the packed pairs.
constexpr int kListFloat4 = kListPairs * (int)sizeof(int2) / (int)sizeof(float4);  // index pairs, per warp
constexpr int kPackFloat4 = 4 * kListPairs;                                          // packed pairs, per warp
__host__ __device__ inline int lists_float4(bool step) { return kListFloat4 + (step ? kPackFloat4 : 0); }
__device__ __forceinline__ WarpLists warp_lists(bool step, float4 *lists) {
  float4 *base = lists + (threadIdx.x >> 5) * lists_float4(step);
  return WarpLists{reinterpret_cast<int2 *>(base), step ? base + kListFloat4 : nullptr, -1, 0u, 0};
}

// Warps of the 128-thread trace blocks.
constexpr int kWarpsPerBlock = 4;
// Chords per bundle when segment tests are bundled (RGEO_FLAG_BUNDLE).
constexpr int kBundle = 4;

// Dense sums of the isotropic graph metric from the bump table packed in pairs (up to this many
// bumps: two float4 per bump more in shared memory).
constexpr int kDensePackBumps = 512;
__host__ __device__ inline bool dense_packed(int mk, const TraceParams &P) {
  return mk == MK_GRAPH_ISO && !P.cull_masks && P.K > 0 && P.K <= kDensePackBumps;
}

// float4s of a trace block's warp lists: index lists for the culled sums, packed pairs too
// for step lists; for packed dense sums, the block's one packed copy of the table.
__host__ __device__ inline int trace_lists_float4(int mk, const TraceParams &P) {
  if (dense_packed(mk, P)) return 2 * iso_pad_index(P.K);
  return (mk == MK_GRAPH_SL || P.cull_masks) ? kWarpsPerBlock * lists_float4(mk == MK_GRAPH_SL) : 0;
}

// The bump table staged in sb, packed in pairs (2 j, 2 j + 1) into pk in the layout of the step
// lists (WarpLists), for the dense sums: every pair read by one paired-FP32 instruction per
// operation.  All threads of the block, then a barrier.
__device__ __forceinline__ void pack_dense_pairs(const float4 *sb, int K, float4 *pk) {
  const int np = iso_pad_index(K) / 2;
  for (int t = threadIdx.x; t < 4 * np; t += blockDim.x) {
    const int j = t >> 2, half = (t >> 1) & 1;  // float4 0, 1 from A, 2, 3 from B
    const float4 a = sb[kIsoBumpStride * (2 * j) + half], b = sb[kIsoBumpStride * (2 * j + 1) + half];
    pk[t] = (t & 1) == 0 ? make_float4(a.x, b.x, a.y, b.y) : make_float4(a.z, b.z, a.w, b.w);
  }
  __syncthreads();
}

// One ray per thread (every metric kind).  MINB 128-thread CTAs per SM at least: seven (72
// registers) for the isotropic graph metric and six (80) for the twist and anisotropic bumps
// by default, five (102 registers) for the local-map jet and, on request
// (rgeo_tuning.ctas_per_sm <= 5), for the isotropic graph metric.  For the
// isotropic graph metric every lane runs every evaluation of the bump sums (a lane without
// a ray joins with empty masks), so that the warp can build its pair list together.
// COUNT false (a launch without work counters) leaves the per-lane counts unread, so the
// compiler drops them.  OOL takes a ray's rare paths out of line (start_ray).
template <int MK, int INTEG, int MINB, int NB, bool COUNT = true, bool OOL = is_iso(MK)>
__global__ void __launch_bounds__(128, MINB) k_trace(const TraceParams P) {
  extern __shared__ float4 smem[];
  const int nb4 = stage_shared<MK>(P, smem);
  const float4 *sb = smem;
  const float4 *ss = smem + nb4;
  float4 *const lists = smem + nb4 + (P.nodes ? 0 : P.S);
  WarpLists wl = warp_lists(MK == MK_GRAPH_SL, lists);
  if (dense_packed(MK, P)) {  // the dense sums take the block's packed copy of the table
    pack_dense_pairs(sb, P.K, lists);
    wl = WarpLists{nullptr, lists, iso_pad_index(P.K) / 2, 0u, 0};
  }
  // the threads' bundle slots (NB > 1), after the warps' lists: slot i of thread t at i * 128 + t
  float4 *const bs = lists + trace_lists_float4(MK, P) + threadIdx.x;
  const float4 ghdr = P.cull_masks ? __ldg(P.cull_hdr) : make_float4(0.f, 0.f, 0.f, 0.f);
  constexpr bool conv = Converged<MK>::value;
  constexpr bool ool = OOL;
  WorkCount evals;
  bool active = false, drained = false;
  Ray r;
  ray_clear(r);
  unsigned cnext = 0u, cend = 0u;
  for (;;) {
    const bool held = active;
    refill_tile<MK, ool>(P, sb, active, drained, r, cnext, cend);
    const unsigned amask = __ballot_sync(0xffffffffu, active);
    if (!amask) {
      if (drained) break;
      continue;
    }
    if (!conv && !active) continue;
    if (MK == MK_GRAPH_SL) step_list_refresh(P, sb, wl, ghdr, active, active && !held, xhi(r));
    bool inside = true;
    F3 a1 = accel<MK, true>(P, sb, SumCtx{ghdr, &wl, active, &evals}, xhi(r), vhi(r), inside);
    const bool go =
        pre_step<MK, Converged<MK>::value, NB, ool>(P, sb, ss, SumCtx{ghdr, &wl, active, &evals}, r, a1, inside, bs);
    if (!go) active = false;
    if (conv ? !__any_sync(0xffffffffu, go) : !go) continue;
    F3 dx, dvel;
    step_increments<MK, INTEG>(P, sb, SumCtx{ghdr, &wl, go, &evals}, xhi(r), vhi(r), a1, dx, dvel);
    if (go) active = post_step<MK, NB, ool>(P, sb, ss, r, dx, dvel, bs);
    ++wl.age;
  }
  if (COUNT) evals.flush(P);
}

// ------------------------------------------------------ Riemannian illumination

// The cull cell of x for the per-lane sums: its mask words, or null when x lies outside the
// grid (which covers every bump's support inflated by kCullInflate + the metric's reach
// margin, so no bump reaches within that margin of x either).
__device__ __forceinline__ const uint32_t *lane_cell(const TraceParams &P, F3 x) {
  const float4 ghdr = __ldg(P.cull_hdr);
  const int G = P.cull_G;
  const float fx = (x.x - ghdr.x) * ghdr.w, fy = (x.y - ghdr.y) * ghdr.w, fz = (x.z - ghdr.z) * ghdr.w;
  if (!(fx >= 0.f && fy >= 0.f && fz >= 0.f && fx < (float)G && fy < (float)G && fz < (float)G)) return nullptr;
  return P.cull_masks + ((size_t)(((int)fz * G + (int)fy) * G + (int)fx)) * (size_t)P.cull_words;
}

// Eq. 5.4 over the bumps of one cull cell's list, with no warp collective: for lanes that
// follow their own paths (the light geodesics), each walks its own list and SIMT serialises
// the differences.  cm is the cell of x, or of a position within the metric's reach margin
// of x (a lane's list serves the steps its reach covers, as the warps' step lists do), or
// null: no bumps.  The
// list's even-numbered bumps are paired with its odd-numbered ones as in the warp-wide
// form, so the sums equal the dense sums.  Other metric kinds, and metrics without a cull
// grid, take the dense sums (cm unused).
template <int MK, bool INSIDE>
__device__ __forceinline__ F3 accel_lane(const TraceParams &P, const float4 *sb, const uint32_t *cm, F3 x, F3 v,
                                         bool &inside, WorkCount &evals) {
  if (MK != MK_GRAPH_ISO || !P.cull_masks) {
    WarpLists nolists{nullptr, nullptr, -1, 0u, 0};
    const SumCtx cx{make_float4(0.f, 0.f, 0.f, 0.f), &nolists, true, &evals};
    return accel<MK, INSIDE>(P, sb, cx, x, v, inside);
  }
  PairAcc a;
  pair_acc_init(a, x, v);
  const int pad = kIsoBumpStride * iso_pad_index(P.K);
  if (cm) {
    // two cursors walk the cell's even-numbered and odd-numbered bumps in increasing order
    const unsigned w0 = __ldg(cm);
    evals.evals += (unsigned)__popc(w0);
    unsigned me = w0 & 0x55555555u, mo = w0 & 0xaaaaaaaau;
    int we = 0, wo = 0;
    for (;;) {
      while (!me && we + 1 < P.cull_words) {  // every word passes the even cursor once
        const unsigned t = __ldg(cm + ++we);
        evals.evals += (unsigned)__popc(t);
        me = t & 0x55555555u;
      }
      while (!mo && wo + 1 < P.cull_words) mo = __ldg(cm + ++wo) & 0xaaaaaaaau;
      if (!(me | mo)) break;
      int ie = pad, io = pad;
      if (me) {
        ie = kIsoBumpStride * ((we << 5) + __ffs(me) - 1);
        me &= me - 1u;
      }
      if (mo) {
        io = kIsoBumpStride * ((wo << 5) + __ffs(mo) - 1);
        mo &= mo - 1u;
      }
      pair_eval<INSIDE>(a, sb, ie, io);
      evals.slots += 2u;
    }
  }
  if (INSIDE) inside = a.in;
  return pair_acc_finish(P, a, x, v);
}

// The list a light geodesic's sums at x take: the cell kept from the step that built it
// while it serves (P.list_steps > 0), else x's own cell.
__device__ __forceinline__ const uint32_t *lane_list(const TraceParams &P, const uint32_t *kept, F3 x) {
  return (P.list_steps > 0 || !P.cull_masks) ? kept : lane_cell(P, x);
}

// One RK4 (or Euler) step's increments with per-lane sums (the light geodesics).
template <int MK, int INTEG>
__device__ __forceinline__ void step_increments_lane(const TraceParams &P, const float4 *sb, const uint32_t *kept,
                                                     F3 x, F3 v, F3 a1, F3 &dx, F3 &dvel, WorkCount &evals) {
  const float h = P.h;
  if (INTEG == 0) {
    bool dummy;
    const float h2 = 0.5f * h;
    const F3 v2 = axpy(h2, a1, v);
    const F3 x2 = axpy(h2, v, x);
    const F3 a2 = accel_lane<MK, false>(P, sb, lane_list(P, kept, x2), x2, v2, dummy, evals);
    const F3 v3 = axpy(h2, a2, v);
    const F3 x3 = axpy(h2, v2, x);
    const F3 a3 = accel_lane<MK, false>(P, sb, lane_list(P, kept, x3), x3, v3, dummy, evals);
    const F3 v4 = axpy(h, a3, v);
    const F3 x4 = axpy(h, v3, x);
    const F3 a4 = accel_lane<MK, false>(P, sb, lane_list(P, kept, x4), x4, v4, dummy, evals);
    const float h6 = h * (1.f / 6.f);
    dx = h6 * (v + 2.f * (v2 + v3) + v4);
    dvel = h6 * (a1 + 2.f * (a2 + a3) + a4);
  } else {
    dx = h * v;
    dvel = h * a1;
  }
}

// g_x(d, d) (Eq. 3.1 with Eq. 5.2, Eq. 5.6 or the composed maps).
template <int MK>
__device__ float metric_dd(const TraceParams &P, const float4 *sb, F3 x, F3 d) {
  if (MK == MK_TWIST) {
    float s, c;
    sincosf(P.twist_k * x.z, &s, &c);
    const float X = c * x.x - s * x.y, Y = s * x.x + c * x.y;
    const float j0 = c * d.x - s * d.y - P.twist_k * Y * d.z;
    const float j1 = s * d.x + c * d.y + P.twist_k * X * d.z;
    return j0 * j0 + j1 * j1 + d.z * d.z;
  }
  if (MK == MK_LOCAL) {
    Jet jt;
    local_jacobian(sb, P.K, x, jt);
    const F3 jd = f3(dot(f3(jt.M[0], jt.M[1], jt.M[2]), d), dot(f3(jt.M[3], jt.M[4], jt.M[5]), d),
                     dot(f3(jt.M[6], jt.M[7], jt.M[8]), d));
    return dot(jd, jd);
  }
  const F3 g = grad_f<MK>(P, sb, x);
  const float gd = dot(g, d);
  return fmaf(gd, gd, dot(d, d));
}

// n^T g_x^-1 n: Sherman-Morrison for the graph metric (g^-1 = I - grad f grad f^T / (1 + |grad f|^2),
// Eq. 5.2), |J^-T n|^2 for a pull-back metric g = J^T J (Eq. 5.6).
template <int MK>
__device__ float metric_inv_nn(const TraceParams &P, const float4 *sb, F3 x, F3 n) {
  if (is_iso(MK) || MK == MK_GRAPH_ANISO) {
    const F3 g = grad_f<MK>(P, sb, x);
    const float gn = dot(g, n);
    return dot(n, n) - gn * gn / fmaf(g.z, g.z, fmaf(g.y, g.y, fmaf(g.x, g.x, 1.f)));
  }
  float M[9];
  if (MK == MK_TWIST) {
    float s, c;
    sincosf(P.twist_k * x.z, &s, &c);
    const float X = c * x.x - s * x.y, Y = s * x.x + c * x.y;
    const float k = P.twist_k;
    M[0] = c; M[1] = -s; M[2] = -k * Y;
    M[3] = s; M[4] = c;  M[5] = k * X;
    M[6] = 0.f; M[7] = 0.f; M[8] = 1.f;
  } else {
    Jet jt;
    local_jacobian(sb, P.K, x, jt);
    for (int i = 0; i < 9; i++) M[i] = jt.M[i];
  }
  // J^-1 has the columns r1 x r2, r2 x r0, r0 x r1 (rows r_i of J) over det J, so
  // y = J^-T n = (c0.n, c1.n, c2.n) / det J
  const F3 r0 = f3(M[0], M[1], M[2]), r1 = f3(M[3], M[4], M[5]), r2 = f3(M[6], M[7], M[8]);
  const F3 c0 = cross(r1, r2), c1 = cross(r2, r0), c2 = cross(r0, r1);
  const F3 y = (1.f / dot(r0, c0)) * f3(dot(c0, n), dot(c1, n), dot(c2, n));
  return dot(y, y);
}

// The light geodesic from q with Euclidean initial direction d, marched (compensated RK4 or
// Euler at the light's step) until its closest approach to L.  Returns false when the step
// budget ran out first; else e = closest point - L.  With SHADOW, every polygon segment (and
// straight advance) up to the closest point is tested against the scene and a hit sets
// blocked.  u: the initial g-unit tangent.
template <int MK, int INTEG, bool SHADOW>
__device__ bool shoot(const TraceParams &P, const float4 *sb, const float4 *ss, F3 L, F3 q, F3 d, F3 &e, F3 &u,
                      bool &blocked, WorkCount &evals) {
  u = rsqrtf(metric_dd<MK>(P, sb, q, d)) * d;
  float xh[3] = {q.x, q.y, q.z}, xl[3] = {0.f, 0.f, 0.f}, vh[3] = {u.x, u.y, u.z}, vl[3] = {0.f, 0.f, 0.f};
  blocked = false;
  const bool keep = MK == MK_GRAPH_ISO && P.cull_masks && P.list_steps > 0;
  const uint32_t *kept = nullptr;  // the lane's list: the cell of the step that built it
  int age = P.list_steps;          // steps it has served
  for (int steps = 0;;) {
    F3 x = f3(xh[0], xh[1], xh[2]);
    const F3 v = f3(vh[0], vh[1], vh[2]);
    if (keep && age >= P.list_steps) {
      kept = lane_cell(P, x);
      age = 0;
    }
    bool inside = true;
    F3 a1 = accel_lane<MK, true>(P, sb, lane_list(P, kept, x), x, v, inside, evals);
    if (MK != MK_TWIST && MK != MK_LOCAL && P.skippable && !inside) {
      // straight line x + t v: closest approach to L at tL, next support ball at te
      const float te = support_entry<MK>(sb, P.K, x, v);
      const F3 w = L - x;
      const float tL = fmaxf(dot(w, v) / dot(v, v), 0.f);
      const float tend = fminf(tL, te);
      if (SHADOW && tend > 0.f) {
        HitRec hr;
        if (scene_hit(P, ss, x, v, tend, hr)) {
          blocked = true;
          return true;
        }
      }
      if (tL <= te) {
        e = axpy(tL, v, x) - L;
        return true;
      }
      for (int c = 0; c < 3; c++) comp_add(xh[c], xl[c], te * comp(v, c));
      x = f3(xh[0], xh[1], xh[2]);
      if (keep) {  // the advance left the list's reach: list afresh
        kept = lane_cell(P, x);
        age = 0;
      }
      bool dummy;
      a1 = accel_lane<MK, false>(P, sb, lane_list(P, kept, x), x, v, dummy, evals);
    }
    if (steps >= P.max_steps) return false;
    F3 dx, dvel;
    step_increments_lane<MK, INTEG>(P, sb, kept, x, v, a1, dx, dvel, evals);
    for (int c = 0; c < 3; c++) {
      comp_add(xh[c], xl[c], comp(dx, c));
      comp_add(vh[c], vl[c], comp(dvel, c));
    }
    ++steps;
    ++age;
    const F3 D = f3(xh[0], xh[1], xh[2]) - x;
    const float t = dot(L - x, D) / dot(D, D);
    if (t < 1.f) {  // the closest approach lies on this segment (or the distance grows)
      const float tc = fmaxf(t, 0.f);
      if (SHADOW && tc > 0.f) {
        HitRec hr;
        if (scene_hit(P, ss, x, D, tc, hr)) {
          blocked = true;
          return true;
        }
      }
      e = axpy(tc, D, x) - L;
      return true;
    }
    if (SHADOW) {
      HitRec hr;
      if (scene_hit(P, ss, x, D, 1.f, hr)) {
        blocked = true;
        return true;
      }
    }
  }
}

#if RGEO_PART(3)
// Riemannian illumination of every hit of a finished trace (Section 4): the geodesic from
// q = hit + 1e-3 n to the light is found by shooting (Gauss-Newton on the initial
// direction d0 + alpha e1 + beta e2, forward-difference Jacobian), and the hit is lit
// when it converged, the Riemannian cosine n.u / sqrt(n^T g^-1 n) is positive and the
// geodesic meets no object on the way; colour albedo (0.1 + 0.9 cos) lit, albedo 0.1 not.
// Each hit takes a group of three lanes (ten hits per warp, hits in 32-pixel tiles): in
// every Gauss-Newton step, lane 0 of the group marches the light geodesic of the current
// direction while lanes 1 and 2 march those of its two difference directions, so a step
// takes the time of one march rather than three (the slowest solves set the kernel's time).
// The lanes then exchange their miss vectors and take the same decision and update, those of
// the solve with its marches one after another, so the result is that solve's bit for bit;
// the difference marches of the step that converges are made and not used.  Each lane sums
// the bumps of its own cull cell (no warp collective): lanes follow their own geodesics.
constexpr unsigned kIllumGroups = 10;  // groups of three lanes per warp

template <int MK, int INTEG>
__global__ void __launch_bounds__(128) k_illuminate(const TraceParams P, const LightParams LP) {
  extern __shared__ float4 smem[];
  const int nb4 = stage_shared<MK>(P, smem);
  const float4 *sb = smem;
  const float4 *ss = smem + nb4;
  const unsigned lane = threadIdx.x & 31u, grp = lane / 3u, role = lane - 3u * grp;
  if (grp >= kIllumGroups) return;
  const unsigned item = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kIllumGroups + grp;
  int p;
  if (item >= P.n_items || !item_pixel(P, item, p)) return;
  const unsigned gmask = 7u << (3u * grp), base = 3u * grp;  // the group's lanes, its lane 0
  const size_t N = (size_t)P.W * P.H;
  const int id = P.id[p];
  if (id < 0) {
    if (role == 0 && LP.lit) LP.lit[p] = 0;
    return;
  }
  const F3 Ph = f3(P.hit[p], P.hit[N + p], P.hit[2 * N + p]);
  const F3 n = f3(P.hit_nrm[p], P.hit_nrm[N + p], P.hit_nrm[2 * N + p]);
  const F3 L = f3(LP.L[0], LP.L[1], LP.L[2]);
  const F3 q = axpy(1e-3f, n, Ph);
  const F3 d0 = normalize(L - q);
  // e1 across the axis least aligned with d0 (lowest index on ties), e2 = d0 x e1
  int ax = 0;
  if (fabsf(d0.y) < fabsf(d0.x)) ax = 1;
  if (fabsf(d0.z) < fabsf(ax == 0 ? d0.x : d0.y)) ax = 2;
  const F3 b1 = normalize(cross(f3(ax == 0 ? 1.f : 0.f, ax == 1 ? 1.f : 0.f, ax == 2 ? 1.f : 0.f), d0));
  const F3 b2 = cross(d0, b1);
  float al = 0.f, be = 0.f;
  bool lit = false, blocked;
  F3 u = d0;
  WorkCount evals;  // work counters
  for (int k = 0;; k++) {
    // this lane's march: the current direction (role 0) or its difference in alpha (1) or beta (2)
    const float aa = role == 1u ? al + LP.delta : al, bb = role == 2u ? be + LP.delta : be;
    F3 e, ud;
    WorkCount w;  // this march's work: counted when the solve uses the march
    const bool ok = shoot<MK, INTEG, false>(P, sb, ss, L, q, normalize(axpy(bb, b2, axpy(aa, b1, d0))), e, ud,
                                            blocked, w);
    F3 eg[3];
    bool okg[3];
    for (unsigned j = 0; j < 3u; ++j) {
      eg[j] = f3(__shfl_sync(gmask, e.x, base + j), __shfl_sync(gmask, e.y, base + j),
                 __shfl_sync(gmask, e.z, base + j));
      okg[j] = __shfl_sync(gmask, ok ? 1 : 0, base + j) != 0;
    }
    const bool conv = okg[0] && sqrtf(dot(eg[0], eg[0])) <= LP.tol;
    const bool more = okg[0] && !conv && k != LP.iters;  // the step goes on to the differences
    if (role == 0u || (more && (role == 1u || okg[1]))) {
      evals.evals += w.evals;
      evals.slots += w.slots;
    }
    if (!okg[0]) break;
    u = ud;  // role 0: the g-unit tangent of the current direction
    if (conv) {
      lit = true;
      break;
    }
    if (!more || !okg[1]) break;
    const F3 J0 = (1.f / LP.delta) * (eg[1] - eg[0]);
    if (!okg[2]) break;
    const F3 J1 = (1.f / LP.delta) * (eg[2] - eg[0]);
    // Gauss-Newton: (J^T J) step = -J^T e, by Cramer's rule
    const float A00 = dot(J0, J0), A01 = dot(J0, J1), A11 = dot(J1, J1);
    const float r0 = -dot(J0, eg[0]), r1 = -dot(J1, eg[0]);
    const float det = A00 * A11 - A01 * A01;
    if (!(det > 1e-12f * (A00 * A11))) break;
    float s0 = (r0 * A11 - r1 * A01) / det, s1 = (A00 * r1 - A01 * r0) / det;
    const float sn = sqrtf(s0 * s0 + s1 * s1);
    if (sn > 0.25f) {
      s0 *= 0.25f / sn;
      s1 *= 0.25f / sn;
    }
    al += s0;
    be += s1;
  }
  if (role == 0u) {
    float cosg = 0.f;
    if (lit) {
      cosg = dot(n, u) * rsqrtf(metric_inv_nn<MK>(P, sb, q, n));
      if (!(cosg > 0.f)) lit = false;
    }
    if (lit) {
      F3 e, uu;
      shoot<MK, INTEG, true>(P, sb, ss, L, q, normalize(axpy(be, b2, axpy(al, b1, d0))), e, uu, blocked, evals);
      if (blocked) lit = false;
    }
    const int obj = id < P.S ? id : P.S;
    const float inten = lit ? fmaf(0.9f, cosg, 0.1f) : 0.1f;
    P.rgba[p] = make_uchar4(to_u8(P.albedo[3 * obj] * inten), to_u8(P.albedo[3 * obj + 1] * inten),
                            to_u8(P.albedo[3 * obj + 2] * inten), 255);
    if (LP.lit) LP.lit[p] = lit ? 1 : 0;
  }
  if (P.bump_evals) atomicAdd(P.bump_evals, evals.evals);
  if (P.bump_slots) atomicAdd(P.bump_slots, evals.slots);
}

// The hits of a finished trace, listed in queue-item order (the trace's 32-pixel tiles) one
// warp's worth at a time: LP.hits[0 .. *LP.n_hits).  Pixels without a hit are marked unlit.
__global__ void __launch_bounds__(128) k_hit_list(const TraceParams P, const LightParams LP) {
  const unsigned item = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31u;
  int p = 0;
  bool hit = false;
  if (item < P.n_items && item_pixel(P, item, p)) {
    hit = P.id[p] >= 0;
    if (!hit && LP.lit) LP.lit[p] = 0;
  }
  const unsigned m = __ballot_sync(0xffffffffu, hit);
  unsigned first = 0;
  if (lane == 0 && m) first = atomicAdd(LP.n_hits, (unsigned)__popc(m));
  first = __shfl_sync(0xffffffffu, first, 0);
  if (hit) LP.hits[first + (unsigned)__popc(m & ((1u << lane) - 1u))] = p;
}

// The same illumination with the warp's light geodesics marched in lockstep, for isotropic
// truncated bumps with a cull grid: every iteration advances each lane's current march by one
// step, and the warp sums the bumps of one list together (the union of the marching lanes' cull
// cells, packed in pairs and kept for LP.list_steps steps, as k_trace does), so the lanes read
// each pair once by broadcast instead of walking their own cells apart.  A lane whose march has
// ended waits for the other two of its group; the group then takes the decision and update of
// k_illuminate and starts its next three marches, or ends its solve (lane 0 then marches the
// shadow geodesic).  Each march takes the steps of shoot: the lists hold every bump that is
// nonzero at a lane's stage points, in the order of the dense sums, so every pixel is the same
// bit for bit as with k_illuminate.  The grid is persistent: a warp takes the next ten hits of
// the hit list (k_hit_list) once its ten solves have ended.  COUNT false (no work counters
// asked for) leaves the counts unread, so the compiler drops them.
template <int INTEG, bool COUNT = true>
__global__ void __launch_bounds__(128, 4) k_illuminate_sl(const TraceParams P, const LightParams LP) {
  extern __shared__ float4 smem[];
  const int nb4 = stage_shared<MK_GRAPH_SL>(P, smem);
  const float4 *sb = smem;
  const float4 *ss = smem + nb4;
  WarpLists wl = warp_lists(true, smem + nb4 + (P.nodes ? 0 : P.S));
  const float4 ghdr = __ldg(P.cull_hdr);
  const unsigned lane = threadIdx.x & 31u, grp = lane / 3u, role = lane - 3u * grp;
  const unsigned base = 3u * min(grp, kIllumGroups - 1u);  // the group's lane 0 (lanes 30, 31: none)
  const unsigned n_hits = *LP.n_hits;
  const size_t N = (size_t)P.W * P.H;
  WorkCount evals;  // the lane's counts over all of its solves
  for (;;) {
    unsigned first = 0;
    if (lane == 0) first = atomicAdd(LP.hit_next, kIllumGroups);
    first = __shfl_sync(0xffffffffu, first, 0);
    if (first >= n_hits) break;
    int p = 0, id = -1;
    if (grp < kIllumGroups && first + grp < n_hits) {
      p = LP.hits[first + grp];
      id = P.id[p];
    }
    constexpr int kMarch = 0, kWait = 1, kDone = 2;
    int phase = id >= 0 ? kMarch : kDone;
    const F3 L = f3(LP.L[0], LP.L[1], LP.L[2]);
    F3 n = f3(0.f, 0.f, 1.f), q = f3(0.f, 0.f, 0.f), d0 = f3(0.f, 0.f, 1.f), b1 = d0, b2 = d0;
    if (phase == kMarch) {
      const F3 Ph = f3(P.hit[p], P.hit[N + p], P.hit[2 * N + p]);
      n = f3(P.hit_nrm[p], P.hit_nrm[N + p], P.hit_nrm[2 * N + p]);
      q = axpy(1e-3f, n, Ph);
      d0 = normalize(L - q);
      int ax = 0;  // e1 across the axis least aligned with d0 (lowest index on ties), e2 = d0 x e1
      if (fabsf(d0.y) < fabsf(d0.x)) ax = 1;
      if (fabsf(d0.z) < fabsf(ax == 0 ? d0.x : d0.y)) ax = 2;
      b1 = normalize(cross(f3(ax == 0 ? 1.f : 0.f, ax == 1 ? 1.f : 0.f, ax == 2 ? 1.f : 0.f), d0));
      b2 = cross(d0, b1);
    }
    float al = 0.f, be = 0.f;
    int k = 0;
    bool lit = false, shadow = false, ok = false, blocked = false, fresh = false;
    F3 u = d0, ud = d0, e = f3(0.f, 0.f, 0.f);
    Ray r;
    ray_clear(r);
    WorkCount w;  // the counts of the lane's current march (counted if the solve uses it)
    // starts this lane's march from q in the Euclidean direction d (shoot's first lines)
    auto start = [&](F3 d) {
      ud = rsqrtf(metric_dd<MK_GRAPH_SL>(P, sb, q, d)) * d;
      for (int c = 0; c < 3; c++) {
        r.xh[c] = comp(q, c);
        r.xl[c] = 0.f;
        r.vh[c] = comp(ud, c);
        r.vl[c] = 0.f;
      }
      r.steps = 0;
      blocked = false;
      fresh = true;
      phase = kMarch;
    };
    // the shaded colour of the hit (lane 0 of its group)
    auto finish = [&](float cosg) {
      const int obj = id < P.S ? id : P.S;
      const float inten = lit ? fmaf(0.9f, cosg, 0.1f) : 0.1f;
      P.rgba[p] = make_uchar4(to_u8(P.albedo[3 * obj] * inten), to_u8(P.albedo[3 * obj + 1] * inten),
                              to_u8(P.albedo[3 * obj + 2] * inten), 255);
      if (LP.lit) LP.lit[p] = lit ? 1 : 0;
      phase = kDone;
    };
    if (phase == kMarch) start(normalize(axpy(role == 2u ? LP.delta : 0.f, b2, axpy(role == 1u ? LP.delta : 0.f, b1, d0))));
    float cosg = 0.f;
    for (;;) {
      // the decision of every group whose three marches have ended (k_illuminate's, in its order)
      const unsigned waiting = __ballot_sync(0xffffffffu, phase == kWait);
      const bool ready = phase == kWait && ((waiting >> base) & 7u) == 7u;
      if (__any_sync(0xffffffffu, ready)) {
        F3 eg[3];
        bool okg[3];
        for (unsigned j = 0; j < 3u; ++j) {
          eg[j] = f3(__shfl_sync(0xffffffffu, e.x, base + j), __shfl_sync(0xffffffffu, e.y, base + j),
                     __shfl_sync(0xffffffffu, e.z, base + j));
          okg[j] = __shfl_sync(0xffffffffu, ok ? 1 : 0, base + j) != 0;
        }
        if (ready) {
          const bool conv = okg[0] && sqrtf(dot(eg[0], eg[0])) <= LP.tol;
          const bool more = okg[0] && !conv && k != LP.iters;
          if (role == 0u || (more && (role == 1u || okg[1]))) {
            evals.evals += w.evals;
            evals.slots += w.slots;
          }
          w = WorkCount{};
          bool next = false;
          if (okg[0]) {
            u = ud;
            if (conv) {
              lit = true;
            } else if (more && okg[1] && okg[2]) {
              const F3 J0 = (1.f / LP.delta) * (eg[1] - eg[0]);
              const F3 J1 = (1.f / LP.delta) * (eg[2] - eg[0]);
              const float A00 = dot(J0, J0), A01 = dot(J0, J1), A11 = dot(J1, J1);
              const float r0 = -dot(J0, eg[0]), r1 = -dot(J1, eg[0]);
              const float det = A00 * A11 - A01 * A01;
              if (det > 1e-12f * (A00 * A11)) {
                float s0 = (r0 * A11 - r1 * A01) / det, s1 = (A00 * r1 - A01 * r0) / det;
                const float sn = sqrtf(s0 * s0 + s1 * s1);
                if (sn > 0.25f) {
                  s0 *= 0.25f / sn;
                  s1 *= 0.25f / sn;
                }
                al += s0;
                be += s1;
                next = true;
              }
            }
          }
          if (next) {
            ++k;
            const float aa = role == 1u ? al + LP.delta : al, bb = role == 2u ? be + LP.delta : be;
            start(normalize(axpy(bb, b2, axpy(aa, b1, d0))));
          } else if (role != 0u) {
            phase = kDone;
          } else {
            if (lit) {
              cosg = dot(n, u) * rsqrtf(metric_inv_nn<MK_GRAPH_SL>(P, sb, q, n));
              if (!(cosg > 0.f)) lit = false;
            }
            if (lit) {
              shadow = true;
              start(normalize(axpy(be, b2, axpy(al, b1, d0))));
            } else {
              finish(cosg);
            }
          }
        }
      }
      if (__all_sync(0xffffffffu, phase == kDone)) break;
      // one step of every lane's march, the warp's sums together
      const bool marching = phase == kMarch;
      WorkCount *wc = marching && !shadow ? &w : &evals;
      step_list_refresh(P, sb, wl, ghdr, marching, fresh, xhi(r));
      fresh = false;
      bool inside = true;
      F3 x = xhi(r);
      const F3 v = vhi(r);
      F3 a1 = accel<MK_GRAPH_SL, true>(P, sb, SumCtx{ghdr, &wl, marching, wc}, x, v, inside);
      bool ended = false, moved = false;
      if (marching && P.skippable && !inside) {
        // straight line x + t v: closest approach to L at tL, next support ball at te
        const float te = support_entry<MK_GRAPH_SL>(sb, P.K, x, v);
        const F3 wv = L - x;
        const float tL = fmaxf(dot(wv, v) / dot(v, v), 0.f);
        const float tend = fminf(tL, te);
        HitRec hr;
        if (shadow && tend > 0.f && scene_hit(P, ss, x, v, tend, hr)) {
          blocked = true;
          ok = ended = true;
        } else if (tL <= te) {
          e = axpy(tL, v, x) - L;
          ok = ended = true;
        } else {
          for (int c = 0; c < 3; c++) comp_add(r.xh[c], r.xl[c], te * comp(v, c));
          x = xhi(r);
          moved = true;
        }
      }
      if (__any_sync(0xffffffffu, moved)) {
        // the advance left the list's reach: list afresh at every marching lane's position
        if (wl.np >= 0) step_list(P, sb, wl, ghdr, marching && !ended, x);
        bool dummy;
        const F3 am = accel<MK_GRAPH_SL, false>(P, sb, SumCtx{ghdr, &wl, moved, wc}, x, v, dummy);
        if (moved) a1 = am;
      }
      if (marching && !ended && r.steps >= P.max_steps) {
        ok = false;
        ended = true;
      }
      const bool go = marching && !ended;
      if (__any_sync(0xffffffffu, go)) {
        F3 dx, dvel;
        step_increments<MK_GRAPH_SL, INTEG>(P, sb, SumCtx{ghdr, &wl, go, wc}, x, v, a1, dx, dvel);
        if (go) {
          for (int c = 0; c < 3; c++) {
            comp_add(r.xh[c], r.xl[c], comp(dx, c));
            comp_add(r.vh[c], r.vl[c], comp(dvel, c));
          }
          ++r.steps;
          const F3 D = xhi(r) - x;
          const float t = dot(L - x, D) / dot(D, D);
          HitRec hr;
          if (t < 1.f) {  // the closest approach lies on this segment (or the distance grows)
            const float tc = fmaxf(t, 0.f);
            if (shadow && tc > 0.f && scene_hit(P, ss, x, D, tc, hr)) blocked = true;
            else e = axpy(tc, D, x) - L;
            ok = ended = true;
          } else if (shadow && scene_hit(P, ss, x, D, 1.f, hr)) {
            blocked = true;
            ok = ended = true;
          }
        }
      }
      ++wl.age;
      if (ended) {
        if (shadow) {  // lane 0's shadow geodesic
          if (blocked) lit = false;
          finish(cosg);
        } else {
          phase = kWait;
        }
      }
    }
  }
  if (COUNT && P.bump_evals) atomicAdd(P.bump_evals, evals.evals);
  if (COUNT && P.bump_slots) atomicAdd(P.bump_slots, evals.slots);
}

#endif

#if RGEO_PART(1)
// Eq. 5.4 for two rays against the same isotropic bumps (dense sums): each pair of
// bumps loaded from shared memory serves both rays, halving shared-memory traffic per ray.
template <bool INSIDE>
__device__ __forceinline__ void accel_graph_iso_x2(const TraceParams &P, const float4 *__restrict__ sb, int K,
                                                   F3 xa, F3 va, F3 xb, F3 vb, F3 &aa, F3 &ab, bool &ina,
                                                   bool &inb) {
  PairAcc A, B;
  pair_acc_init(A, xa, va);
  pair_acc_init(B, xb, vb);
  const int n4 = kIsoBumpStride * iso_pad_index(K);
#pragma unroll 1
  for (int i = 0; i < n4; i += 2 * kIsoBumpStride) {
    pair_eval<INSIDE>(A, sb, i, i + kIsoBumpStride);
    pair_eval<INSIDE>(B, sb, i, i + kIsoBumpStride);
  }
  aa = pair_acc_finish(P, A, xa, va);
  ab = pair_acc_finish(P, B, xb, vb);
  if (INSIDE) {
    ina = A.in;
    inb = B.in;
  }
}

// Two rays per thread (isotropic graph metric): both rays step together and share
// every bump pair read from shared memory; each has its own refill, skip and
// termination.  An empty slot keeps evaluating its last state (results unused).
template <int INTEG>
__global__ void __launch_bounds__(128) k_trace_x2(const TraceParams P) {
  extern __shared__ float4 smem[];
  const int nb4 = stage_shared<MK_GRAPH_ISO>(P, smem);
  const float4 *sb = smem;
  const float4 *ss = smem + nb4;
  bool act0 = false, act1 = false, drained = false;
  WorkCount evals;
  Ray r0, r1;
  for (int c = 0; c < 3; c++) {
    r0.xh[c] = r0.vh[c] = r1.xh[c] = r1.vh[c] = 0.f;
    r0.xl[c] = r0.vl[c] = r1.xl[c] = r1.vl[c] = 0.f;
  }
  const float h = P.h;
  for (;;) {
    refill<MK_GRAPH_ISO>(P, sb, act0, drained, r0);
    refill<MK_GRAPH_ISO>(P, sb, act1, drained, r1);
    const unsigned m0 = __ballot_sync(0xffffffffu, act0), m1 = __ballot_sync(0xffffffffu, act1);
    if (!(m0 | m1)) {
      if (drained) break;
      continue;
    }
    if (!act0 && !act1) continue;
    bool in0 = true, in1 = true;
    F3 a10, a11;
    accel_graph_iso_x2<true>(P, sb, P.K, xhi(r0), vhi(r0), xhi(r1), vhi(r1), a10, a11, in0, in1);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);  // this kernel sums densely (no cull grid)
    WarpLists nolists{nullptr, nullptr, -1, 0u, 0};
    evals.evals += 2ull * (unsigned)P.K;
    evals.slots += 2u * (unsigned)iso_pad_index(P.K);
    if (act0) act0 = pre_step<MK_GRAPH_ISO, false>(P, sb, ss, SumCtx{z4, &nolists, true, &evals}, r0, a10, in0);
    if (act1) act1 = pre_step<MK_GRAPH_ISO, false>(P, sb, ss, SumCtx{z4, &nolists, true, &evals}, r1, a11, in1);
    if (!act0 && !act1) continue;
    const F3 x0 = xhi(r0), v0 = vhi(r0), x1 = xhi(r1), v1 = vhi(r1);
    F3 dx0, dv0, dx1, dv1;
    if (INTEG == 0) {
      bool dummy0, dummy1;
      const float h2 = 0.5f * h;
      const F3 v20 = axpy(h2, a10, v0), v21 = axpy(h2, a11, v1);
      F3 a20, a21;
      accel_graph_iso_x2<false>(P, sb, P.K, axpy(h2, v0, x0), v20, axpy(h2, v1, x1), v21, a20, a21, dummy0,
                                dummy1);
      const F3 v30 = axpy(h2, a20, v0), v31 = axpy(h2, a21, v1);
      F3 a30, a31;
      accel_graph_iso_x2<false>(P, sb, P.K, axpy(h2, v20, x0), v30, axpy(h2, v21, x1), v31, a30, a31, dummy0,
                                dummy1);
      const F3 v40 = axpy(h, a30, v0), v41 = axpy(h, a31, v1);
      F3 a40, a41;
      accel_graph_iso_x2<false>(P, sb, P.K, axpy(h, v30, x0), v40, axpy(h, v31, x1), v41, a40, a41, dummy0,
                                dummy1);
      evals.evals += 6ull * (unsigned)P.K;
      evals.slots += 6u * (unsigned)iso_pad_index(P.K);
      const float h6 = h * (1.f / 6.f);
      dx0 = h6 * (v0 + 2.f * (v20 + v30) + v40);
      dv0 = h6 * (a10 + 2.f * (a20 + a30) + a40);
      dx1 = h6 * (v1 + 2.f * (v21 + v31) + v41);
      dv1 = h6 * (a11 + 2.f * (a21 + a31) + a41);
    } else {
      dx0 = h * v0;
      dv0 = h * a10;
      dx1 = h * v1;
      dv1 = h * a11;
    }
    if (act0) act0 = post_step<MK_GRAPH_ISO>(P, sb, ss, r0, dx0, dv0);
    if (act1) act1 = post_step<MK_GRAPH_ISO>(P, sb, ss, r1, dx1, dv1);
  }
  evals.flush(P);
}

#endif

// Many instances (frames, views or metrics of uneven size) in one persistent launch.
// Each warp serves one instance at a time: its lanes refill from that instance's
// queue (the instance's own counter), and once the instance is drained and the
// warp's lanes are idle it moves to the next instance.  Bump tables, cull masks
// and spheres are read through L1 because warps of one block may be on
// different instances.  All instances share the metric kind and integrator.
// Shared-memory slot of one warp in the batch kernel: a copy of the current
// instance's parameters, then (when it fits) its packed bump table.
constexpr int kParamWords = (int)((sizeof(TraceParams) + 15) / 16) * 4;

// Copies instance i's bump table into the warp's shared-memory table (SMEM: the
// launcher made it large enough for every instance) or reads it through L1.  Keeping
// the two cases apart lets the compiler see that sb points to shared memory.
template <bool SMEM>
__device__ __forceinline__ void warp_load_table(const TraceParams &P, float4 *tab, const float4 *&sb) {
  if (SMEM) {
    const unsigned lane = threadIdx.x & 31u;
    const int need = table_float4s(P.kind, P.K, P.aniso);
    __syncwarp();  // every lane is done with the previous table
    for (int k = (int)lane; k < need; k += 32) tab[k] = __ldg(P.bumps + k);
    sb = tab;
  } else {
    sb = P.bumps;
  }
  __syncwarp();
}

// Instance parameters from a per-warp shared-memory copy (any number of instances).  The
// warp's slot holds the parameters, then (when it fits) the bump table, then its pair list.
struct SmemInstances {
  const TraceParams *inst;
  uint32_t *slot;
  int table_f4;
  bool step;
  __device__ __forceinline__ const TraceParams &get(int) const {
    return *reinterpret_cast<const TraceParams *>(slot);
  }
  __device__ __forceinline__ float4 *table() const { return reinterpret_cast<float4 *>(slot + kParamWords); }
  __device__ __forceinline__ WarpLists lists() const {
    float4 *b = table() + table_f4;
    return WarpLists{reinterpret_cast<int2 *>(b), step ? b + kListFloat4 : nullptr, -1, 0u, 0};
  }
  __device__ __forceinline__ void load(int i) const {
    const unsigned lane = threadIdx.x & 31u;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(inst + i);
    __syncwarp();  // every lane is done with the previous instance's parameters
    for (int k = (int)lane; k < (int)(sizeof(TraceParams) / 4); k += 32) slot[k] = __ldg(src + k);
    __syncwarp();
  }
};

// Instance parameters from the kernel's parameter space (up to kMaxParamInstances),
// where field reads are constant-cache loads shared by the whole warp; the warp's slot in
// shared memory holds the bump table (when it fits) and the pair list.
struct ParamInstances {
  const BatchTable *T;
  float4 *tab;
  int table_f4;
  bool step;
  __device__ __forceinline__ const TraceParams &get(int i) const { return T->inst[i]; }
  __device__ __forceinline__ float4 *table() const { return tab; }
  __device__ __forceinline__ WarpLists lists() const {
    float4 *b = tab + table_f4;
    return WarpLists{reinterpret_cast<int2 *>(b), step ? b + kListFloat4 : nullptr, -1, 0u, 0};
  }
  __device__ __forceinline__ void load(int) const {}
};

// The batch loop: every warp starts on instance 0 (the launcher orders instances by
// decreasing cost) and moves to the next one once the current instance's queue is
// drained, reloading parameters and bump table; the end of one instance overlaps the
// start of the next, and only one instance's structures are hot at a time.
template <int MK, int INTEG, bool SMEM, class Src>
__device__ __forceinline__ void batch_loop(const Src &src, int n) {
  constexpr bool conv = Converged<MK>::value;
  int i = 0;
  int visited = 0;
  WorkCount evals;
  bool active = false, drained = false;
  Ray r;
  ray_clear(r);
  unsigned cnext = 0u, cend = 0u;
  const float4 *sb = nullptr;
  WarpLists wl = src.lists();
  src.load(i);
  warp_load_table<SMEM>(src.get(i), src.table(), sb);
  for (;;) {
    const TraceParams &P = src.get(i);
    const float4 *ss = P.spheres;
    const bool held = active;
    refill_tile<MK>(P, sb, active, drained, r, cnext, cend);
    const unsigned amask = __ballot_sync(0xffffffffu, active);
    if (!amask) {
      if (drained) {
        evals.flush(P);
        if (++visited >= n) break;
        i = (i + 1) % n;
        drained = false;
        cnext = cend = 0u;
        wl.np = -1;  // the next instance's lists start afresh
        src.load(i);
        warp_load_table<SMEM>(src.get(i), src.table(), sb);
      }
      continue;
    }
    if (!conv && !active) continue;
    const float4 ghdr = P.cull_masks ? __ldg(P.cull_hdr) : make_float4(0.f, 0.f, 0.f, 0.f);
    if (MK == MK_GRAPH_SL) step_list_refresh(P, sb, wl, ghdr, active, active && !held, xhi(r));
    bool inside = true;
    F3 a1 = accel<MK, true>(P, sb, SumCtx{ghdr, &wl, active, &evals}, xhi(r), vhi(r), inside);
    const bool go = pre_step<MK>(P, sb, ss, SumCtx{ghdr, &wl, active, &evals}, r, a1, inside);
    if (!go) active = false;
    if (conv ? !__any_sync(0xffffffffu, go) : !go) continue;
    F3 dx, dvel;
    step_increments<MK, INTEG>(P, sb, SumCtx{ghdr, &wl, go, &evals}, xhi(r), vhi(r), a1, dx, dvel);
    if (go) active = post_step<MK>(P, sb, ss, r, dx, dvel);
    ++wl.age;
  }
}

template <int MK, int INTEG, bool SMEM>
__global__ void __launch_bounds__(128, 5) k_trace_batch(const TraceParams *__restrict__ inst, int n, int table_f4) {
  extern __shared__ float4 bsmem[];
  constexpr bool step = MK == MK_GRAPH_SL;
  uint32_t *slot = reinterpret_cast<uint32_t *>(bsmem) +
                   (threadIdx.x >> 5) * (kParamWords + 4 * table_f4 + 4 * lists_float4(step));
  batch_loop<MK, INTEG, SMEM>(SmemInstances{inst, slot, table_f4, step}, n);
}

template <int MK, int INTEG, bool SMEM>
__global__ void __launch_bounds__(128, 5) k_trace_batch_param(const __grid_constant__ BatchTable T, int n,
                                                           int table_f4) {
  extern __shared__ float4 bsmem[];
  constexpr bool step = MK == MK_GRAPH_SL;
  float4 *tab = bsmem + (threadIdx.x >> 5) * (table_f4 + lists_float4(step));
  batch_loop<MK, INTEG, SMEM>(ParamInstances{&T, tab, table_f4, step}, n);
}

// ------------------------------------------------------- surrogate tracer
// Rays advance in rounds.  In a round each ray runs RK4 steps (as k_trace) until it
// finishes or reaches a point from which a surrogate jump is allowed; it then saves
// its state and joins the jump queue.  Between rounds the network evaluates the
// queue (tensor cores) and k_wave_apply takes each jump whose predicted error is
// within the threshold; a rejected ray integrates that segment by RK4 instead.

__device__ __forceinline__ void wave_store(const WaveArgs &W, const Ray &r, int cool) {
  const size_t N = (size_t)W.N, p = (size_t)r.pix;
  for (int c = 0; c < 3; c++) {
    W.st[c * N + p] = r.xh[c];
    W.st[(3 + c) * N + p] = r.xl[c];
    W.st[(6 + c) * N + p] = r.vh[c];
    W.st[(9 + c) * N + p] = r.vl[c];
  }
  W.st[12 * N + p] = r.dleft;
  W.st[13 * N + p] = r.e0m1;
  W.st[14 * N + p] = r.arc;
  W.steps[p] = r.steps;
  W.cool[p] = cool;
}

__device__ __forceinline__ void wave_load(const WaveArgs &W, int pix, Ray &r, int &cool) {
  const size_t N = (size_t)W.N, p = (size_t)pix;
  for (int c = 0; c < 3; c++) {
    r.xh[c] = W.st[c * N + p];
    r.xl[c] = W.st[(3 + c) * N + p];
    r.vh[c] = W.st[(6 + c) * N + p];
    r.vl[c] = W.st[(9 + c) * N + p];
  }
  r.dleft = W.st[12 * N + p];
  r.e0m1 = W.st[13 * N + p];
  r.arc = W.st[14 * N + p];
  r.steps = W.steps[p];
  r.pix = pix;
  r.nb = 0;
  cool = W.cool[p];
}

// As refill, but a ray of a later round resumes from its saved state.
template <int MK>
__device__ __forceinline__ void wave_refill(const TraceParams &P, const WaveArgs &W, const float4 *sb,
                                            bool &active, bool &drained, Ray &r, int &cool, unsigned &cnext,
                                            unsigned &cend) {
  const unsigned lane = threadIdx.x & 31u;
  for (int pass = 0; pass < 2; ++pass) {
    const unsigned need = __ballot_sync(0xffffffffu, !active && !drained);
    if (!need) return;
    if (cnext >= cend) {  // a warp-private chunk of 32 items (in the first round, one tile)
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(P.counter, 32u);
      base = __shfl_sync(0xffffffffu, base, 0);
      cnext = base;
      cend = base + 32u;
      if (base >= P.n_items) {
        drained = true;
        return;
      }
    }
    const unsigned take = min((unsigned)__popc(need), cend - cnext);
    const unsigned rank = (unsigned)__popc(need & ((1u << lane) - 1u));
    if (((need >> lane) & 1u) && rank < take) {
      const unsigned item = cnext + rank;
      if (item < P.n_items) {
        int pix;
        if (W.first) {
          if (item_pixel(P, item, pix)) {
            init_ray<MK>(P, sb, pix, r);
            cool = 0;
            active = true;
          }
        } else {
          wave_load(W, W.list_in[item], r, cool);
          active = true;
        }
      }
    }
    cnext += take;
  }
}

// Queue a jump of k steps (arc length s = k h) when it is certified free of the
// scene: g = I + grad f grad f^T >= I (Eq. 5.2), so a geodesic of g-length s with a
// g-unit tangent stays within Euclidean distance s of x, and the safe distance at x
// bounds the distance to every scene point from below.  The network was trained on
// |x_i| <= box; k is at least k_min and fits the step budget.  Under a far-field
// bound, k is halved (up to twice) until the bound holds over the jump.
template <int MK>
__device__ __forceinline__ bool wave_try_queue(const TraceParams &P, const WaveArgs &W, const float4 *sb, Ray &r,
                                               int &cool) {
  const F3 x = xhi(r), v = vhi(r);
  int k = -1;
  if (fabsf(x.x) <= W.box && fabsf(x.y) <= W.box && fabsf(x.z) <= W.box) {
    const float reach = fminf(W.s_max, (safe_distance(P, x) - 1e-4f) * (1.f / 1.01f));
    if (reach > 0.f) k = min((int)(reach / P.h), P.max_steps - r.steps);
  }
  if (is_iso(MK) && W.accel_bound > 0.f) {
    bool ok = false;
    for (int t = 0; t < 3 && k >= W.k_min && !ok; ++t) {
      ok = far_field_bound(sb, P.K, x, k * P.h) <= W.accel_bound;
      if (!ok) k >>= 1;
    }
    if (!ok) k = -1;
  }
  if (k < W.k_min) {
    cool = W.cool_check;
    return false;
  }
  const unsigned lane = threadIdx.x & 31u;
  const unsigned m = __activemask();
  const int leader = __ffs(m) - 1;
  unsigned base = 0;
  if ((int)lane == leader) base = atomicAdd(W.n_queue, (unsigned)__popc(m));
  base = __shfl_sync(m, base, leader);
  const unsigned slot = base + (unsigned)__popc(m & ((1u << lane) - 1u));
  W.queue[slot] = r.pix;
  W.jump_k[slot] = k;
  const float inv = rsqrtf(dot(v, v));
  float *xi = W.X + (size_t)slot * 7;
  const float ib = 1.f / W.box;
  xi[0] = x.x * ib;
  xi[1] = x.y * ib;
  xi[2] = x.z * ib;
  xi[3] = v.x * inv;
  xi[4] = v.y * inv;
  xi[5] = v.z * inv;
  xi[6] = (k * P.h) / W.s_max;
  wave_store(W, r, 0);
  return true;
}

// One round of the surrogate tracer (graph metrics, RK4).
template <int MK>
__global__ void __launch_bounds__(128, 5) k_wave_trace(const TraceParams P, const WaveArgs W) {
  extern __shared__ float4 smem[];
  const int nb4 = stage_shared<MK>(P, smem);
  const float4 *sb = smem;
  const float4 *ss = smem + nb4;
  WarpLists wl = warp_lists(MK == MK_GRAPH_SL, smem + nb4 + (P.nodes ? 0 : P.S));
  const float4 ghdr = P.cull_masks ? __ldg(P.cull_hdr) : make_float4(0.f, 0.f, 0.f, 0.f);
  constexpr bool conv = Converged<MK>::value;
  WorkCount evals;
  bool active = false, drained = false;
  Ray r;
  ray_clear(r);
  int cool = 0;
  unsigned cnext = 0u, cend = 0u;
  for (;;) {
    const bool held = active;
    wave_refill<MK>(P, W, sb, active, drained, r, cool, cnext, cend);
    const unsigned amask = __ballot_sync(0xffffffffu, active);
    if (!amask) {
      if (drained) break;
      continue;
    }
    if (!conv && !active) continue;
    if (MK == MK_GRAPH_SL) step_list_refresh(P, sb, wl, ghdr, active, active && !held, xhi(r));
    bool inside = true;
    F3 a1 = accel<MK, true>(P, sb, SumCtx{ghdr, &wl, active, &evals}, xhi(r), vhi(r), inside);
    if (active && inside && r.steps < P.max_steps) {
      bool queued = false;
      if (cool <= 0) queued = wave_try_queue<MK>(P, W, sb, r, cool);
      else --cool;
      if (queued) active = false;
    }
    if (!conv && !active) continue;
    const bool go = pre_step<MK>(P, sb, ss, SumCtx{ghdr, &wl, active, &evals}, r, a1, inside);
    if (!go) active = false;
    if (conv ? !__any_sync(0xffffffffu, go) : !go) continue;
    F3 dx, dvel;
    step_increments<MK, 0>(P, sb, SumCtx{ghdr, &wl, go, &evals}, xhi(r), vhi(r), a1, dx, dvel);
    if (go) active = post_step<MK>(P, sb, ss, r, dx, dvel);
    ++wl.age;
  }
  evals.flush(P);
}

#if RGEO_PART(3)
// The network's jump for queue slot i: x_s = x + s v + s^2 r_x, v_s = v + s r_v
// (scaled residuals of Eq. 3.5's exp map), taken when the predicted log squared
// error (output 6) is at most log tau^2; otherwise the ray integrates the segment.
__global__ void k_wave_apply(const WaveArgs W, unsigned n, float h) {
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  int acc = 0, rej = 0;
  if (i < n) {
    const int p = W.queue[i], k = W.jump_k[i];
    const float *y = W.Y + (size_t)i * 7;
    float yv[7];
    bool finite = true;
    for (int o = 0; o < 7; o++) {
      yv[o] = y[o];
      finite = finite && isfinite(yv[o]);
    }
    const size_t N = (size_t)W.N;
    const float sc = W.accel_bound > 0.f ? W.accel_bound : 1.f;  // targets were divided by the bound
    for (int o = 0; o < 6; o++) yv[o] *= sc;
    if (finite && yv[6] <= W.log_tau2) {
      const float s = k * h, s2 = s * s;
      for (int c = 0; c < 3; c++) {
        float xh = W.st[c * N + p], xl = W.st[(3 + c) * N + p];
        float vh = W.st[(6 + c) * N + p], vl = W.st[(9 + c) * N + p];
        const float v = vh;
        comp_add(xh, xl, fmaf(s2, yv[c], s * v));
        comp_add(vh, vl, s * yv[3 + c]);
        W.st[c * N + p] = xh;
        W.st[(3 + c) * N + p] = xl;
        W.st[(6 + c) * N + p] = vh;
        W.st[(9 + c) * N + p] = vl;
      }
      W.st[12 * N + p] = 0.f;  // the next chord queries the safe distance afresh
      W.st[14 * N + p] += s;   // arc length of the jump
      W.steps[p] += k;
      W.cool[p] = 0;
      acc = 1;
    } else {
      W.cool[p] = k;
      rej = 1;
    }
  }
  const int na = __syncthreads_count(acc), nr = __syncthreads_count(rej);
  if (threadIdx.x == 0 && (na | nr)) {
    atomicAdd(&W.stats[0], (unsigned long long)na);
    atomicAdd(&W.stats[1], (unsigned long long)nr);
  }
}

#endif

#if RGEO_PART(1)
// Bump motion c_k(t) = c0_k + A_k sin(2 pi f_k t + phi_k) (per axis), then the packed
// table; t is read from and advanced in device memory so that a captured graph
// animates without host input.  motion = [K*3 c0 | K*3 A | K f | K phi].
__global__ void k_advance_motion(const float *motion, int K, int aniso, const int32_t *perm, float *raw,
                                 float4 *bumps, float *t, float dt) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;  // table slot k holds bump u
  const float tt = *t;
  if (k < K) {
    const int u = perm ? perm[k] : k;
    const float f = motion[6 * K + u], ph = motion[7 * K + u];
    const float s = sinf(6.283185307179586f * f * tt + ph);
    float c[3];
    for (int a = 0; a < 3; a++) {
      c[a] = motion[3 * u + a] + motion[3 * K + 3 * u + a] * s;
      raw[3 * u + a] = c[a];
    }
    if (aniso) {
      float4 b = bumps[kAnisoStride * k];
      b.x = c[0];
      b.y = c[1];
      b.z = c[2];
      bumps[kAnisoStride * k] = b;
    } else {
      float4 b = bumps[kIsoBumpStride * k];
      b.x = -c[0];
      b.y = -c[1];
      b.z = -c[2];
      bumps[kIsoBumpStride * k] = b;
    }
  }
}

#endif

#if RGEO_PART(3)
// Counter-based uniform in [0, 1): SplitMix64 (Steele, Lea, Flood 2014) output for the
// state seed + (i + 1) golden, top 24 bits.
__device__ __forceinline__ float u01(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)(z >> 40) * (1.f / 16777216.f);
}

// Training segments of the learned exponential map (Eq. 3.5): sample i draws a
// position x ~ U[-box, box]^3, a direction d uniform on S^2 and an arc length
// s = n h with n uniform in 1..round(s_max / h); its g-unit tangent v then follows the
// geodesic flow for n RK4 steps (dense sums) to (x_s, v_s).  Written per sample:
//   X = (x / box, d, s / s_max)                    (the network input)
//   T = ((x_s - x - s v) / s^2, (v_s - v) / s)     (scaled residuals of the straight line)
template <int MK>
__global__ void k_segments(const TraceParams P, long long n, unsigned long long seed, float box, float s_max,
                           float accel_bound, float *X, float *T) {
  const int nmax = max(1, (int)roundf(s_max / P.h));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    // candidate j of sample i draws counters 8 (j n + i) .. + 5; with a far-field bound
    // the first candidate within it is kept (the last one if none of kSegTries is)
    F3 x0, d;
    int steps = 1;
    const int tries = accel_bound > 0.f ? kSegTries : 1;
    for (int j = 0; j < tries; ++j) {
      const unsigned long long base = ((unsigned long long)j * (unsigned long long)n + (unsigned long long)i) * 8ull;
      x0 = f3(box * (2.f * u01(seed, base) - 1.f), box * (2.f * u01(seed, base + 1) - 1.f),
              box * (2.f * u01(seed, base + 2) - 1.f));
      const float z = 2.f * u01(seed, base + 3) - 1.f, ph = 6.283185307179586f * u01(seed, base + 4);
      const float rxy = sqrtf(fmaxf(0.f, 1.f - z * z));
      d = f3(rxy * cosf(ph), rxy * sinf(ph), z);
      steps = min(nmax, 1 + (int)(u01(seed, base + 5) * nmax));
      if (accel_bound <= 0.f || far_field_bound(P.bumps, P.K, x0, steps * P.h) <= accel_bound) break;
    }
    const float s = steps * P.h;
    F3 g = grad_f<MK>(P, P.bumps, x0);
    const float gd = dot(g, d);
    const F3 v0 = rsqrtf(fmaf(gd, gd, dot(d, d))) * d;
    float xh[3] = {x0.x, x0.y, x0.z}, xl[3] = {0.f, 0.f, 0.f}, vh[3] = {v0.x, v0.y, v0.z}, vl[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < steps; ++k) {
      const F3 x = f3(xh[0], xh[1], xh[2]), v = f3(vh[0], vh[1], vh[2]);
      bool dummy;
      const F3 a1 = MK == MK_GRAPH_ISO ? accel_graph_iso<false>(P, P.bumps, P.K, x, v, dummy)
                                       : accel_graph_aniso<false>(P, P.bumps, P.K, x, v, dummy);
      const float h = P.h, h2 = 0.5f * h;
      const F3 v2 = axpy(h2, a1, v);
      const F3 a2 = MK == MK_GRAPH_ISO ? accel_graph_iso<false>(P, P.bumps, P.K, axpy(h2, v, x), v2, dummy)
                                       : accel_graph_aniso<false>(P, P.bumps, P.K, axpy(h2, v, x), v2, dummy);
      const F3 v3 = axpy(h2, a2, v);
      const F3 a3 = MK == MK_GRAPH_ISO ? accel_graph_iso<false>(P, P.bumps, P.K, axpy(h2, v2, x), v3, dummy)
                                       : accel_graph_aniso<false>(P, P.bumps, P.K, axpy(h2, v2, x), v3, dummy);
      const F3 v4 = axpy(h, a3, v);
      const F3 a4 = MK == MK_GRAPH_ISO ? accel_graph_iso<false>(P, P.bumps, P.K, axpy(h, v3, x), v4, dummy)
                                       : accel_graph_aniso<false>(P, P.bumps, P.K, axpy(h, v3, x), v4, dummy);
      const float h6 = h * (1.f / 6.f);
      const F3 dx = h6 * (v + 2.f * (v2 + v3) + v4), dv = h6 * (a1 + 2.f * (a2 + a3) + a4);
      for (int c = 0; c < 3; c++) {
        comp_add(xh[c], xl[c], comp(dx, c));
        comp_add(vh[c], vl[c], comp(dv, c));
      }
    }
    float *xo = X + i * 7, *to = T + i * 6;
    xo[0] = x0.x / box;
    xo[1] = x0.y / box;
    xo[2] = x0.z / box;
    xo[3] = d.x;
    xo[4] = d.y;
    xo[5] = d.z;
    xo[6] = s / s_max;
    const float tsc = accel_bound > 0.f ? 1.f / accel_bound : 1.f;
    const float is2 = tsc / (s * s), is = tsc / s;
    for (int c = 0; c < 3; c++) {
      // (x_s - x - s v) from the compensated pair: (hi - x) + lo - s v
      const float dxs = (xh[c] - comp(x0, c)) + xl[c] - s * comp(v0, c);
      to[c] = dxs * is2;
      to[3 + c] = ((vh[c] - comp(v0, c)) + vl[c]) * is;
    }
  }
}

#endif

#if RGEO_PART(1)
__global__ void k_tick(float *t, float dt) { *t += dt; }
__global__ void k_set_time(float *t, float value) { *t = value; }

// Packs table slot k (isotropic: one thread per slot of the padded table, so the inert pad
// bumps K .. Ke are written too) from bump perm[k] (k without a permutation).
__global__ void k_pack_bumps(const float *raw, int K, float cutoff, int aniso, const int32_t *perm, float4 *out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int limit = aniso ? K : iso_pad_index(K) + 1;
  if (k >= limit) return;
  const bool pad = k >= K;
  const int u = pad ? 0 : (perm ? perm[k] : k);
  const float *c = raw + 3 * u;
  const float a = pad ? 0.f : raw[3 * K + u];
  const float *sg = raw + 4 * K + 3 * u;
  if (!aniso) {
    pack_iso_bump(out, k, c[0], c[1], c[2], a, sg[0], cutoff);
    return;
  }
  const bool inert = a == 0.f;
  const float la = inert ? -__int_as_float(0x7f800000) : log2f(fabsf(a));
  const float sgn = a > 0.f ? 1.f : (a < 0.f ? -1.f : 0.f);
  const float inf = __int_as_float(0x7f800000);
  const float smax = fmaxf(sg[0], fmaxf(sg[1], sg[2]));
  float Rb = cutoff > 0.f ? (cutoff * smax) * (cutoff * smax) : inf;
  float c2 = cutoff > 0.f ? cutoff * cutoff : inf;
  if (inert) {
    Rb = -1.f;
    c2 = -1.f;
  }
  out[3 * k] = make_float4(c[0], c[1], c[2], Rb);
  out[3 * k + 1] = make_float4(1.f / (sg[0] * sg[0]), 1.f / (sg[1] * sg[1]), 1.f / (sg[2] * sg[2]), sgn);
  out[3 * k + 2] = make_float4(la, c2, 0.f, 0.f);
}

// Table slot k takes the centre of bump perm[k] (k without a permutation) from c [K*3].
__global__ void k_set_centers(const float *c, int K, int aniso, const int32_t *perm, float4 *bumps) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const float *cu = c + 3 * (perm ? perm[k] : k);
  if (aniso) {
    float4 b = bumps[kAnisoStride * k];
    b.x = cu[0];
    b.y = cu[1];
    b.z = cu[2];
    bumps[kAnisoStride * k] = b;
  } else {
    float4 b = bumps[kIsoBumpStride * k];
    b.x = -cu[0];
    b.y = -cu[1];
    b.z = -cu[2];
    bumps[kIsoBumpStride * k] = b;
  }
}

// Cull grid, step 1 (one block): bounding box of every live support ball, inflated
// by kCullInflate + reach; hdr[0] = (min corner, 1 / cell), hdr[1].x = cell (cubic cells, G
// along the longest axis).  With no live bump, hdr[0].w = 0 and every mask is empty.
__global__ void k_cull_bounds(const float4 *bumps, int K, int G, float reach, float4 *hdr) {
  __shared__ float red[6][256];
  float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const IsoBump b = iso_bump(bumps, k);
    if (!(b.R2 >= 0.f) || isinf(b.R2)) continue;
    const float R = sqrtf(b.R2) + kCullInflate + reach;
    for (int c = 0; c < 3; c++) {
      lo[c] = fminf(lo[c], comp(b.c, c) - R);
      hi[c] = fmaxf(hi[c], comp(b.c, c) + R);
    }
  }
  for (int c = 0; c < 3; c++) {
    red[c][threadIdx.x] = lo[c];
    red[3 + c][threadIdx.x] = hi[c];
  }
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int c = 0; c < 3; c++) {
        red[c][threadIdx.x] = fminf(red[c][threadIdx.x], red[c][threadIdx.x + s]);
        red[3 + c][threadIdx.x] = fmaxf(red[3 + c][threadIdx.x], red[3 + c][threadIdx.x + s]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    float ext = 0.f;
    for (int c = 0; c < 3; c++) ext = fmaxf(ext, red[3 + c][0] - red[c][0]);
    if (!(ext > 0.f) || !(red[0][0] < FLT_MAX)) {
      hdr[0] = make_float4(0.f, 0.f, 0.f, 0.f);
      hdr[1] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      const float cell = ext / (float)G;
      hdr[0] = make_float4(red[0][0], red[1][0], red[2][0], 1.f / cell);
      hdr[1] = make_float4(cell, 0.f, 0.f, 0.f);
    }
  }
}

// Cull grid, step 2 (one thread per cell): bit k of the cell's words is set when the
// live support ball of bump k (radius + kCullInflate + reach) meets the cell box.
__global__ void k_cull_masks(const float4 *bumps, int K, int G, int words, float reach, const float4 *hdr,
                             uint32_t *masks) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= (long long)G * G * G) return;
  uint32_t *out = masks + cell * words;
  const float4 h0 = hdr[0];
  if (h0.w == 0.f) {
    for (int w = 0; w < words; ++w) out[w] = 0u;
    return;
  }
  const float cs = hdr[1].x;
  const int ix = (int)(cell % G), iy = (int)((cell / G) % G), iz = (int)(cell / ((long long)G * G));
  const float lo[3] = {h0.x + ix * cs, h0.y + iy * cs, h0.z + iz * cs};
  for (int w = 0; w < words; ++w) {
    uint32_t bits = 0u;
    for (int b = 0; b < 32; ++b) {
      const int k = w * 32 + b;
      if (k >= K) break;
      const IsoBump bb = iso_bump(bumps, k);
      if (!(bb.R2 >= 0.f) || isinf(bb.R2)) continue;
      const float R = sqrtf(bb.R2) + kCullInflate + reach;
      float d2 = 0.f;
      for (int c = 0; c < 3; c++) {
        const float cc = comp(bb.c, c);
        const float e = fmaxf(fmaxf(lo[c] - cc, cc - (lo[c] + cs)), 0.f);
        d2 = fmaf(e, e, d2);
      }
      if (d2 <= R * R) bits |= 1u << b;
    }
    out[w] = bits;
  }
}

// FP32 throughput probe: 8 independent FMA chains per thread, scalar (mode 0) or
// paired f32x2 (mode 1, 16 chains' worth of flops per loop), 2 flops per FMA.
__global__ void k_ffma(float *out, int iters, int mode) {
  float a0 = threadIdx.x * 1e-3f, a1 = a0 + 1.f, a2 = a0 + 2.f, a3 = a0 + 3.f;
  float a4 = a0 + 4.f, a5 = a0 + 5.f, a6 = a0 + 6.f, a7 = a0 + 7.f;
  const float b = 0.999999f, c = 1e-7f;
  if (mode == 0) {
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        a0 = fmaf(a0, b, c); a1 = fmaf(a1, b, c); a2 = fmaf(a2, b, c); a3 = fmaf(a3, b, c);
        a4 = fmaf(a4, b, c); a5 = fmaf(a5, b, c); a6 = fmaf(a6, b, c); a7 = fmaf(a7, b, c);
      }
    }
  } else {
    float2 p0 = make_float2(a0, a1), p1 = make_float2(a2, a3), p2 = make_float2(a4, a5),
           p3 = make_float2(a6, a7);
    const float2 B = make_float2(b, b), C = make_float2(c, c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        p0 = __ffma2_rn(p0, B, C); p1 = __ffma2_rn(p1, B, C);
        p2 = __ffma2_rn(p2, B, C); p3 = __ffma2_rn(p3, B, C);
      }
    }
    a0 = p0.x + p0.y; a1 = p1.x + p1.y; a2 = p2.x + p2.y; a3 = p3.x + p3.y;
    a4 = a5 = a6 = a7 = 0.f;
  }
  const float s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == 12345.f) out[threadIdx.x] = s;  // keeps the loop alive
}

#endif

#if RGEO_PART(1)
template <int MK, int INTEG>
cudaError_t launch_one(const TraceParams &p, cudaStream_t st) {
  const int cap = tuning().ctas_per_sm;
  const bool five = MK == MK_LOCAL || (is_iso(MK) && cap > 0 && cap <= 5);
  const bool bundle = INTEG == 0 && p.bundle;
  const size_t smem = (size_t)(table_float4s(p.kind, p.K, MK == MK_GRAPH_ANISO) + (p.nodes ? 0 : p.S) +
                               trace_lists_float4(MK, p) + (bundle ? (kBundle + 1) * 128 : 0)) *
                      sizeof(float4);
  if (smem > 227u * 1024u) return cudaErrorInvalidValue;  // bump table + spheres must fit on chip
  const bool x2 = is_iso(MK) && p.rays_per_thread == 2 && p.cull_masks == nullptr && !bundle;
  // CTAs per SM at least (the register budget): 7 (72 registers) for the isotropic graph metric,
  // measured 3 % faster at 1080p than 6 and 8; 5 (102) for the local-map jet and on request
  constexpr int kDefaultMinb = is_iso(MK) ? 7 : 6;
  // The step-list kernel without work counters when the launch asks for none (1 % faster at
  // 1080p).  The isotropic graph metric with an affine or quadratic part (the lattice
  // showcases) takes its rays' rare paths inline in RK4: 6 % faster there, where out of line
  // is 4 % faster at 1080p / 64 bumps.
  const bool count = p.bump_evals != nullptr || p.bump_slots != nullptr;
  const bool inl = INTEG == 0 && (p.has_affine || p.has_quad);
  void (*kern)(const TraceParams) = k_trace<MK, INTEG, kDefaultMinb, 1>;
  if (bundle) {
    kern = five ? k_trace<MK, 0, 5, kBundle> : k_trace<MK, 0, kDefaultMinb, kBundle>;
  } else if (five) {
    kern = k_trace<MK, INTEG, 5, 1>;
  } else if constexpr (MK == MK_GRAPH_SL) {
    if (inl) kern = count ? k_trace<MK, 0, kDefaultMinb, 1, true, false> : k_trace<MK, 0, kDefaultMinb, 1, false, false>;
    else if (!count) kern = k_trace<MK, INTEG, kDefaultMinb, 1, false>;
  } else if constexpr (MK == MK_GRAPH_ISO) {
    if (inl) kern = k_trace<MK, 0, kDefaultMinb, 1, true, false>;
  }
  if (x2) kern = k_trace_x2<INTEG>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (cap > 0 && cap < per_sm) per_sm = cap;
  long long blocks = (long long)sms * per_sm;
  const long long rays_per_block = x2 ? 256 : 128;
  const long long need = ((long long)p.n_items + rays_per_block - 1) / rays_per_block;
  if (blocks > need) blocks = need > 0 ? need : 1;
  kern<<<(unsigned)blocks, 128, smem, st>>>(p);
  return cudaGetLastError();
}

#endif

#if RGEO_PART(2)
template <int MK, int INTEG>
cudaError_t launch_batch_t(const TraceParams *dev_inst, const TraceParams *host_inst, int n, int table_f4,
                           long long total_items, cudaStream_t st) {
  const bool param = host_inst != nullptr && n <= kMaxParamInstances && tuning().batch_params == 0;
  const size_t lf4 = (size_t)lists_float4(MK == MK_GRAPH_SL);
  const size_t smem = param ? (size_t)kWarpsPerBlock * ((size_t)table_f4 + lf4) * 16
                            : (size_t)kWarpsPerBlock * (kParamWords * 4 + ((size_t)table_f4 + lf4) * 16);
  const bool in_smem = table_f4 > 0 || MK == MK_TWIST;
  void (*kern_s)(const TraceParams *, int, int) =
      in_smem ? k_trace_batch<MK, INTEG, true> : k_trace_batch<MK, INTEG, false>;
  void (*kern_p)(const BatchTable, int, int) =
      in_smem ? k_trace_batch_param<MK, INTEG, true> : k_trace_batch_param<MK, INTEG, false>;
  const void *kern = param ? (const void *)kern_p : (const void *)kern_s;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (tuning().ctas_per_sm > 0 && tuning().ctas_per_sm < per_sm) per_sm = tuning().ctas_per_sm;
  long long blocks = (long long)sms * per_sm;
  const long long need = (total_items + 127) / 128;
  if (blocks > need) blocks = need > 0 ? need : 1;
  if (param) {
    static thread_local BatchTable table;  // 23.5 KB: kept off the stack
    std::memset(&table, 0, sizeof(table));
    std::memcpy(table.inst, host_inst, sizeof(TraceParams) * (size_t)n);
    kern_p<<<(unsigned)blocks, 128, smem, st>>>(table, n, table_f4);
  } else {
    kern_s<<<(unsigned)blocks, 128, smem, st>>>(dev_inst, n, table_f4);
  }
  return cudaGetLastError();
}

#endif

}  // namespace

#if RGEO_PART(2)
cudaError_t launch_batch(const TraceParams *dev_inst, const TraceParams *host_inst, int n, int kind, int aniso,
                         int integrator, int max_table_f4, long long total_items, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  // per-warp bump tables of up to 512 isotropic bumps (1026 float4); larger tables are read
  // through L1
  const int table_f4 = max_table_f4 <= packed_float4s(512, 0) ? max_table_f4 : 0;
  const int mk = kind == 2 ? MK_LOCAL : (kind == 1 ? MK_TWIST : (aniso ? MK_GRAPH_ANISO : MK_GRAPH_ISO));
  if (mk == MK_LOCAL)
    return integrator == 0 ? launch_batch_t<MK_LOCAL, 0>(dev_inst, host_inst, n, table_f4, total_items, st)
                           : launch_batch_t<MK_LOCAL, 1>(dev_inst, host_inst, n, table_f4, total_items, st);
  if (mk == MK_GRAPH_ISO) {
    // step lists when every culled instance takes them (instances without a cull grid sum densely)
    bool sl = integrator == 0 && host_inst != nullptr;
    for (int i = 0; sl && i < n; ++i) sl = !host_inst[i].cull_masks || host_inst[i].step_lists;
    if (sl) return launch_batch_t<MK_GRAPH_SL, 0>(dev_inst, host_inst, n, table_f4, total_items, st);
    return integrator == 0 ? launch_batch_t<MK_GRAPH_ISO, 0>(dev_inst, host_inst, n, table_f4, total_items, st)
                           : launch_batch_t<MK_GRAPH_ISO, 1>(dev_inst, host_inst, n, table_f4, total_items, st);
  }
  if (mk == MK_GRAPH_ANISO)
    return integrator == 0 ? launch_batch_t<MK_GRAPH_ANISO, 0>(dev_inst, host_inst, n, table_f4, total_items, st)
                           : launch_batch_t<MK_GRAPH_ANISO, 1>(dev_inst, host_inst, n, table_f4, total_items, st);
  return integrator == 0 ? launch_batch_t<MK_TWIST, 0>(dev_inst, host_inst, n, table_f4, total_items, st)
                         : launch_batch_t<MK_TWIST, 1>(dev_inst, host_inst, n, table_f4, total_items, st);
}

#endif

#if RGEO_PART(1)
cudaError_t launch_advance_motion(const float *motion, int K, int aniso, const int32_t *perm, float *raw,
                                  float4 *bumps, float *t, float dt, cudaStream_t st) {
  if (K > 0) {
    k_advance_motion<<<(K + 127) / 128, 128, 0, st>>>(motion, K, aniso, perm, raw, bumps, t, dt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_tick<<<1, 1, 0, st>>>(t, dt);
  return cudaGetLastError();
}

#endif

#if RGEO_PART(3)
cudaError_t launch_segments(const TraceParams &p, long long n, unsigned long long seed, float box, float s_max,
                            float accel_bound, float *X, float *T, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const long long want = (n + 127) / 128;
  const unsigned blocks = (unsigned)(want < (long long)sms * 8 ? want : (long long)sms * 8);
  if (p.aniso) k_segments<MK_GRAPH_ANISO><<<blocks, 128, 0, st>>>(p, n, seed, box, s_max, accel_bound, X, T);
  else k_segments<MK_GRAPH_ISO><<<blocks, 128, 0, st>>>(p, n, seed, box, s_max, accel_bound, X, T);
  return cudaGetLastError();
}

cudaError_t launch_wave_trace(const TraceParams &p, const WaveArgs &w, cudaStream_t st) {
  if (p.kind != 0) return cudaErrorInvalidValue;
  const bool aniso = p.aniso != 0;
  const size_t smem = (size_t)(packed_float4s(p.K, aniso) + (p.nodes ? 0 : p.S) +
                               (p.cull_masks ? kWarpsPerBlock * lists_float4(p.step_lists != 0 && !aniso) : 0)) *
                      sizeof(float4);
  if (smem > 227u * 1024u) return cudaErrorInvalidValue;
  void (*kern)(const TraceParams, const WaveArgs) =
      aniso ? k_wave_trace<MK_GRAPH_ANISO> : (p.step_lists ? k_wave_trace<MK_GRAPH_SL> : k_wave_trace<MK_GRAPH_ISO>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long blocks = (long long)sms * per_sm;
  const long long need = ((long long)p.n_items + 127) / 128;
  if (blocks > need) blocks = need > 0 ? need : 1;
  kern<<<(unsigned)blocks, 128, smem, st>>>(p, w);
  return cudaGetLastError();
}

cudaError_t launch_wave_apply(const WaveArgs &w, unsigned n, float h, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_wave_apply<<<(n + 255) / 256, 256, 0, st>>>(w, n, h);
  return cudaGetLastError();
}

#endif

#if RGEO_PART(1)
cudaError_t launch_set_time(float *t, float value, cudaStream_t st) {
  k_set_time<<<1, 1, 0, st>>>(t, value);
  return cudaGetLastError();
}

cudaError_t launch_trace(const TraceParams &p, cudaStream_t st) {
  const int mk = p.kind == 2 ? MK_LOCAL : (p.kind == 1 ? MK_TWIST : (p.aniso ? MK_GRAPH_ANISO : MK_GRAPH_ISO));
  if (mk == MK_LOCAL) return p.integrator == 0 ? launch_one<MK_LOCAL, 0>(p, st) : launch_one<MK_LOCAL, 1>(p, st);
  if (mk == MK_GRAPH_ISO && p.step_lists) return launch_one<MK_GRAPH_SL, 0>(p, st);  // RK4 only
  if (mk == MK_GRAPH_ISO) return p.integrator == 0 ? launch_one<MK_GRAPH_ISO, 0>(p, st) : launch_one<MK_GRAPH_ISO, 1>(p, st);
  if (mk == MK_GRAPH_ANISO) return p.integrator == 0 ? launch_one<MK_GRAPH_ANISO, 0>(p, st) : launch_one<MK_GRAPH_ANISO, 1>(p, st);
  return p.integrator == 0 ? launch_one<MK_TWIST, 0>(p, st) : launch_one<MK_TWIST, 1>(p, st);
}

#endif

#if RGEO_PART(3)
template <int MK, int INTEG>
cudaError_t launch_illuminate_t(const TraceParams &p, const LightParams &l, cudaStream_t st) {
  const size_t smem =
      (size_t)(table_float4s(p.kind, p.K, MK == MK_GRAPH_ANISO) + (p.nodes ? 0 : p.S)) * sizeof(float4);
  if (smem > 227u * 1024u) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_illuminate<MK, INTEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned per_block = 4u * kIllumGroups;  // hits per 128-thread block
  const unsigned blocks = (p.n_items + per_block - 1u) / per_block;
  if (blocks == 0) return cudaSuccess;
  k_illuminate<MK, INTEG><<<blocks, 128, smem, st>>>(p, l);
  return cudaGetLastError();
}

// The lockstep form: the warps' lists after the bump table and the spheres.
template <int INTEG>
cudaError_t launch_illuminate_sl(const TraceParams &p, const LightParams &l, cudaStream_t st) {
  const size_t smem =
      (size_t)(table_float4s(p.kind, p.K, 0) + (p.nodes ? 0 : p.S) + kWarpsPerBlock * lists_float4(true)) *
      sizeof(float4);
  if (smem > 227u * 1024u) return cudaErrorInvalidValue;
  if (p.n_items == 0) return cudaSuccess;
  k_hit_list<<<(p.n_items + 127u) / 128u, 128, 0, st>>>(p, l);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // without work counters when the launch asks for none
  void (*kern)(const TraceParams, const LightParams) =
      p.bump_evals || p.bump_slots ? k_illuminate_sl<INTEG, true> : k_illuminate_sl<INTEG, false>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // persistent: as many blocks as fit, at most one per 40 queue items
  long long blocks = (long long)sms * per_sm;
  const long long need = ((long long)p.n_items + 4 * kIllumGroups - 1) / (4 * kIllumGroups);
  if (blocks > need) blocks = need;
  kern<<<(unsigned)blocks, 128, smem, st>>>(p, l);
  return cudaGetLastError();
}

cudaError_t launch_illuminate(const TraceParams &p0, const LightParams &l, cudaStream_t st) {
  if (!p0.hit_nrm) return cudaErrorInvalidValue;
  TraceParams p = p0;  // keeps the cull grid
  p.h = l.h;
  p.max_steps = l.max_steps;
  p.energy = 0;
  p.list_steps = l.list_steps;
  const int mk = p.kind == 2 ? MK_LOCAL : (p.kind == 1 ? MK_TWIST : (p.aniso ? MK_GRAPH_ANISO : MK_GRAPH_ISO));
  const bool rk4 = p.integrator == 0;
  // isotropic truncated bumps with lists that serve several steps: the warp's marches in lockstep
  // over shared lists (k_illuminate_sl), unless the light asks for one list walk per lane
  if (mk == MK_GRAPH_ISO && p.cull_masks && l.list_steps > 0 && p.K <= kStepListBumps && !l.per_lane) {
    p.step_lists = 1;
    return rk4 ? launch_illuminate_sl<0>(p, l, st) : launch_illuminate_sl<1>(p, l, st);
  }
  p.step_lists = 0;  // the light geodesics keep per-lane lists (shoot), for l.list_steps steps
  if (mk == MK_LOCAL) return rk4 ? launch_illuminate_t<MK_LOCAL, 0>(p, l, st) : launch_illuminate_t<MK_LOCAL, 1>(p, l, st);
  if (mk == MK_TWIST) return rk4 ? launch_illuminate_t<MK_TWIST, 0>(p, l, st) : launch_illuminate_t<MK_TWIST, 1>(p, l, st);
  if (mk == MK_GRAPH_ANISO)
    return rk4 ? launch_illuminate_t<MK_GRAPH_ANISO, 0>(p, l, st) : launch_illuminate_t<MK_GRAPH_ANISO, 1>(p, l, st);
  return rk4 ? launch_illuminate_t<MK_GRAPH_ISO, 0>(p, l, st) : launch_illuminate_t<MK_GRAPH_ISO, 1>(p, l, st);
}

#endif

#if RGEO_PART(1)
cudaError_t launch_pack_bumps(const float *raw, int K, float cutoff, int aniso, const int32_t *perm, float4 *out,
                              cudaStream_t st) {
  if (K <= 0) return cudaSuccess;
  k_pack_bumps<<<(iso_pad_index(K) + 1 + 127) / 128, 128, 0, st>>>(raw, K, cutoff, aniso, perm, out);
  return cudaGetLastError();
}

cudaError_t launch_build_cull(const float4 *bumps, int K, int G, int words, float reach, float4 *hdr,
                              uint32_t *masks, cudaStream_t st) {
  if (K <= 0 || G <= 0) return cudaSuccess;
  k_cull_bounds<<<1, 256, 0, st>>>(bumps, K, G, reach, hdr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long cells = (long long)G * G * G;
  k_cull_masks<<<(unsigned)((cells + 127) / 128), 128, 0, st>>>(bumps, K, G, words, reach, hdr, masks);
  return cudaGetLastError();
}

cudaError_t launch_set_centers(const float *c, int K, int aniso, const int32_t *perm, float4 *bumps, cudaStream_t st) {
  if (K <= 0) return cudaSuccess;
  k_set_centers<<<(K + 127) / 128, 128, 0, st>>>(c, K, aniso, perm, bumps);
  return cudaGetLastError();
}

#endif

// This part's error word, read and cleared.
cudaError_t RGEO_PART_NAME(read_and_clear_trace_error_, RGEO_TRACE_PART)(unsigned *word, cudaStream_t st) {
  cudaError_t e = cudaMemcpyFromSymbolAsync(word, g_rgeo_error, sizeof(unsigned), 0,
                                            cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  const unsigned zero = 0;
  e = cudaMemcpyToSymbolAsync(g_rgeo_error, &zero, sizeof(unsigned), 0, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

#if RGEO_PART(1)
cudaError_t read_and_clear_device_error(unsigned *word, cudaStream_t st) {
  unsigned w[3] = {0u, 0u, 0u};
  cudaError_t e = read_and_clear_trace_error_1(&w[0], st);
  if (e == cudaSuccess) e = read_and_clear_trace_error_2(&w[1], st);
  if (e == cudaSuccess) e = read_and_clear_trace_error_3(&w[2], st);
  *word = w[0] | w[1] | w[2];
  return e;
}

cudaError_t run_ffma_probe(int mode, float *tflops, float *ms) {
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  float *out = nullptr;
  if ((e = cudaMalloc(&out, 1024 * sizeof(float))) != cudaSuccess) return e;
  const int blocks = sms * 8, threads = 256, iters = 4096;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  k_ffma<<<blocks, threads>>>(out, 64, mode);  // warm-up
  cudaEventRecord(a);
  k_ffma<<<blocks, threads>>>(out, iters, mode);
  cudaEventRecord(b);
  e = cudaEventSynchronize(b);
  float t = 0.f;
  cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess) return e;
  const double flops = 2.0 * 8.0 * 16.0 * iters * (double)blocks * threads;
  *ms = t;
  *tflops = (float)(flops / (t * 1e-3) / 1e12);
  return cudaGetLastError();
}

#endif  // RGEO_PART(1)

}  // namespace rgeo
