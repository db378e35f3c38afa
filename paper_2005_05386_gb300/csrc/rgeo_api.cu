// rgeo_api.cu -- the C ABI of librgeo: argument validation, handle ownership,
// scene construction and kernel launches.  See include/rgeo.h for the contract.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "rgeo.h"
#include "rgeo_internal.h"

struct rgeo_metric {
  rgeo::MetricDev d;
  int device;
};

struct rgeo_scene {
  rgeo::SceneDev d;
  int device;
};

struct rgeo_batch {
  rgeo::TraceParams *table;  // device instance table
  std::vector<rgeo::TraceParams> host_table;  // the same, passed by value when it fits the parameter space
  uint32_t *counters;        // device, one work counter per instance
  int n, kind, aniso, integrator;
  int max_table_f4;  // largest packed bump table of the instances, in float4
  long long total_items;
};

namespace {

thread_local std::string g_last_error;

rgeo_status fail(rgeo_status s, const std::string &msg) {
  g_last_error = msg;
  return s;
}

rgeo_status cuda_fail(cudaError_t e, const char *what) {
  return fail(e == cudaErrorMemoryAllocation ? RGEO_ENOMEM : RGEO_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define RGEO_CUDA(call, what)                 \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

bool finite_all(const float *p, size_t n) {
  for (size_t i = 0; i < n; i++)
    if (!std::isfinite(p[i])) return false;
  return true;
}

template <typename T>
cudaError_t upload(T **dst, const T *src, size_t n) {
  *dst = nullptr;
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc((void **)dst, n * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
}

void free_metric(rgeo_metric *m) {
  if (!m) return;
  cudaFree(m->d.bumps);
  cudaFree(m->d.raw);
  cudaFree(m->d.cull_masks);
  cudaFree(m->d.perm);
  cudaFree(m->d.cull_hdr);
  cudaFree(m->d.motion);
  cudaFree(m->d.time);
  delete m;
}

void free_scene(rgeo_scene *s) {
  if (!s) return;
  cudaFree(s->d.spheres);
  cudaFree(s->d.albedo);
  cudaFree(s->d.nodes);
  cudaFree(s->d.prims);
  cudaFree(s->d.grid);
  delete s;
}

rgeo_status validate_trace(const rgeo_metric *metric, const rgeo_scene *scene, const rgeo_camera *cam,
                           int32_t W, int32_t H, float h, int32_t max_steps, int32_t integrator,
                           int32_t shading, uint32_t flags, const rgeo_outputs *out) {
  if (!metric || !scene || !cam || !out) return fail(RGEO_EINVAL, "rgeo_trace: NULL handle, camera or outputs");
  if (W < 1 || H < 1 || (int64_t)W * H >= (int64_t(1) << 31))
    return fail(RGEO_EINVAL, "rgeo_trace: width and height must be >= 1 with W*H < 2^31");
  if (!std::isfinite(h) || h <= 0.f) return fail(RGEO_EINVAL, "rgeo_trace: step h must be finite and > 0");
  if (max_steps < 1) return fail(RGEO_EINVAL, "rgeo_trace: max_steps must be >= 1");
  if (integrator != RGEO_RK4 && integrator != RGEO_EULER)
    return fail(RGEO_EINVAL, "rgeo_trace: unknown integrator");
  if (shading != RGEO_SHADE_LAMBERT && shading != RGEO_SHADE_PSEUDO)
    return fail(RGEO_EINVAL, "rgeo_trace: unknown shading mode");
  if (flags & ~(RGEO_FLAG_ENERGY_DIAG | RGEO_FLAG_NO_SAFE_SKIP | RGEO_FLAG_DENSE | RGEO_FLAG_BUNDLE))
    return fail(RGEO_EINVAL, "rgeo_trace: unknown flag bits");
  if (!out->id || !out->hit || !out->steps || !out->rgba)
    return fail(RGEO_EINVAL, "rgeo_trace: id, hit, steps and rgba outputs are required");
  if ((flags & RGEO_FLAG_ENERGY_DIAG) && !out->drift)
    return fail(RGEO_EINVAL, "rgeo_trace: RGEO_FLAG_ENERGY_DIAG needs a drift buffer");
  if (!finite_all(cam->pos, 3) || !finite_all(cam->forward, 3) || !finite_all(cam->up, 3) ||
      !std::isfinite(cam->vfov_deg) || cam->vfov_deg <= 0.f || cam->vfov_deg >= 180.f)
    return fail(RGEO_EINVAL, "rgeo_trace: camera values must be finite, 0 < vfov < 180");
  const float *f = cam->forward, *u = cam->up;
  const float cx = u[1] * f[2] - u[2] * f[1], cy = u[2] * f[0] - u[0] * f[2], cz = u[0] * f[1] - u[1] * f[0];
  if (f[0] * f[0] + f[1] * f[1] + f[2] * f[2] == 0.f || cx * cx + cy * cy + cz * cz == 0.f)
    return fail(RGEO_EINVAL, "rgeo_trace: forward must be nonzero and not parallel to up");
  return RGEO_OK;
}

// Steps one culled-sum list serves at step h, 0 when a single step can leave its reach (the
// sums then look up each right-hand side's own cell).  A list built at x holds every bump
// whose support, inflated by kCullInflate + the masks' reach margin m.cull_reach, meets x's
// cell, so it serves every point within m.cull_reach of x: a step's stage points stay within
// h (|v| + h |x''| / 2) of its start, with |v| <= 1 for a g-unit tangent (g >= I; 1 % for its
// float32 drift) and |x''| <= accel_max, and n steps within n times that.  Tuning: sum_lists
// 1 takes no lists, 2 one list per step.
int list_steps_for(const rgeo::MetricDev &m, float h) {
  const double reach = (double)h * (1.01 + 0.5 * (double)h * m.accel_max) * 1.001 + 1e-5;
  const int mode = rgeo::tuning().sum_lists;
  if (mode == 1 || !(m.cull_reach > 0.f) || reach > m.cull_reach) return 0;
  return mode == 2 ? 1 : std::max(1, std::min(8, (int)std::floor(m.cull_reach / reach)));
}

rgeo::TraceParams make_params(const rgeo_metric *metric, const rgeo_scene *scene, const rgeo_camera *cam,
                              int32_t W, int32_t H, float h, int32_t max_steps, int32_t integrator,
                              int32_t shading, uint32_t flags, const rgeo_outputs *out) {
  rgeo::TraceParams p;
  std::memset(&p, 0, sizeof(p));
  const rgeo::MetricDev &m = metric->d;
  p.bumps = m.bumps;
  if (m.cull_G > 0 && !(flags & RGEO_FLAG_DENSE)) {
    p.cull_masks = m.cull_masks;
    p.cull_hdr = m.cull_hdr;
    p.cull_G = m.cull_G;
    p.cull_words = m.cull_words;
    // warp step lists (RK4, up to kStepListBumps bumps: the warp's packed pairs in shared memory)
    const int n = list_steps_for(m, h);
    p.step_lists = integrator == RGEO_RK4 && n > 0 && m.K <= rgeo::kStepListBumps;
    p.list_steps = p.step_lists ? n : 0;
  }
  p.K = m.kind == RGEO_METRIC_DIFFEO_TWIST ? 0 : m.K;
  p.kind = m.kind;
  p.aniso = m.aniso;
  p.skippable = m.skippable;
  std::memcpy(p.b, m.b, sizeof(p.b));
  std::memcpy(p.A, m.A, sizeof(p.A));
  p.has_affine = m.has_affine;
  p.has_quad = m.has_quad;
  p.twist_k = m.twist_k;
  const rgeo::SceneDev &s = scene->d;
  p.spheres = s.spheres;
  p.S = s.S;
  p.albedo = s.albedo;
  p.nodes = s.nodes;
  p.prims = s.prims;
  p.T = s.T;
  p.grid = s.grid;
  std::memcpy(p.gdim, s.gdim, sizeof(p.gdim));
  std::memcpy(p.gmin, s.gmin, sizeof(p.gmin));
  p.ginv = s.ginv;
  std::memcpy(p.smin, s.smin, sizeof(p.smin));
  std::memcpy(p.smax, s.smax, sizeof(p.smax));
  p.has_grid = s.has_grid;
  p.safe_skip = s.has_grid && !(flags & RGEO_FLAG_NO_SAFE_SKIP);
  p.fog = s.fog;
  std::memcpy(p.fog_rgb, s.fog_rgb, sizeof(p.fog_rgb));
  std::memcpy(p.cam_pos, cam->pos, sizeof(p.cam_pos));
  std::memcpy(p.cam_fwd, cam->forward, sizeof(p.cam_fwd));
  std::memcpy(p.cam_up, cam->up, sizeof(p.cam_up));
  p.vfov_deg = cam->vfov_deg;
  p.W = W;
  p.H = H;
  p.tile_lw = rgeo::tuning().tile_lw;
  p.tiles_x = (W + (1 << p.tile_lw) - 1) >> p.tile_lw;
  const int th = 32 >> p.tile_lw;
  const int tiles_y = (H + th - 1) / th;
  p.tile0 = 0;
  p.tile_step = 1;
  p.n_items = (uint32_t)p.tiles_x * (uint32_t)tiles_y * 32u;
  p.h = h;
  p.max_steps = max_steps;
  p.integrator = integrator;
  p.shading = shading;
  p.energy = (flags & RGEO_FLAG_ENERGY_DIAG) ? 1 : 0;
  p.bundle = (flags & RGEO_FLAG_BUNDLE) && !p.energy && integrator == RGEO_RK4 ? 1 : 0;
  p.id = out->id;
  p.hit = out->hit;
  p.steps = out->steps;
  p.rgba = reinterpret_cast<uchar4 *>(out->rgba);
  p.drift = out->drift;
  p.bump_evals = out->bump_evals;
  p.bump_slots = out->bump_slots;
  p.rays_per_thread = rgeo::tuning().rays_per_thread;
  p.refill_lanes = rgeo::tuning().refill;
  return p;
}

}  // namespace

namespace rgeo {
Tuning &tuning() {
  static Tuning t;
  return t;
}

void set_last_error(const char *msg) { g_last_error = msg; }
}  // namespace rgeo

extern "C" {

int32_t rgeo_abi_version(void) { return RGEO_ABI_VERSION; }

const char *rgeo_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace {

// Table order of isotropic bumps for the culled sums.  A warp pairs the even-numbered bumps
// of its list with the odd-numbered ones, so a list with more of one parity than the other
// pays pad slots.  Bumps are numbered so that the lists are balanced: at up to 4096 seeded
// points in the union of the supports, the bumps whose inflated support meets the point's
// grid cell form a list; bumps are taken by decreasing support radius, and each joins the
// parity (even or odd table slots, ceil(K/2) and floor(K/2) of them) that lowers the summed
// imbalance of its lists (greedy discrepancy balancing).  Returns perm, the bump of each
// table slot; the numbering changes the summation order only.  The sample cells are those
// of a fixed 192^3 grid over the supports whatever grid the metric is culled on (or none),
// so the numbering, and with it every result bit, is a function of the bumps alone: dense
// sums and culled sums on any grid give the same frame.
constexpr int kParityCells = 192;

std::vector<int32_t> balanced_parity_order(const float *center, const float *sigma, int K, float cutoff) {
  std::vector<int32_t> perm(K);
  for (int k = 0; k < K; k++) perm[k] = k;
  if (K < 2 || !(cutoff > 0.f)) return perm;
  std::vector<double> R(K);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int k = 0; k < K; k++) {
    R[k] = (double)cutoff * sigma[3 * k] + rgeo::kCullInflate + rgeo::cull_reach_for(K);
    for (int c = 0; c < 3; c++) {
      lo[c] = std::min(lo[c], (double)center[3 * k + c] - R[k]);
      hi[c] = std::max(hi[c], (double)center[3 * k + c] + R[k]);
    }
  }
  const double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
  const double cell = ext / kParityCells;
  uint64_t state = 0x5EEDBA5Eull + (uint64_t)K;
  auto u01 = [&state]() {  // SplitMix64 (Steele, Lea and Flood 2014)
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return (double)((z ^ (z >> 31)) >> 11) * (1.0 / 9007199254740992.0);
  };
  std::vector<std::vector<int>> member(K);  // the sample lists each bump belongs to
  int n_lists = 0;
  for (int tries = 0; tries < 65536 && n_lists < 4096; tries++) {
    double p[3];
    for (int c = 0; c < 3; c++) p[c] = lo[c] + u01() * (hi[c] - lo[c]);
    bool in = false;
    for (int k = 0; k < K && !in; k++) {
      double d2 = 0.0;
      for (int c = 0; c < 3; c++) d2 += (p[c] - center[3 * k + c]) * (p[c] - center[3 * k + c]);
      in = d2 < (double)cutoff * sigma[3 * k] * cutoff * sigma[3 * k];
    }
    if (!in) continue;
    double clo[3];
    for (int c = 0; c < 3; c++) clo[c] = lo[c] + std::floor((p[c] - lo[c]) / cell) * cell;
    for (int k = 0; k < K; k++) {
      double d2 = 0.0;
      for (int c = 0; c < 3; c++) {
        const double e = std::max(std::max(clo[c] - center[3 * k + c], center[3 * k + c] - (clo[c] + cell)), 0.0);
        d2 += e * e;
      }
      if (d2 <= R[k] * R[k]) member[k].push_back(n_lists);
    }
    n_lists++;
  }
  std::vector<int> order(K);
  for (int k = 0; k < K; k++) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return R[a] > R[b]; });
  std::vector<int> balance(n_lists, 0);  // even minus odd bumps of each list so far
  std::vector<int32_t> even, odd;
  const int n_even = (K + 1) / 2, n_odd = K / 2;
  for (int k : order) {
    long ce = 0, co = 0;
    for (int l : member[k]) {
      ce += std::abs(balance[l] + 1);
      co += std::abs(balance[l] - 1);
    }
    const bool to_even = ((int)even.size() < n_even && (ce <= co || (int)odd.size() >= n_odd));
    for (int l : member[k]) balance[l] += to_even ? 1 : -1;
    (to_even ? even : odd).push_back(k);
  }
  std::sort(even.begin(), even.end());
  std::sort(odd.begin(), odd.end());
  for (int i = 0; i < (int)even.size(); i++) perm[2 * i] = even[i];
  for (int i = 0; i < (int)odd.size(); i++) perm[2 * i + 1] = odd[i];
  return perm;
}

// The composition of local maps (kind 2): validated, packed five float4 per map
// (the layout in rgeo_internal.h) and uploaded.
rgeo_status create_local_metric(const rgeo_metric_desc *desc, rgeo_metric **out) {
  const int K = desc->n_bumps;
  if (K < 1 || K > RGEO_MAX_LOCAL_MAPS)
    return fail(RGEO_EINVAL, "rgeo_metric_create: local maps need 1 <= n_bumps <= RGEO_MAX_LOCAL_MAPS");
  for (int i = 0; i < 3; i++)
    if (desc->reserved[i] != 0) return fail(RGEO_EINVAL, "rgeo_metric_create: reserved fields must be zero");
  if (!desc->center || !desc->amplitude || !desc->sigma || !desc->direction)
    return fail(RGEO_EINVAL, "rgeo_metric_create: local maps need center, amplitude, sigma and direction");
  for (int i = 0; i < 3; i++)
    if (desc->affine_b[i] != 0.f) return fail(RGEO_EINVAL, "rgeo_metric_create: local maps take no affine_b");
  for (int i = 0; i < 9; i++)
    if (desc->quad_A[i] != 0.f) return fail(RGEO_EINVAL, "rgeo_metric_create: local maps take no quad_A");
  if (!finite_all(desc->center, 3 * (size_t)K) || !finite_all(desc->amplitude, K) ||
      !finite_all(desc->sigma, 3 * (size_t)K) || !finite_all(desc->direction, 3 * (size_t)K) ||
      (desc->field && !finite_all(desc->field, 9 * (size_t)K)))
    return fail(RGEO_EINVAL, "rgeo_metric_create: non-finite local-map value");
  std::vector<float4> table((size_t)rgeo::kLocalStride * K);
  bool any_field = false;
  for (int k = 0; k < K; k++) {
    const float *sg = desc->sigma + 3 * k, *c = desc->center + 3 * k, *v = desc->direction + 3 * k;
    if (!(sg[0] > 0.f) || sg[1] != sg[0] || sg[2] != sg[0])
      return fail(RGEO_EINVAL, "rgeo_metric_create: local maps need isotropic sigma > 0");
    const float *B = desc->field ? desc->field + 9 * k : nullptr;
    bool field = false;
    if (B)
      for (int i = 0; i < 9; i++) field |= B[i] != 0.f;
    any_field |= field;
    const double vn = std::sqrt((double)v[0] * v[0] + (double)v[1] * v[1] + (double)v[2] * v[2]);
    if (!field && std::fabs((double)desc->amplitude[k]) * vn * std::exp(-0.5) / sg[0] >= 1.0)
      return fail(RGEO_EINVAL, "rgeo_metric_create: local map is not a diffeomorphism "
                               "(|a| |v| e^-1/2 / sigma must be < 1)");
    const float q = 1.f / (sg[0] * sg[0]);
    float4 *t = table.data() + (size_t)rgeo::kLocalStride * k;
    t[0] = make_float4(c[0], c[1], c[2], desc->amplitude[k]);
    t[1] = make_float4(v[0], v[1], v[2], (float)(-0.5 * q * 1.4426950408889634));
    t[2] = make_float4(B ? B[0] : 0.f, B ? B[1] : 0.f, B ? B[2] : 0.f, q);
    t[3] = make_float4(B ? B[3] : 0.f, B ? B[4] : 0.f, B ? B[5] : 0.f, field ? 1.f : 0.f);
    t[4] = make_float4(B ? B[6] : 0.f, B ? B[7] : 0.f, B ? B[8] : 0.f, 0.f);
  }
  (void)any_field;
  rgeo_metric *m = new rgeo_metric();
  std::memset(&m->d, 0, sizeof(m->d));
  cudaGetDevice(&m->device);
  m->d.kind = desc->kind;
  m->d.K = K;
  cudaError_t e = upload(&m->d.bumps, table.data(), table.size());
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) {
    free_metric(m);
    return cuda_fail(e, "rgeo_metric_create");
  }
  *out = m;
  return RGEO_OK;
}

}  // namespace

extern "C" {

rgeo_status rgeo_metric_create(const rgeo_metric_desc *desc, rgeo_metric **out) {
  g_last_error.clear();
  if (!out) return fail(RGEO_EINVAL, "rgeo_metric_create: out is NULL");
  *out = nullptr;
  if (!desc) return fail(RGEO_EINVAL, "rgeo_metric_create: desc is NULL");
  const int K = desc->n_bumps;
  if (desc->kind != RGEO_METRIC_GRAPH_BUMPS && desc->kind != RGEO_METRIC_DIFFEO_TWIST &&
      desc->kind != RGEO_METRIC_DIFFEO_LOCAL)
    return fail(RGEO_EINVAL, "rgeo_metric_create: unknown metric kind");
  if (desc->kind == RGEO_METRIC_DIFFEO_LOCAL) return create_local_metric(desc, out);
  if (K < 0 || K > RGEO_MAX_BUMPS) return fail(RGEO_EINVAL, "rgeo_metric_create: n_bumps out of range");
  for (int i = 0; i < 3; i++)
    if (desc->reserved[i] != 0) return fail(RGEO_EINVAL, "rgeo_metric_create: reserved fields must be zero");
  if (desc->cull_grid != 0 && desc->cull_grid != -1 && (desc->cull_grid < 4 || desc->cull_grid > 256))
    return fail(RGEO_EINVAL, "rgeo_metric_create: cull_grid must be 0, -1 or in [4, 256]");
  if (desc->kind == RGEO_METRIC_DIFFEO_TWIST && K != 0)
    return fail(RGEO_EINVAL, "rgeo_metric_create: the twist metric takes no bumps");
  if (!finite_all(desc->affine_b, 3) || !finite_all(desc->quad_A, 9) || !std::isfinite(desc->cutoff_sigmas) ||
      !std::isfinite(desc->twist_rate))
    return fail(RGEO_EINVAL, "rgeo_metric_create: non-finite parameter");
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < i; j++)
      if (desc->quad_A[3 * i + j] != desc->quad_A[3 * j + i])
        return fail(RGEO_EINVAL, "rgeo_metric_create: quad_A must be symmetric");
  if (K > 0) {
    if (!desc->center || !desc->amplitude || !desc->sigma)
      return fail(RGEO_EINVAL, "rgeo_metric_create: NULL bump arrays");
    if (!finite_all(desc->center, 3 * (size_t)K) || !finite_all(desc->amplitude, K) ||
        !finite_all(desc->sigma, 3 * (size_t)K))
      return fail(RGEO_EINVAL, "rgeo_metric_create: non-finite bump value");
    for (int i = 0; i < 3 * K; i++)
      if (!(desc->sigma[i] > 0.f)) return fail(RGEO_EINVAL, "rgeo_metric_create: sigma must be > 0");
  }
  rgeo_metric *m = new rgeo_metric();
  std::memset(&m->d, 0, sizeof(m->d));
  cudaGetDevice(&m->device);
  m->d.kind = desc->kind;
  m->d.K = K;
  int aniso = 0;
  for (int k = 0; k < K; k++)
    if (desc->sigma[3 * k] != desc->sigma[3 * k + 1] || desc->sigma[3 * k] != desc->sigma[3 * k + 2]) aniso = 1;
  m->d.aniso = aniso;
  bool quad = false, affine = false;
  for (int i = 0; i < 9; i++) {
    m->d.A[i] = desc->quad_A[i];
    quad |= desc->quad_A[i] != 0.f;
  }
  for (int i = 0; i < 3; i++) {
    m->d.b[i] = desc->affine_b[i];
    affine |= desc->affine_b[i] != 0.f;
  }
  m->d.has_quad = quad;
  m->d.has_affine = affine;
  m->d.cutoff = desc->cutoff_sigmas;
  m->d.twist_k = desc->twist_rate;
  m->d.skippable = desc->kind == RGEO_METRIC_GRAPH_BUMPS && desc->cutoff_sigmas > 0.f && !quad;
  {
    double hs = 0.0, a2 = 0.0;  // sum |a_k| / sigma_k^2 (largest sigma per bump), ||A||_F
    for (int k = 0; k < K; k++) {
      const double sg = std::min(desc->sigma[3 * k], std::min(desc->sigma[3 * k + 1], desc->sigma[3 * k + 2]));
      hs += std::fabs((double)desc->amplitude[k]) / (sg * sg);
    }
    for (int i = 0; i < 9; i++) a2 += (double)desc->quad_A[i] * desc->quad_A[i];
    m->d.accel_max = (float)(0.5 * (hs + std::sqrt(a2)) * 1.0001);
  }
  if (K > 0) {
    std::vector<float> raw(7 * (size_t)K);
    std::memcpy(raw.data(), desc->center, sizeof(float) * 3 * K);
    std::memcpy(raw.data() + 3 * K, desc->amplitude, sizeof(float) * K);
    std::memcpy(raw.data() + 4 * K, desc->sigma, sizeof(float) * 3 * K);
    // bump-support cull grid: isotropic truncated bumps only
    int G = 0;
    if (desc->kind == RGEO_METRIC_GRAPH_BUMPS && !aniso && desc->cutoff_sigmas > 0.f)
      // automatic: 192^3 cells up to 64 bumps (57 MB of masks; 1 % faster at 1080p than 128^3),
      // 128^3 up to 1024 bumps (masks of 128^3 x ceil(K / 32) words), 64^3 above
      G = desc->cull_grid == 0 ? (K >= 16 ? (K <= 64 ? 192 : (K <= 1024 ? 128 : 64)) : 0)
                               : (desc->cull_grid < 0 ? 0 : desc->cull_grid);
    cudaError_t e = upload(&m->d.raw, raw.data(), raw.size());
    if (e == cudaSuccess && desc->kind == RGEO_METRIC_GRAPH_BUMPS && !aniso && desc->cutoff_sigmas > 0.f) {
      const std::vector<int32_t> perm = balanced_parity_order(desc->center, desc->sigma, K, desc->cutoff_sigmas);
      e = upload(&m->d.perm, perm.data(), perm.size());
    }
    if (e == cudaSuccess) e = cudaMalloc(&m->d.bumps, sizeof(float4) * (size_t)rgeo::packed_float4s(K, aniso));
    if (e == cudaSuccess)
      e = rgeo::launch_pack_bumps(m->d.raw, K, desc->cutoff_sigmas, aniso, m->d.perm, m->d.bumps, 0);
    if (e == cudaSuccess && G > 0) {
      const int words = rgeo::cull_words_for(K);
      m->d.cull_G = G;
      m->d.cull_words = words;
      m->d.cull_reach = rgeo::cull_reach_for(K);
      e = cudaMalloc(&m->d.cull_masks, sizeof(uint32_t) * (size_t)G * G * G * words);
      if (e == cudaSuccess) e = cudaMalloc(&m->d.cull_hdr, sizeof(float4) * 2);
      if (e == cudaSuccess)
        e = rgeo::launch_build_cull(m->d.bumps, K, G, words, m->d.cull_reach, m->d.cull_hdr, m->d.cull_masks, 0);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
      free_metric(m);
      return cuda_fail(e, "rgeo_metric_create");
    }
  }
  *out = m;
  return RGEO_OK;
}

rgeo_status rgeo_metric_set_centers(rgeo_metric *metric, const float *center, void *cuda_stream) {
  g_last_error.clear();
  if (!metric || !center) return fail(RGEO_EINVAL, "rgeo_metric_set_centers: NULL argument");
  if (metric->d.kind != RGEO_METRIC_GRAPH_BUMPS)
    return fail(RGEO_EINVAL, "rgeo_metric_set_centers: not a graph metric");
  const int K = metric->d.K;
  if (K == 0) return RGEO_OK;
  if (!finite_all(center, 3 * (size_t)K)) return fail(RGEO_EINVAL, "rgeo_metric_set_centers: non-finite centre");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  RGEO_CUDA(cudaMemcpyAsync(metric->d.raw, center, sizeof(float) * 3 * K, cudaMemcpyHostToDevice, st),
            "rgeo_metric_set_centers: copy");
  RGEO_CUDA(rgeo::launch_set_centers(metric->d.raw, K, metric->d.aniso, metric->d.perm, metric->d.bumps, st),
            "rgeo_metric_set_centers: launch");
  if (metric->d.cull_G > 0)
    RGEO_CUDA(rgeo::launch_build_cull(metric->d.bumps, K, metric->d.cull_G, metric->d.cull_words, metric->d.cull_reach,
                                      metric->d.cull_hdr, metric->d.cull_masks, st),
              "rgeo_metric_set_centers: cull grid");
  return RGEO_OK;
}

void rgeo_metric_destroy(rgeo_metric *metric) { free_metric(metric); }

rgeo_status rgeo_scene_create(const float *spheres, int32_t S, const float *verts, int32_t V,
                              const int32_t *tris, int32_t T, const float *albedo, rgeo_scene **out) {
  g_last_error.clear();
  if (!out) return fail(RGEO_EINVAL, "rgeo_scene_create: out is NULL");
  *out = nullptr;
  if (S < 0 || V < 0 || T < 0) return fail(RGEO_EINVAL, "rgeo_scene_create: negative count");
  if ((S > 0 && !spheres) || (T > 0 && (!verts || !tris)) || !albedo)
    return fail(RGEO_EINVAL, "rgeo_scene_create: NULL array");
  if (T > (1 << 26) || S > (1 << 20)) return fail(RGEO_EINVAL, "rgeo_scene_create: scene too large");
  if (S > 0 && !finite_all(spheres, 4 * (size_t)S)) return fail(RGEO_EINVAL, "rgeo_scene_create: non-finite sphere");
  for (int s = 0; s < S; s++)
    if (!(spheres[4 * s + 3] > 0.f)) return fail(RGEO_EINVAL, "rgeo_scene_create: sphere radius must be > 0");
  if (V > 0 && !finite_all(verts, 3 * (size_t)V)) return fail(RGEO_EINVAL, "rgeo_scene_create: non-finite vertex");
  for (int t = 0; t < 3 * T; t++)
    if (tris[t] < 0 || tris[t] >= V) return fail(RGEO_EINVAL, "rgeo_scene_create: vertex index out of range");
  for (int i = 0; i < 3 * (S + 1); i++)
    if (!(albedo[i] >= 0.f && albedo[i] <= 1.f)) return fail(RGEO_EINVAL, "rgeo_scene_create: albedo outside [0, 1]");

  rgeo::HostBVH bvh;
  if (!rgeo::build_bvh(spheres, S, verts, V, tris, T, bvh, rgeo::kMaxBvhDepth))
    return fail(RGEO_EINVAL, "rgeo_scene_create: BVH build failed");
  rgeo::HostGrid grid;
  // 192 cells along the scene's longest axis (about 30 MB for the 1080p scene): a finer grid
  // gives tighter lower bounds and fewer BVH queries (lattice scenes: 1.9x faster than 64)
  rgeo::build_safe_grid(spheres, S, verts, tris, T, 192, grid);

  rgeo_scene *sc = new rgeo_scene();
  std::memset(&sc->d, 0, sizeof(sc->d));
  cudaGetDevice(&sc->device);
  sc->d.S = S;
  sc->d.T = T;
  sc->d.n_nodes = (int)bvh.nodes.size() / 2;
  std::vector<float4> sph(S);
  for (int s = 0; s < S; s++)
    sph[s] = make_float4(spheres[4 * s], spheres[4 * s + 1], spheres[4 * s + 2], spheres[4 * s + 3]);
  cudaError_t e = upload(&sc->d.spheres, sph.data(), sph.size());
  if (e == cudaSuccess) e = upload(&sc->d.albedo, albedo, 3 * (size_t)(S + 1));
  if (e == cudaSuccess) e = upload(&sc->d.nodes, bvh.nodes.data(), bvh.nodes.size());
  if (e == cudaSuccess) e = upload(&sc->d.prims, bvh.prims.data(), bvh.prims.size());
  if (e == cudaSuccess && !grid.dist.empty()) {
    e = upload(&sc->d.grid, grid.dist.data(), grid.dist.size());
    sc->d.has_grid = 1;
    for (int i = 0; i < 3; i++) {
      sc->d.gdim[i] = grid.dim[i];
      sc->d.gmin[i] = grid.gmin[i];
      sc->d.smin[i] = grid.smin[i];
      sc->d.smax[i] = grid.smax[i];
    }
    sc->d.ginv = 1.0f / grid.cell;
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_scene(sc);
    return cuda_fail(e, "rgeo_scene_create");
  }
  *out = sc;
  return RGEO_OK;
}

rgeo_status rgeo_scene_set_fog(rgeo_scene *scene, float density, const float *rgb) {
  g_last_error.clear();
  if (!scene) return fail(RGEO_EINVAL, "rgeo_scene_set_fog: NULL scene");
  if (!std::isfinite(density) || density < 0.f || (rgb && !finite_all(rgb, 3)))
    return fail(RGEO_EINVAL, "rgeo_scene_set_fog: density must be finite and >= 0, rgb finite");
  scene->d.fog = density;
  for (int c = 0; c < 3; c++) scene->d.fog_rgb[c] = rgb ? rgb[c] : 0.f;
  return RGEO_OK;
}

void rgeo_scene_destroy(rgeo_scene *scene) { free_scene(scene); }

rgeo_status rgeo_trace(const rgeo_metric *metric, const rgeo_scene *scene, const rgeo_camera *camera,
                       int32_t width, int32_t height, float h, int32_t max_steps, int32_t integrator,
                       int32_t shading, uint32_t flags, const rgeo_outputs *out, void *cuda_stream) {
  return rgeo_trace_tiles(metric, scene, camera, width, height, h, max_steps, integrator, shading, flags, 0, -1, 1,
                          out, cuda_stream);
}

int32_t rgeo_frame_tiles(int32_t width, int32_t height) {
  if (width < 1 || height < 1) return 0;
  const int lw = rgeo::tuning().tile_lw;
  return (int32_t)(((width + (1 << lw) - 1) >> lw) * ((height + (32 >> lw) - 1) / (32 >> lw)));
}

int32_t rgeo_frame_tile_pixels(int32_t width, int32_t height, int32_t tile, int32_t *pixels) {
  if (width < 1 || height < 1 || tile < 0 || tile >= rgeo_frame_tiles(width, height) || !pixels) return -1;
  const int lw = rgeo::tuning().tile_lw;
  const int tiles_x = (width + (1 << lw) - 1) >> lw;
  int n = 0;
  for (unsigned sub = 0; sub < 32u; ++sub) {
    int pix;
    if (rgeo::tile_pixel(width, height, tiles_x, lw, (unsigned)tile, sub, pix)) pixels[n++] = pix;
  }
  return n;
}

rgeo_status rgeo_trace_tiles(const rgeo_metric *metric, const rgeo_scene *scene, const rgeo_camera *camera,
                             int32_t width, int32_t height, float h, int32_t max_steps, int32_t integrator,
                             int32_t shading, uint32_t flags, int32_t tile_begin, int32_t tile_end,
                             int32_t tile_step, const rgeo_outputs *out, void *cuda_stream) {
  g_last_error.clear();
  rgeo_status s = validate_trace(metric, scene, camera, width, height, h, max_steps, integrator, shading,
                                 flags, out);
  if (s != RGEO_OK) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  rgeo::TraceParams p = make_params(metric, scene, camera, width, height, h, max_steps, integrator, shading,
                                    flags, out);
  const int64_t tiles = (int64_t)p.n_items / 32;
  if (tile_end < 0) tile_end = (int32_t)tiles;
  if (tile_begin < 0 || tile_begin > tile_end || tile_end > tiles || tile_step < 1)
    return fail(RGEO_EINVAL, "rgeo_trace_tiles: need 0 <= tile_begin <= tile_end <= rgeo_frame_tiles(width, height) "
                             "and tile_step >= 1");
  if (tile_begin == tile_end) return RGEO_OK;
  p.tile0 = (uint32_t)tile_begin;
  p.tile_step = (uint32_t)tile_step;
  p.n_items = (uint32_t)((tile_end - tile_begin + tile_step - 1) / tile_step) * 32u;
  uint32_t *counter = nullptr;
  RGEO_CUDA(cudaMallocAsync((void **)&counter, sizeof(uint32_t), st), "rgeo_trace: work counter");
  p.counter = counter;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = rgeo::launch_trace(p, st);
  cudaError_t e2 = cudaFreeAsync(counter, st);
  if (e != cudaSuccess) return cuda_fail(e, "rgeo_trace: launch");
  if (e2 != cudaSuccess) return cuda_fail(e2, "rgeo_trace: free");
  return RGEO_OK;
}

rgeo_status rgeo_trace_lit(const rgeo_metric *metric, const rgeo_scene *scene, const rgeo_camera *camera,
                           int32_t width, int32_t height, float h, int32_t max_steps, int32_t integrator,
                           const rgeo_light *light, const rgeo_outputs *out, int32_t *lit, void *cuda_stream) {
  g_last_error.clear();
  rgeo_status s = validate_trace(metric, scene, camera, width, height, h, max_steps, integrator, RGEO_SHADE_LAMBERT,
                                 0u, out);
  if (s != RGEO_OK) return s;
  if (!light) return fail(RGEO_EINVAL, "rgeo_trace_lit: light is NULL");
  if (!finite_all(light->pos, 3) || !std::isfinite(light->h) || !(light->h > 0.f) || light->max_steps < 1 ||
      light->iters < 0 || !std::isfinite(light->tol) || !(light->tol > 0.f) || !std::isfinite(light->delta) ||
      !(light->delta > 0.f))
    return fail(RGEO_EINVAL, "rgeo_trace_lit: light position, h, tol and delta must be finite, h, tol, delta > 0, "
                             "max_steps >= 1, iters >= 0");
  if (light->schedule != 0 && light->schedule != 1) return fail(RGEO_EINVAL, "rgeo_trace_lit: schedule must be 0 or 1");
  for (int i = 0; i < 3; i++)
    if (light->reserved[i] != 0) return fail(RGEO_EINVAL, "rgeo_trace_lit: reserved fields must be zero");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  rgeo::TraceParams p = make_params(metric, scene, camera, width, height, h, max_steps, integrator,
                                    RGEO_SHADE_LAMBERT, 0u, out);
  p.fog = 0.f;
  const size_t N = (size_t)width * height;
  char *buf = nullptr;
  RGEO_CUDA(cudaMallocAsync((void **)&buf, 16 + 16 * N, st), "rgeo_trace_lit: work counters, normals, hit list");
  p.counter = (uint32_t *)buf;
  p.hit_nrm = (float *)(buf + 16);
  rgeo::LightParams l;
  for (int c = 0; c < 3; c++) l.L[c] = light->pos[c];
  l.h = light->h;
  l.max_steps = light->max_steps;
  l.iters = light->iters;
  l.tol = light->tol;
  l.delta = light->delta;
  l.lit = lit;
  l.list_steps = p.cull_masks ? list_steps_for(metric->d, light->h) : 0;
  l.per_lane = light->schedule;
  l.n_hits = (uint32_t *)buf + 1;
  l.hit_next = (uint32_t *)buf + 2;
  l.hits = (int32_t *)(buf + 16 + 12 * N);
  cudaError_t e = cudaMemsetAsync(buf, 0, 16, st);
  if (e == cudaSuccess) e = rgeo::launch_trace(p, st);
  if (e == cudaSuccess) e = rgeo::launch_illuminate(p, l, st);
  cudaError_t e2 = cudaFreeAsync(buf, st);
  if (e != cudaSuccess) return cuda_fail(e, "rgeo_trace_lit: launch");
  if (e2 != cudaSuccess) return cuda_fail(e2, "rgeo_trace_lit: free");
  return RGEO_OK;
}

rgeo_status rgeo_trace_host(const rgeo_metric *metric, const rgeo_scene *scene, const rgeo_camera *camera,
                            int32_t width, int32_t height, float h, int32_t max_steps, int32_t integrator,
                            int32_t shading, uint32_t flags, const rgeo_outputs *host_out,
                            void *cuda_stream) {
  g_last_error.clear();
  rgeo_status s = validate_trace(metric, scene, camera, width, height, h, max_steps, integrator, shading,
                                 flags, host_out);
  if (s != RGEO_OK) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t N = (size_t)width * height;
  const bool drift = host_out->drift != nullptr;
  const size_t bytes = N * (4 + 12 + 4 + 4) + (drift ? N * 8 : 0);
  char *buf = nullptr;
  RGEO_CUDA(cudaMallocAsync((void **)&buf, bytes, st), "rgeo_trace_host: staging");
  rgeo_outputs d;
  d.bump_evals = nullptr;
  d.bump_slots = nullptr;
  d.drift = drift ? (double *)buf : nullptr;
  char *q = buf + (drift ? N * 8 : 0);
  d.hit = (float *)q;
  q += N * 12;
  d.id = (int32_t *)q;
  q += N * 4;
  d.steps = (int32_t *)q;
  q += N * 4;
  d.rgba = (uint8_t *)q;
  s = rgeo_trace(metric, scene, camera, width, height, h, max_steps, integrator, shading, flags, &d, st);
  cudaError_t e = cudaSuccess;
  if (s == RGEO_OK) {
    e = cudaMemcpyAsync(host_out->id, d.id, N * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out->hit, d.hit, N * 12, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out->steps, d.steps, N * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out->rgba, d.rgba, N * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && drift) e = cudaMemcpyAsync(host_out->drift, d.drift, N * 8, cudaMemcpyDeviceToHost, st);
  }
  cudaFreeAsync(buf, st);
  if (s != RGEO_OK) return s;
  if (e != cudaSuccess) return cuda_fail(e, "rgeo_trace_host: copy back");
  RGEO_CUDA(cudaStreamSynchronize(st), "rgeo_trace_host: synchronise");
  return RGEO_OK;
}

rgeo_status rgeo_sync(void *cuda_stream) {
  g_last_error.clear();
  cudaStream_t st = (cudaStream_t)cuda_stream;
  RGEO_CUDA(cudaStreamSynchronize(st), "rgeo_sync: stream");
  unsigned word = 0, mlp_word = 0;
  RGEO_CUDA(rgeo::read_and_clear_device_error(&word, st), "rgeo_sync: error word");
  RGEO_CUDA(rgeo::read_and_clear_mlp_error(&mlp_word), "rgeo_sync: error word");
  word |= mlp_word;
  if (word & rgeo::kErrTimeout) return fail(RGEO_ETIMEOUT, "a bounded device-side wait timed out");
  if (word & rgeo::kErrStackOverflow)
    return fail(RGEO_EDEVICE, "BVH traversal stack exhausted (the affected segment tests were cut short)");
  return RGEO_OK;
}

rgeo_status rgeo_set_tuning(const rgeo_tuning *t) {
  g_last_error.clear();
  if (!t) return fail(RGEO_EINVAL, "rgeo_set_tuning: NULL");
  if (t->reserved[0] != 0) return fail(RGEO_EINVAL, "rgeo_set_tuning: reserved fields must be zero");
  if (t->rays_per_thread != 0 && t->rays_per_thread != 1 && t->rays_per_thread != 2)
    return fail(RGEO_EINVAL, "rgeo_set_tuning: rays_per_thread must be 0, 1 or 2");
  if (t->batch_params != 0 && t->batch_params != 1)
    return fail(RGEO_EINVAL, "rgeo_set_tuning: batch_params must be 0 or 1");
  if (t->wait_limit < -1) return fail(RGEO_EINVAL, "rgeo_set_tuning: wait_limit must be >= -1");
  if (t->ctas_per_sm < 0 || t->ctas_per_sm > 32) return fail(RGEO_EINVAL, "rgeo_set_tuning: ctas_per_sm must be in [0, 32]");
  if (t->tile_shape < 0 || t->tile_shape > 3)
    return fail(RGEO_EINVAL, "rgeo_set_tuning: tile_shape must be 0 (default), 1 (8x4), 2 (4x8) or 3 (16x2)");
  if (t->batch_order != 0 && t->batch_order != 1)
    return fail(RGEO_EINVAL, "rgeo_set_tuning: batch_order must be 0 or 1");
  if (t->sum_lists < 0 || t->sum_lists > 2) return fail(RGEO_EINVAL, "rgeo_set_tuning: sum_lists must be 0, 1 or 2");
  if (t->refill != 0 && t->refill != 1) return fail(RGEO_EINVAL, "rgeo_set_tuning: refill must be 0 or 1");
  rgeo::Tuning &g = rgeo::tuning();
  const rgeo::Tuning d;
  g.rays_per_thread = t->rays_per_thread == 0 ? d.rays_per_thread : t->rays_per_thread;
  g.batch_params = t->batch_params;
  g.wait_limit = t->wait_limit;
  g.ctas_per_sm = t->ctas_per_sm;
  g.tile_lw = t->tile_shape == 0 ? d.tile_lw : (t->tile_shape == 1 ? 3 : (t->tile_shape == 2 ? 2 : 4));
  g.batch_order = t->batch_order;
  g.sum_lists = t->sum_lists;
  g.refill = t->refill;
  return RGEO_OK;
}

rgeo_status rgeo_get_tuning(rgeo_tuning *t) {
  g_last_error.clear();
  if (!t) return fail(RGEO_EINVAL, "rgeo_get_tuning: NULL");
  std::memset(t, 0, sizeof(*t));
  const rgeo::Tuning &g = rgeo::tuning();
  t->rays_per_thread = g.rays_per_thread;
  t->batch_params = g.batch_params;
  t->wait_limit = g.wait_limit;
  t->ctas_per_sm = g.ctas_per_sm;
  t->tile_shape = g.tile_lw == 3 ? 1 : (g.tile_lw == 2 ? 2 : 3);
  t->batch_order = g.batch_order;
  t->sum_lists = g.sum_lists;
  t->refill = g.refill;
  return RGEO_OK;
}

rgeo_status rgeo_ffma_probe(int32_t mode, float *tflops, float *ms) {
  g_last_error.clear();
  if (!tflops || !ms) return fail(RGEO_EINVAL, "rgeo_ffma_probe: NULL output");
  if (mode != 0 && mode != 1) return fail(RGEO_EINVAL, "rgeo_ffma_probe: mode must be 0 or 1");
  RGEO_CUDA(rgeo::run_ffma_probe(mode, tflops, ms), "rgeo_ffma_probe");
  return RGEO_OK;
}

rgeo_status rgeo_batch_create(int32_t n, const rgeo_instance *inst, rgeo_batch **out) {
  g_last_error.clear();
  if (!out) return fail(RGEO_EINVAL, "rgeo_batch_create: out is NULL");
  *out = nullptr;
  if (n < 1 || !inst) return fail(RGEO_EINVAL, "rgeo_batch_create: need n >= 1 instances");
  std::vector<rgeo::TraceParams> table(n);
  long long total = 0;
  int max_f4 = 0;
  for (int i = 0; i < n; i++) {
    const rgeo_instance &q = inst[i];
    rgeo_status s = validate_trace(q.metric, q.scene, &q.camera, q.width, q.height, q.h, q.max_steps, q.integrator,
                                   q.shading, q.flags, &q.out);
    if (s != RGEO_OK) return fail(s, "rgeo_batch_create: instance " + std::to_string(i) + ": " + g_last_error);
    if (q.metric->d.kind != inst[0].metric->d.kind || q.metric->d.aniso != inst[0].metric->d.aniso ||
        q.integrator != inst[0].integrator)
      return fail(RGEO_EINVAL, "rgeo_batch_create: instances must share metric kind, bump layout and integrator");
    table[i] = make_params(q.metric, q.scene, &q.camera, q.width, q.height, q.h, q.max_steps, q.integrator,
                           q.shading, q.flags, &q.out);
    table[i].rays_per_thread = 1;
    table[i].bundle = 0;  // the batch kernel tests every chord alone
    total += table[i].n_items;
    max_f4 = std::max(max_f4, rgeo::table_float4s(q.metric->d.kind, q.metric->d.K, q.metric->d.aniso));
  }
  // instances in order of decreasing cost (pixels x bump terms per point, roughly), so that
  // the last instance the warps drain is a short one; each keeps its own outputs
  if (rgeo::tuning().batch_order == 0) {
    std::vector<std::pair<double, int>> cost(n);
    for (int i = 0; i < n; i++)
      cost[i] = {-(double)inst[i].width * inst[i].height * (1.0 + inst[i].metric->d.K), i};
    std::stable_sort(cost.begin(), cost.end());
    std::vector<rgeo::TraceParams> sorted(n);
    for (int i = 0; i < n; i++) sorted[i] = table[cost[i].second];
    table.swap(sorted);
  }
  rgeo_batch *b = new rgeo_batch();
  b->n = n;
  b->kind = inst[0].metric->d.kind;
  b->aniso = inst[0].metric->d.aniso;
  b->integrator = inst[0].integrator;
  b->total_items = total;
  b->max_table_f4 = max_f4;
  cudaError_t e = cudaMalloc(&b->counters, sizeof(uint32_t) * n);
  if (e == cudaSuccess) {
    for (int i = 0; i < n; i++) table[i].counter = b->counters + i;
    e = upload(&b->table, table.data(), table.size());
    b->host_table = table;
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(b->counters);
    cudaFree(b->table);
    delete b;
    return cuda_fail(e, "rgeo_batch_create");
  }
  *out = b;
  return RGEO_OK;
}

rgeo_status rgeo_batch_launch(rgeo_batch *b, void *cuda_stream) {
  g_last_error.clear();
  if (!b) return fail(RGEO_EINVAL, "rgeo_batch_launch: NULL batch");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  RGEO_CUDA(cudaMemsetAsync(b->counters, 0, sizeof(uint32_t) * b->n, st), "rgeo_batch_launch: counters");
  RGEO_CUDA(rgeo::launch_batch(b->table, b->host_table.data(), b->n, b->kind, b->aniso, b->integrator,
                               b->max_table_f4, b->total_items, st),
            "rgeo_batch_launch: launch");
  return RGEO_OK;
}

void rgeo_batch_destroy(rgeo_batch *b) {
  if (!b) return;
  cudaFree(b->counters);
  cudaFree(b->table);
  delete b;
}

rgeo_status rgeo_metric_set_motion(rgeo_metric *m, const float *amplitude, const float *frequency,
                                   const float *phase) {
  g_last_error.clear();
  if (!m || !amplitude || !frequency || !phase) return fail(RGEO_EINVAL, "rgeo_metric_set_motion: NULL argument");
  if (m->d.kind != RGEO_METRIC_GRAPH_BUMPS) return fail(RGEO_EINVAL, "rgeo_metric_set_motion: not a graph metric");
  const int K = m->d.K;
  if (!finite_all(amplitude, 3 * (size_t)K) || !finite_all(frequency, K) || !finite_all(phase, K))
    return fail(RGEO_EINVAL, "rgeo_metric_set_motion: non-finite value");
  if (!m->d.motion && K > 0) RGEO_CUDA(cudaMalloc(&m->d.motion, sizeof(float) * 8 * (size_t)K), "rgeo_metric_set_motion");
  if (!m->d.time) RGEO_CUDA(cudaMalloc(&m->d.time, sizeof(float)), "rgeo_metric_set_motion");
  if (K > 0) {
    RGEO_CUDA(cudaMemcpy(m->d.motion, m->d.raw, sizeof(float) * 3 * K, cudaMemcpyDeviceToDevice), "set_motion: c0");
    RGEO_CUDA(cudaMemcpy(m->d.motion + 3 * K, amplitude, sizeof(float) * 3 * K, cudaMemcpyHostToDevice), "set_motion: A");
    RGEO_CUDA(cudaMemcpy(m->d.motion + 6 * K, frequency, sizeof(float) * K, cudaMemcpyHostToDevice), "set_motion: f");
    RGEO_CUDA(cudaMemcpy(m->d.motion + 7 * K, phase, sizeof(float) * K, cudaMemcpyHostToDevice), "set_motion: phi");
  }
  RGEO_CUDA(cudaMemset(m->d.time, 0, sizeof(float)), "rgeo_metric_set_motion: t");
  RGEO_CUDA(cudaDeviceSynchronize(), "rgeo_metric_set_motion");
  return RGEO_OK;
}

rgeo_status rgeo_metric_set_time(rgeo_metric *m, float t, void *cuda_stream) {
  g_last_error.clear();
  if (!m || !m->d.time) return fail(RGEO_EINVAL, "rgeo_metric_set_time: no motion set");
  if (!std::isfinite(t)) return fail(RGEO_EINVAL, "rgeo_metric_set_time: non-finite t");
  RGEO_CUDA(rgeo::launch_set_time(m->d.time, t, (cudaStream_t)cuda_stream), "rgeo_metric_set_time");
  return RGEO_OK;
}

rgeo_status rgeo_metric_advance(rgeo_metric *m, float dt, void *cuda_stream) {
  g_last_error.clear();
  if (!m || !m->d.time) return fail(RGEO_EINVAL, "rgeo_metric_advance: no motion set");
  if (!std::isfinite(dt)) return fail(RGEO_EINVAL, "rgeo_metric_advance: non-finite dt");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  RGEO_CUDA(rgeo::launch_advance_motion(m->d.motion, m->d.K, m->d.aniso, m->d.perm, m->d.raw, m->d.bumps, m->d.time,
                                        dt, st),
            "rgeo_metric_advance: motion");
  if (m->d.cull_G > 0)
    RGEO_CUDA(rgeo::launch_build_cull(m->d.bumps, m->d.K, m->d.cull_G, m->d.cull_words, m->d.cull_reach, m->d.cull_hdr,
                                      m->d.cull_masks, st),
              "rgeo_metric_advance: cull grid");
  return RGEO_OK;
}

rgeo_status rgeo_expmap_generate(const rgeo_metric *metric, int64_t n, uint64_t seed, float box, float s_max,
                                 float h, float accel_bound, float *inputs, float *targets, void *cuda_stream) {
  g_last_error.clear();
  if (!metric || n < 0 || (n > 0 && (!inputs || !targets)))
    return fail(RGEO_EINVAL, "rgeo_expmap_generate: bad argument");
  if (metric->d.kind != RGEO_METRIC_GRAPH_BUMPS) return fail(RGEO_EINVAL, "rgeo_expmap_generate: graph metrics only");
  if (!std::isfinite(accel_bound) || accel_bound < 0.f)
    return fail(RGEO_EINVAL, "rgeo_expmap_generate: accel_bound must be finite and >= 0");
  if (accel_bound > 0.f && (metric->d.aniso || metric->d.has_affine || metric->d.has_quad))
    return fail(RGEO_EINVAL, "rgeo_expmap_generate: a far-field bound needs isotropic bumps without polynomial part");
  if (!(box > 0.f) || !(s_max > 0.f) || !(h > 0.f) || !std::isfinite(box) || !std::isfinite(s_max) ||
      !std::isfinite(h) || s_max < h)
    return fail(RGEO_EINVAL, "rgeo_expmap_generate: need finite box > 0, h > 0, s_max >= h");
  rgeo::TraceParams p;
  std::memset(&p, 0, sizeof(p));
  const rgeo::MetricDev &m = metric->d;
  p.bumps = m.bumps;
  p.K = m.K;
  p.kind = m.kind;
  p.aniso = m.aniso;
  std::memcpy(p.b, m.b, sizeof(p.b));
  std::memcpy(p.A, m.A, sizeof(p.A));
  p.has_affine = m.has_affine;
  p.has_quad = m.has_quad;
  p.h = h;
  RGEO_CUDA(rgeo::launch_segments(p, n, seed, box, s_max, accel_bound, inputs, targets, (cudaStream_t)cuda_stream),
            "rgeo_expmap_generate");
  return RGEO_OK;
}


rgeo_status rgeo_expmap_train(rgeo_expmap *expmap, const rgeo_metric *metric, const rgeo_train_cfg *cfg,
                              float *loss, void *cuda_stream) {
  g_last_error.clear();
  if (!expmap || !metric || !cfg) return fail(RGEO_EINVAL, "rgeo_expmap_train: NULL argument");
  for (int i = 0; i < 4; i++)
    if (cfg->reserved[i] != 0) return fail(RGEO_EINVAL, "rgeo_expmap_train: reserved fields must be zero");
  if (cfg->steps < 1 || cfg->batch < 128 || cfg->batch % 128 != 0 || cfg->n_segments < cfg->batch ||
      !(cfg->lr_max > 0.f) || !(cfg->lr_min >= 0.f) || !(cfg->lr_min <= cfg->lr_max) || !std::isfinite(cfg->lr_max))
    return fail(RGEO_EINVAL, "rgeo_expmap_train: need steps >= 1, batch a multiple of 128, n_segments >= batch, "
                             "0 <= lr_min <= lr_max, lr_max > 0 finite");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t n = (size_t)cfg->n_segments, B = (size_t)cfg->batch;
  float *buf = nullptr;
  RGEO_CUDA(cudaMallocAsync((void **)&buf, sizeof(float) * (13 * n + 13 * B + (size_t)cfg->steps), st),
            "rgeo_expmap_train: buffers");
  float *X = buf, *T = X + 7 * n, *Xb = T + 6 * n, *Tb = Xb + 7 * B, *losses = Tb + 6 * B;
  rgeo_status s = rgeo_expmap_generate(metric, cfg->n_segments, cfg->seed, cfg->box, cfg->s_max, cfg->h,
                                       cfg->accel_bound, X, T, cuda_stream);
  const unsigned long long bseed = cfg->seed ^ 0xD1B54A32D192ED03ull;  // batch draws apart from the segments
  for (int it = 0; s == RGEO_OK && it < cfg->steps; ++it) {
    // cosine schedule from lr_max (first step) to lr_min (last step)
    const double c = cfg->steps > 1 ? (double)it / (cfg->steps - 1) : 0.0;
    const float lr = (float)(cfg->lr_min + 0.5 * (cfg->lr_max - cfg->lr_min) * (1.0 + std::cos(3.141592653589793 * c)));
    cudaError_t e = rgeo::launch_gather_batch(X, T, (long long)n, (int)B, bseed, it, Xb, Tb, st);
    if (e != cudaSuccess) {
      s = cuda_fail(e, "rgeo_expmap_train: batch");
      break;
    }
    s = rgeo_expmap_train_step(expmap, Xb, Tb, (int32_t)B, lr, losses + it, cuda_stream);
  }
  if (s == RGEO_OK && loss) {
    // mean loss over the last 1 % of the steps (at least one)
    const int tail = std::max(1, cfg->steps / 100);
    std::vector<float> h(tail);
    cudaError_t e = cudaMemcpyAsync(h.data(), losses + (cfg->steps - tail), sizeof(float) * tail,
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      s = cuda_fail(e, "rgeo_expmap_train: loss");
    } else {
      double acc = 0.0;
      for (float v : h) acc += v;
      *loss = (float)(acc / tail);
    }
  }
  cudaError_t e2 = cudaFreeAsync(buf, st);
  if (s != RGEO_OK) return s;
  if (e2 != cudaSuccess) return cuda_fail(e2, "rgeo_expmap_train: free");
  return RGEO_OK;
}

rgeo_status rgeo_trace_surrogate(const rgeo_metric *metric, const rgeo_scene *scene, const rgeo_camera *camera,
                                 int32_t width, int32_t height, float h, int32_t max_steps, int32_t shading,
                                 uint32_t flags, const rgeo_surrogate *sur, const rgeo_outputs *out,
                                 rgeo_surrogate_stats *stats, void *cuda_stream) {
  g_last_error.clear();
  rgeo_status s = validate_trace(metric, scene, camera, width, height, h, max_steps, RGEO_RK4, shading, flags, out);
  if (s != RGEO_OK) return s;
  if (metric->d.kind != RGEO_METRIC_GRAPH_BUMPS)
    return fail(RGEO_EINVAL, "rgeo_trace_surrogate: graph metrics only");
  if (sur && (!std::isfinite(sur->accel_bound) || sur->accel_bound < 0.f))
    return fail(RGEO_EINVAL, "rgeo_trace_surrogate: accel_bound must be finite and >= 0");
  if (sur && sur->accel_bound > 0.f && (metric->d.aniso || metric->d.has_affine || metric->d.has_quad))
    return fail(RGEO_EINVAL, "rgeo_trace_surrogate: a far-field bound needs isotropic bumps without polynomial part");
  if (!sur || !sur->expmap) return fail(RGEO_EINVAL, "rgeo_trace_surrogate: NULL surrogate or network");
  if (!(sur->box > 0.f) || !std::isfinite(sur->box) || !(sur->s_max >= h) || !std::isfinite(sur->s_max) ||
      !(sur->tau >= 0.f) || !std::isfinite(sur->tau) || sur->k_min < 1 || sur->cool_check < 1 || sur->max_rounds < 0 ||
      sur->reserved != 0)
    return fail(RGEO_EINVAL,
                "rgeo_trace_surrogate: need finite box > 0, s_max >= h, tau >= 0, k_min >= 1, cool_check >= 1, "
                "max_rounds >= 0, zero reserved fields");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  rgeo::TraceParams p = make_params(metric, scene, camera, width, height, h, max_steps, RGEO_RK4, shading, flags, out);
  const size_t N = (size_t)width * height;
  // one device block: state 15 N floats, steps, cool, two queues, jump_k (N ints each),
  // X and Y (7 N floats each), the work counter, the queue length and two statistics
  const size_t words = 15 * N + 5 * N + 14 * N;
  char *buf = nullptr;
  RGEO_CUDA(cudaMallocAsync((void **)&buf, words * 4 + 64, st), "rgeo_trace_surrogate: state");
  float *fw = (float *)buf;
  rgeo::WaveArgs w;
  std::memset(&w, 0, sizeof(w));
  w.st = fw;
  w.steps = (int32_t *)(fw + 15 * N);
  w.cool = w.steps + N;
  int32_t *qa = w.cool + N, *qb = qa + N;
  w.jump_k = qb + N;
  w.X = (float *)(w.jump_k + N);
  float *Y = w.X + 7 * N;
  w.Y = Y;
  uint32_t *counter = (uint32_t *)(Y + 7 * N);
  w.n_queue = counter + 1;
  w.stats = (unsigned long long *)(buf + words * 4 + 16);
  w.box = sur->box;
  w.s_max = sur->s_max;
  w.log_tau2 = sur->tau > 0.f ? 2.f * std::log(sur->tau) : -INFINITY;
  w.cool_check = sur->cool_check;
  w.accel_bound = sur->accel_bound;
  w.N = (long long)N;
  const long long natural = (long long)max_steps / sur->k_min + 2;
  const long long max_rounds = sur->max_rounds > 0 ? sur->max_rounds : natural;
  p.counter = counter;
  cudaError_t e = cudaMemsetAsync(w.stats, 0, 16, st);
  uint32_t n_in = p.n_items, nq = 0;
  int rounds = 0;
  for (long long round = 0; e == cudaSuccess; ++round) {
    w.first = round == 0;
    w.list_in = qa;
    w.queue = qb;
    w.k_min = round + 1 >= max_rounds ? 0x7fffffff : sur->k_min;
    p.n_items = n_in;
    if ((e = cudaMemsetAsync(counter, 0, 8, st)) != cudaSuccess) break;
    if ((e = rgeo::launch_wave_trace(p, w, st)) != cudaSuccess) break;
    ++rounds;
    if ((e = cudaMemcpyAsync(&nq, w.n_queue, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
    if (nq == 0) break;
    if ((e = rgeo::expmap_infer(sur->expmap, w.X, nq, Y, st)) != cudaSuccess) break;
    if ((e = rgeo::launch_wave_apply(w, nq, h, st)) != cudaSuccess) break;
    std::swap(qa, qb);
    n_in = nq;
  }
  unsigned long long hs[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hs, w.stats, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaError_t e2 = cudaFreeAsync(buf, st);
  if (e != cudaSuccess) return cuda_fail(e, "rgeo_trace_surrogate");
  if (e2 != cudaSuccess) return cuda_fail(e2, "rgeo_trace_surrogate: free");
  if (stats) {
    stats->jumps_accepted = (int64_t)hs[0];
    stats->jumps_rejected = (int64_t)hs[1];
    stats->rounds = rounds;
    stats->reserved = 0;
  }
  return RGEO_OK;
}

}  // extern "C"
