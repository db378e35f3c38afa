// rgeo_noalloc.cu -- an allocation-free variant of the trace entry point.
//
// rgeo_trace allocates its work counter with cudaMallocAsync on every call, and
// the metric and scene handles allocate their tables when they are created.
// Some callers cannot allocate device memory at all: a plugin whose host
// application owns the whole device memory budget, a real-time frame loop in
// which cudaMalloc (which may synchronise the device) is not allowed, or code
// that hands out memory only from its own fixed arena.  rgeo_trace_noalloc
// serves them: the caller passes its inputs and outputs in device memory it
// already owns, and the packed bump table and the work counter live in the
// file-scope device array below, which every GPU that loads this library holds
// until the process exits.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "rgeo.h"
#include "rgeo_internal.h"

namespace rgeo {
namespace {

// Scratch: the packed isotropic bump table (two float4 per bump, plus the inert pad
// bump) for up to RGEO_NOALLOC_MAX_BUMPS bumps, then 16 float4 whose first word is the
// work counter.  33,056 bytes per device.
constexpr int kNaTableFloat4 = kIsoBumpStride * (RGEO_NOALLOC_MAX_BUMPS + 1);
constexpr int kNaScratchFloat4 = kNaTableFloat4 + 16;
static __device__ __align__(256) float4 g_noalloc_scratch[kNaScratchFloat4];

// Host-side device addresses of the scratch, one per device, filled on first use
// with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
float4 *g_na_ptr[kMaxDevices] = {nullptr};

cudaError_t scratch_for_current_device(float4 **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = static_cast<float4 *>(p);
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

// Packs bump k of the padded table (layout of rgeo_internal.h).  A bump with a
// non-finite value or a spread <= 0 is written as an inert bump.
__global__ void k_pack_noalloc(const float *center, const float *amplitude, const float *sigma, int K,
                               float cutoff, float4 *table) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > iso_pad_index(K)) return;
  float c0 = 0.f, c1 = 0.f, c2 = 0.f, a = 0.f, s = 1.f;
  if (k < K) {
    c0 = center[3 * k];
    c1 = center[3 * k + 1];
    c2 = center[3 * k + 2];
    a = amplitude[k];
    s = sigma[k];
  }
  const bool bad = !isfinite(c0) || !isfinite(c1) || !isfinite(c2) || !isfinite(a) || !isfinite(s) || !(s > 0.f);
  if (bad) {
    c0 = c1 = c2 = a = 0.f;
    s = 1.f;
  }
  pack_iso_bump(table, k, c0, c1, c2, a, s, cutoff);
}

rgeo_status na_fail(rgeo_status s, const char *msg) {
  set_last_error(msg);
  return s;
}

// Whether p is memory that kernels on the current device can read and write: device
// memory of that device or managed memory.  A host pointer (pageable or pinned) is
// refused.  Queries only; allocates nothing.
bool device_accessible(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the (non-sticky) error the query recorded
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  if (at.type != cudaMemoryTypeDevice) return false;
  int dev = -1;
  return cudaGetDevice(&dev) == cudaSuccess && at.device == dev;
}

}  // namespace
}  // namespace rgeo

extern "C" rgeo_status rgeo_trace_noalloc(const float *center, const float *amplitude, const float *sigma,
                                          int32_t n_bumps, float cutoff_sigmas, const float *spheres,
                                          int32_t n_spheres, const float *albedo, const rgeo_camera *camera,
                                          int32_t width, int32_t height, float h, int32_t max_steps,
                                          int32_t integrator, int32_t shading, const rgeo_outputs *out,
                                          void *cuda_stream) {
  using namespace rgeo;
  set_last_error("");
  if (n_bumps < 0 || n_bumps > RGEO_NOALLOC_MAX_BUMPS)
    return na_fail(RGEO_EINVAL, "rgeo_trace_noalloc: n_bumps must be in [0, RGEO_NOALLOC_MAX_BUMPS]");
  if (n_spheres < 0 || n_spheres > RGEO_NOALLOC_MAX_SPHERES)
    return na_fail(RGEO_EINVAL, "rgeo_trace_noalloc: n_spheres must be in [0, RGEO_NOALLOC_MAX_SPHERES]");
  if ((n_bumps > 0 && (!center || !amplitude || !sigma)) || (n_spheres > 0 && !spheres) || !albedo)
    return na_fail(RGEO_EINVAL, "rgeo_trace_noalloc: NULL device array");
  if (n_spheres > 0 && reinterpret_cast<uintptr_t>(spheres) % 16 != 0)
    return na_fail(RGEO_EINVAL, "rgeo_trace_noalloc: spheres must be 16-byte aligned (read as float4)");
  if (!std::isfinite(cutoff_sigmas)) return na_fail(RGEO_EINVAL, "rgeo_trace_noalloc: non-finite cutoff");
  if (!camera || !out || !out->id || !out->hit || !out->steps || !out->rgba)
    return na_fail(RGEO_EINVAL, "rgeo_trace_noalloc: NULL camera or output");
  if (width < 1 || height < 1 || (int64_t)width * height >= (int64_t(1) << 31))
    return na_fail(RGEO_EINVAL, "rgeo_trace_noalloc: width and height must be >= 1 with W*H < 2^31");
  if (!std::isfinite(h) || h <= 0.f || max_steps < 1)
    return na_fail(RGEO_EINVAL, "rgeo_trace_noalloc: h must be finite and > 0, max_steps >= 1");
  if ((integrator != RGEO_RK4 && integrator != RGEO_EULER) ||
      (shading != RGEO_SHADE_LAMBERT && shading != RGEO_SHADE_PSEUDO))
    return na_fail(RGEO_EINVAL, "rgeo_trace_noalloc: unknown integrator or shading mode");
  for (int i = 0; i < 3; i++)
    if (!std::isfinite(camera->pos[i]) || !std::isfinite(camera->forward[i]) || !std::isfinite(camera->up[i]))
      return na_fail(RGEO_EINVAL, "rgeo_trace_noalloc: non-finite camera");
  {
    const void *arrays[] = {n_bumps > 0 ? center : nullptr, n_bumps > 0 ? amplitude : nullptr,
                            n_bumps > 0 ? sigma : nullptr,  n_spheres > 0 ? spheres : nullptr,
                            albedo,  out->id,  out->hit,  out->steps,  out->rgba};
    for (const void *a : arrays)
      if (a && !device_accessible(a))
        return na_fail(RGEO_EINVAL, "rgeo_trace_noalloc: every array must be device (or managed) memory of the "
                                    "current device");
  }
  const float *f = camera->forward, *u = camera->up;
  const float cx = u[1] * f[2] - u[2] * f[1], cy = u[2] * f[0] - u[0] * f[2], cz = u[0] * f[1] - u[1] * f[0];
  if (!(camera->vfov_deg > 0.f && camera->vfov_deg < 180.f) || cx * cx + cy * cy + cz * cz == 0.f)
    return na_fail(RGEO_EINVAL, "rgeo_trace_noalloc: bad field of view or forward parallel to up");

  cudaStream_t st = (cudaStream_t)cuda_stream;
  float4 *scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return na_fail(RGEO_ECUDA, "rgeo_trace_noalloc: cudaGetSymbolAddress failed");
  float4 *table = scratch;
  uint32_t *counter = reinterpret_cast<uint32_t *>(scratch + kNaTableFloat4);
  if (n_bumps > 0) {
    k_pack_noalloc<<<(iso_pad_index(n_bumps) + 1 + 127) / 128, 128, 0, st>>>(center, amplitude, sigma, n_bumps,
                                                                              cutoff_sigmas, table);
    if ((e = cudaGetLastError()) != cudaSuccess) return na_fail(RGEO_ECUDA, "rgeo_trace_noalloc: pack launch");
  }
  if ((e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), st)) != cudaSuccess)
    return na_fail(RGEO_ECUDA, "rgeo_trace_noalloc: counter reset");

  TraceParams p;
  std::memset(&p, 0, sizeof(p));
  p.bumps = table;
  p.K = n_bumps;
  p.kind = RGEO_METRIC_GRAPH_BUMPS;
  p.skippable = cutoff_sigmas > 0.f ? 1 : 0;
  p.spheres = reinterpret_cast<const float4 *>(spheres);
  p.S = n_spheres;
  p.albedo = albedo;
  for (int i = 0; i < 3; i++) {
    p.cam_pos[i] = camera->pos[i];
    p.cam_fwd[i] = camera->forward[i];
    p.cam_up[i] = camera->up[i];
  }
  p.vfov_deg = camera->vfov_deg;
  p.W = width;
  p.H = height;
  p.tile_lw = 3;  // 8 x 4 pixel tiles
  p.tile_step = 1;
  p.tiles_x = (width + 7) / 8;
  p.n_items = (uint32_t)p.tiles_x * (uint32_t)((height + 3) / 4) * 32u;
  p.h = h;
  p.max_steps = max_steps;
  p.integrator = integrator;
  p.shading = shading;
  p.id = out->id;
  p.hit = out->hit;
  p.steps = out->steps;
  p.rgba = reinterpret_cast<uchar4 *>(out->rgba);
  p.counter = counter;
  p.rays_per_thread = 1;
  if ((e = launch_trace(p, st)) != cudaSuccess) return na_fail(RGEO_ECUDA, "rgeo_trace_noalloc: trace launch");
  return RGEO_OK;
}
