/*
 * rgeo.h -- C ABI of librgeo, a geodesic ray tracer for (R^3, g) on sm_103a.
 *
 * The library traces one geodesic per pixel through R^3 endowed with a
 * designed Riemannian metric and intersects every step's segment with a scene
 * of spheres and triangles ("Design and visualization of Riemannian metrics",
 * Novello, da Silva, Velho 2020):
 *   - metric: the graph metric g = I + grad f grad f^T of a sum of Gaussian
 *     bumps (Eq. 5.2, Eq. 6.1, Section 6 "Summing functions"), or the
 *     pull-back metric g = J^T J of the twist diffeomorphism (Eq. 5.6,
 *     Section 5.2);
 *   - geodesics: the geodesic flow of Eq. 3.3 with the Christoffel symbols of
 *     Eq. 5.3 (graph) or Theorem 5.1 (diffeomorphism), i.e. the accelerations
 *     of Eq. 5.4 and Eq. 5.8, integrated by classical RK4 (Section 4.1 names it)
 *     or by Euler marching (Eq. 4.1);
 *   - shading: Riemannian shading (Section 4): each direction of the observer's
 *     view field gets the colour of the first object its geodesic meets; the
 *     polygon's segments are tested in order (Section 4.1).
 *
 * Conventions (apply to every entry point):
 *   - All entry points return an rgeo_status.  On a non-OK status a message
 *     describing the failure is available from rgeo_last_error() on the same
 *     host thread.  No C++ exception crosses this boundary.
 *   - Pointers documented as HOST are read during the call only.  Pointers
 *     documented as DEVICE must be device-accessible allocations on the
 *     current CUDA device; they are used asynchronously on the given stream.
 *   - A NULL stream means the legacy default stream.  Every launch is
 *     asynchronous with respect to the host unless stated otherwise.
 *   - Device-side errors (an exhausted traversal stack, a wait that timed
 *     out) are recorded in a per-device sticky error word; rgeo_sync() waits
 *     for the stream, reads and clears it, and maps it to a status.
 *   - float is IEEE binary32; all arithmetic on the device path is FP32 except
 *     the optional energy-drift diagnostic, which is FP64.
 */
#ifndef RGEO_H
#define RGEO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RGEO_ABI_VERSION 4 /* 4: rgeo_trace_tiles, tuning knobs, bundles, bump_slots; 3: rgeo_trace_lit; 2: local maps */

typedef enum {
  RGEO_OK = 0,
  RGEO_EINVAL = 1,       /* an argument failed validation */
  RGEO_ENOMEM = 2,       /* a device or host allocation failed */
  RGEO_ECUDA = 3,        /* a CUDA runtime call failed */
  RGEO_ETIMEOUT = 4,     /* a bounded device-side wait gave up */
  RGEO_EUNSUPPORTED = 5, /* valid request this build does not implement */
  RGEO_EDEVICE = 6       /* a kernel recorded a device-side error */
} rgeo_status;

typedef enum {
  RGEO_METRIC_GRAPH_BUMPS = 0, /* graph of f (Eq. 5.2), f a sum of Gaussian bumps (Eq. 6.1) */
  RGEO_METRIC_DIFFEO_TWIST = 1, /* pull-back through the twist of Section 5.2 (Eq. 5.6) */
  RGEO_METRIC_DIFFEO_LOCAL = 2  /* pull-back through a composition of local maps (Section 6) */
} rgeo_metric_kind;

typedef enum { RGEO_RK4 = 0, RGEO_EULER = 1 } rgeo_integrator;
typedef enum { RGEO_SHADE_LAMBERT = 0, RGEO_SHADE_PSEUDO = 1 } rgeo_shading;

/* rgeo_trace flags */
#define RGEO_FLAG_ENERGY_DIAG 1u /* write drift[p] = g(v_end, v_end) / g(v_0, v_0) - 1 (FP64) */
#define RGEO_FLAG_NO_SAFE_SKIP 2u /* test every segment (disables the exact safe-distance skip) */
#define RGEO_FLAG_DENSE 4u        /* sum over every bump even when the metric has a cull grid */
#define RGEO_FLAG_BUNDLE 8u       /* test the segments that need a test in bundles of four chords per
                                     scene query (Section 4.1: many segments per query); same results;
                                     rgeo_trace and rgeo_trace_tiles with RK4 only, ignored with
                                     RGEO_FLAG_ENERGY_DIAG */

/* Object ids written to rgeo_outputs.id */
#define RGEO_ID_MISS (-1)   /* the geodesic left every bump support and met nothing */
#define RGEO_ID_BUDGET (-2) /* max_steps integration steps without a hit */

typedef struct rgeo_metric rgeo_metric; /* opaque, owns device memory */
typedef struct rgeo_scene rgeo_scene;   /* opaque, owns device memory */

/* Metric description.  For the graph metric
 *   f(x) = b.x + 1/2 x^T A x + sum_k a_k exp(-sum_i (x_i - c_ki)^2 / (2 sigma_ki^2))
 * (Eq. 6.1 summed).  Each bump is truncated to ||(x - c_k) / sigma_k|| < cutoff_sigmas;
 * cutoff_sigmas <= 0 keeps every bump untruncated.  Where no truncated support
 * contains the ray and A = 0, Hess f = 0 and the geodesic is a straight line
 * (Eq. 5.4); the tracer then advances in closed form to the next support.
 * Bumps with a_k = 0 are inert.  With a cull grid (isotropic truncated bumps),
 * each cell records which bumps' supports meet it, and a point's sums run over
 * its cell's bumps only; excluded bumps are exactly zero there, so the result is
 * the same sum up to float32 summation order.  For the twist, twist_rate k gives
 * Phi(x, y, z) = (cos(kz) x - sin(kz) y, sin(kz) x + cos(kz) y, z) (k = 1 in the paper).
 *
 * For RGEO_METRIC_DIFFEO_LOCAL, n_bumps = K (1..RGEO_MAX_LOCAL_MAPS) local maps
 *   Phi_k(p) = p + f_k(p) V_k(p),  f_k(p) = a_k exp(-|p - c_k|^2 / (2 sigma_k^2)),
 *   V_k(p) = v_k + B_k (p - c_k)
 * (Section 6, "Using diffeomorphism", with the vector field V affine) are composed as
 * Phi = Phi_0 o Phi_1 o ... o Phi_{K-1} (map K - 1 acts first; Section 6, "Composing
 * diffeomorphisms") and the metric is g = J(Phi)^T J(Phi) (Eq. 5.6).  center, amplitude
 * and sigma (isotropic: equal triple) describe f_k, untruncated (cutoff_sigmas, affine_b
 * and quad_A unused; the last two must be zero); direction [K*3] holds v_k and field
 * [K*9] (row-major B_k, may be NULL for B_k = 0) the linear part of V_k.  With no field,
 * each map must satisfy |a_k| |v_k| e^{-1/2} / sigma_k < 1 (then p -> p + f_k(p) v_k is a
 * diffeomorphism of R^3); with a field, keeping each map a diffeomorphism is up to the
 * caller. */
typedef struct {
  int32_t kind;            /* rgeo_metric_kind */
  int32_t n_bumps;         /* K >= 0 (graph only); at most RGEO_MAX_BUMPS */
  const float *center;     /* HOST [K*3] bump centres c_k */
  const float *amplitude;  /* HOST [K] amplitudes a_k, finite */
  const float *sigma;      /* HOST [K*3] spreads sigma_k per axis, > 0; equal triple = isotropic */
  float affine_b[3];       /* b */
  float quad_A[9];         /* A, row-major, must be symmetric */
  float cutoff_sigmas;     /* c; 4 is the default used by the workloads */
  float twist_rate;        /* k (twist only) */
  int32_t cull_grid;       /* bump-support cull grid of G^3 cells: 0 = automatic (for >= 16
                              isotropic truncated bumps, G = 192 up to 64 bumps, 128 up to 1024, else 64; the
                              masks take G^3 x ceil(K / 32) x 4 bytes), -1 = none, 4..256 = that G */
  int32_t reserved[3];     /* must be zero */
  const float *direction;  /* HOST [K*3] v_k (local maps only; else ignored) */
  const float *field;      /* HOST [K*9] B_k or NULL (local maps only; else ignored) */
} rgeo_metric_desc;

#define RGEO_MAX_BUMPS 4096
#define RGEO_MAX_LOCAL_MAPS 64

/* Pinhole observer: position p, forward and up vectors (need not be unit or
 * orthogonal; up must not be parallel to forward), vertical field of view in
 * degrees (0, 180).  Pixel (i, j), row 0 at the top, looks along
 * normalize(F + u R + w U) with R = normalize(up x F), U = F x R,
 * u = (2 (i + 1/2) / W - 1) tan(fov/2) W / H and w = (1 - 2 (j + 1/2) / H) tan(fov/2);
 * its initial tangent is that direction scaled to g-unit length, a point of
 * the unit sphere S^2_p of Section 4. */
typedef struct {
  float pos[3];
  float forward[3];
  float up[3];
  float vfov_deg;
} rgeo_camera;

/* Per-pixel outputs, caller-owned DEVICE buffers, pixel p = j * W + i.
 *   id    [W*H] int32: sphere index in [0, S), S + t for triangle t, or RGEO_ID_*
 *   hit   [3*W*H] float, planar: hit[p], hit[N + p], hit[2N + p] = x, y, z of the hit
 *         point on the polygon segment (for MISS / BUDGET: the last position)
 *   steps [W*H] int32: integration steps taken (closed-form flat advances not counted)
 *   rgba  [4*W*H] uint8: shaded colour, alpha 255 on a hit, all zero otherwise
 *   drift [W*H] double, may be NULL: energy drift when RGEO_FLAG_ENERGY_DIAG is set
 *   bump_evals, bump_slots: optional work counters (below) */
typedef struct {
  int32_t *id;
  float *hit;
  int32_t *steps;
  uint8_t *rgba;
  double *drift;
  unsigned long long *bump_evals; /* DEVICE, may be NULL: one counter that receives (added to
                                     its current value) the number of bump terms summed, over
                                     all rays and RHS stages: K per stage for dense sums, the
                                     bumps of the ray's cull-grid cell otherwise */
  unsigned long long *bump_slots; /* DEVICE, may be NULL: as bump_evals, the bump terms the
                                     lanes evaluated (every lane of a warp evaluates the pairs
                                     of the warp's list, pads and other lanes' bumps included);
                                     bump_evals / bump_slots is the bump loop's SIMD efficiency */
} rgeo_outputs;

/* Library version and device capability check.  Returns RGEO_ABI_VERSION. */
int32_t rgeo_abi_version(void);

/* Message for the last non-OK status returned on this host thread ("" if none).
 * The string stays valid until the next rgeo_* call on this thread. */
const char *rgeo_last_error(void);

/* Build a metric on the current device (Eq. 5.2 / Eq. 6.1 or Eq. 5.6).  The
 * HOST arrays of desc are copied; the handle owns its device copies.  Packing
 * of the bump table runs on the device; the call synchronises before returning.
 * Errors: RGEO_EINVAL (NULL out/desc, unknown kind, K < 0 or > RGEO_MAX_BUMPS,
 * NULL arrays with K > 0, sigma <= 0, non-finite value, asymmetric A, twist
 * with bumps), RGEO_ENOMEM, RGEO_ECUDA.  On error *out is set to NULL. */
rgeo_status rgeo_metric_create(const rgeo_metric_desc *desc, rgeo_metric **out);

/* Replace the bump centres of a graph metric in place (HOST [K*3], same K),
 * enqueued on the stream (no synchronisation).  Used for animated metrics.
 * Errors: RGEO_EINVAL (NULL, not a graph metric, non-finite), RGEO_ECUDA. */
rgeo_status rgeo_metric_set_centers(rgeo_metric *metric, const float *center, void *cuda_stream);

void rgeo_metric_destroy(rgeo_metric *metric);

/* Build a scene on the current device: S spheres (HOST [S*4]: cx, cy, cz, r > 0),
 * a triangle mesh (HOST verts [V*3], HOST tris [T*3] vertex indices in [0, V)),
 * and albedo (HOST [(S+1)*3], one RGB per sphere then one for the whole mesh,
 * each in [0, 1]).  Builds a binned-SAH BVH over the triangles and a grid of
 * lower bounds of the distance to the scene on the host, then uploads them.
 * S and T may be zero.  Synchronises before returning.
 * Errors: RGEO_EINVAL, RGEO_ENOMEM, RGEO_ECUDA.  On error *out is set to NULL. */
rgeo_status rgeo_scene_create(const float *spheres, int32_t n_spheres, const float *verts,
                              int32_t n_verts, const int32_t *tris, int32_t n_tris,
                              const float *albedo, rgeo_scene **out);

/* Fog (Section 6 renders its grid figures with a faint black fog; the paper gives no
 * formula, so this is exponential attenuation along the ray): a hit's colour c
 * (Lambert or pseudo-colour) becomes
 * c T + rgb (1 - T), T = exp(-density * L), with L the arc length travelled to the hit
 * (h per integration step, the fraction of h on the hit segment, and the length of
 * each closed-form advance through flat space).  density = 0 (the default) turns it
 * off; rgb NULL is black.  Applies to traces enqueued afterwards.
 * Errors: RGEO_EINVAL (NULL scene, density < 0 or not finite, rgb not finite). */
rgeo_status rgeo_scene_set_fog(rgeo_scene *scene, float density, const float *rgb);

void rgeo_scene_destroy(rgeo_scene *scene);

/* Riemannian shading of a W x H view field (Section 4): for each pixel, march
 * its geodesic with step h (Section 4.1; RK4 or Euler per `integrator`) for at
 * most max_steps steps, test each segment against the scene, shade the first
 * hit.  Enqueued on `cuda_stream`; returns after enqueueing (asynchronous).
 * Allocates a 4-byte work counter with cudaMallocAsync on the stream per call.
 * Errors (synchronous): RGEO_EINVAL (NULL handles/outputs, W or H < 1,
 * W*H >= 2^31, h not finite or <= 0, max_steps < 1, bad enum, drift NULL with
 * RGEO_FLAG_ENERGY_DIAG), RGEO_ECUDA.  Device-side errors surface at rgeo_sync. */
rgeo_status rgeo_trace(const rgeo_metric *metric, const rgeo_scene *scene,
                       const rgeo_camera *camera, int32_t width, int32_t height, float h,
                       int32_t max_steps, int32_t integrator, int32_t shading, uint32_t flags,
                       const rgeo_outputs *out, void *cuda_stream);

/* One part of a frame (Section 4: the view field V of the observer, one geodesic
 * per direction), for splitting a frame across GPUs or calls: the pixels of
 * the frame tiles tile_begin, tile_begin + tile_step, ... below tile_end, in
 * the row-major order of the frame's tiles of 32 pixels in the tuning's tile
 * shape (rgeo_frame_tiles gives their number, rgeo_frame_tile_pixels their
 * pixels; tile_end = -1 means all).  Part r of N is (r, -1, N): interleaved
 * tiles spread the costly regions of a frame evenly.  Only the pixels of the
 * part are written in the full-frame output buffers; each pixel's result equals
 * that of rgeo_trace bit for bit, and the parts (r, -1, N), r = 0 .. N - 1,
 * write every pixel exactly once.  Otherwise as rgeo_trace.  Errors: as
 * rgeo_trace, and RGEO_EINVAL for tile_step < 1 or a range outside
 * [0, rgeo_frame_tiles(width, height)]. */
rgeo_status rgeo_trace_tiles(const rgeo_metric *metric, const rgeo_scene *scene, const rgeo_camera *camera,
                             int32_t width, int32_t height, float h, int32_t max_steps, int32_t integrator,
                             int32_t shading, uint32_t flags, int32_t tile_begin, int32_t tile_end,
                             int32_t tile_step, const rgeo_outputs *out, void *cuda_stream);

/* Number of queue tiles of a width x height frame in the current tile shape
 * (0 for an empty frame).  Host only. */
int32_t rgeo_frame_tiles(int32_t width, int32_t height);

/* The pixel indices (j * width + i) of frame tile `tile` in the current tile
 * shape, written to pixels[0 .. n) (at most 32; fewer at the frame's right and
 * bottom edges).  Returns n, or -1 for a bad argument.  Host only (the kernels
 * use the same mapping). */
int32_t rgeo_frame_tile_pixels(int32_t width, int32_t height, int32_t tile, int32_t *pixels);

/* rgeo_trace with HOST output buffers (same layout as rgeo_outputs; drift may be
 * NULL).  Stages the outputs in device memory, traces on the stream, copies the
 * results back and synchronises the stream before returning.  Host buffers
 * that are page-locked give asynchronous copies. */
rgeo_status rgeo_trace_host(const rgeo_metric *metric, const rgeo_scene *scene,
                            const rgeo_camera *camera, int32_t width, int32_t height, float h,
                            int32_t max_steps, int32_t integrator, int32_t shading,
                            uint32_t flags, const rgeo_outputs *host_out, void *cuda_stream);

/* Riemannian illumination (Section 4): a surface point q is lit by a light source
 * through the geodesics that connect q to it, and its radiant intensity is
 * Lambertian with an angle measured by the metric.  rgeo_trace_lit traces the view
 * field as rgeo_trace does (Lambert shading, no flags) and then re-shades every hit
 * from one point light:
 *   - q = hit + 1e-3 n, with n the unit surface normal facing the segment that hit;
 *   - the light geodesic from q is found by shooting: Gauss-Newton on the initial
 *     direction d0 + alpha e1 + beta e2 (d0 = (L - q) / |L - q|, e1 across the axis
 *     least aligned with d0, e2 = d0 x e1) for a zero miss vector (the closest
 *     approach of the marched polygon to L, minus L), with forward differences of
 *     step `delta`, at most `iters` steps, each clamped to 0.25;
 *   - each light geodesic is marched like a view ray (g-unit start, step h, the
 *     flat-space advance of truncated bumps) for at most max_steps steps;
 *   - the hit is lit when the miss fell to `tol` or below, the Riemannian cosine
 *     n.u / sqrt(n^T g^-1 n) of the initial g-unit tangent u is positive, and no
 *     segment of the light geodesic up to its closest approach meets the scene;
 *   - colour albedo * (0.1 + 0.9 cos) when lit, albedo * 0.1 otherwise (no fog).
 * The light geodesics sum, at each point, the bumps of its cull-grid cell (every bump
 * when the metric has no cull grid).  For isotropic truncated bumps with a cull grid (up
 * to 512 bumps) a warp's 30 light geodesics advance in lockstep by default and sum one
 * shared list of bumps, the union of their cells; schedule = 1, and every other metric,
 * has each lane walk its own cell's list.  Both give the same image bit for bit.
 * out->bump_evals, when given, receives the bump terms of the view rays and of the light
 * geodesics together.
 * `lit` (DEVICE [W*H] int32, may be NULL) receives 1 for lit hits, else 0.
 * Allocates work counters and a 16-byte-per-pixel buffer (normals, hit list) with
 * cudaMallocAsync on the stream.  Asynchronous on the stream.
 * Errors: those of rgeo_trace, and RGEO_EINVAL for a NULL light, a non-finite
 * light position, h or tol or delta not finite or <= 0, max_steps < 1, iters < 0,
 * a schedule other than 0 or 1, or nonzero reserved fields. */
typedef struct {
  float pos[3];      /* the point light L */
  float h;           /* step of the light geodesics */
  int32_t max_steps; /* step budget of each light geodesic */
  int32_t iters;     /* Gauss-Newton steps at most */
  float tol;         /* miss distance that counts as reaching the light */
  float delta;       /* forward-difference step of the Jacobian */
  int32_t schedule;  /* 0 (default): lockstep marches where they apply; 1: each lane on its own */
  int32_t reserved[3]; /* must be zero */
} rgeo_light;

rgeo_status rgeo_trace_lit(const rgeo_metric *metric, const rgeo_scene *scene, const rgeo_camera *camera,
                           int32_t width, int32_t height, float h, int32_t max_steps, int32_t integrator,
                           const rgeo_light *light, const rgeo_outputs *out, int32_t *lit,
                           void *cuda_stream);

/* ---------------------------------------------------------------- batches
 * Time- or user-dependent metrics (Introduction) and many views at once: a batch
 * traces several instances -- each its own metric, scene, camera, resolution,
 * step and outputs -- in one persistent launch whose warps move between
 * instances as their queues drain, so uneven sizes keep the GPU full.  Every
 * instance of a batch must share the metric kind, the bump layout (isotropic or
 * not) and the integrator.  Instances read their metric and scene at launch
 * time, so metrics animated with rgeo_metric_advance between launches are
 * traced at their new state.  rgeo_batch_launch enqueues only device work (a
 * memset of the per-instance counters and one kernel), so a stream capture of
 * [rgeo_metric_advance..., rgeo_batch_launch] replays as a CUDA graph. */
typedef struct rgeo_batch rgeo_batch; /* opaque, owns device memory */

typedef struct {
  const rgeo_metric *metric;
  const rgeo_scene *scene;
  rgeo_camera camera;
  int32_t width, height;
  float h;
  int32_t max_steps;
  int32_t integrator; /* rgeo_integrator */
  int32_t shading;    /* rgeo_shading */
  uint32_t flags;     /* RGEO_FLAG_* as for rgeo_trace */
  rgeo_outputs out;   /* DEVICE buffers of this instance */
} rgeo_instance;

/* Validate n >= 1 instances (each as rgeo_trace would), upload the instance
 * table and allocate per-instance work counters.  Synchronises.  The handles and
 * output buffers must outlive the batch.  Errors: RGEO_EINVAL (n < 1, NULL,
 * invalid instance, mixed metric kinds / layouts / integrators), RGEO_ENOMEM,
 * RGEO_ECUDA. */
rgeo_status rgeo_batch_create(int32_t n, const rgeo_instance *instances, rgeo_batch **out);

/* Trace every instance of the batch in one launch on the stream (asynchronous). */
rgeo_status rgeo_batch_launch(rgeo_batch *batch, void *cuda_stream);

void rgeo_batch_destroy(rgeo_batch *batch);

/* Sinusoidal motion of the bump centres of a graph metric:
 *   c_k(t) = c_k(0) + A_k sin(2 pi f_k t + phi_k), per axis of A_k,
 * with c_k(0) the centres the metric holds when this is called.  HOST arrays
 * amplitude [K*3], frequency [K], phase [K].  Sets t = 0.  Synchronises.
 * Errors: RGEO_EINVAL (NULL, not a graph metric, non-finite), RGEO_ENOMEM, RGEO_ECUDA. */
rgeo_status rgeo_metric_set_motion(rgeo_metric *metric, const float *amplitude, const float *frequency,
                                   const float *phase);

/* Set the motion time t (stream-ordered). */
rgeo_status rgeo_metric_set_time(rgeo_metric *metric, float t, void *cuda_stream);

/* Move the centres to c_k(t), rebuild the cull grid, then advance t by dt; t
 * lives in device memory, so a captured graph of this call animates frame after
 * frame without host input.  Asynchronous.  Errors: RGEO_EINVAL (no motion set,
 * non-finite dt), RGEO_ECUDA. */
rgeo_status rgeo_metric_advance(rgeo_metric *metric, float dt, void *cuda_stream);

/* -------------------------------------------------- learned exponential map
 * A surrogate of exp_p (Eq. 3.5) over short arcs: an MLP 7 -> 256 -> 256 -> 256 -> 7
 * (ReLU) maps a segment's start (x / box, unit direction d, s / s_max) to the
 * scaled residuals of its endpoint and tangent with respect to the straight line,
 *   r_x = (x_s - x - s v) / s^2,   r_v = (v_s - v) / s   (v the g-unit tangent along d),
 * plus a seventh output estimating log of its own squared error.  The two
 * 256 x 256 layers, forward and backward, run as BF16 tcgen05 tensor-core GEMMs
 * with FP32 accumulation; the 7-wide layers run in FP32.  Parameters are kept in
 * FP32 (Adam moments too): W1 [256 x 7], b1 [256], W2 [256 x 256], b2, W3, b3,
 * W4 [7 x 256], b4 [7], each W row-major (out x in), in this order.
 * Loss: mean squared error of outputs 0..5 against the targets, plus 0.1 x the
 * squared error of output 6 against log(sum of the six squared errors + 1e-6). */
typedef struct rgeo_expmap rgeo_expmap; /* opaque, owns device memory */

int64_t rgeo_expmap_param_count(void);

/* Allocate the network for batches of up to max_batch rows (a multiple of 128)
 * and initialise it (He-uniform weights from the seed, zero biases). Synchronises. */
rgeo_status rgeo_expmap_create(int32_t max_batch, uint64_t seed, rgeo_expmap **out);
void rgeo_expmap_destroy(rgeo_expmap *expmap);

/* Training segments generated by the integrator: n samples with x ~ U[-box, box]^3,
 * d uniform on S^2, s = k h with k uniform in 1..round(s_max / h), integrated by
 * RK4 at step h under the metric (graph metrics).  DEVICE inputs [n*7] =
 * (x / box, d, s / s_max), DEVICE targets [n*6] = (r_x, r_v).
 * accel_bound > 0 restricts the samples to the far field: a candidate is kept when
 * an upper bound on |x''| along every path of Euclidean length s from x (summed
 * per-bump bounds on |grad f| and ||Hess f|| of Eq. 6.1 at the nearest reachable
 * distance) is at most accel_bound, and the targets are divided by accel_bound, so
 * |r_x| <= 1/2 and |r_v| <= 1.  Up to 4096 candidates are drawn per sample (the last
 * is kept if none passes).  It needs isotropic bumps without affine or quadratic
 * part.  Asynchronous. */
rgeo_status rgeo_expmap_generate(const rgeo_metric *metric, int64_t n, uint64_t seed, float box, float s_max,
                                 float h, float accel_bound, float *inputs, float *targets, void *cuda_stream);

/* outputs [n*7] (DEVICE) for inputs [n*7] (DEVICE); any n >= 0.  Asynchronous. */
rgeo_status rgeo_expmap_forward(const rgeo_expmap *expmap, const float *inputs, int64_t n, float *outputs,
                                void *cuda_stream);

/* Loss and its gradient w.r.t. every parameter for one batch (a multiple of 128,
 * at most max_batch): grads (DEVICE [param_count], may be NULL) and loss (DEVICE
 * [1], may be NULL).  One persistent kernel runs the forward and backward pass of
 * every 128-row tile (the 256-wide layers' products on the tensor cores); its CTAs'
 * partial gradients are summed in a fixed order, so the same inputs give the same
 * bits on every call on a given device.  Asynchronous. */
rgeo_status rgeo_expmap_gradients(rgeo_expmap *expmap, const float *inputs, const float *targets, int32_t batch,
                                  float *grads, float *loss, void *cuda_stream);

/* One Adam step (beta 0.9, 0.999, eps 1e-8) at learning rate lr (finite, > 0) on the
 * gradient of rgeo_expmap_gradients: two kernel launches.  Asynchronous. */
rgeo_status rgeo_expmap_train_step(rgeo_expmap *expmap, const float *inputs, const float *targets,
                                   int32_t batch, float lr, float *loss, void *cuda_stream);

/* HOST copies of the FP32 parameters (n must equal rgeo_expmap_param_count()). */
rgeo_status rgeo_expmap_get_params(const rgeo_expmap *expmap, float *params, int64_t n);
rgeo_status rgeo_expmap_set_params(rgeo_expmap *expmap, const float *params, int64_t n);

/* Checkpoint: parameters, Adam moments and step count to / from a file. */
rgeo_status rgeo_expmap_save(const rgeo_expmap *expmap, const char *path);
rgeo_status rgeo_expmap_load(rgeo_expmap *expmap, const char *path);

/* Training in one call: n_segments segments from rgeo_expmap_generate (seed, box,
 * s_max, h, accel_bound as there), then `steps` Adam steps (rgeo_expmap_train_step) on
 * batches of `batch` rows drawn uniformly with replacement (counter-based), the learning
 * rate following a cosine from lr_max at the first step to lr_min at the last.  Writes
 * the mean loss of the last 1 % of the steps (at least one) to *loss (HOST, may be NULL)
 * and synchronises the stream when it does; otherwise asynchronous.  Scratch:
 * 52 (n_segments + batch) + 4 steps bytes of stream-ordered device memory. */
typedef struct {
  int64_t n_segments;  /* >= batch */
  int32_t steps;       /* >= 1 */
  int32_t batch;       /* multiple of 128, at most the network's max_batch */
  float lr_max, lr_min;
  uint64_t seed;
  float box, s_max, h, accel_bound;
  int32_t reserved[4]; /* must be zero */
} rgeo_train_cfg;

rgeo_status rgeo_expmap_train(rgeo_expmap *expmap, const rgeo_metric *metric, const rgeo_train_cfg *cfg,
                              float *loss, void *cuda_stream);

/* Tracing with surrogate jumps (Section 3, Eq. 3.5; graph metrics, RK4).
 * As rgeo_trace, except that a ray inside the bumps' supports may replace k RK4
 * steps (k_min <= k, k h <= s_max) by one evaluation of the trained network:
 *   x <- x + s v + s^2 r_x,   v <- v + s r_v,   s = k h.
 * A jump is attempted only where it cannot reach the scene: g = I + grad f grad f^T
 * >= I (Eq. 5.2) bounds the Euclidean length of a geodesic arc by its g-length s,
 * so the jump is queued when the scene's safe distance at x exceeds 1.01 s + 1e-4,
 * |x_i| <= box, and the step budget allows k steps.  The network evaluates the
 * queue in batches on the tensor cores; a jump is taken when its predicted error
 * satisfies exp(output 6) <= tau^2 (tau = 0 takes none), otherwise the ray
 * integrates those k steps by RK4 before it may try again.  With accel_bound > 0
 * the jump must also lie in the far field of rgeo_expmap_generate (k is halved up
 * to twice to find such a jump) and the network's outputs are multiplied by
 * accel_bound; tau is then in units of accel_bound.  Rays that found no
 * certified jump retry after cool_check steps.  steps[p] counts a jump as its k
 * steps.  Rays advance in rounds; each round ends with a host wait on the stream,
 * so this call returns when the image is complete (it is not graph-capturable).
 * The last round (max_rounds, or 0 for max_steps / k_min + 2) takes no jumps.
 * stats may be NULL.  Errors: as rgeo_trace, plus RGEO_EINVAL for a metric that
 * is not a graph metric, an integrator other than RK4, or bad surrogate values. */
typedef struct {
  const rgeo_expmap *expmap; /* trained network (its max_batch is the inference chunk) */
  float box;                 /* input scale of positions; jumps only where |x_i| <= box */
  float s_max;               /* input scale of arc length; longest jump */
  float tau;                 /* threshold on the predicted root-sum-square error of (r_x, r_v) */
  int32_t k_min;             /* shortest jump in steps, >= 1 */
  int32_t cool_check;        /* steps between attempts where no jump is certified, >= 1 */
  int32_t max_rounds;        /* 0: max_steps / k_min + 2 */
  float accel_bound;         /* > 0: far-field domain, as in rgeo_expmap_generate; 0: none */
  int32_t reserved;          /* must be zero */
} rgeo_surrogate;

typedef struct {
  int64_t jumps_accepted;
  int64_t jumps_rejected;
  int32_t rounds;
  int32_t reserved;
} rgeo_surrogate_stats;

rgeo_status rgeo_trace_surrogate(const rgeo_metric *metric, const rgeo_scene *scene, const rgeo_camera *camera,
                                 int32_t width, int32_t height, float h, int32_t max_steps, int32_t shading,
                                 uint32_t flags, const rgeo_surrogate *surrogate, const rgeo_outputs *out,
                                 rgeo_surrogate_stats *stats, void *cuda_stream);

/* The tensor-core GEMM of the surrogate, C = A B^T (+ bias), for testing and
 * measurement: A DEVICE bf16 [M x K] row-major, B DEVICE bf16 [N x K] row-major,
 * 16 <= N <= 256 with N % 16 == 0, K % 64 == 0, A and B 16-byte aligned.  mode 0: C float [M x ldc] with
 * bias; mode 1: relu(C + bias) as bf16 [M x ldc] and, if ct != NULL, transposed
 * bf16 [N x ldt]; mode 2: C added atomically to float [M x ldc], K split over
 * `splits` CTAs.  Asynchronous; a tensor-core wait that gives up is reported by
 * rgeo_sync as RGEO_ETIMEOUT. */
rgeo_status rgeo_gemm_bf16(const void *A, const void *B, int32_t M, int32_t N, int32_t K, int32_t splits,
                           const float *bias, int32_t mode, void *C, int32_t ldc, void *ct, int32_t ldt,
                           void *cuda_stream);

/* Wait for the stream, then read and clear the device error word of the
 * current device.  Returns RGEO_OK, RGEO_EDEVICE or RGEO_ETIMEOUT (message in
 * rgeo_last_error), or RGEO_ECUDA if the stream itself failed. */
rgeo_status rgeo_sync(void *cuda_stream);

/* Allocation-free tracing (the paper has no counterpart; this serves callers).
 *
 * Some callers cannot allocate device memory: a plugin whose host application
 * owns the whole device memory budget, a real-time frame loop in which
 * cudaMalloc (which may synchronise the device) is not allowed, or code that
 * hands out memory only from its own fixed arena.  They also cannot create the
 * metric and scene handles, which allocate.  rgeo_trace_noalloc takes the
 * inputs as DEVICE arrays the caller owns and allocates nothing: it calls no
 * cudaMalloc, cudaMallocAsync, cudaFree or other allocating routine.  Its
 * scratch (the packed bump table and the work counter) is a file-scope device
 * array of 33,056 bytes that every GPU loading the library holds until the
 * process exits.
 *
 * Scope: the graph metric of up to RGEO_NOALLOC_MAX_BUMPS isotropic Gaussian
 * bumps (no affine or quadratic part), up to RGEO_NOALLOC_MAX_SPHERES spheres,
 * no triangle mesh, no energy diagnostic; results equal those of rgeo_trace on
 * the same inputs.
 *   center    DEVICE [K*3] bump centres       amplitude DEVICE [K]
 *   sigma     DEVICE [K] isotropic spreads (> 0)
 *   spheres   DEVICE [S*4] cx, cy, cz, r (16-byte aligned)
 *   albedo    DEVICE [(S+1)*3]
 * Other arguments as for rgeo_trace (out->drift is ignored).  A bump whose
 * device values are non-finite or whose spread is <= 0 is treated as inert.
 *
 * The first call on a device looks up the scratch address with that device
 * current (cudaGetSymbolAddress) and keeps it for the life of the process;
 * make that first call before any stream capture, and do not use this entry
 * point across a cudaDeviceReset (the module reloads and the kept address goes
 * stale).  Every call shares the one scratch array per device and it keeps the
 * last call's contents: calls whose work overlaps on the GPU (different streams
 * without ordering between them) race and must not be issued.  Asynchronous on
 * the stream.  Errors: RGEO_EINVAL (counts beyond the maxima, NULL pointers,
 * spheres not 16-byte aligned, an array that is not device or managed memory of
 * the current device, bad camera, size, step or enum), RGEO_ECUDA. */
#define RGEO_NOALLOC_MAX_BUMPS 1024
#define RGEO_NOALLOC_MAX_SPHERES 1024

rgeo_status rgeo_trace_noalloc(const float *center, const float *amplitude, const float *sigma,
                               int32_t n_bumps, float cutoff_sigmas, const float *spheres,
                               int32_t n_spheres, const float *albedo, const rgeo_camera *camera,
                               int32_t width, int32_t height, float h, int32_t max_steps,
                               int32_t integrator, int32_t shading, const rgeo_outputs *out,
                               void *cuda_stream);

/* Process-wide launch tuning (the knobs the autotuner searches).  None of them
 * changes a result bit of a trace: every lane sums its own bumps in the same
 * order whatever shares its warp.
 *   rays_per_thread  1 or 2 rays advanced together by each thread (2 applies to
 *                    isotropic graph metrics with dense sums only); 0 restores 1.
 *   batch_params     where a batch's warps read their instance's parameters: 0
 *                    (default) from the kernel's parameter space when the batch
 *                    has at most 64 instances, else from a per-warp shared-memory
 *                    copy; 1 always from the shared-memory copy.
 *   wait_limit       polls of each bounded barrier wait in the tensor-core kernels'
 *                    work (rgeo_gemm_bf16, the surrogate's inference): 0 the
 *                    default, n > 0 that many, -1 none, so that every such wait
 *                    gives up at once (for testing the timeout path).  A wait that
 *                    gives up makes the kernel drain its own copies and MMAs, free
 *                    its tensor memory and return; rgeo_sync then reports
 *                    RGEO_ETIMEOUT.
 *   ctas_per_sm      persistent trace launches: 0 (default) as many 128-thread
 *                    CTAs per SM as fit, else at most this many (1 .. 32).
 *   tile_shape       pixels a warp takes from the queue at a time (32 per tile):
 *                    0 default (4 x 8), 1 8 x 4, 2 4 x 8, 3 16 x 2; read by
 *                    rgeo_frame_tiles and every trace.
 *   batch_order      rgeo_batch_create's instance order: 0 (default) by
 *                    decreasing cost (pixels x bumps), 1 as given.
 *   sum_lists        culled bump sums of a warp: 0 (default) one list of bumps for
 *                    as many RK4 steps (up to 8) as stay within 0.04 of where it
 *                    was made (metrics of up to 512 bumps, whose cull masks carry
 *                    that margin), else a list per right-hand side; 1 always per
 *                    right-hand side; 2 one list per RK4 step.
 *   refill           when the lanes of a trace warp take new rays from the queue:
 *                    0 (default) in generations, the warp taking the next 32
 *                    items once all of its rays have finished: its rays start
 *                    from one tile together and stay close, so the bump lists
 *                    its lanes share stay short, and its lanes take the same
 *                    branches longer; 1 each lane as soon as its ray has finished.
 * A setting is read when a trace or batch is enqueued or created (a captured
 * graph keeps the choice made at capture); it is not synchronised between host
 * threads.  Errors: RGEO_EINVAL (NULL, bad value, nonzero reserved fields). */
typedef struct {
  int32_t rays_per_thread;
  int32_t batch_params;
  int32_t wait_limit;
  int32_t ctas_per_sm;
  int32_t tile_shape;
  int32_t batch_order;
  int32_t sum_lists;
  int32_t refill;
  int32_t reserved[1]; /* must be zero */
} rgeo_tuning;

rgeo_status rgeo_set_tuning(const rgeo_tuning *tuning);
rgeo_status rgeo_get_tuning(rgeo_tuning *tuning);

/* Measurement helper: time an FP32 fused multiply-add loop on the current
 * device (mode 0: scalar FFMA; mode 1: paired f32x2 FMA) and write the achieved
 * rate in TFLOP/s (2 flops per multiply-add) to *tflops and the loop time to
 * *ms.  Synchronous.  Errors: RGEO_EINVAL (NULL output, unknown mode), RGEO_ECUDA. */
rgeo_status rgeo_ffma_probe(int32_t mode, float *tflops, float *ms);

#ifdef __cplusplus
}
#endif

#endif /* RGEO_H */
