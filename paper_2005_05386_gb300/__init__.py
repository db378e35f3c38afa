"""Python binding of librgeo, a geodesic ray tracer for designed Riemannian metrics on GB300.

The functions ``rgeo_*`` below carry the names of the C entry points declared in
``include/rgeo.h`` and only marshal arguments: every step of the traced path
runs in the library's CUDA kernels.  PyTorch provides device memory and streams.
There is no CPU fallback: when the library is missing or cannot be loaded, the
first call raises.

Convenience wrappers (``Metric``, ``Scene``, ``trace``) build the C structs from
the seeded workloads of :mod:`paper_2005_05386_gb300.scenes` and allocate the
output buffers as torch tensors.
"""
from __future__ import annotations

import ctypes
import os

from . import scenes

_HERE = os.path.dirname(os.path.abspath(__file__))
# the in-tree build; RGEO_LIBRARY names another build of the same sources to load instead
LIB_PATH = os.environ.get("RGEO_LIBRARY") or os.path.join(_HERE, "librgeo.so")

RGEO_OK, RGEO_EINVAL, RGEO_ENOMEM, RGEO_ECUDA, RGEO_ETIMEOUT, RGEO_EUNSUPPORTED, RGEO_EDEVICE = range(7)
RGEO_METRIC_GRAPH_BUMPS, RGEO_METRIC_DIFFEO_TWIST, RGEO_METRIC_DIFFEO_LOCAL = 0, 1, 2
RGEO_MAX_LOCAL_MAPS = 64
RGEO_ABI_VERSION = 4  # include/rgeo.h; the loaded library must report the same
RGEO_RK4, RGEO_EULER = 0, 1
RGEO_SHADE_LAMBERT, RGEO_SHADE_PSEUDO = 0, 1
RGEO_FLAG_ENERGY_DIAG = 1
RGEO_FLAG_NO_SAFE_SKIP = 2
RGEO_FLAG_DENSE = 4
RGEO_FLAG_BUNDLE = 8
RGEO_ID_MISS, RGEO_ID_BUDGET = -1, -2
RGEO_MAX_BUMPS = 4096

# Every symbol include/rgeo.h declares (checked by the tests).
EXPORTS = ("rgeo_abi_version", "rgeo_last_error", "rgeo_metric_create", "rgeo_metric_set_centers",
           "rgeo_metric_destroy", "rgeo_scene_create", "rgeo_scene_destroy", "rgeo_trace",
           "rgeo_trace_host", "rgeo_sync", "rgeo_set_tuning", "rgeo_get_tuning", "rgeo_ffma_probe",
           "rgeo_trace_noalloc", "rgeo_batch_create", "rgeo_batch_launch", "rgeo_batch_destroy",
           "rgeo_metric_set_motion", "rgeo_metric_set_time", "rgeo_metric_advance", "rgeo_expmap_param_count",
           "rgeo_expmap_create", "rgeo_expmap_destroy", "rgeo_expmap_generate", "rgeo_expmap_forward",
           "rgeo_expmap_gradients", "rgeo_expmap_train_step", "rgeo_expmap_get_params", "rgeo_expmap_set_params",
           "rgeo_expmap_save", "rgeo_expmap_load", "rgeo_gemm_bf16", "rgeo_trace_surrogate", "rgeo_expmap_train", "rgeo_scene_set_fog",
           "rgeo_trace_lit", "rgeo_trace_tiles", "rgeo_frame_tiles", "rgeo_frame_tile_pixels")
RGEO_NOALLOC_MAX_BUMPS = 1024
RGEO_NOALLOC_MAX_SPHERES = 1024


class RgeoError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where} failed with status {status}: {message}")
        self.status = status


class rgeo_metric_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_bumps", ctypes.c_int32),
                ("center", ctypes.POINTER(ctypes.c_float)), ("amplitude", ctypes.POINTER(ctypes.c_float)),
                ("sigma", ctypes.POINTER(ctypes.c_float)), ("affine_b", ctypes.c_float * 3),
                ("quad_A", ctypes.c_float * 9), ("cutoff_sigmas", ctypes.c_float),
                ("twist_rate", ctypes.c_float), ("cull_grid", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3),
                ("direction", ctypes.POINTER(ctypes.c_float)), ("field", ctypes.POINTER(ctypes.c_float))]


class rgeo_camera(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_float * 3), ("forward", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("vfov_deg", ctypes.c_float)]


class rgeo_light(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_float * 3), ("h", ctypes.c_float), ("max_steps", ctypes.c_int32),
                ("iters", ctypes.c_int32), ("tol", ctypes.c_float), ("delta", ctypes.c_float),
                ("schedule", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class rgeo_tuning(ctypes.Structure):
    _fields_ = [("rays_per_thread", ctypes.c_int32), ("batch_params", ctypes.c_int32),
                ("wait_limit", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("tile_shape", ctypes.c_int32), ("batch_order", ctypes.c_int32), ("sum_lists", ctypes.c_int32),
                ("refill", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


TUNING_FIELDS = ("rays_per_thread", "batch_params", "wait_limit", "ctas_per_sm", "tile_shape", "batch_order",
                 "sum_lists", "refill")


class rgeo_outputs(ctypes.Structure):
    _fields_ = [("id", ctypes.c_void_p), ("hit", ctypes.c_void_p), ("steps", ctypes.c_void_p),
                ("rgba", ctypes.c_void_p), ("drift", ctypes.c_void_p), ("bump_evals", ctypes.c_void_p),
                ("bump_slots", ctypes.c_void_p)]


class rgeo_train_cfg(ctypes.Structure):
    _fields_ = [("n_segments", ctypes.c_int64), ("steps", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("lr_max", ctypes.c_float), ("lr_min", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("box", ctypes.c_float), ("s_max", ctypes.c_float), ("h", ctypes.c_float),
                ("accel_bound", ctypes.c_float), ("reserved", ctypes.c_int32 * 4)]


class rgeo_surrogate(ctypes.Structure):
    _fields_ = [("expmap", ctypes.c_void_p), ("box", ctypes.c_float), ("s_max", ctypes.c_float),
                ("tau", ctypes.c_float), ("k_min", ctypes.c_int32), ("cool_check", ctypes.c_int32),
                ("max_rounds", ctypes.c_int32), ("accel_bound", ctypes.c_float), ("reserved", ctypes.c_int32)]


class rgeo_surrogate_stats(ctypes.Structure):
    _fields_ = [("jumps_accepted", ctypes.c_int64), ("jumps_rejected", ctypes.c_int64), ("rounds", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class rgeo_instance(ctypes.Structure):
    _fields_ = [("metric", ctypes.c_void_p), ("scene", ctypes.c_void_p), ("camera", rgeo_camera),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("h", ctypes.c_float),
                ("max_steps", ctypes.c_int32), ("integrator", ctypes.c_int32), ("shading", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("out", rgeo_outputs)]


_lib = None


def library() -> ctypes.CDLL:
    """Load librgeo.so (built in-tree by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"librgeo.so not found at {LIB_PATH}; build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, u32, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_float
    fp = ctypes.POINTER(ctypes.c_float)
    ip = ctypes.POINTER(ctypes.c_int32)
    L.rgeo_abi_version.restype = i32
    L.rgeo_abi_version.argtypes = []
    L.rgeo_last_error.restype = ctypes.c_char_p
    L.rgeo_last_error.argtypes = []
    L.rgeo_metric_create.restype = i32
    L.rgeo_metric_create.argtypes = [ctypes.POINTER(rgeo_metric_desc), ctypes.POINTER(vp)]
    L.rgeo_metric_set_centers.restype = i32
    L.rgeo_metric_set_centers.argtypes = [vp, fp, vp]
    L.rgeo_metric_destroy.restype = None
    L.rgeo_metric_destroy.argtypes = [vp]
    L.rgeo_scene_create.restype = i32
    L.rgeo_scene_create.argtypes = [fp, i32, fp, i32, ip, i32, fp, ctypes.POINTER(vp)]
    L.rgeo_scene_destroy.restype = None
    L.rgeo_scene_destroy.argtypes = [vp]
    trace_args = [vp, vp, ctypes.POINTER(rgeo_camera), i32, i32, f32, i32, i32, i32, u32,
                  ctypes.POINTER(rgeo_outputs), vp]
    L.rgeo_trace.restype = i32
    L.rgeo_trace.argtypes = trace_args
    L.rgeo_trace_host.restype = i32
    L.rgeo_trace_host.argtypes = trace_args
    L.rgeo_trace_tiles.restype = i32
    L.rgeo_trace_tiles.argtypes = trace_args[:10] + [i32, i32, i32] + trace_args[10:]
    L.rgeo_frame_tiles.restype = i32
    L.rgeo_frame_tiles.argtypes = [i32, i32]
    L.rgeo_frame_tile_pixels.restype = i32
    L.rgeo_frame_tile_pixels.argtypes = [i32, i32, i32, ctypes.POINTER(i32)]
    L.rgeo_trace_lit.restype = i32
    L.rgeo_trace_lit.argtypes = [vp, vp, ctypes.POINTER(rgeo_camera), i32, i32, f32, i32, i32,
                                 ctypes.POINTER(rgeo_light), ctypes.POINTER(rgeo_outputs), vp, vp]
    L.rgeo_sync.restype = i32
    L.rgeo_sync.argtypes = [vp]
    i64, u64 = ctypes.c_int64, ctypes.c_uint64
    L.rgeo_expmap_param_count.restype = i64
    L.rgeo_expmap_param_count.argtypes = []
    L.rgeo_expmap_create.restype = i32
    L.rgeo_expmap_create.argtypes = [i32, u64, ctypes.POINTER(vp)]
    L.rgeo_expmap_destroy.restype = None
    L.rgeo_expmap_destroy.argtypes = [vp]
    L.rgeo_expmap_generate.restype = i32
    L.rgeo_expmap_generate.argtypes = [vp, i64, u64, f32, f32, f32, f32, vp, vp, vp]
    L.rgeo_expmap_forward.restype = i32
    L.rgeo_expmap_forward.argtypes = [vp, vp, i64, vp, vp]
    L.rgeo_expmap_gradients.restype = i32
    L.rgeo_expmap_gradients.argtypes = [vp, vp, vp, i32, vp, vp, vp]
    L.rgeo_expmap_train_step.restype = i32
    L.rgeo_expmap_train_step.argtypes = [vp, vp, vp, i32, f32, vp, vp]
    L.rgeo_expmap_get_params.restype = i32
    L.rgeo_expmap_get_params.argtypes = [vp, fp, i64]
    L.rgeo_expmap_set_params.restype = i32
    L.rgeo_expmap_set_params.argtypes = [vp, fp, i64]
    L.rgeo_expmap_save.restype = i32
    L.rgeo_expmap_save.argtypes = [vp, ctypes.c_char_p]
    L.rgeo_expmap_load.restype = i32
    L.rgeo_expmap_load.argtypes = [vp, ctypes.c_char_p]
    L.rgeo_scene_set_fog.restype = i32
    L.rgeo_scene_set_fog.argtypes = [vp, f32, fp]
    L.rgeo_expmap_train.restype = i32
    L.rgeo_expmap_train.argtypes = [vp, vp, ctypes.POINTER(rgeo_train_cfg), fp, vp]
    L.rgeo_trace_surrogate.restype = i32
    L.rgeo_trace_surrogate.argtypes = [vp, vp, ctypes.POINTER(rgeo_camera), i32, i32, f32, i32, i32, ctypes.c_uint32,
                                       ctypes.POINTER(rgeo_surrogate), ctypes.POINTER(rgeo_outputs),
                                       ctypes.POINTER(rgeo_surrogate_stats), vp]
    L.rgeo_gemm_bf16.restype = i32
    L.rgeo_gemm_bf16.argtypes = [vp, vp, i32, i32, i32, i32, vp, i32, vp, i32, vp, i32, vp]
    L.rgeo_batch_create.restype = i32
    L.rgeo_batch_create.argtypes = [i32, ctypes.POINTER(rgeo_instance), ctypes.POINTER(vp)]
    L.rgeo_batch_launch.restype = i32
    L.rgeo_batch_launch.argtypes = [vp, vp]
    L.rgeo_batch_destroy.restype = None
    L.rgeo_batch_destroy.argtypes = [vp]
    L.rgeo_metric_set_motion.restype = i32
    L.rgeo_metric_set_motion.argtypes = [vp, fp, fp, fp]
    L.rgeo_metric_set_time.restype = i32
    L.rgeo_metric_set_time.argtypes = [vp, f32, vp]
    L.rgeo_metric_advance.restype = i32
    L.rgeo_metric_advance.argtypes = [vp, f32, vp]
    L.rgeo_trace_noalloc.restype = i32
    L.rgeo_trace_noalloc.argtypes = [vp, vp, vp, i32, f32, vp, i32, vp, ctypes.POINTER(rgeo_camera), i32, i32,
                                     f32, i32, i32, i32, ctypes.POINTER(rgeo_outputs), vp]
    L.rgeo_set_tuning.restype = i32
    L.rgeo_set_tuning.argtypes = [ctypes.POINTER(rgeo_tuning)]
    L.rgeo_get_tuning.restype = i32
    L.rgeo_get_tuning.argtypes = [ctypes.POINTER(rgeo_tuning)]
    L.rgeo_ffma_probe.restype = i32
    L.rgeo_ffma_probe.argtypes = [i32, fp, fp]
    _lib = L
    return L


def _check(status: int, where: str):
    if status != RGEO_OK:
        raise RgeoError(status, where, rgeo_last_error())


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if a is not None else None


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------- raw C entry points
def rgeo_abi_version() -> int:
    return library().rgeo_abi_version()


def rgeo_last_error() -> str:
    return library().rgeo_last_error().decode()


def rgeo_metric_create(desc: rgeo_metric_desc) -> int:
    out = ctypes.c_void_p()
    _check(library().rgeo_metric_create(ctypes.byref(desc), ctypes.byref(out)), "rgeo_metric_create")
    return out.value


def rgeo_metric_set_centers(metric: int, center, stream=None):
    import numpy as np
    c = np.ascontiguousarray(center, dtype=np.float32)
    _check(library().rgeo_metric_set_centers(metric, _fptr(c), _stream_handle(stream)), "rgeo_metric_set_centers")


def rgeo_metric_destroy(metric: int):
    library().rgeo_metric_destroy(metric)


def rgeo_scene_create(spheres, verts, tris, albedo) -> int:
    import numpy as np
    s = np.ascontiguousarray(spheres, dtype=np.float32).reshape(-1, 4)
    v = np.ascontiguousarray(verts, dtype=np.float32).reshape(-1, 3)
    t = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
    a = np.ascontiguousarray(albedo, dtype=np.float32).reshape(-1, 3)
    out = ctypes.c_void_p()
    _check(library().rgeo_scene_create(_fptr(s), s.shape[0], _fptr(v), v.shape[0],
                                       t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), t.shape[0],
                                       _fptr(a), ctypes.byref(out)), "rgeo_scene_create")
    return out.value


def rgeo_scene_destroy(scene: int):
    library().rgeo_scene_destroy(scene)


def rgeo_trace(metric: int, scene: int, camera: rgeo_camera, width: int, height: int, h: float,
               max_steps: int, integrator: int, shading: int, flags: int, out: rgeo_outputs, stream=None):
    _check(library().rgeo_trace(metric, scene, ctypes.byref(camera), width, height, h, max_steps, integrator,
                                shading, flags, ctypes.byref(out), _stream_handle(stream)), "rgeo_trace")


def rgeo_trace_tiles(metric: int, scene: int, camera: rgeo_camera, width: int, height: int, h: float,
                     max_steps: int, integrator: int, shading: int, flags: int, tile_begin: int, tile_end: int,
                     tile_step: int, out: rgeo_outputs, stream=None):
    _check(library().rgeo_trace_tiles(metric, scene, ctypes.byref(camera), width, height, h, max_steps, integrator,
                                      shading, flags, tile_begin, tile_end, tile_step, ctypes.byref(out),
                                      _stream_handle(stream)), "rgeo_trace_tiles")


def rgeo_frame_tiles(width: int, height: int) -> int:
    return int(library().rgeo_frame_tiles(width, height))


def rgeo_frame_tile_pixels(width: int, height: int, tile: int):
    """Pixel indices of one frame tile (numpy int32 array), as the kernels map them."""
    import numpy as np
    buf = np.empty(32, np.int32)
    n = library().rgeo_frame_tile_pixels(width, height, tile, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if n < 0:
        raise RgeoError(RGEO_EINVAL, "rgeo_frame_tile_pixels", "bad argument")
    return buf[:n].copy()


def part_pixels(width: int, height: int, part: int, n_parts: int):
    """Pixels of part `part` of `n_parts` (interleaved tiles part, part + n_parts, ...)."""
    import numpy as np
    tiles = range(part, rgeo_frame_tiles(width, height), n_parts)
    return np.concatenate([rgeo_frame_tile_pixels(width, height, t) for t in tiles] or [np.empty(0, np.int32)])


def rgeo_trace_lit(metric: int, scene: int, camera: rgeo_camera, width: int, height: int, h: float,
                   max_steps: int, integrator: int, light: rgeo_light, out: rgeo_outputs, lit: int = 0,
                   stream=None):
    _check(library().rgeo_trace_lit(metric, scene, ctypes.byref(camera), width, height, h, max_steps, integrator,
                                    ctypes.byref(light), ctypes.byref(out), lit or None, _stream_handle(stream)),
           "rgeo_trace_lit")


def rgeo_trace_host(metric: int, scene: int, camera: rgeo_camera, width: int, height: int, h: float,
                    max_steps: int, integrator: int, shading: int, flags: int, out: rgeo_outputs, stream=None):
    _check(library().rgeo_trace_host(metric, scene, ctypes.byref(camera), width, height, h, max_steps,
                                     integrator, shading, flags, ctypes.byref(out), _stream_handle(stream)),
           "rgeo_trace_host")


def rgeo_trace_noalloc(center: int, amplitude: int, sigma: int, n_bumps: int, cutoff: float, spheres: int,
                       n_spheres: int, albedo: int, camera: rgeo_camera, width: int, height: int, h: float,
                       max_steps: int, integrator: int, shading: int, out: rgeo_outputs, stream=None):
    """Allocation-free trace: every array argument is a device pointer the caller owns
    (isotropic spreads, spheres only); see include/rgeo.h."""
    _check(library().rgeo_trace_noalloc(center, amplitude, sigma, n_bumps, cutoff, spheres, n_spheres, albedo,
                                        ctypes.byref(camera), width, height, h, max_steps, integrator, shading,
                                        ctypes.byref(out), _stream_handle(stream)), "rgeo_trace_noalloc")


def rgeo_batch_create(instances) -> int:
    arr = (rgeo_instance * len(instances))(*instances)
    out = ctypes.c_void_p()
    _check(library().rgeo_batch_create(len(instances), arr, ctypes.byref(out)), "rgeo_batch_create")
    return out.value


def rgeo_batch_launch(batch: int, stream=None):
    _check(library().rgeo_batch_launch(batch, _stream_handle(stream)), "rgeo_batch_launch")


def rgeo_batch_destroy(batch: int):
    library().rgeo_batch_destroy(batch)


def rgeo_metric_set_motion(metric: int, amplitude, frequency, phase):
    import numpy as np
    a = np.ascontiguousarray(amplitude, np.float32).reshape(-1)
    f = np.ascontiguousarray(frequency, np.float32).reshape(-1)
    p = np.ascontiguousarray(phase, np.float32).reshape(-1)
    _check(library().rgeo_metric_set_motion(metric, _fptr(a), _fptr(f), _fptr(p)), "rgeo_metric_set_motion")


def rgeo_metric_set_time(metric: int, t: float, stream=None):
    _check(library().rgeo_metric_set_time(metric, t, _stream_handle(stream)), "rgeo_metric_set_time")


def rgeo_metric_advance(metric: int, dt: float, stream=None):
    _check(library().rgeo_metric_advance(metric, dt, _stream_handle(stream)), "rgeo_metric_advance")


def trace_surrogate(work: scenes.Workload, expmap: "Expmap", tau: float, box: float = 4.0, s_max: float = 0.5,
                    k_min: int = 20, cool_check: int = 16, max_rounds: int = 0, accel_bound: float = 0.0,
                    metric: "Metric" = None, scene: "Scene" = None, out=None, stream=None, flags: int = 0):
    """Trace a workload with surrogate jumps (RK4 only; returns when the image is done).
    Returns (outputs, stats dict)."""
    metric = metric or Metric(work.metric)
    scene = scene or Scene(work.scene)
    if out is None:
        out = alloc_outputs(work.n_pixels, drift=bool(flags & RGEO_FLAG_ENERGY_DIAG))
    sur = rgeo_surrogate(expmap.handle, box, s_max, tau, k_min, cool_check, max_rounds, accel_bound)
    st = rgeo_surrogate_stats()
    _check(library().rgeo_trace_surrogate(metric.handle, scene.handle, ctypes.byref(camera_struct(work.camera)),
                                          work.width, work.height, work.h, work.max_steps, work.shading, flags,
                                          ctypes.byref(sur), ctypes.byref(outputs_struct(out)), ctypes.byref(st),
                                          _stream_handle(stream)), "rgeo_trace_surrogate")
    out["_handles"] = (metric, scene)
    return out, dict(accepted=st.jumps_accepted, rejected=st.jumps_rejected, rounds=st.rounds)


def rgeo_gemm_bf16(A, B, M, N, K, splits, bias, mode, C, ldc, ct, ldt, stream=None):
    """Pointers are device addresses (ints) or None."""
    _check(library().rgeo_gemm_bf16(A, B, M, N, K, splits, bias, mode, C, ldc, ct, ldt, _stream_handle(stream)),
           "rgeo_gemm_bf16")


def rgeo_expmap_param_count() -> int:
    return library().rgeo_expmap_param_count()


class Expmap:
    """The learned exponential map (device weights, Adam state and scratch)."""

    IN, OUT, WIDTH = 7, 7, 256

    def __init__(self, max_batch: int = 8192, seed: int = 1):
        out = ctypes.c_void_p()
        _check(library().rgeo_expmap_create(max_batch, seed, ctypes.byref(out)), "rgeo_expmap_create")
        self.handle, self.max_batch = out.value, max_batch

    def close(self):
        if getattr(self, "handle", None):
            library().rgeo_expmap_destroy(self.handle)
            self.handle = None

    __del__ = close

    @staticmethod
    def generate(metric: "Metric", n: int, seed: int, box: float = 4.0, s_max: float = 0.5, h: float = 0.005,
                 accel_bound: float = 0.0, stream=None):
        """(inputs [n, 7], targets [n, 6]) device tensors of integrator-generated segments
        (far-field segments with targets divided by accel_bound when it is > 0)."""
        import torch
        X = torch.empty(n, 7, dtype=torch.float32, device="cuda")
        T = torch.empty(n, 6, dtype=torch.float32, device="cuda")
        _check(library().rgeo_expmap_generate(metric.handle, n, seed, box, s_max, h, accel_bound, X.data_ptr(),
                                              T.data_ptr(), _stream_handle(stream)), "rgeo_expmap_generate")
        return X, T

    def forward(self, X, out=None, stream=None):
        import torch
        Y = out if out is not None else torch.empty(X.shape[0], 7, dtype=torch.float32, device="cuda")
        _check(library().rgeo_expmap_forward(self.handle, X.data_ptr(), X.shape[0], Y.data_ptr(),
                                             _stream_handle(stream)), "rgeo_expmap_forward")
        return Y

    def gradients(self, X, T, stream=None):
        import torch
        G = torch.empty(rgeo_expmap_param_count(), dtype=torch.float32, device="cuda")
        L = torch.empty(1, dtype=torch.float32, device="cuda")
        _check(library().rgeo_expmap_gradients(self.handle, X.data_ptr(), T.data_ptr(), X.shape[0], G.data_ptr(),
                                               L.data_ptr(), _stream_handle(stream)), "rgeo_expmap_gradients")
        return G, L

    def train_step(self, X, T, lr: float, loss=None, stream=None):
        _check(library().rgeo_expmap_train_step(self.handle, X.data_ptr(), T.data_ptr(), X.shape[0], lr,
                                                loss.data_ptr() if loss is not None else None,
                                                _stream_handle(stream)), "rgeo_expmap_train_step")

    def train(self, metric: "Metric", n_segments: int, steps: int, batch: int = 8192, lr_max: float = 2e-3,
              lr_min: float = 1e-4, seed: int = 11, box: float = 4.0, s_max: float = 0.5, h: float = 0.005,
              accel_bound: float = 0.0, stream=None) -> float:
        """Generate segments and train in one call; returns the mean loss of the last 1 % of steps."""
        cfg = rgeo_train_cfg(n_segments, steps, batch, lr_max, lr_min, seed, box, s_max, h, accel_bound)
        loss = ctypes.c_float(0.0)
        _check(library().rgeo_expmap_train(self.handle, metric.handle, ctypes.byref(cfg), ctypes.byref(loss),
                                           _stream_handle(stream)), "rgeo_expmap_train")
        return loss.value

    def get_params(self):
        import numpy as np
        p = np.empty(rgeo_expmap_param_count(), np.float32)
        _check(library().rgeo_expmap_get_params(self.handle, _fptr(p), p.size), "rgeo_expmap_get_params")
        return p

    def set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, np.float32)
        _check(library().rgeo_expmap_set_params(self.handle, _fptr(p), p.size), "rgeo_expmap_set_params")

    def save(self, path: str):
        _check(library().rgeo_expmap_save(self.handle, os.fsencode(path)), "rgeo_expmap_save")

    def load(self, path: str):
        _check(library().rgeo_expmap_load(self.handle, os.fsencode(path)), "rgeo_expmap_load")


def rgeo_sync(stream=None):
    _check(library().rgeo_sync(_stream_handle(stream)), "rgeo_sync")


def rgeo_set_tuning(rays_per_thread: int = 0, batch_params: int = 0, wait_limit: int = 0, ctas_per_sm: int = 0,
                    tile_shape: int = 0, batch_order: int = 0, sum_lists: int = 0, refill: int = 0):
    t = rgeo_tuning()
    t.rays_per_thread, t.batch_params, t.wait_limit = rays_per_thread, batch_params, wait_limit
    t.ctas_per_sm, t.tile_shape, t.batch_order, t.sum_lists = ctas_per_sm, tile_shape, batch_order, sum_lists
    t.refill = refill
    _check(library().rgeo_set_tuning(ctypes.byref(t)), "rgeo_set_tuning")


def rgeo_get_tuning() -> dict:
    t = rgeo_tuning()
    _check(library().rgeo_get_tuning(ctypes.byref(t)), "rgeo_get_tuning")
    return {k: getattr(t, k) for k in TUNING_FIELDS}


def rgeo_ffma_probe(mode: int = 0):
    t, ms = ctypes.c_float(), ctypes.c_float()
    _check(library().rgeo_ffma_probe(mode, ctypes.byref(t), ctypes.byref(ms)), "rgeo_ffma_probe")
    return t.value, ms.value


# ------------------------------------------------------------------ conveniences
def metric_desc(m: scenes.Metric):
    """C descriptor for a ``scenes.Metric``; returns (desc, keep-alive arrays)."""
    import numpy as np
    c = np.ascontiguousarray(m.center, np.float32).reshape(-1)
    a = np.ascontiguousarray(m.amplitude, np.float32).reshape(-1)
    s = np.ascontiguousarray(m.sigma, np.float32).reshape(-1)
    d = rgeo_metric_desc()
    d.kind = m.kind
    d.n_bumps = a.shape[0] if m.kind != RGEO_METRIC_DIFFEO_TWIST else 0
    d.center, d.amplitude, d.sigma = (_fptr(c), _fptr(a), _fptr(s)) if d.n_bumps else (None, None, None)
    keep = [c, a, s]
    if m.kind == RGEO_METRIC_DIFFEO_LOCAL:
        dv = np.ascontiguousarray(m.direction, np.float32).reshape(-1)
        keep.append(dv)
        d.direction = _fptr(dv)
        if getattr(m, "field", None) is not None:
            fb = np.ascontiguousarray(m.field, np.float32).reshape(-1)
            keep.append(fb)
            d.field = _fptr(fb)
    d.affine_b = (ctypes.c_float * 3)(*m.affine_b)
    d.quad_A = (ctypes.c_float * 9)(*m.quad_A)
    d.cutoff_sigmas = m.cutoff
    d.twist_rate = m.twist_rate
    d.cull_grid = getattr(m, "cull_grid", 0)
    return d, tuple(keep)


def camera_struct(cam: scenes.Camera) -> rgeo_camera:
    return rgeo_camera((ctypes.c_float * 3)(*cam.pos), (ctypes.c_float * 3)(*cam.forward),
                       (ctypes.c_float * 3)(*cam.up), cam.vfov_deg)


class Metric:
    """Owning handle of a device metric."""

    def __init__(self, m: scenes.Metric):
        desc, self._keep = metric_desc(m)
        self.handle = rgeo_metric_create(desc)

    def close(self):
        if getattr(self, "handle", None):
            rgeo_metric_destroy(self.handle)
            self.handle = None

    __del__ = close


class Scene:
    """Owning handle of a device scene (spheres + triangle BVH + safe-distance grid)."""

    def __init__(self, s: scenes.Scene):
        self.handle = rgeo_scene_create(s.spheres, s.verts, s.tris, s.albedo)
        if getattr(s, "fog", 0.0) > 0.0:
            self.set_fog(s.fog, s.fog_rgb)

    def set_fog(self, density: float, rgb=(0.0, 0.0, 0.0)):
        import numpy as np
        c = np.ascontiguousarray(rgb, np.float32)
        _check(library().rgeo_scene_set_fog(self.handle, density, _fptr(c)), "rgeo_scene_set_fog")

    def close(self):
        if getattr(self, "handle", None):
            rgeo_scene_destroy(self.handle)
            self.handle = None

    __del__ = close


def alloc_outputs(n_pixels: int, device="cuda", drift: bool = False, pin: bool = False, count: bool = False):
    """Output tensors: id, hit (planar [3, N]), steps, rgba ([N, 4]), drift (optional) and
    bump_evals (optional device work counter, zeroed)."""
    import torch
    kw = dict(device=device)
    if pin:
        kw = dict(device="cpu", pin_memory=True)
    out = dict(id=torch.empty(n_pixels, dtype=torch.int32, **kw),
               hit=torch.empty(3, n_pixels, dtype=torch.float32, **kw),
               steps=torch.empty(n_pixels, dtype=torch.int32, **kw),
               rgba=torch.empty(n_pixels, 4, dtype=torch.uint8, **kw))
    out["drift"] = torch.empty(n_pixels, dtype=torch.float64, **kw) if drift else None
    out["bump_evals"] = torch.zeros(1, dtype=torch.int64, device=device) if count and not pin else None
    out["bump_slots"] = torch.zeros(1, dtype=torch.int64, device=device) if count and not pin else None
    return out


def outputs_struct(out) -> rgeo_outputs:
    def ptr(k):
        t = out.get(k)
        return t.data_ptr() if t is not None else None
    return rgeo_outputs(out["id"].data_ptr(), out["hit"].data_ptr(), out["steps"].data_ptr(),
                        out["rgba"].data_ptr(), ptr("drift"), ptr("bump_evals"), ptr("bump_slots"))


def instance(work: scenes.Workload, metric: Metric, scene: Scene, out, flags: int = 0) -> rgeo_instance:
    """One batch instance: a workload's camera and stepping with its own handles and outputs."""
    return rgeo_instance(metric.handle, scene.handle, camera_struct(work.camera), work.width, work.height,
                         work.h, work.max_steps, work.integrator, work.shading, flags, outputs_struct(out))


class Batch:
    """Owning handle of a batch of instances traced in one launch."""

    def __init__(self, instances):
        self._instances = list(instances)
        self.handle = rgeo_batch_create(self._instances)

    def launch(self, stream=None):
        rgeo_batch_launch(self.handle, stream)

    def close(self):
        if getattr(self, "handle", None):
            rgeo_batch_destroy(self.handle)
            self.handle = None

    __del__ = close


def trace(work: scenes.Workload, metric: Metric = None, scene: Scene = None, out=None, stream=None,
          flags: int = 0, tiles=None):
    """Trace a workload on the current CUDA device into torch tensors (asynchronous on ``stream``).
    ``tiles`` = (begin, end, step): only those of the frame's queue tiles (rgeo_trace_tiles)."""
    metric = metric or Metric(work.metric)
    scene = scene or Scene(work.scene)
    if out is None:
        out = alloc_outputs(work.n_pixels, drift=bool(flags & RGEO_FLAG_ENERGY_DIAG))
    if tiles is None:
        rgeo_trace(metric.handle, scene.handle, camera_struct(work.camera), work.width, work.height, work.h,
                   work.max_steps, work.integrator, work.shading, flags, outputs_struct(out), stream)
    else:
        rgeo_trace_tiles(metric.handle, scene.handle, camera_struct(work.camera), work.width, work.height, work.h,
                         work.max_steps, work.integrator, work.shading, flags, int(tiles[0]), int(tiles[1]),
                         int(tiles[2]) if len(tiles) > 2 else 1, outputs_struct(out), stream)
    out["_handles"] = (metric, scene)
    return out


def light_struct(light: scenes.Light) -> rgeo_light:
    return rgeo_light((ctypes.c_float * 3)(*light.pos), light.h, light.max_steps, light.iters, light.tol,
                      light.delta, light.schedule, (ctypes.c_int32 * 3)())


def trace_lit(work: scenes.Workload, light: scenes.Light, metric: Metric = None, scene: Scene = None, out=None,
              stream=None):
    """Trace a workload with Riemannian illumination of its hits by a point light (torch tensors,
    asynchronous on ``stream``); out["lit"] holds 1 for lit hits."""
    import torch
    metric = metric or Metric(work.metric)
    scene = scene or Scene(work.scene)
    if out is None:
        out = alloc_outputs(work.n_pixels)
    if out.get("lit") is None:
        out["lit"] = torch.zeros(work.n_pixels, dtype=torch.int32, device=out["id"].device)
    rgeo_trace_lit(metric.handle, scene.handle, camera_struct(work.camera), work.width, work.height, work.h,
                   work.max_steps, work.integrator, light_struct(light), outputs_struct(out),
                   out["lit"].data_ptr(), stream)
    out["_handles"] = (metric, scene)
    return out
