"""FP64 CPU oracle for the geodesic ray tracer (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it, and it imports nothing of the product
path: the two sides share only the seeded input arrays of
``paper_2005_05386_gb300.scenes``.

The arithmetic lives in ``rgeo_oracle.c`` (plain C, FP64, no blocking or
fusion); this module builds it with gcc and wraps it with ctypes.

Parity status of each function (what pins it, see tests/test_oracle_pins.py):
  field              closed-form values of Eq. 6.1, finite differences of f and grad f
  christoffel        finite-difference Christoffel symbols of Eq. 3.4 (graph and twist)
  accel              contraction of the pinned symbols (Eq. 3.3); straight lines for affine f
  twist maps         closed-form rotation values; finite differences of Phi and J
  step / integrate   straight lines (f = 0, affine f); twist geodesics = Phi^-1 of lines;
                     (x - c) x x' conservation for a radial bump; g(v, v) conservation;
                     convergence orders 4 (RK4) and 1 (Euler) against dopri5
  dopri5             closed-form twist geodesics to 1e-9
  scene_hit          analytic ray-sphere hits, BVH vs brute force, closed-mesh watertightness
  trace              straight-line scenes against analytic hits; curved frames by step
                     refinement (fourth-order convergence of the hit points untruncated,
                     first order with a constant below 1e-7 truncated); the paper prints
                     no worked image or number
  illuminate         light geodesics by shooting: the segment q -> L in flat space, the
                     Riemannian cosine under affine f (Sherman-Morrison), preimages of lines
                     under the twist, the axis of a radial bump, re-integration to the light;
                     shadows by analytic occluders (tests/test_oracle_illum.py)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rgeo_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# Tests that plant a mistake in a copy of the oracle point this at the copy.
_LIB_OVERRIDE = os.environ.get("RGEO_ORACLE_LIB")

GRAPH, TWIST, LOCAL = 0, 1, 2
RK4, EULER = 0, 1
LAMBERT, PSEUDO = 0, 1
MISS, BUDGET = -1, -2

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so results match across hosts)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        if _LIB_OVERRIDE:
            L = ctypes.CDLL(_LIB_OVERRIDE)
        else:
            build()
            L = ctypes.CDLL(_LIB)
        L.or_metric_create.restype = ctypes.c_void_p
        L.or_metric_create.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp,
                                       ctypes.c_double, ctypes.c_double]
        L.or_metric_destroy.argtypes = [ctypes.c_void_p]
        L.or_scene_create.restype = ctypes.c_void_p
        L.or_scene_create.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, ctypes.c_int]
        L.or_scene_destroy.argtypes = [ctypes.c_void_p]
        L.or_scene_set_fog.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp]
        L.or_field.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
        L.or_christoffel.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.or_accel.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
        L.or_metric_tensor.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.or_inner.restype = ctypes.c_double
        L.or_inner.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
        L.or_step.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, _dp, _dp]
        L.or_integrate.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                   _dp, _dp, _dp, _dp]
        L.or_dopri5.restype = ctypes.c_int
        L.or_dopri5.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, _dp, _dp]
        for name in ("or_twist_phi", "or_twist_phi_inv", "or_twist_jacobian", "or_twist_hessian"):
            getattr(L, name).argtypes = [ctypes.c_double, _dp, _dp]
        L.or_inverse_by_minors.argtypes = [_dp, _dp]
        L.or_metric_set_local.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.or_local_map.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp, _dp, _dp]
        L.or_local_compose.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
        L.or_local_jinv.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.or_hit_sphere.restype = ctypes.c_int
        L.or_hit_sphere.argtypes = [_dp, _dp, ctypes.c_double, _dp, _dp]
        L.or_hit_triangle.restype = ctypes.c_int
        L.or_hit_triangle.argtypes = [_dp, _dp, ctypes.c_double, _dp, _dp]
        L.or_scene_hit.restype = ctypes.c_int
        L.or_scene_hit.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_double, _dp, _ip]
        L.or_camera_dir.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, _dp]
        L.or_trace.restype = ctypes.c_int
        L.or_trace.argtypes = [ctypes.c_void_p, ctypes.c_void_p, _dp, _dp, _dp, ctypes.c_double,
                               ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, _i64p, ctypes.c_int64, _ip, _dp, _ip,
                               _u8p, _dp, _dp, ctypes.c_int, ctypes.c_int]
        L.or_trace_dirs.restype = ctypes.c_int
        L.or_trace_dirs.argtypes = [ctypes.c_void_p, ctypes.c_void_p, _dp, _dp, ctypes.c_int64, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, _ip, _dp, _ip, _u8p, ctypes.c_int]
        L.or_trace_lit.restype = ctypes.c_int
        L.or_trace_lit.argtypes = [ctypes.c_void_p, ctypes.c_void_p, _dp, _dp, _dp, ctypes.c_double,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                   _dp, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_double, _i64p, ctypes.c_int64, _ip, _dp, _ip, _u8p, _ip, ctypes.c_int]
        L.or_illuminate.restype = ctypes.c_int
        L.or_illuminate.argtypes = [ctypes.c_void_p, ctypes.c_void_p, _dp, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                    _dp, _dp, _u8p, _dp, _ip, _dp]
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


class Metric:
    """FP64 copy of a metric description: graph of summed bumps, twist, or a composition of
    local diffeomorphisms p + f_i(p) (v_i + B_i (p - c_i)) (kind LOCAL; direction [K,3], field
    [K,3,3] or None)."""

    def __init__(self, kind=GRAPH, center=None, amplitude=None, sigma=None, affine_b=(0, 0, 0),
                 quad_A=(0,) * 9, cutoff=4.0, twist_rate=1.0, direction=None, field=None):
        center = np.zeros((0, 3)) if center is None else np.asarray(center, np.float64).reshape(-1, 3)
        amplitude = np.zeros((0,)) if amplitude is None else np.asarray(amplitude, np.float64).reshape(-1)
        sigma = np.zeros((0, 3)) if sigma is None else np.asarray(sigma, np.float64).reshape(-1, 3)
        K = amplitude.shape[0]
        self._keep = [_d(center), _d(amplitude), _d(sigma), _d(affine_b), _d(quad_A)]
        (_, pc), (_, pa), (_, ps), (_, pb), (_, pA) = self._keep
        self.kind = kind
        self.K = K
        self.ptr = lib().or_metric_create(kind, K, pc, pa, ps, pb, pA, float(cutoff), float(twist_rate))
        if kind == LOCAL:
            dv = _d(np.zeros((K, 3)) if direction is None else np.asarray(direction, np.float64).reshape(-1, 3))
            fb = _d(np.asarray(field, np.float64).reshape(-1, 9)) if field is not None else (None, None)
            self._keep += [dv, fb]
            lib().or_metric_set_local(self.ptr, dv[1], fb[1])

    @classmethod
    def from_desc(cls, m):
        """From a ``scenes.Metric`` (float32 arrays converted exactly to float64)."""
        return cls(m.kind, m.center, m.amplitude, m.sigma, m.affine_b, m.quad_A, m.cutoff,
                   m.twist_rate, getattr(m, "direction", None), getattr(m, "field", None))

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.or_metric_destroy(self.ptr)
            self.ptr = None


class Scene:
    def __init__(self, spheres, verts=None, tris=None, albedo=None, use_bvh=True, fog=0.0, fog_rgb=(0, 0, 0)):
        spheres = np.asarray(spheres, np.float64).reshape(-1, 4)
        S = spheres.shape[0]
        if verts is None or tris is None or len(tris) == 0:
            tri9 = np.zeros((0, 9))
        else:
            v = np.asarray(verts, np.float64).reshape(-1, 3)
            tri9 = v[np.asarray(tris, np.int64).reshape(-1, 3)].reshape(-1, 9)
        if albedo is None:
            albedo = np.full((S + 1, 3), 0.8)
        self.S, self.T = S, tri9.shape[0]
        self.tri9 = tri9
        self._keep = [_d(spheres), _d(tri9), _d(np.asarray(albedo, np.float64).reshape(-1, 3))]
        (_, ps), (_, pt), (_, pa) = self._keep
        self.ptr = lib().or_scene_create(S, ps, self.T, pt, pa, int(bool(use_bvh)))
        if fog > 0.0:
            rgb = _d(fog_rgb)
            self._keep.append(rgb)
            lib().or_scene_set_fog(self.ptr, float(fog), rgb[1])

    @classmethod
    def from_desc(cls, s, use_bvh=True):
        return cls(s.spheres, s.verts, s.tris, s.albedo, use_bvh, getattr(s, "fog", 0.0),
                   getattr(s, "fog_rgb", (0.0, 0.0, 0.0)))

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.or_scene_destroy(self.ptr)
            self.ptr = None


def field(m: Metric, x):
    x, px = _d(x)
    f = np.zeros(1); g = np.zeros(3); H = np.zeros(9)
    lib().or_field(m.ptr, px, f.ctypes.data_as(_dp), g.ctypes.data_as(_dp), H.ctypes.data_as(_dp))
    return f[0], g, H.reshape(3, 3)


def christoffel(m: Metric, x):
    """Gamma[m, i, j] at x (Eq. 5.3 for graphs, Theorem 5.1 for the twist)."""
    x, px = _d(x)
    G = np.zeros(27)
    lib().or_christoffel(m.ptr, px, G.ctypes.data_as(_dp))
    return G.reshape(3, 3, 3)


def accel(m: Metric, x, v):
    x, px = _d(x); v, pv = _d(v)
    a = np.zeros(3)
    lib().or_accel(m.ptr, px, pv, a.ctypes.data_as(_dp))
    return a


def metric_tensor(m: Metric, x):
    x, px = _d(x)
    g = np.zeros(9)
    lib().or_metric_tensor(m.ptr, px, g.ctypes.data_as(_dp))
    return g.reshape(3, 3)


def inner(m: Metric, p, u, v):
    p, pp = _d(p); u, pu = _d(u); v, pv = _d(v)
    return lib().or_inner(m.ptr, pp, pu, pv)


def integrate(m: Metric, integrator: int, h: float, n: int, p, v):
    """Polygon of n fixed steps: returns (xs [n+1,3], vs [n+1,3])."""
    p, pp = _d(p); v, pv = _d(v)
    xs = np.zeros((n + 1, 3)); vs = np.zeros((n + 1, 3))
    lib().or_integrate(m.ptr, integrator, float(h), int(n), pp, pv, xs.ctypes.data_as(_dp),
                       vs.ctypes.data_as(_dp))
    return xs, vs


def dopri5(m: Metric, p, v, T: float, rtol=1e-12, atol=1e-12):
    p, pp = _d(p); v, pv = _d(v)
    x = np.zeros(3); w = np.zeros(3)
    n = lib().or_dopri5(m.ptr, pp, pv, float(T), float(rtol), float(atol), x.ctypes.data_as(_dp),
                        w.ctypes.data_as(_dp))
    if n < 0:
        raise RuntimeError("dopri5 step size collapsed")
    return x, w


def _twist_call(name, k, p, n_out):
    p, pp = _d(p)
    out = np.zeros(n_out)
    getattr(lib(), name)(float(k), pp, out.ctypes.data_as(_dp))
    return out


def twist_phi(k, p):
    return _twist_call("or_twist_phi", k, p, 3)


def twist_phi_inv(k, p):
    return _twist_call("or_twist_phi_inv", k, p, 3)


def twist_jacobian(k, p):
    return _twist_call("or_twist_jacobian", k, p, 9).reshape(3, 3)


def twist_hessian(k, p):
    return _twist_call("or_twist_hessian", k, p, 27).reshape(3, 3, 3)


def local_map(m: Metric, i: int, p):
    """(Phi_i(p), J [3,3], H [3,3,3] with H[s, i, j] = d_i d_j (Phi_i)_s) of one local map."""
    p, pp = _d(p)
    out, J, H = np.zeros(3), np.zeros(9), np.zeros(27)
    lib().or_local_map(m.ptr, int(i), pp, out.ctypes.data_as(_dp), J.ctypes.data_as(_dp), H.ctypes.data_as(_dp))
    return out, J.reshape(3, 3), H.reshape(3, 3, 3)


def local_compose(m: Metric, p):
    """(Phi(p), J, H) of the composition Phi = Phi_1 o ... o Phi_K."""
    p, pp = _d(p)
    out, J, H = np.zeros(3), np.zeros(9), np.zeros(27)
    lib().or_local_compose(m.ptr, pp, out.ctypes.data_as(_dp), J.ctypes.data_as(_dp), H.ctypes.data_as(_dp))
    return out, J.reshape(3, 3), H.reshape(3, 3, 3)


def local_jinv(m: Metric, p):
    """J^-1 of the composition as the product of the maps' inverses in reverse order."""
    p, pp = _d(p)
    out = np.zeros(9)
    lib().or_local_jinv(m.ptr, pp, out.ctypes.data_as(_dp))
    return out.reshape(3, 3)


def inverse_by_minors(J):
    J, pJ = _d(J)
    out = np.zeros(9)
    lib().or_inverse_by_minors(pJ, out.ctypes.data_as(_dp))
    return out.reshape(3, 3)


def hit_sphere(O, D, smax, sphere):
    O, pO = _d(O); D, pD = _d(D); sp, ps = _d(sphere)
    s = np.zeros(1)
    ok = lib().or_hit_sphere(pO, pD, float(smax), ps, s.ctypes.data_as(_dp))
    return (s[0] if ok else None)


def hit_triangle(O, D, smax, tri9):
    O, pO = _d(O); D, pD = _d(D); t, pt = _d(tri9)
    s = np.zeros(1)
    ok = lib().or_hit_triangle(pO, pD, float(smax), pt, s.ctypes.data_as(_dp))
    return (s[0] if ok else None)


def scene_hit(sc: Scene, O, D, smax):
    """(s, id) of the earliest hit of O + s D, s in [0, smax), or None."""
    O, pO = _d(O); D, pD = _d(D)
    s = np.zeros(1); i = np.zeros(1, np.int32)
    ok = lib().or_scene_hit(sc.ptr, pO, pD, float(smax), s.ctypes.data_as(_dp), i.ctypes.data_as(_ip))
    return (s[0], int(i[0])) if ok else None


class _Cam(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_double * 3), ("fwd", ctypes.c_double * 3),
                ("up", ctypes.c_double * 3), ("vfov", ctypes.c_double)]


def camera_dir(cam, W, H, i, j):
    c = _Cam((ctypes.c_double * 3)(*cam.pos), (ctypes.c_double * 3)(*cam.forward),
             (ctypes.c_double * 3)(*cam.up), float(cam.vfov_deg))
    d = np.zeros(3)
    lib().or_camera_dir(ctypes.byref(c), W, H, i, j, d.ctypes.data_as(_dp))
    return d


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def trace(work, pixels=None, nthreads=None, metric: Metric = None, scene: Scene = None,
          no_skip: bool = False):
    """Trace ``work`` (a ``scenes.Workload``) on the listed pixels (all when None).

    Returns a dict of numpy arrays: id, hit [n,3], steps, rgba [n,4], drift, xend [n,3].
    """
    m = metric or Metric.from_desc(work.metric)
    sc = scene or Scene.from_desc(work.scene)
    if pixels is None:
        pixels = np.arange(work.width * work.height, dtype=np.int64)
    pixels = np.ascontiguousarray(pixels, dtype=np.int64)
    n = pixels.shape[0]
    out = dict(id=np.zeros(n, np.int32), hit=np.zeros((n, 3)), steps=np.zeros(n, np.int32),
               rgba=np.zeros((n, 4), np.uint8), drift=np.zeros(n), xend=np.zeros((n, 3)))
    cam = work.camera
    _, pp = pos = _d(cam.pos)
    _, pf = fwd = _d(cam.forward)
    _, pu = up = _d(cam.up)
    nt = nthreads or default_threads()
    lib().or_trace(m.ptr, sc.ptr, pp, pf, pu, float(cam.vfov_deg), work.width, work.height,
                   float(work.h), int(work.max_steps), int(work.integrator), int(work.shading),
                   pixels.ctypes.data_as(_i64p), n, out["id"].ctypes.data_as(_ip),
                   out["hit"].ctypes.data_as(_dp), out["steps"].ctypes.data_as(_ip),
                   out["rgba"].ctypes.data_as(_u8p), out["drift"].ctypes.data_as(_dp),
                   out["xend"].ctypes.data_as(_dp), int(bool(no_skip)), int(nt))
    del pos, fwd, up
    out["pixels"] = pixels
    out["threads"] = nt
    return out


def trace_dirs(work, dirs, nthreads=None, metric: Metric = None, scene: Scene = None):
    """Trace rays from ``work``'s camera position with the given Euclidean initial directions
    ``dirs`` [n, 3] (normalised by the oracle) instead of the pixels' own: the same marching,
    segment tests and shading as ``trace``.  Returns id, hit [n,3], steps, rgba [n,4]."""
    m = metric or Metric.from_desc(work.metric)
    sc = scene or Scene.from_desc(work.scene)
    dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    n = dirs.shape[0]
    out = dict(id=np.zeros(n, np.int32), hit=np.zeros((n, 3)), steps=np.zeros(n, np.int32),
               rgba=np.zeros((n, 4), np.uint8))
    _, pp = pos = _d(work.camera.pos)
    lib().or_trace_dirs(m.ptr, sc.ptr, pp, dirs.ctypes.data_as(_dp), n, float(work.h), int(work.max_steps),
                        int(work.integrator), int(work.shading), out["id"].ctypes.data_as(_ip),
                        out["hit"].ctypes.data_as(_dp), out["steps"].ctypes.data_as(_ip),
                        out["rgba"].ctypes.data_as(_u8p), int(nthreads or default_threads()))
    del pos
    return out


def conditioning(work, pixels, eps=2.0 ** -23, nthreads=None, metric: Metric = None, scene: Scene = None):
    """How far each listed pixel's answer moves when its initial direction turns by eps radians
    (default one float32 ulp at 1): the ray is re-traced in FP64 with the direction tilted by
    eps along +-e1 and +-e2 (an orthonormal frame across it).  Returns (same_object [n] bool,
    largest hit-point move [n]) over the four tilts; a MISS or BUDGET answer counts as an
    object."""
    m = metric or Metric.from_desc(work.metric)
    sc = scene or Scene.from_desc(work.scene)
    pixels = np.asarray(pixels, np.int64)
    base = trace(work, pixels, nthreads=nthreads, metric=m, scene=sc)
    dirs = []
    for p in pixels:
        d = camera_dir(work.camera, work.width, work.height, int(p % work.width), int(p // work.width))
        a = np.eye(3)[int(np.argmin(np.abs(d)))]
        e1 = np.cross(d, a)
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(d, e1)
        dirs += [d + eps * e1, d - eps * e1, d + eps * e2, d - eps * e2]
    t = trace_dirs(work, np.array(dirs), nthreads=nthreads, metric=m, scene=sc)
    S = sc.S
    obj = lambda i: np.where(np.asarray(i) >= S, S, np.asarray(i))  # noqa: E731
    n = len(pixels)
    tid = obj(t["id"]).reshape(n, 4)
    same = (tid == obj(base["id"])[:, None]).all(axis=1)
    move = np.abs(t["hit"].reshape(n, 4, 3) - base["hit"][:, None, :]).max(axis=(1, 2))
    return same, move


def trace_lit(work, light, pixels=None, nthreads=None, metric: Metric = None, scene: Scene = None):
    """Trace ``work`` with Riemannian illumination of every hit by the point light ``light``
    (a ``scenes.Light``): the hits are shaded by the light geodesics (Section 4).

    Returns a dict of numpy arrays: id, hit [n,3], steps, rgba [n,4], lit."""
    m = metric or Metric.from_desc(work.metric)
    sc = scene or Scene.from_desc(work.scene)
    if pixels is None:
        pixels = np.arange(work.width * work.height, dtype=np.int64)
    pixels = np.ascontiguousarray(pixels, dtype=np.int64)
    n = pixels.shape[0]
    out = dict(id=np.zeros(n, np.int32), hit=np.zeros((n, 3)), steps=np.zeros(n, np.int32),
               rgba=np.zeros((n, 4), np.uint8), lit=np.zeros(n, np.int32))
    cam = work.camera
    keep = [_d(cam.pos), _d(cam.forward), _d(cam.up), _d(light.pos)]
    (_, pp), (_, pf), (_, pu), (_, pl) = keep
    nt = nthreads or default_threads()
    lib().or_trace_lit(m.ptr, sc.ptr, pp, pf, pu, float(cam.vfov_deg), work.width, work.height, float(work.h),
                       int(work.max_steps), int(work.integrator), pl, float(light.h), int(light.max_steps),
                       int(light.iters), float(light.tol), float(light.delta), pixels.ctypes.data_as(_i64p), n,
                       out["id"].ctypes.data_as(_ip), out["hit"].ctypes.data_as(_dp),
                       out["steps"].ctypes.data_as(_ip), out["rgba"].ctypes.data_as(_u8p),
                       out["lit"].ctypes.data_as(_ip), int(nt))
    del keep
    out["pixels"] = pixels
    out["threads"] = nt
    return out


def illuminate(m: Metric, sc: Scene, light, integrator: int, obj_id: int, P, D):
    """Illumination of one hit (point P on object obj_id, reached along direction D).

    Returns (lit, rgba [4], Riemannian cosine, Gauss-Newton steps, initial g-unit tangent [3])."""
    keep = [_d(light.pos), _d(P), _d(D)]
    (_, pl), (_, pp), (_, pd) = keep
    rgba = np.zeros(4, np.uint8)
    cosg = np.zeros(1)
    it = np.zeros(1, np.int32)
    u = np.zeros(3)
    lit = lib().or_illuminate(m.ptr, sc.ptr, pl, float(light.h), int(light.max_steps), int(light.iters),
                              float(light.tol), float(light.delta), int(integrator), int(obj_id), pp, pd,
                              rgba.ctypes.data_as(_u8p), cosg.ctypes.data_as(_dp), it.ctypes.data_as(_ip),
                              u.ctypes.data_as(_dp))
    del keep
    return bool(lit), rgba, float(cosg[0]), int(it[0]), u
