"""Seeded synthetic workloads for the geodesic ray tracer.

This module only draws numbers: bump tables, sphere lists, a displaced
lat-long sphere mesh, cameras and pixel samples.  It holds none of the
method's arithmetic (no metric, no Christoffel symbols, no integration, no
intersection), so both the CUDA path and the FP64 oracle consume the same
generated arrays without sharing any code of the method.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the state advances by the
golden-ratio increment 0x9E3779B97F4A7C15 and each output is the state passed
through the two xor-shift-multiply rounds with multipliers
0xBF58476D1CE4E5B9 and 0x94D049BB133111EB.  A uniform double in [0, 1) is
(u >> 11) * 2**-53.  Each component draws from its own stream, seeded with
``seed * 16 + {1: bumps, 2: spheres, 3: mesh, 4: animation, 5: pixel sample}``.

Workload shapes follow the paper's experiments: Gaussian bumps of Eq. 6.1
summed as in Section 6 ("Summing functions"), observer and view field of
Section 4 ("Riemannian shading"), twist map of Section 5.2.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MASK64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB

STREAM_BUMPS, STREAM_SPHERES, STREAM_MESH, STREAM_ANIM, STREAM_PIXELS = 1, 2, 3, 4, 5

METRIC_GRAPH_BUMPS = 0
METRIC_DIFFEO_TWIST = 1
METRIC_DIFFEO_LOCAL = 2
INTEGRATOR_RK4 = 0
INTEGRATOR_EULER = 1
SHADING_LAMBERT = 0
SHADING_PSEUDO = 1


class SplitMix64:
    """Sequential SplitMix64 stream (Steele, Lea and Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + _GOLDEN) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * _M1) & MASK64
        z = ((z ^ (z >> 27)) * _M2) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        u = (self.next_u64() >> 11) * (2.0 ** -53)
        return lo + (hi - lo) * u


def splitmix64_hash(x: np.ndarray) -> np.ndarray:
    """One SplitMix64 output for each state in ``x`` (uint64, vectorised)."""
    z = (np.asarray(x, dtype=np.uint64) + np.uint64(_GOLDEN))
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
    return z ^ (z >> np.uint64(31))


def sub_seed(seed: int, stream: int) -> int:
    return (seed * 16 + stream) & MASK64


def pixel_sample(n_pixels: int, seed: int, fraction: float) -> np.ndarray:
    """Seeded pixel sample: idx is kept iff hash(idx xor seed5) < fraction * 2**64."""
    idx = np.arange(n_pixels, dtype=np.uint64)
    h = splitmix64_hash(idx ^ np.uint64(sub_seed(seed, STREAM_PIXELS)))
    thresh = np.uint64(min(int(fraction * 2.0 ** 64), MASK64))
    return np.nonzero(h < thresh)[0].astype(np.int64)


@dataclasses.dataclass
class Camera:
    pos: tuple = (0.0, 0.0, -6.0)
    forward: tuple = (0.0, 0.0, 1.0)
    up: tuple = (0.0, 1.0, 0.0)
    vfov_deg: float = 60.0


@dataclasses.dataclass
class Light:
    """A point light for Riemannian illumination and the parameters of the geodesic shooting
    toward it: step h and step budget of each light geodesic, at most ``iters`` Gauss-Newton
    steps to a miss of at most ``tol`` scene units, forward-difference step ``delta``;
    ``schedule`` 1 has each lane march on its own instead of the warp's lockstep marches."""
    pos: tuple = (1.0, 6.0, -3.0)
    h: float = 0.005
    max_steps: int = 4000
    iters: int = 24
    tol: float = 1e-4
    delta: float = 1e-3
    schedule: int = 0


@dataclasses.dataclass
class Metric:
    """Metric description: graph of a sum of Gaussian bumps, or the twist diffeomorphism.

    For the graph metric f(x) = b.x + 1/2 x^T A x + sum_k a_k exp(-sum_i (x_i - c_ki)^2 / (2 sigma_ki^2)),
    each bump truncated at ||(x - c_k) / sigma_k|| < cutoff (no truncation when cutoff <= 0).
    """
    kind: int = METRIC_GRAPH_BUMPS
    center: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 3), np.float32))
    amplitude: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0,), np.float32))
    sigma: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 3), np.float32))
    affine_b: tuple = (0.0, 0.0, 0.0)
    quad_A: tuple = (0.0,) * 9
    cutoff: float = 4.0
    twist_rate: float = 1.0
    cull_grid: int = 0          # bump-support cull grid: 0 automatic, -1 none, G in [4, 128]
    direction: np.ndarray = None  # local maps: [K, 3] v_k of p + f_k(p) (v_k + B_k (p - c_k))
    field: np.ndarray = None      # local maps: [K, 3, 3] B_k, or None

    @property
    def n_bumps(self) -> int:
        return int(self.amplitude.shape[0])


@dataclasses.dataclass
class Scene:
    spheres: np.ndarray   # [S, 4] float32: cx, cy, cz, r
    verts: np.ndarray     # [V, 3] float32
    tris: np.ndarray      # [T, 3] int32
    albedo: np.ndarray    # [S + 1, 3] float32: one colour per sphere, then one for the mesh
    fog: float = 0.0      # fog density per unit of arc length (the grid figures use a little black fog)
    fog_rgb: tuple = (0.0, 0.0, 0.0)

    @property
    def n_spheres(self) -> int:
        return int(self.spheres.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


@dataclasses.dataclass
class Workload:
    name: str
    width: int
    height: int
    h: float
    max_steps: int
    metric: Metric
    scene: Scene
    camera: Camera
    integrator: int = INTEGRATOR_RK4
    shading: int = SHADING_LAMBERT
    seed: int = 0

    @property
    def n_pixels(self) -> int:
        return self.width * self.height


# --------------------------------------------------------------------------- bumps
def random_bumps(seed: int, n: int, box: float = 4.0, amp: float = 1.0,
                 sigma_lo: float = 0.2, sigma_hi: float = 1.0, isotropic: bool = True):
    """n bumps: centres U[-box, box]^3, amplitudes U[-amp, amp], spreads U[sigma_lo, sigma_hi]."""
    rng = SplitMix64(sub_seed(seed, STREAM_BUMPS))
    c = np.zeros((n, 3), np.float64)
    a = np.zeros((n,), np.float64)
    s = np.zeros((n, 3), np.float64)
    for k in range(n):
        c[k] = [rng.uniform(-box, box) for _ in range(3)]
        a[k] = rng.uniform(-amp, amp)
        if isotropic:
            s[k] = rng.uniform(sigma_lo, sigma_hi)
        else:
            s[k] = [rng.uniform(sigma_lo, sigma_hi) for _ in range(3)]
    return c.astype(np.float32), a.astype(np.float32), s.astype(np.float32)


# --------------------------------------------------------------------------- scene
def displaced_sphere_mesh(seed: int, n_lon: int, n_lat: int, centre=(0.0, 0.0, 2.0),
                          radius: float = 1.5, n_modes: int = 4, alpha_max: float = 0.08):
    """Closed lat-long sphere, radius R0 (1 + sum_m alpha_m sin(omega_m . n + psi_m)).

    One vertex per pole and n_lat - 1 rings of n_lon vertices give
    2 n_lon (n_lat - 1) triangles (n_lon = 100, n_lat = 51 -> 10,000).
    Returns (verts [V,3] f32, tris [T,3] i32, max radius).
    """
    rng = SplitMix64(sub_seed(seed, STREAM_MESH))
    alpha = [rng.uniform(0.0, alpha_max) for _ in range(n_modes)]
    omega = [[rng.uniform(-4.0, 4.0) for _ in range(3)] for _ in range(n_modes)]
    psi = [rng.uniform(0.0, 2.0 * math.pi) for _ in range(n_modes)]

    def rad(n):
        return radius * (1.0 + sum(alpha[m] * math.sin(omega[m][0] * n[0] + omega[m][1] * n[1]
                                                         + omega[m][2] * n[2] + psi[m])
                                   for m in range(n_modes)))

    cx, cy, cz = centre
    verts = []
    for n in ([0.0, 1.0, 0.0],):
        r = rad(n)
        verts.append([cx + r * n[0], cy + r * n[1], cz + r * n[2]])
    for j in range(1, n_lat):
        th = math.pi * j / n_lat
        for i in range(n_lon):
            ph = 2.0 * math.pi * i / n_lon
            n = [math.sin(th) * math.cos(ph), math.cos(th), math.sin(th) * math.sin(ph)]
            r = rad(n)
            verts.append([cx + r * n[0], cy + r * n[1], cz + r * n[2]])
    n = [0.0, -1.0, 0.0]
    r = rad(n)
    verts.append([cx + r * n[0], cy + r * n[1], cz + r * n[2]])
    south = len(verts) - 1

    def ring(j, i):  # j in 1..n_lat-1
        return 1 + (j - 1) * n_lon + (i % n_lon)

    tris = []
    for i in range(n_lon):
        tris.append([0, ring(1, i + 1), ring(1, i)])
    for j in range(1, n_lat - 1):
        for i in range(n_lon):
            a, b = ring(j, i), ring(j, i + 1)
            c, d = ring(j + 1, i), ring(j + 1, i + 1)
            tris.append([a, b, d])
            tris.append([a, d, c])
    for i in range(n_lon):
        tris.append([south, ring(n_lat - 1, i), ring(n_lat - 1, i + 1)])
    rmax = radius * (1.0 + sum(alpha))
    return (np.asarray(verts, np.float32), np.asarray(tris, np.int32), rmax)


# the 12 triangles of an axis-aligned box whose corner k has x from bit 0, y from bit 1, z from bit 2
_BOX_TRIS = ((0, 2, 6), (0, 6, 4), (1, 5, 7), (1, 7, 3), (0, 4, 5), (0, 5, 1),
             (2, 3, 7), (2, 7, 6), (0, 1, 3), (0, 3, 2), (4, 6, 7), (4, 7, 5))


def lattice_mesh(half: float = 4.0, spacing: float = 1.0, width: float = 0.08):
    """The regular grid of R^3 the paper renders (Section 4, Figures of Sections 5-6): an
    axis-parallel square bar of the given width through every grid line {-half, -half +
    spacing, ..., half}^2 along each axis, each bar a closed box of 12 triangles extending
    to +-(half + width / 2).  Spacing 1 and half 4: 243 bars, 2,916 triangles.
    Returns (verts [V,3] f32, tris [T,3] i32)."""
    ticks = np.arange(-half, half + 1e-9, spacing)
    hw, ext = width / 2.0, half + width / 2.0
    verts, tris = [], []
    for axis in range(3):
        o1, o2 = [a for a in range(3) if a != axis]
        for p in ticks:
            for q in ticks:
                lo, hi = np.empty(3), np.empty(3)
                lo[axis], hi[axis] = -ext, ext
                lo[o1], hi[o1] = p - hw, p + hw
                lo[o2], hi[o2] = q - hw, q + hw
                base = len(verts)
                for k in range(8):
                    verts.append([hi[0] if k & 1 else lo[0], hi[1] if k & 2 else lo[1], hi[2] if k & 4 else lo[2]])
                tris.extend([base + a, base + b, base + c] for a, b, c in _BOX_TRIS)
    return np.asarray(verts, np.float32), np.asarray(tris, np.int32)


def random_spheres(seed: int, n: int, box: float, r_lo: float, r_hi: float, avoid):
    """n non-overlapping spheres (centres U[-box, box]^3, radii U[r_lo, r_hi]).

    ``avoid`` is a list of (centre, radius) balls a sphere must stay clear of.
    Returns (spheres [n,4] f32, albedo [n,3] f32).
    """
    rng = SplitMix64(sub_seed(seed, STREAM_SPHERES))
    out, alb = [], []
    attempts = 0
    while len(out) < n:
        attempts += 1
        if attempts > 200000:
            raise RuntimeError("sphere rejection sampling did not converge")
        c = np.array([rng.uniform(-box, box) for _ in range(3)])
        r = rng.uniform(r_lo, r_hi)
        col = [rng.uniform(0.2, 1.0) for _ in range(3)]
        ok = all(np.linalg.norm(c - np.asarray(o[:3])) > r + o[3] for o in out)
        ok = ok and all(np.linalg.norm(c - np.asarray(ac)) > r + ar for ac, ar in avoid)
        if ok:
            out.append([c[0], c[1], c[2], r])
            alb.append(col)
    return np.asarray(out, np.float32).reshape(-1, 4), np.asarray(alb, np.float32).reshape(-1, 3)


# --------------------------------------------------------------------------- configs
def config_parity_64(seed: int = 0) -> Workload:
    """64x64, one bump f = 0.5 exp(-|x|^2 / (2 * 0.5^2)), 4 spheres r=0.5 at (+-1.5, +-1.5, 2), h=0.01, 256 steps."""
    metric = Metric(center=np.zeros((1, 3), np.float32), amplitude=np.array([0.5], np.float32),
                    sigma=np.full((1, 3), 0.5, np.float32))
    sph = np.array([[sx * 1.5, sy * 1.5, 2.0, 0.5] for sx in (-1, 1) for sy in (-1, 1)], np.float32)
    albedo = np.array([[0.9, 0.3, 0.3], [0.3, 0.9, 0.3], [0.3, 0.3, 0.9], [0.9, 0.9, 0.3],
                       [0.7, 0.7, 0.7]], np.float32)
    scene = Scene(sph, np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), albedo)
    return Workload("parity_64x64_1bump", 64, 64, 0.01, 256, metric, scene, Camera(), seed=seed)


def _random_scene(seed, n_spheres, n_lon, n_lat, mesh_radius, cam):
    verts, tris, rmax = displaced_sphere_mesh(seed, n_lon, n_lat, radius=mesh_radius)
    avoid = [((0.0, 0.0, 2.0), rmax), (tuple(cam.pos), 1.0)]
    sph, alb = random_spheres(seed, n_spheres, 4.0, 0.2, 0.8, avoid)
    albedo = np.concatenate([alb, np.array([[0.8, 0.8, 0.8]], np.float32)], 0)
    return Scene(sph, verts, tris, albedo)


def config_1080p_64(seed: int = 1, width: int = 1920, height: int = 1080) -> Workload:
    """1920x1080, 64 bumps (centres U[-4,4]^3, a U[-1,1], sigma U[0.2,1]), 32 spheres + 10k-triangle mesh."""
    cam = Camera()
    c, a, s = random_bumps(seed, 64)
    metric = Metric(center=c, amplitude=a, sigma=s)
    scene = _random_scene(seed, 32, 100, 51, 1.5, cam)
    return Workload("1080p_64bumps_32spheres_10ktris", width, height, 0.005, 2000, metric, scene, cam,
                    seed=seed)


def config_1080p_twist(seed: int = 1, width: int = 1920, height: int = 1080, rate: float = 1.0) -> Workload:
    """The 1080p scene under the pull-back metric of the twist map (rate 1, Section 5.2)."""
    w = config_1080p_64(seed, width, height)
    w.metric = Metric(kind=METRIC_DIFFEO_TWIST, twist_rate=rate, cutoff=0.0)
    w.name = "1080p_twist_32spheres_10ktris"
    return w


def config_4k_1024(seed: int = 4) -> Workload:
    """3840x2160, 1024 bumps, 128 spheres + 100k-triangle mesh (radius 2), h=0.005, 4000 steps."""
    cam = Camera()
    c, a, s = random_bumps(seed, 1024)
    metric = Metric(center=c, amplitude=a, sigma=s)
    scene = _random_scene(seed, 128, 250, 201, 2.0, cam)
    return Workload("4k_1024bumps_128spheres_100ktris", 3840, 2160, 0.005, 4000, metric, scene, cam,
                    seed=seed)


BATCH_RESOLUTIONS = ((256, 256), (512, 512), (1280, 720), (1920, 1080))


def _lattice_scene():
    verts, tris = lattice_mesh()
    return Scene(np.zeros((0, 4), np.float32), verts, tris, np.array([[0.85, 0.85, 0.85]], np.float32))


def config_quad_lattice(width: int = 1920, height: int = 1080, look: str = "x") -> Workload:
    """Section 5.1's example: the graph metric of f(x, y, z) = x^2 + y^2 - z^2 (A = diag(2, 2, -2)),
    seen from the centre of a lattice cell looking along x (or z), through the regular grid
    (spacing 1, bars 0.08 wide, |x_i| <= 4); pseudo-colour shading, h = 0.005, <= 2000 steps."""
    metric = Metric(quad_A=(2.0, 0.0, 0.0, 0.0, 2.0, 0.0, 0.0, 0.0, -2.0), cutoff=0.0)
    fwd, up = ((1.0, 0.0, 0.0), (0.0, 0.0, 1.0)) if look == "x" else ((0.0, 0.0, 1.0), (0.0, 1.0, 0.0))
    cam = Camera(pos=(0.5, 0.5, 0.5), forward=fwd, up=up)
    return Workload(f"quad_lattice_look_{look}", width, height, 0.005, 2000, metric, _lattice_scene(), cam,
                    shading=SHADING_PSEUDO)


def config_paraboloid_lattice(width: int = 1920, height: int = 1080) -> Workload:
    """The paraboloid f = x^2 + y^2 + z^2 (Section 3.3: its exponential map is not injective, so
    grid points appear more than once) through the same lattice, looking along x."""
    w = config_quad_lattice(width, height, "x")
    w.metric = Metric(quad_A=(2.0, 0.0, 0.0, 0.0, 2.0, 0.0, 0.0, 0.0, 2.0), cutoff=0.0)
    w.name = "paraboloid_lattice_look_x"
    return w


def local_maps(seed: int, K: int, lo=(-2.0, -2.0, -1.5), hi=(2.0, 2.0, 2.5), sigma=(0.5, 1.0),
               slope: float = 0.6, field_scale: float = 0.1, with_field: bool = True) -> Metric:
    """K local maps p + f_k(p) (v_k + B_k (p - c_k)) (Section 6): centres U[lo, hi], spreads
    U[sigma], unit directions v_k, amplitudes a_k = +-slope sigma_k e^{1/2} (so that |a| |v|
    e^{-1/2} / sigma = slope < 1), and for every other map a field B_k with entries
    U[-field_scale, field_scale] (none when with_field is False)."""
    rng = SplitMix64(sub_seed(seed, STREAM_BUMPS))
    c = np.zeros((K, 3)); a = np.zeros(K); s = np.zeros((K, 3)); v = np.zeros((K, 3)); B = np.zeros((K, 3, 3))
    for k in range(K):
        c[k] = [rng.uniform(lo[i], hi[i]) for i in range(3)]
        sg = rng.uniform(*sigma)
        s[k] = sg
        d = np.array([rng.uniform(-1.0, 1.0) for _ in range(3)])
        v[k] = d / max(np.linalg.norm(d), 1e-6)
        a[k] = (1.0 if rng.uniform(0.0, 1.0) < 0.5 else -1.0) * slope * sg * math.exp(0.5)
        if with_field and k % 2 == 1:
            B[k] = [[rng.uniform(-field_scale, field_scale) for _ in range(3)] for _ in range(3)]
    return Metric(kind=METRIC_DIFFEO_LOCAL, center=c.astype(np.float32), amplitude=a.astype(np.float32),
                  sigma=s.astype(np.float32), cutoff=0.0, direction=v.astype(np.float32),
                  field=B.astype(np.float32) if with_field else None)


def config_local_lattice(K: int = 8, seed: int = 5, width: int = 1920, height: int = 1080) -> Workload:
    """The lattice under the pull-back metric of K composed local maps (Section 6): camera in a
    cell at (0.5, 0.5, -2.5) looking +z, pseudo-colour, h = 0.005, <= 2000 steps."""
    cam = Camera(pos=(0.5, 0.5, -2.5), forward=(0.0, 0.0, 1.0), up=(0.0, 1.0, 0.0))
    return Workload(f"local{K}_lattice", width, height, 0.005, 2000, local_maps(seed, K), _lattice_scene(), cam,
                    shading=SHADING_PSEUDO, seed=seed)


def config_batch16(seed: int = 3, n: int = 16):
    """n instances over the 1080p scene: resolution uniform from BATCH_RESOLUTIONS, bump count
    floor(exp(U[ln 8, ln 257))) with the 1080p bump distributions, each instance its own bumps."""
    base = config_1080p_64()
    rng = SplitMix64(sub_seed(seed, STREAM_BUMPS))
    out = []
    for i in range(n):
        W, H = BATCH_RESOLUTIONS[min(int(rng.uniform(0, 4)), 3)]
        K = int(math.floor(math.exp(rng.uniform(math.log(8.0), math.log(257.0)))))
        c, a, s = random_bumps(seed * 1000 + i, K)
        w = dataclasses.replace(base, width=W, height=H, metric=Metric(center=c, amplitude=a, sigma=s),
                                name=f"batch{i}_{W}x{H}_{K}bumps", seed=seed * 1000 + i)
        out.append(w)
    return out


def motion(seed: int, K: int):
    """Seeded sinusoidal motion of K centres: A ~ U[0, 0.5]^3, f ~ U[0.1, 0.5] Hz, phi ~ U[0, 2 pi)."""
    rng = SplitMix64(sub_seed(seed, STREAM_ANIM))
    A = np.array([[rng.uniform(0.0, 0.5) for _ in range(3)] for _ in range(K)], np.float32).reshape(K, 3)
    f = np.array([rng.uniform(0.1, 0.5) for _ in range(K)], np.float32)
    ph = np.array([rng.uniform(0.0, 2.0 * math.pi) for _ in range(K)], np.float32)
    return A, f, ph


def scaled(w: Workload, width: int, height: int) -> Workload:
    """Same metric and scene at another resolution."""
    return dataclasses.replace(w, width=width, height=height)
