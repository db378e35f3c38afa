"""Pins for the FP64 oracle: each test checks the oracle against something the
paper or the mathematics fixes independently of the oracle's own formulas
(closed-form values, finite differences of a lower-level quantity, exact
invariants, closed-form geodesics, convergence orders, brute force).

CPU only.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2005_05386_gb300 import scenes

RNG = np.random.default_rng(12345)


def _random_graph_metric(K, aniso=True, affine=False, quad=False, cutoff=0.0, seed=0):
    r = np.random.default_rng(seed)
    c = r.uniform(-1, 1, (K, 3))
    a = r.uniform(-1, 1, K)
    s = r.uniform(0.4, 1.0, (K, 3)) if aniso else np.repeat(r.uniform(0.4, 1.0, (K, 1)), 3, 1)
    b = r.uniform(-0.5, 0.5, 3) if affine else np.zeros(3)
    A = np.zeros((3, 3))
    if quad:
        M = r.uniform(-0.3, 0.3, (3, 3))
        A = M + M.T
    return oracle.Metric(oracle.GRAPH, c, a, s, b, A.reshape(-1), cutoff)


def _fd_grad(fun, x, eps):
    x = np.asarray(x, float)
    out = []
    for k in range(3):
        e = np.zeros(3); e[k] = eps
        out.append((np.asarray(fun(x + e)) - np.asarray(fun(x - e))) / (2 * eps))
    return np.array(out)  # out[k] = d/dx_k fun


def _gamma_from_metric_fd(m, x, eps=1e-5):
    """Eq. 3.4 (read with the standard index placement) from finite differences of g_ij."""
    g = oracle.metric_tensor(m, x)
    ginv = np.linalg.inv(g)
    dg = _fd_grad(lambda y: oracle.metric_tensor(m, y), x, eps)  # dg[k, i, j] = d_k g_ij
    G = np.zeros((3, 3, 3))
    for mm in range(3):
        for i in range(3):
            for j in range(3):
                G[mm, i, j] = 0.5 * sum(ginv[mm, k] * (dg[i, j, k] + dg[j, i, k] - dg[k, i, j])
                                        for k in range(3))
    return G


# ----------------------------------------------------------------- Eq. 6.1
def test_bump_closed_form_values():
    """Eq. 6.1: f(x0) = a; one spread away along axis i, f = a e^{-1/2}; zero past the cutoff."""
    c = np.array([[0.3, -0.2, 0.7]])
    s = np.array([[0.5, 0.8, 1.1]])
    m = oracle.Metric(oracle.GRAPH, c, [0.9], s, cutoff=4.0)
    f, g, H = oracle.field(m, c[0])
    assert f == pytest.approx(0.9, abs=1e-15)
    assert np.allclose(g, 0, atol=1e-15)
    # Hessian at the centre: -a / sigma_i^2 on the diagonal
    assert np.allclose(H, np.diag(-0.9 / s[0] ** 2), atol=1e-14)
    for i in range(3):
        x = c[0].copy(); x[i] += s[0, i]
        f, g, _ = oracle.field(m, x)
        assert f == pytest.approx(0.9 * math.exp(-0.5), rel=1e-14)
        # d f / d x_i = -f / sigma_i at one spread
        assert g[i] == pytest.approx(-0.9 * math.exp(-0.5) / s[0, i], rel=1e-13)
    x = c[0].copy(); x[1] += 4.0 * s[0, 1] * (1 + 1e-9)
    f, g, H = oracle.field(m, x)
    assert f == 0.0 and not g.any() and not H.any()
    x = c[0].copy(); x[1] += 4.0 * s[0, 1] * (1 - 1e-9)
    f, _, _ = oracle.field(m, x)
    assert f == pytest.approx(0.9 * math.exp(-8.0), rel=1e-6)


def test_affine_and_quadratic_part():
    b = np.array([0.3, -0.1, 0.2])
    M = np.array([[1.0, 0.2, 0.0], [0.2, -0.5, 0.1], [0.0, 0.1, 0.3]])
    m = oracle.Metric(oracle.GRAPH, None, None, None, b, M.reshape(-1), 4.0)
    x = np.array([0.7, -1.1, 2.0])
    f, g, H = oracle.field(m, x)
    assert f == pytest.approx(b @ x + 0.5 * x @ M @ x, rel=1e-14)
    assert np.allclose(g, b + M @ x, atol=1e-14)
    assert np.allclose(H, M, atol=0)


@pytest.mark.parametrize("K", [1, 2, 4])
def test_gradient_and_hessian_by_finite_differences(K):
    m = _random_graph_metric(K, aniso=True, affine=True, quad=True, seed=K)
    for _ in range(5):
        x = RNG.uniform(-1, 1, 3)
        f, g, H = oracle.field(m, x)
        gfd = _fd_grad(lambda y: oracle.field(m, y)[0], x, 1e-5)
        Hfd = _fd_grad(lambda y: oracle.field(m, y)[1], x, 1e-5)
        assert np.allclose(g, gfd, atol=1e-8, rtol=1e-7)
        assert np.allclose(H, Hfd, atol=1e-8, rtol=1e-7)
        assert np.allclose(H, H.T, atol=1e-14)


def test_summation_is_linear():
    """Section 6, "Summing functions": derivatives of the sum are the sums of the derivatives."""
    r = np.random.default_rng(7)
    c = r.uniform(-1, 1, (5, 3)); a = r.uniform(-1, 1, 5); s = r.uniform(0.3, 1, (5, 3))
    whole = oracle.Metric(oracle.GRAPH, c, a, s, cutoff=0.0)
    parts = [oracle.Metric(oracle.GRAPH, c[k:k + 1], a[k:k + 1], s[k:k + 1], cutoff=0.0) for k in range(5)]
    for _ in range(5):
        x = r.uniform(-1.5, 1.5, 3)
        f, g, H = oracle.field(whole, x)
        fs = [oracle.field(p, x) for p in parts]
        assert f == pytest.approx(sum(t[0] for t in fs), abs=1e-14)
        assert np.allclose(g, sum(t[1] for t in fs), atol=1e-14)
        assert np.allclose(H, sum(t[2] for t in fs), atol=1e-13)


# -------------------------------------------------------- Eq. 5.2, 5.3, 3.4
def test_graph_metric_inverse_is_sherman_morrison():
    """g = I + grad f grad f^T (Eq. 5.2); its inverse I - grad f grad f^T / (1 + |grad f|^2),
    and det g = 1 + |grad f|^2 (both stated with Eq. 5.2)."""
    m = _random_graph_metric(3, seed=3)
    for _ in range(5):
        x = RNG.uniform(-1, 1, 3)
        _, g, _ = oracle.field(m, x)
        G = oracle.metric_tensor(m, x)
        n2 = g @ g
        assert np.allclose(np.linalg.inv(G), np.eye(3) - np.outer(g, g) / (1 + n2), atol=1e-13)
        assert np.linalg.det(G) == pytest.approx(1 + n2, rel=1e-12)


@pytest.mark.parametrize("K", [1, 2, 3, 4])
def test_graph_christoffel_matches_general_formula(K):
    """Eq. 5.3 against Eq. 3.4 evaluated with finite differences of g."""
    m = _random_graph_metric(K, aniso=True, affine=(K % 2 == 0), quad=(K == 3), seed=10 + K)
    for _ in range(4):
        x = RNG.uniform(-1, 1, 3)
        G = oracle.christoffel(m, x)
        Gfd = _gamma_from_metric_fd(m, x)
        scale = max(1.0, np.abs(G).max())
        assert np.abs(G - Gfd).max() <= 2e-7 * scale


def test_accel_is_minus_gamma_contracted():
    """Eq. 3.3 for the graph metric reduces to Eq. 5.4: a = -(v^T Hess f v) / (1 + |grad f|^2) grad f."""
    m = _random_graph_metric(3, aniso=True, seed=21)
    for _ in range(5):
        x = RNG.uniform(-1, 1, 3); v = RNG.normal(size=3)
        _, g, H = oracle.field(m, x)
        a = oracle.accel(m, x, v)
        assert np.allclose(a, -(v @ H @ v) / (1 + g @ g) * g, atol=1e-14)


# --------------------------------------------------- twist: Eq. 5.6, Thm 5.1
@pytest.mark.parametrize("k", [1.0, 0.6])
def test_twist_map_closed_forms(k):
    p = np.array([1.0, 0.0, math.pi / (2 * k)])
    assert np.allclose(oracle.twist_phi(k, p), [0.0, 1.0, math.pi / (2 * k)], atol=1e-15)
    for _ in range(5):
        p = RNG.uniform(-3, 3, 3)
        q = oracle.twist_phi(k, p)
        assert np.hypot(q[0], q[1]) == pytest.approx(np.hypot(p[0], p[1]), rel=1e-14)
        assert q[2] == p[2]
        assert np.allclose(oracle.twist_phi_inv(k, q), p, atol=1e-14)
        J = oracle.twist_jacobian(k, p)
        Jfd = _fd_grad(lambda y: oracle.twist_phi(k, y), p, 1e-6).T  # J[s, i] = d x_s / d x_i
        assert np.allclose(J, Jfd, atol=1e-8)
        assert np.linalg.det(J) == pytest.approx(1.0, abs=1e-13)
        H = oracle.twist_hessian(k, p)
        Hfd = np.stack([_fd_grad(lambda y, s=s: oracle.twist_jacobian(k, y)[s], p, 1e-6).T
                        for s in range(3)])  # H[s, i, j] = d_j (J[s, i])
        assert np.allclose(H, Hfd, atol=1e-7)
        assert np.allclose(H, H.transpose(0, 2, 1), atol=0)


def test_inverse_by_minors():
    """[J^-1]_ms = (-1)^(s+m) det J_sm / det J (the formula before Theorem 5.1)."""
    for _ in range(5):
        J = RNG.normal(size=(3, 3)) + 3 * np.eye(3)
        Ji = oracle.inverse_by_minors(J)
        assert np.allclose(Ji @ J, np.eye(3), atol=1e-13)
        assert np.allclose(J @ Ji, np.eye(3), atol=1e-13)


@pytest.mark.parametrize("k", [1.0, 0.7])
def test_twist_christoffel_matches_general_formula(k):
    """Theorem 5.1 against Eq. 3.4 with finite differences of g = J^T J (Eq. 5.6)."""
    m = oracle.Metric(oracle.TWIST, twist_rate=k, cutoff=0.0)
    for _ in range(4):
        x = RNG.uniform(-2, 2, 3)
        J = oracle.twist_jacobian(k, x)
        assert np.allclose(oracle.metric_tensor(m, x), J.T @ J, atol=1e-14)
        G = oracle.christoffel(m, x)
        Gfd = _gamma_from_metric_fd(m, x)
        assert np.abs(G - Gfd).max() <= 2e-7 * max(1.0, np.abs(G).max())


# ------------------------------------------------------- straight geodesics
@pytest.mark.parametrize("integrator", [oracle.RK4, oracle.EULER])
@pytest.mark.parametrize("affine", [False, True])
def test_flat_or_affine_f_gives_straight_lines(integrator, affine):
    """Hess f = 0 makes every Christoffel symbol of Eq. 5.3 vanish: polygons are straight."""
    b = (0.4, -0.3, 0.2) if affine else (0, 0, 0)
    m = oracle.Metric(oracle.GRAPH, None, None, None, b, (0,) * 9, cutoff=0.0)
    p = np.array([0.1, -0.2, -6.0]); v = np.array([0.3, 0.1, 0.9])
    xs, vs = oracle.integrate(m, integrator, 0.01, 500, p, v)
    n = np.arange(501)[:, None]
    assert np.allclose(xs, p + 0.01 * n * v, atol=1e-12)
    assert np.allclose(vs, v, atol=0)


@pytest.mark.parametrize("k", [1.0, 0.5])
def test_twist_geodesics_are_preimages_of_lines(k):
    """Eq. 5.8 <=> (Phi o gamma)'' = 0: gamma(t) = Phi^-1(Phi(p) + t J(p) v); RK4 error O(h^4)."""
    m = oracle.Metric(oracle.TWIST, twist_rate=k, cutoff=0.0)
    p = np.array([0.8, -0.5, -1.0]); v = np.array([0.2, 0.6, 0.7])
    Jv = oracle.twist_jacobian(k, p) @ v
    P = oracle.twist_phi(k, p)
    T = 3.0
    errs = []
    for h in (0.02, 0.01, 0.005):
        n = int(round(T / h))
        xs, vs = oracle.integrate(m, oracle.RK4, h, n, p, v)
        exact = np.array([oracle.twist_phi_inv(k, P + (i * h) * Jv) for i in range(n + 1)])
        errs.append(np.abs(xs - exact).max())
    assert errs[1] < 1e-7
    assert 10 < errs[0] / errs[1] < 24 and 10 < errs[1] / errs[2] < 24
    x, _ = oracle.dopri5(m, p, v, T)
    assert np.allclose(x, oracle.twist_phi_inv(k, P + T * Jv), atol=1e-9)


def test_radial_bump_keeps_plane_and_central_line():
    """Isotropic bump: the acceleration of Eq. 5.4 is parallel to x - c, so the polygon
    stays in the plane through c spanned by p - c and v, and (x - c) x v is a first integral."""
    c = np.array([0.2, -0.1, 0.3])
    m = oracle.Metric(oracle.GRAPH, c[None], [0.7], [[0.5, 0.5, 0.5]], cutoff=0.0)
    p = np.array([0.9, 0.5, -1.6]); v = np.array([-0.2, -0.25, 0.9])
    nrm = np.cross(p - c, v); nrm /= np.linalg.norm(nrm)
    L0 = np.cross(p - c, v)
    dL = []
    for h in (0.01, 0.005):
        xs, vs = oracle.integrate(m, oracle.RK4, h, int(round(3.0 / h)), p, v)
        assert np.abs((xs - c) @ nrm).max() < 1e-12
        dL.append(np.abs(np.cross(xs - c, vs) - L0).max())
    assert dL[0] < 1e-6 and dL[0] / dL[1] > 10
    # a ray aimed at the centre stays on its line
    v2 = (c - p) / np.linalg.norm(c - p)
    xs, _ = oracle.integrate(m, oracle.RK4, 0.01, 300, p, v2)
    assert np.abs(np.cross(xs - p, v2)).max() < 1e-12


def test_energy_is_conserved_to_order_four():
    """g(gamma', gamma') is constant along a geodesic (Eq. 3.3 is the geodesic flow)."""
    m = _random_graph_metric(3, aniso=True, seed=5)
    p = np.array([-0.3, 0.2, -2.0]); d = np.array([0.1, -0.05, 1.0])
    v = d / math.sqrt(oracle.inner(m, p, d, d))
    drift = []
    for h in (0.02, 0.01):
        xs, vs = oracle.integrate(m, oracle.RK4, h, int(round(4.0 / h)), p, v)
        e = np.array([oracle.inner(m, x, w, w) for x, w in zip(xs, vs)])
        drift.append(np.abs(e - 1.0).max())
    assert drift[0] < 1e-5
    assert drift[0] / drift[1] > 10


@pytest.mark.parametrize("integrator,order", [(oracle.RK4, 4), (oracle.EULER, 1)])
def test_convergence_order_against_dopri5(integrator, order):
    m = _random_graph_metric(2, aniso=True, seed=9)
    p = np.array([-0.4, 0.3, -2.0]); d = np.array([0.2, -0.1, 1.0])
    v = d / math.sqrt(oracle.inner(m, p, d, d))
    T = 3.2
    ref, _ = oracle.dopri5(m, p, v, T)
    hs = (0.04, 0.02, 0.01) if integrator == oracle.RK4 else (0.004, 0.002, 0.001)
    errs = []
    for h in hs:
        xs, _ = oracle.integrate(m, integrator, h, int(round(T / h)), p, v)
        errs.append(np.linalg.norm(xs[-1] - ref))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    for r in rates:
        assert abs(r - order) < 0.35, (errs, rates)


# ------------------------------------------------------------ intersections
def test_sphere_hits_analytic():
    sp = [0.0, 0.0, 2.0, 0.5]
    O = [0.0, 0.0, -6.0]
    assert oracle.hit_sphere(O, [0, 0, 2.0], 100.0, sp) == pytest.approx(7.5 / 2.0, rel=1e-15)
    assert oracle.hit_sphere(O, [0, 0, 2.0], 3.75, sp) is None          # s_max is exclusive
    assert oracle.hit_sphere(O, [0, 0, -1.0], 100.0, sp) is None        # behind
    s = oracle.hit_sphere([0.5, 0.0, -6.0], [0, 0, 1.0], 100.0, sp)     # grazing counts
    assert s == pytest.approx(8.0, rel=1e-12)
    assert oracle.hit_sphere([0.0, 0.1, 2.0], [1, 0, 0], 1.0, sp) == 0.0  # starts inside
    assert oracle.hit_sphere([0.0, 0.0, 2.5], [0, 0, 1.0], 1.0, sp) == 0.0  # starts on the surface
    # oblique: closest approach b, hit at sqrt(L^2 - b^2) - sqrt(r^2 - b^2) along a unit direction
    d = np.array([0.03, 0.0, 1.0]); d /= np.linalg.norm(d)
    oc = np.array(sp[:3]) - np.array(O)
    tca = oc @ d; b2 = oc @ oc - tca ** 2
    assert oracle.hit_sphere(O, d, 100.0, sp) == pytest.approx(tca - math.sqrt(0.25 - b2), rel=1e-13)


def test_triangle_hits_edges_inclusive():
    tri = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0], float)
    D = [0, 0, 1.0]
    assert oracle.hit_triangle([0.2, 0.2, -1], D, 2.0, tri) == pytest.approx(1.0)
    assert oracle.hit_triangle([0.5, 0.5, -1], D, 2.0, tri) == pytest.approx(1.0)   # on the hypotenuse
    assert oracle.hit_triangle([0.0, 0.0, -1], D, 2.0, tri) == pytest.approx(1.0)   # on a vertex
    assert oracle.hit_triangle([0.6, 0.6, -1], D, 2.0, tri) is None
    assert oracle.hit_triangle([0.2, 0.2, 1], [0, 0, -1.0], 2.0, tri) == pytest.approx(1.0)  # two-sided
    assert oracle.hit_triangle([0.2, 0.2, -1], [1.0, 0, 0], 2.0, tri) is None      # parallel
    assert oracle.hit_triangle([0.2, 0.2, -1], D, 1.0, tri) is None                 # s_max exclusive


@pytest.fixture(scope="module")
def mesh_scene():
    w = scenes.config_1080p_64()
    return w.scene


def test_bvh_matches_brute_force(mesh_scene):
    bvh = oracle.Scene.from_desc(mesh_scene, use_bvh=True)
    brute = oracle.Scene.from_desc(mesh_scene, use_bvh=False)
    r = np.random.default_rng(3)
    n_hit = 0
    for q in range(400):
        O = r.uniform(-3, 3, 3) + np.array([0, 0, 2.0])
        if q % 2:
            D = r.normal(size=3) * 0.05      # short chords, like the polygon's
            smax = 1.0
        else:
            D = r.normal(size=3)
            smax = 1e6
        a = bvh and oracle.scene_hit(bvh, O, D, smax)
        b = oracle.scene_hit(brute, O, D, smax)
        assert a == b
        n_hit += a is not None
    assert n_hit > 20


def test_closed_mesh_is_watertight(mesh_scene):
    """Rays from inside the closed displaced sphere always hit it, also through vertices and edges."""
    sc = oracle.Scene(np.zeros((0, 4)), mesh_scene.verts, mesh_scene.tris, None, use_bvh=True)
    O = np.array([0.0, 0.0, 2.0])
    r = np.random.default_rng(4)
    dirs = list(r.normal(size=(300, 3)))
    V = mesh_scene.verts.astype(np.float64)
    T = mesh_scene.tris
    dirs += [V[i] - O for i in range(0, V.shape[0], 37)]                          # through vertices
    dirs += [0.5 * (V[T[t, 0]] + V[T[t, 1]]) - O for t in range(0, T.shape[0], 53)]  # through edges
    for D in dirs:
        assert oracle.scene_hit(sc, O, D, 1e9) is not None


# ------------------------------------------------------------------ camera
def test_camera_directions():
    cam = scenes.Camera()
    W = H = 65
    d = oracle.camera_dir(cam, W, H, 32, 32)
    assert np.allclose(d, [0, 0, 1], atol=1e-15)
    t = math.tan(math.radians(30))
    d = oracle.camera_dir(cam, 64, 32, 0, 0)   # top-left pixel: left is -x, top is +y
    assert d[0] / d[2] == pytest.approx((2 * 0.5 / 64 - 1) * t * 2, rel=1e-13)
    assert d[1] / d[2] == pytest.approx((1 - 2 * 0.5 / 32) * t, rel=1e-13)
    assert np.linalg.norm(d) == pytest.approx(1.0, rel=1e-15)


# ------------------------------------------------------------- whole trace
def _flat_workload(h=0.05, steps=400, shading=scenes.SHADING_LAMBERT):
    w = scenes.config_parity_64()
    w.metric = scenes.Metric(cutoff=0.0)            # flat, and no closed-form skip
    w.h, w.max_steps, w.shading = h, steps, shading
    return w


def test_flat_trace_hits_are_analytic():
    """A flat metric marched in chords of length h must find the analytic first hits."""
    w = _flat_workload()
    o = oracle.trace(w)
    O = np.array(w.camera.pos)
    n_hit = 0
    for p in range(w.n_pixels):
        i, j = p % w.width, p // w.width
        d = oracle.camera_dir(w.camera, w.width, w.height, i, j)
        best, bid = np.inf, -1
        for k, sp in enumerate(w.scene.spheres.astype(float)):
            oc = sp[:3] - O
            tca = oc @ d; b2 = oc @ oc - tca * tca
            if b2 <= sp[3] ** 2 and tca > 0:
                t = tca - math.sqrt(sp[3] ** 2 - b2)
                if t < best:
                    best, bid = t, k
        if bid < 0:
            assert o["id"][p] == oracle.BUDGET   # never curved, never flat-skipped: runs out
        else:
            n_hit += 1
            assert o["id"][p] == bid
            assert np.allclose(o["hit"][p], O + best * d, atol=1e-11)
            assert o["steps"][p] == math.floor(best / w.h) + 1
    assert n_hit > 100


def test_affine_metric_marches_at_g_unit_speed():
    """With f = b.x the metric is constant, g = I + b b^T (Eq. 5.2): a g-unit tangent along the
    Euclidean unit d has Euclidean speed 1 / sqrt(1 + (b.d)^2), which sets the step count."""
    w = _flat_workload(h=0.05, steps=600)
    b = np.array([0.6, -0.3, 0.8])
    w.metric = scenes.Metric(affine_b=tuple(b), cutoff=0.0)
    flat = oracle.trace(_flat_workload(h=0.05, steps=600))
    o = oracle.trace(w)
    hit = np.nonzero(flat["id"] >= 0)[0]
    assert len(hit) > 100
    for p in hit[::7]:
        d = oracle.camera_dir(w.camera, w.width, w.height, p % w.width, p // w.width)
        speed = 1.0 / math.sqrt(1.0 + (b @ d) ** 2)
        t = np.linalg.norm(flat["hit"][p] - np.array(w.camera.pos))
        assert o["id"][p] == flat["id"][p]
        assert np.allclose(o["hit"][p], flat["hit"][p], atol=1e-11)
        assert o["steps"][p] == math.floor(t / (w.h * speed)) + 1


def test_skip_matches_marching_through_flat_space():
    """Advancing in closed form outside the truncated supports equals marching there
    (marching spends steps in flat space, so it gets a larger step budget)."""
    w = scenes.config_parity_64()
    a = oracle.trace(w)
    w.max_steps += 1500
    b = oracle.trace(w, no_skip=True)
    hit = a["id"] >= 0
    assert hit.sum() > 50
    assert (a["id"][hit] == b["id"][hit]).mean() > 0.99
    both = hit & (b["id"] == a["id"])
    assert np.abs(a["hit"][both] - b["hit"][both]).max() < 1e-4
    assert (b["id"][a["id"] == oracle.MISS] < 0).all()


def test_shading_rules():
    w = scenes.config_parity_64()
    w.width = w.height = 65
    w.metric = scenes.Metric(cutoff=0.0)
    w.h, w.max_steps = 0.05, 400
    w.scene = scenes.Scene(np.array([[0, 0, 2.0, 1.0]], np.float32), np.zeros((0, 3), np.float32),
                           np.zeros((0, 3), np.int32), np.array([[0.4, 0.6, 0.8], [1, 1, 1]], np.float32))
    centre = np.array([32 * 65 + 32])
    o = oracle.trace(w, centre)
    # head-on: intensity 0.1 + 0.9 * 1
    assert o["id"][0] == 0
    assert list(o["rgba"][0]) == [math.floor(255 * c + 0.5) for c in (0.4, 0.6, 0.8)] + [255]
    w.shading = scenes.SHADING_PSEUDO
    o = oracle.trace(w, centre)
    assert np.allclose(o["hit"][0], [0, 0, 1.0], atol=1e-12)
    assert list(o["rgba"][0]) == [128, 128, 159, 255]      # 0.5 + hit / 8
    w.scene.spheres[0, 0] = 5.0                              # nothing in view: runs out of steps
    o = oracle.trace(w, centre)
    assert o["id"][0] == oracle.BUDGET and list(o["rgba"][0]) == [0, 0, 0, 0]


def test_miss_when_no_support_ahead():
    w = scenes.config_parity_64()
    w.scene = scenes.Scene(np.zeros((0, 4), np.float32), np.zeros((0, 3), np.float32),
                           np.zeros((0, 3), np.int32), np.ones((1, 3), np.float32))
    o = oracle.trace(w, np.array([0, 63, 64 * 64 - 1]))   # corner rays pass outside the bump
    assert list(o["id"]) == [oracle.MISS] * 3
    assert list(o["steps"]) == [0, 0, 0]


def test_quadratic_metric_axis_geodesic_closed_form():
    """f = x^2 + y^2 - z^2 (A = diag(2, 2, -2), Section 5.1's example).  From the origin along x
    the geodesic stays on the x-axis (the metric is symmetric under y -> -y and z -> -z), where
    g_xx = 1 + f_x^2 = 1 + 4 x^2, so its arc length is s(x) = x sqrt(1 + 4x^2) / 2 + asinh(2x) / 4."""
    m = oracle.Metric(oracle.GRAPH, None, None, None, (0, 0, 0), (2, 0, 0, 0, 2, 0, 0, 0, -2), cutoff=0.0)
    h, n = 0.005, 400
    xs, vs = oracle.integrate(m, oracle.RK4, h, n, [0.0, 0.0, 0.0], [1.0, 0.0, 0.0])
    assert np.abs(xs[:, 1:]).max() == 0.0
    x = xs[-1, 0]
    s = x * np.sqrt(1 + 4 * x * x) / 2 + np.arcsinh(2 * x) / 4
    assert abs(s - n * h) < 1e-9, (s, n * h)
    # and the tangent stays g-unit: (1 + 4x^2) x'^2 = 1
    assert abs((1 + 4 * x * x) * vs[-1, 0] ** 2 - 1) < 1e-9


def _local_metric(K=3, seed=1, field=True):
    """K local maps p + f_i(p) (v_i + B_i (p - c_i)) with |a_i| |v_i| e^{-1/2} / sigma_i = 0.6."""
    r = np.random.default_rng(seed)
    c = r.uniform(-1, 1, (K, 3))
    sig = r.uniform(0.4, 0.8, K)
    d = r.normal(size=(K, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    a = 0.6 * sig / np.exp(-0.5)
    B = r.normal(size=(K, 3, 3)) * 0.1 if field else None
    return oracle.Metric(oracle.LOCAL, c, a, np.repeat(sig[:, None], 3, 1), cutoff=0.0, direction=d, field=B)


@pytest.mark.parametrize("K", [1, 3])
def test_local_composition_derivatives_match_finite_differences(K):
    """J and H of Phi = Phi_1 o ... o Phi_K (chain rule and Eq. 6.3) against central differences
    of Phi itself and of J."""
    m = _local_metric(K)
    p = np.array([0.2, -0.1, 0.3])
    q, J, H = oracle.local_compose(m, p)
    eps = 1e-5
    for j in range(3):
        e = np.zeros(3)
        e[j] = eps
        qp, Jp, _ = oracle.local_compose(m, p + e)
        qm, Jm, _ = oracle.local_compose(m, p - e)
        np.testing.assert_allclose(J[:, j], (qp - qm) / (2 * eps), atol=1e-8)
        np.testing.assert_allclose(H[:, :, j], (Jp - Jm) / (2 * eps), atol=1e-8)
    assert np.abs(q - p).max() > 1e-3  # the maps actually move p


def test_local_jinv_product_inverts_the_jacobian():
    """The paper's J^-1(Phi) = J^-1(Phi_K) ... J^-1(Phi_1) is the inverse of the composed J."""
    m = _local_metric(4, seed=2)
    for p in ([0.0, 0.0, 0.0], [0.5, -0.7, 0.1]):
        _, J, _ = oracle.local_compose(m, p)
        np.testing.assert_allclose(oracle.local_jinv(m, p) @ J, np.eye(3), atol=1e-12)


@pytest.mark.parametrize("field", [False, True])
def test_local_geodesics_are_preimages_of_lines(field):
    """Under the pull-back metric g = J^T J of a diffeomorphism, Phi maps geodesics to straight
    lines (Section 5.2): Phi(x(s)) = Phi(p) + s J(p) v with |J(p) v| = 1, to O(h^4) for RK4."""
    m = _local_metric(3, field=field)
    x0, d0 = np.array([-1.0, 0.2, -0.5]), np.array([0.3, 0.5, -0.8])
    v0 = d0 / np.sqrt(oracle.inner(m, x0, d0, d0))
    q0, J0, _ = oracle.local_compose(m, x0)
    assert abs(np.linalg.norm(J0 @ v0) - 1.0) < 1e-12
    errs = []
    for h, n in ((0.01, 200), (0.005, 400)):
        xs, _ = oracle.integrate(m, oracle.RK4, h, n, x0, v0)
        errs.append(max(np.linalg.norm(oracle.local_compose(m, xs[i])[0] - (q0 + i * h * J0 @ v0))
                        for i in range(n + 1)))
        bend = np.linalg.norm(xs[-1] - (x0 + n * h * v0))
    assert errs[1] < 1e-9 and errs[0] / errs[1] > 10, errs
    assert bend > 1e-2  # the geodesic is not itself a straight line


def test_local_zero_amplitude_is_flat():
    m = oracle.Metric(oracle.LOCAL, [[0.0, 0.0, 0.0]], [0.0], [[0.5] * 3], cutoff=0.0,
                      direction=[[1.0, 0.0, 0.0]])
    xs, _ = oracle.integrate(m, oracle.RK4, 0.01, 50, [0.1, 0.2, 0.3], [0.0, 0.6, 0.8])
    np.testing.assert_allclose(xs[-1], [0.1, 0.2 + 0.3, 0.3 + 0.4], atol=1e-14)


@pytest.mark.parametrize("no_skip", [False, True])
def test_fog_attenuates_by_arc_length_on_straight_rays(no_skip):
    """Fog (the grid figures' black fog): colour c exp(-d * arc length).  One bump of amplitude
    1e-12 leaves the rays straight lines of unit speed (to ~1e-12) while its support ball makes
    them advance in closed form, march through the ball and advance again, so the arc length
    to a hit must be its distance from the camera along every path (or when marching only)."""
    from paper_2005_05386_gb300 import scenes
    w = scenes.scaled(scenes.config_parity_64(), 48, 48)
    w.metric = scenes.Metric(center=np.zeros((1, 3), np.float32), amplitude=np.array([1e-12], np.float32),
                             sigma=np.full((1, 3), 0.5, np.float32))
    w.h, w.max_steps = 0.01, 2000
    base = oracle.trace(w, no_skip=no_skip)
    d = 0.15
    w.scene.fog = d
    fogged = oracle.trace(w, no_skip=no_skip)
    hit = base["id"] >= 0
    assert hit.sum() > 40
    np.testing.assert_array_equal(base["id"], fogged["id"])
    dist = np.linalg.norm(base["hit"][hit] - np.asarray(w.camera.pos), axis=1)
    expect = base["rgba"][hit][:, :3] / 255.0 * np.exp(-d * dist)[:, None]
    got = fogged["rgba"][hit][:, :3] / 255.0
    assert np.abs(got - expect).max() <= 1.0 / 255.0 + 1e-9
    assert (fogged["rgba"][hit][:, :3] < base["rgba"][hit][:, :3]).any()
    assert (fogged["rgba"][~hit] == 0).all()


def _refined_hits(w, steps_h, pixels=None, arc=None):
    """Hit points of the same frame traced at each step in steps_h (budget arc / h, or the frame's
    own arc length budget), on the pixels that hit the same object every time."""
    import dataclasses
    arc = arc if arc is not None else w.max_steps * w.h
    res = [oracle.trace(dataclasses.replace(w, h=h, max_steps=int(round(arc / h))), pixels) for h in steps_h]
    same = np.all([r["id"] == res[0]["id"] for r in res], axis=0) & (res[0]["id"] >= 0)
    return [r["hit"][same] for r in res], int(same.sum())


def test_full_trace_converges_at_fourth_order_without_truncation():
    """The whole pipeline (camera, RK4 marching, segment tests) on a curved frame: with the bump
    untruncated the metric is smooth, so hit points converge at the order of RK4 (Eq. 3.3):
    halving h divides their change by 16."""
    import dataclasses
    w = scenes.config_parity_64()
    w.metric = dataclasses.replace(w.metric, cutoff=0.0)
    hits, n = _refined_hits(w, (0.04, 0.02, 0.01), np.arange(0, 4096, 3), arc=12.0)
    assert n >= 40
    e1 = np.abs(hits[0] - hits[1]).max()
    e2 = np.abs(hits[1] - hits[2]).max()
    assert 11.0 < e1 / e2 < 22.0, (e1, e2)
    assert e2 < 1e-10


def test_truncation_costs_one_order_with_a_tiny_constant():
    """With truncated bumps (reading R4) the acceleration jumps where a ray crosses a support
    sphere, so RK4 converges at first order there; the jump is of size a e^-8, and the hit points
    move by less than 1e-7 between h = 0.02 and 0.01."""
    w = scenes.config_parity_64()
    hits, n = _refined_hits(w, (0.02, 0.01, 0.005))
    assert n >= 60
    e1 = np.abs(hits[0] - hits[1]).max()
    e2 = np.abs(hits[1] - hits[2]).max()
    assert 1.4 < e1 / e2 < 3.0, (e1, e2)
    assert e1 < 1e-7


def test_twist_frame_hits_lie_on_preimages_of_lines():
    """The full trace under the twist metric against its closed form (Section 5.2): every view
    geodesic is Phi^-1(Phi(p) + t J(p) v), so a sphere hit has an exact position, the first
    crossing of that curve with the sphere.  The oracle's hit lies on the marched polygon (the
    nodes are exact to RK4's order), off the curve by the segment's sagitta over the sine of
    the angle at which the path meets the sphere: within the 1e-4 parity tolerance at the
    frame's step h = 0.005, and at least 1.8 times closer when h is halved.  (Halving keeps the
    node before the crossing, so the sagitta at the crossing, about kappa h d / 2 at a distance
    d past that node, falls in proportion to h.)"""
    import dataclasses
    from scipy.optimize import brentq
    k = 1.0
    w = scenes.config_1080p_twist(width=12, height=8, rate=k)
    m = oracle.Metric(oracle.TWIST, twist_rate=k)
    sph = np.asarray(w.scene.spheres, np.float64)
    res = {h: oracle.trace(dataclasses.replace(w, h=h, max_steps=int(round(10.0 / h)))) for h in (0.005, 0.0025)}
    P0 = np.array(w.camera.pos, np.float64)
    Q0 = oracle.twist_phi(k, P0)
    J = oracle.twist_jacobian(k, P0)
    checked = 0
    for p in range(w.n_pixels):
        sid = int(res[0.005]["id"][p])
        if sid < 0 or sid >= len(sph) or int(res[0.0025]["id"][p]) != sid:
            continue
        d = oracle.camera_dir(w.camera, w.width, w.height, p % w.width, p // w.width)
        v = d / np.sqrt(oracle.inner(m, P0, d, d))
        Jv = J @ v
        c, r = sph[sid, :3], sph[sid, 3]
        f = lambda t: np.linalg.norm(oracle.twist_phi_inv(k, Q0 + t * Jv) - c) - r
        ts = np.linspace(0.0, 10.0, 4001)
        inside = np.nonzero(np.array([f(t) for t in ts]) < 0.0)[0]
        assert len(inside), p
        t_hit = brentq(f, ts[inside[0] - 1], ts[inside[0]], xtol=1e-14)
        X = oracle.twist_phi_inv(k, Q0 + t_hit * Jv)
        e_h = np.abs(res[0.005]["hit"][p] - X).max()
        e_h2 = np.abs(res[0.0025]["hit"][p] - X).max()
        assert e_h < 1e-4 and e_h2 * 1.8 < e_h + 1e-10, (p, e_h, e_h2)
        checked += 1
    assert checked >= 20


def test_trace_dirs_equals_trace_and_conditioning_of_straight_rays():
    """trace_dirs with the pixels' own directions is trace; in flat space a ray that meets a
    sphere head-on at distance t moves its hit by about eps t when its direction turns by
    eps (the conditioning measure the 4K parity test uses), and a grazing ray may change
    object."""
    w = scenes.config_parity_64()
    px = np.arange(0, w.n_pixels, 13)
    a = oracle.trace(w, px)
    dirs = np.array([oracle.camera_dir(w.camera, w.width, w.height, int(p % w.width), int(p // w.width))
                     for p in px])
    b = oracle.trace_dirs(w, dirs)
    for k in ("id", "steps", "rgba", "hit"):
        assert np.array_equal(a[k], b[k]), k
    flat = scenes.config_parity_64()
    flat.metric = scenes.Metric()          # no bumps: straight rays, closed-form miss or hit
    flat.scene = scenes.Scene(np.array([[0.0, 0.0, 4.0, 1.0]], np.float32), np.zeros((0, 3), np.float32),
                              np.zeros((0, 3), np.int32), np.ones((2, 3), np.float32))
    centre = (flat.height // 2) * flat.width + flat.width // 2
    eps = 1e-6
    same, move = oracle.conditioning(flat, [centre], eps=eps)
    t = oracle.trace(flat, [centre])
    dist = np.linalg.norm(t["hit"][0] - np.array(flat.camera.pos))
    assert same[0] and 0.5 * eps * dist <= move[0] <= 3 * eps * dist, (move[0], eps * dist)
    # a ray that grazes the sphere's rim: a tilt of eps decides between hit and miss
    r = oracle.trace(flat)
    hit = (r["id"] == 0).reshape(flat.height, flat.width)
    row = flat.height // 2
    cols = np.nonzero(hit[row])[0]
    rim = row * flat.width + int(cols.max())
    same, move = oracle.conditioning(flat, [rim], eps=0.05)
    assert not same[0] or move[0] > 1e-2
