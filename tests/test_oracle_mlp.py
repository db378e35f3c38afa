"""Pins for the FP64 reference of the learned exponential map (CPU)."""
import numpy as np

from oracle import mlp


def _net(seed):
    r = np.random.default_rng(seed)
    d = {}
    for name, shape in mlp.SHAPES:
        fan = shape[1] if len(shape) == 2 else 1
        d[name] = r.uniform(-1, 1, shape) * np.sqrt(6.0 / fan) if len(shape) == 2 else r.uniform(-0.1, 0.1, shape)
    return mlp.pack(d)


def test_parameter_count():
    assert mlp.N_PARAMS == 135431


def test_gradients_match_finite_differences():
    """Central differences of the loss, its error-head target held fixed, on sampled
    coordinates of every parameter block."""
    r = np.random.default_rng(3)
    params = _net(1)
    X = r.uniform(-1, 1, (16, 7))
    T = r.normal(size=(16, 6))
    L, g = mlp.loss_and_grads(params, X, T)
    assert abs(L - mlp.loss(params, X, T)) < 1e-12
    e = mlp.error_target(params, X, T)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])
    for b in range(len(mlp.SHAPES)):
        for idx in r.integers(offs[b], offs[b + 1], 4):
            eps = 1e-6
            pp, pm = params.copy(), params.copy()
            pp[idx] += eps
            pm[idx] -= eps
            fd = (mlp.loss(pp, X, T, e=e) - mlp.loss(pm, X, T, e=e)) / (2 * eps)
            assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), (mlp.SHAPES[b][0], idx, fd, g[idx])


def test_zero_network_predicts_zero():
    params = np.zeros(mlp.N_PARAMS)
    Y, _ = mlp.forward(params, np.ones((3, 7)))
    assert not Y.any()


def _segments(n, seed, s_max=0.5):
    r = np.random.default_rng(seed)
    X = np.zeros((n, 7))
    X[:, :3] = r.uniform(-1, 1, (n, 3))
    d = r.normal(size=(n, 3))
    X[:, 3:6] = d / np.linalg.norm(d, axis=1, keepdims=True)
    X[:, 6] = r.integers(1, 101, n) * 0.005 / s_max
    return X


def test_segment_residuals_vanish_when_geodesics_are_lines():
    """f = 0 and f linear (Eq. 5.4 with Hess f = 0): the exp map is x + s v, so both residuals are zero."""
    import oracle
    X = _segments(6, 1)
    for m in (oracle.Metric(oracle.GRAPH, cutoff=0.0),
              oracle.Metric(oracle.GRAPH, None, None, None, (0.3, -0.2, 0.5), (0,) * 9, 0.0)):
        R = mlp.segment_residuals(m, X, 4.0, 0.5, 0.005)
        assert np.abs(R).max() < 1e-12


def test_segment_residuals_match_adaptive_reference():
    """RK4 at h = 0.005 against Dormand-Prince at 1e-12 over the same arc: the residuals
    agree to O(h^4) / s^2, far below the surrogate's error scale.  The field is left
    untruncated so that the right-hand side is smooth and RK4 keeps its order."""
    import oracle
    from paper_2005_05386_gb300 import scenes
    c, a, s = scenes.random_bumps(1, 64)
    m = oracle.Metric(oracle.GRAPH, c, a, s, cutoff=0.0)
    X = _segments(8, 2)
    R = mlp.segment_residuals(m, X, 4.0, 0.5, 0.005)
    for row, r in zip(X, R):
        x, d = row[:3] * 4.0, row[3:6]
        sl = round(row[6] * 0.5 / 0.005) * 0.005
        v = d / np.sqrt(oracle.inner(m, x, d, d))
        xe, ve = oracle.dopri5(m, x, v, sl)
        ref = np.concatenate([(xe - x - sl * v) / sl ** 2, (ve - v) / sl])
        assert np.abs(ref - r).max() < 1e-5 * max(1.0, np.abs(ref).max()), (row, ref, r)
    assert np.abs(R).max() > 1e-3  # the field actually bends these segments


def test_far_field_bound_dominates_sampled_accelerations():
    """Along RK4 geodesics of g-length s from x (g-unit tangent), |x''| at every vertex
    stays below the bound for (x, s); points whose reach misses every support get 0."""
    import oracle
    from paper_2005_05386_gb300 import scenes
    c, a, s = scenes.random_bumps(1, 64)
    m = oracle.Metric(oracle.GRAPH, c, a, s, cutoff=4.0)
    r = np.random.default_rng(5)
    tight = []
    for _ in range(60):
        x = r.uniform(-4, 4, 3)
        d = r.normal(size=3)
        d /= np.linalg.norm(d)
        k = int(r.integers(1, 101))
        sl = k * 0.005
        B = mlp.far_field_bound(c, a, s, 4.0, x, sl)
        v = d / np.sqrt(oracle.inner(m, x, d, d))
        xs, vs = oracle.integrate(m, oracle.RK4, 0.005, k, x, v)
        amax = max(np.linalg.norm(oracle.accel(m, xi, vi)) for xi, vi in zip(xs, vs))
        assert amax <= B * (1 + 1e-9) + 1e-15, (x, d, sl, amax, B)
        if amax > 0:
            tight.append(amax / B)
    assert len(tight) > 30 and max(tight) > 1e-2  # not vacuous
    far = np.array([40.0, 0.0, 0.0])
    assert mlp.far_field_bound(c, a, s, 4.0, far, 0.5) == 0.0
    assert np.linalg.norm(oracle.accel(m, far, np.array([1.0, 0, 0]))) == 0.0


def test_far_field_bound_single_bump_is_attained_in_gradient_direction():
    """One bump, s = 0, at distance r = 2 sigma: the gradient factor is exact and the
    Hessian factor is attained by v along the gradient, so the bound equals
    |grad f| ||Hess f|| evaluated there (before the min with 1/2)."""
    sig, amp = 0.5, 0.3
    x = np.array([2 * sig, 0.0, 0.0])
    B = mlp.far_field_bound([[0.0, 0.0, 0.0]], [amp], [[sig] * 3], 0.0, x, 0.0)
    q, u = 1 / sig ** 2, 4.0
    grad = amp * q * (2 * sig) * np.exp(-u / 2)           # |df/dr| of a Gaussian
    hess_rr = amp * q * (u - 1) * np.exp(-u / 2)          # d2f/dr2
    assert grad < 0.5
    assert B >= grad * hess_rr
    assert B <= grad * hess_rr * (1 + u) / (u - 1) + 1e-15
