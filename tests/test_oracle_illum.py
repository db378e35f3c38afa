"""Pins of the oracle's Riemannian illumination (Section 4): the light geodesic found by
shooting, the Riemannian Lambert cosine and the shadow test, against closed forms.

- flat space: the geodesic to the light is the segment q -> L, the solve stops at once and
  the cosine is the Euclidean n . (L - q) / |L - q|; an occluder on the segment shadows;
- affine f: straight lines again, but g = I + b b^T, so the initial tangent is
  d / sqrt(1 + (b.d)^2) and n^T g^-1 n = 1 - (n.b)^2 / (1 + |b|^2) (Sherman-Morrison, Eq. 5.2);
- twist metric: geodesics are preimages of straight lines (Section 5.2), so the direction
  to the light is J(q)^-1 (Phi(L) - Phi(q)) normalised;
- radial bump: the geodesic along a line through the centre stays on it, and there the
  normal and the tangent are parallel, so the Riemannian cosine is exactly 1; off the axis
  the solved direction, integrated again at a finer step, passes through the light.
"""
import numpy as np
import pytest

import oracle
from paper_2005_05386_gb300 import scenes

RK4 = 0


def _scene(spheres, albedo=None):
    spheres = np.asarray(spheres, np.float64).reshape(-1, 4)
    if albedo is None:
        albedo = np.tile([[0.6, 0.7, 0.8]], (spheres.shape[0] + 1, 1))
    return oracle.Scene(spheres, albedo=albedo)


def _rgba(albedo, inten):
    return np.floor(255.0 * np.clip(np.asarray(albedo) * inten, 0, 1) + 0.5).astype(np.uint8)


def test_flat_space_direct_segment_and_shadow():
    m = oracle.Metric(oracle.GRAPH)
    sc = _scene([[0.0, 0.0, 0.0, 1.0]])
    P = np.array([0.0, 0.0, -1.0])
    D = np.array([0.0, 0.0, 1.0])  # the viewer looks along +z and hits the sphere's -z pole
    lt = scenes.Light(pos=(2.0, 1.0, -4.0), tol=1e-9)
    lit, rgba, cosg, iters, u = oracle.illuminate(m, sc, lt, RK4, 0, P, D)
    q = P + 1e-3 * np.array([0.0, 0.0, -1.0])
    d = (np.array(lt.pos) - q) / np.linalg.norm(np.array(lt.pos) - q)
    assert lit and iters == 0
    assert np.allclose(u, d, atol=1e-15)
    assert cosg == pytest.approx(-d[2], abs=1e-14)
    assert np.array_equal(rgba[:3], _rgba([0.6, 0.7, 0.8], 0.1 + 0.9 * (-d[2])))
    # an occluder halfway along q -> L shadows the point; moved aside, it does not
    mid = 0.5 * (q + np.array(lt.pos))
    for centre, expect in ((mid, False), (mid + np.array([0.0, 3.0, 0.0]), True)):
        sc2 = _scene([[0.0, 0.0, 0.0, 1.0], [*centre, 0.3]])
        lit2, rgba2, cos2, _, _ = oracle.illuminate(m, sc2, lt, RK4, 0, P, D)
        assert lit2 == expect
        assert cos2 == pytest.approx(cosg, abs=1e-14)
        if not expect:
            assert np.array_equal(rgba2[:3], _rgba([0.6, 0.7, 0.8], 0.1))
    # a light behind the surface does not light it
    lt_back = scenes.Light(pos=(0.0, 0.0, 3.0))
    assert not oracle.illuminate(m, sc, lt_back, RK4, 0, P, D)[0]


def test_affine_f_riemannian_cosine():
    b = np.array([0.3, -0.5, 0.4])
    m = oracle.Metric(oracle.GRAPH, affine_b=b)
    sc = _scene([[0.0, 0.0, 0.0, 1.0]])
    P = np.array([0.0, -1.0, 0.0])
    D = np.array([0.1, 1.0, 0.0])
    lt = scenes.Light(pos=(-1.0, -5.0, 2.0), tol=1e-9)
    lit, rgba, cosg, iters, u = oracle.illuminate(m, sc, lt, RK4, 0, P, D)
    n = np.array([0.0, -1.0, 0.0])
    q = P + 1e-3 * n
    d = (np.array(lt.pos) - q) / np.linalg.norm(np.array(lt.pos) - q)
    assert lit and iters == 0
    assert np.allclose(u, d / np.sqrt(1.0 + b.dot(d) ** 2), atol=1e-14)
    expect = n.dot(u) / np.sqrt(1.0 - n.dot(b) ** 2 / (1.0 + b.dot(b)))
    assert cosg == pytest.approx(expect, abs=1e-13)
    assert cosg != pytest.approx(n.dot(d), abs=1e-3)  # the metric changes the cosine


@pytest.mark.parametrize("k", [0.5, 1.0])
def test_twist_direction_is_preimage_of_a_line(k):
    m = oracle.Metric(oracle.TWIST, twist_rate=k)
    sc = _scene([[0.0, 0.0, -3.0, 0.5]])
    P = np.array([0.0, 0.0, -2.5])
    D = np.array([0.0, 0.0, -1.0])
    lt = scenes.Light(pos=(1.0, 0.8, 1.5), tol=1e-9, iters=12)
    lit, rgba, cosg, iters, u = oracle.illuminate(m, sc, lt, RK4, 0, P, D)
    q = P + 1e-3 * np.array([0.0, 0.0, 1.0])
    J = oracle.twist_jacobian(k, q)
    w = np.linalg.solve(J, oracle.twist_phi(k, np.array(lt.pos)) - oracle.twist_phi(k, q))
    assert lit and iters >= 1  # the straight guess misses: the solve had to work
    assert np.allclose(u / np.linalg.norm(u), w / np.linalg.norm(w), atol=2e-7)


def _radial():
    return oracle.Metric(oracle.GRAPH, center=[[0.0, 0.0, 0.0]], amplitude=[0.8], sigma=[[0.9] * 3], cutoff=4.0)


def test_radial_bump_on_axis_cosine_is_one():
    m = _radial()
    sc = _scene([[0.0, 0.0, -4.0, 1.0]])
    P = np.array([0.0, 0.0, -3.0])
    D = np.array([0.0, 0.0, -1.0])
    lt = scenes.Light(pos=(0.0, 0.0, 3.0), tol=1e-9)
    lit, rgba, cosg, iters, u = oracle.illuminate(m, sc, lt, RK4, 0, P, D)
    assert lit and iters == 0
    assert u[0] == 0.0 and u[1] == 0.0
    assert cosg == pytest.approx(1.0, abs=1e-14)
    assert u[2] < 1.0 - 1e-5  # g-unit, not Euclidean-unit: the metric is not flat at q


def test_radial_bump_off_axis_geodesic_reaches_the_light():
    m = _radial()
    sc = _scene([[-0.5, 0.2, -4.0, 1.0]])
    P = np.array([-0.5, 0.2, -3.0])
    D = np.array([0.0, 0.0, -1.0])
    L = np.array([0.4, -0.3, 3.0])
    lt = scenes.Light(pos=tuple(L), tol=1e-9, iters=12)
    lit, rgba, cosg, iters, u = oracle.illuminate(m, sc, lt, RK4, 0, P, D)
    assert lit and iters >= 1
    q = P + 1e-3 * np.array([0.0, 0.0, 1.0])
    xs, _ = oracle.integrate(m, RK4, 0.001, 8000, q, u)
    assert np.min(np.linalg.norm(xs - L, axis=1)) < 5e-4  # within one fine step of the light
    straight = (L - q) / np.linalg.norm(L - q)
    assert np.linalg.norm(u / np.linalg.norm(u) - straight) > 1e-3  # and the path is curved
