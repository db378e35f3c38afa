"""Riemannian illumination on the GPU (rgeo_trace_lit) against the FP64 oracle.

Every hit is re-shaded from a point light through the light geodesic found by shooting
(Section 4, "Riemannian illumination").  The view rays must agree as in the other parity
tests (object and hit point within 1e-4 on at least 99.9 % of the pixels).  A hit's colour
(2/255, which separates lit from unlit) must agree too, except where several geodesics
join the hit point to the light (the exponential map is not injective, Section 3.3): there
the solution the shooting finds depends on rounding, and the FP32 and FP64 solves may land
on different ones.  Such a pixel is accepted only when the oracle's own answer changes
under a 2 % change of the light step or a doubled difference step, and at most 2 % of the
hits may be such pixels.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2005_05386_gb300 import scenes
from parity import assert_parity, compare, gpu_arrays

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rg():
    import torch
    import paper_2005_05386_gb300 as rg
    torch.cuda.set_device(0)
    return rg


def _lit(rg, w, light, pixels=None):
    out = rg.trace_lit(w, light)
    rg.rgeo_sync()
    g = gpu_arrays(out, pixels)
    lit = out["lit"].cpu().numpy()
    g["lit"] = lit[pixels] if pixels is not None else lit
    return g


def _check(w, light, pixels, g, ref, min_hits, min_lit):
    S = w.scene.n_spheres
    # the view rays: same object and hit point as the oracle
    view = compare(g, dict(ref, rgba=g["rgba"]), S)
    assert_parity(view, min_hits=min_hits)
    go, ro = np.where(g["id"] >= S, S, g["id"]), np.where(ref["id"] >= S, S, ref["id"])
    hit = (go == ro) & (ro >= 0)
    cerr = np.abs(g["rgba"].astype(np.int64) - ref["rgba"].astype(np.int64)).max(axis=1)
    bad = np.nonzero(hit & (cerr > 2))[0]
    assert len(bad) <= max(2, int(0.02 * hit.sum())), (len(bad), int(hit.sum()))
    if len(bad):
        # every disagreement must be a pixel whose light geodesic is ambiguous for the oracle itself
        px = pixels[bad] if pixels is not None else bad
        ambiguous = np.zeros(len(bad), bool)
        for lt in (dataclasses.replace(light, h=light.h * 0.98), dataclasses.replace(light, h=light.h * 1.02),
                   dataclasses.replace(light, delta=light.delta * 2)):
            r = oracle.trace_lit(w, lt, px)
            ambiguous |= np.abs(r["rgba"].astype(np.int64) - ref["rgba"][bad].astype(np.int64)).max(axis=1) > 2
        assert ambiguous.all(), [int(p) for p in px[~ambiguous]]
    assert ref["lit"].sum() >= min_lit and (ref["lit"][ref["id"] >= 0] == 0).sum() > 0  # lit and unlit hits
    assert np.all(g["lit"][g["id"] < 0] == 0)
    return view, len(bad)


def test_lit_parity_one_bump_full_frame(rg):
    w = scenes.config_parity_64()
    light = scenes.Light(pos=(1.0, 4.0, -3.0))
    g = _lit(rg, w, light)
    ref = oracle.trace_lit(w, light)
    _check(w, light, None, g, ref, min_hits=60, min_lit=30)


def test_lit_parity_twist_frame(rg):
    w = scenes.config_1080p_twist(width=32, height=24)
    light = scenes.Light(pos=(1.0, 6.0, -3.0))
    g = _lit(rg, w, light)
    ref = oracle.trace_lit(w, light)
    _check(w, light, None, g, ref, min_hits=200, min_lit=20)


def test_lit_parity_1080p_64_bumps_sample(rg):
    """The full 1920x1080 frame of 64 bumps, 32 spheres and the 10k-triangle mesh, lit, against
    the oracle on a seeded sample of the pixels."""
    w = scenes.config_1080p_64()
    light = scenes.Light()
    px = scenes.pixel_sample(w.n_pixels, 13, 400.0 / w.n_pixels)
    g = _lit(rg, w, light, px)
    ref = oracle.trace_lit(w, light, px)
    _check(w, light, px, g, ref, min_hits=50, min_lit=15)


def test_lit_flat_space_is_the_euclidean_lambert_law(rg):
    """No bumps: light geodesics are segments, so a lit hit's colour is albedo (0.1 + 0.9 n.l)
    with l the unit direction to the light from q = hit + 1e-3 n (oracle-free)."""
    w = scenes.config_parity_64()
    w.metric = scenes.Metric(center=np.zeros((0, 3), np.float32), amplitude=np.zeros(0, np.float32),
                             sigma=np.zeros((0, 3), np.float32))
    light = scenes.Light(pos=(1.0, 4.0, -3.0))
    g = _lit(rg, w, light)
    sph = np.asarray(w.scene.spheres, np.float64)
    hits = np.nonzero(g["id"] >= 0)[0]
    assert len(hits) >= 60
    L = np.array(light.pos)
    checked = 0
    for p in hits:
        P = g["hit"][p].astype(np.float64)
        c = sph[g["id"][p]]
        n = (P - c[:3]) / np.linalg.norm(P - c[:3])
        q = P + 1e-3 * n
        cos = n.dot((L - q) / np.linalg.norm(L - q))
        if g["lit"][p]:
            alb = np.asarray(w.scene.albedo, np.float64)[g["id"][p]]
            expect = np.floor(255.0 * np.clip(alb * (0.1 + 0.9 * cos), 0, 1) + 0.5)
            assert np.abs(g["rgba"][p, :3].astype(np.int64) - expect).max() <= 1, (p, cos)
            checked += 1
    assert checked >= 30


def test_lit_ragged_frame(rg):
    """A frame that leaves partial 8x4 tiles on both edges, against the oracle."""
    w = scenes.scaled(scenes.config_parity_64(), 67, 29)
    light = scenes.Light(pos=(1.0, 4.0, -3.0))
    g = _lit(rg, w, light)
    ref = oracle.trace_lit(w, light)
    _check(w, light, None, g, ref, min_hits=15, min_lit=10)


def test_lit_single_pixel(rg):
    """A 1x1 frame (one partial tile): its ray misses every object, so nothing is lit."""
    w = scenes.scaled(scenes.config_parity_64(), 1, 1)
    g = _lit(rg, w, scenes.Light(pos=(1.0, 4.0, -3.0)))
    ref = oracle.trace_lit(w, scenes.Light(pos=(1.0, 4.0, -3.0)))
    assert np.array_equal(g["id"], ref["id"]) and ref["id"][0] < 0
    assert g["lit"][0] == 0 and np.all(g["rgba"] == 0)


def test_lit_without_hits(rg):
    """An empty scene: no hit, nothing lit, every pixel black."""
    w = scenes.config_parity_64()
    w.scene = scenes.Scene(np.zeros((0, 4), np.float32), np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32),
                           np.full((1, 3), 0.8, np.float32))
    g = _lit(rg, w, scenes.Light())
    assert np.all(g["id"] < 0) and np.all(g["lit"] == 0) and np.all(g["rgba"] == 0)


def test_lit_parity_anisotropic_bump(rg):
    """An anisotropic bump (three spreads, Eq. 6.1): the light geodesics sum the anisotropic
    field and the Riemannian cosine uses its gradient."""
    w = scenes.config_parity_64()
    w.metric.sigma = np.array([[0.5, 0.6, 0.45]], np.float32)
    w.max_steps = 1000
    light = scenes.Light(pos=(1.0, 4.0, -3.0))
    g = _lit(rg, w, light)
    ref = oracle.trace_lit(w, light)
    _check(w, light, None, g, ref, min_hits=100, min_lit=50)


def test_lit_parity_composed_local_maps(rg):
    """Eight composed local diffeomorphisms through the lattice (Eq. 6.3, Theorem 5.1): the light
    geodesics march the pull-back metric and the cosine uses n^T (J^T J)^-1 n."""
    w = scenes.scaled(scenes.config_local_lattice(K=8), 32, 18)
    light = scenes.Light(pos=(0.5, 0.5, -1.5), max_steps=1500)
    g = _lit(rg, w, light)
    ref = oracle.trace_lit(w, light)
    _check(w, light, None, g, ref, min_hits=300, min_lit=100)


@pytest.mark.parametrize("config", ["parity_64", "1080p_64_320x180", "1080p_64_ragged"])
def test_lockstep_marches_give_the_per_lane_image(rg, config):
    """The warp's light geodesics marched in lockstep over shared bump lists (the default for
    isotropic bumps with a cull grid) and each lane marching on its own (schedule 1) give the
    same image bit for bit: every list holds the bumps nonzero at a lane's stage points in the
    order of the dense sums, and the Gauss-Newton decisions are the same."""
    if config == "parity_64":
        w, light = scenes.config_parity_64(), scenes.Light(pos=(1.0, 4.0, -3.0))
    elif config == "1080p_64_320x180":
        w, light = scenes.config_1080p_64(width=320, height=180), scenes.Light()
    else:
        w, light = scenes.config_1080p_64(width=83, height=45), scenes.Light(pos=(1.0, 4.0, -3.0))
    a = _lit(rg, w, light)
    b = _lit(rg, w, dataclasses.replace(light, schedule=1))
    for k in ("id", "hit", "rgba", "lit"):
        assert np.array_equal(a[k], b[k]), k
    assert a["lit"].sum() > 0 and (a["lit"][a["id"] >= 0] == 0).sum() > 0
