"""Compositions of local diffeomorphisms (Section 6) on the GPU against the FP64 oracle.

The GPU pushes a second-order jet through the maps (the chain rule and Eq. 6.3 taken along
the velocity) and solves J a = -D^2 Phi[v, v]; the oracle forms the full Hessians by Eq. 6.3
and J^-1 as the paper's product of inverses.  Same bar as every image: >= 99.9 % of pixels
with the same object and hit points within 1e-4.
"""
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


def _run(rg, w, flags=0):
    out = rg.trace(w, flags=flags)
    rg.rgeo_sync()
    return gpu_arrays(out)


def test_single_local_map_full_frame(rg):
    """One local deformation p + f(p) v (Section 6, "Using diffeomorphism")."""
    w = scenes.scaled(scenes.config_local_lattice(K=1, seed=9), 64, 64)
    w.metric = scenes.local_maps(9, 1, lo=(0.0, 0.0, 0.5), hi=(1.0, 1.0, 1.5), with_field=False)
    st = compare(_run(rg, w), oracle.trace(w), w.scene.n_spheres)
    assert_parity(st, min_hits=1000)


@pytest.mark.parametrize("W,H", [(64, 64), (37, 21)])
def test_composition_of_eight_maps(rg, W, H):
    w = scenes.scaled(scenes.config_local_lattice(K=8), W, H)
    g = _run(rg, w)
    st = compare(g, oracle.trace(w), w.scene.n_spheres)
    assert_parity(st, min_hits=W * H // 3)


def test_composition_energy_is_conserved(rg):
    """g(v, v) = |J v|^2 is constant along a geodesic; the composition is smooth (untruncated),
    so the FP64 drift after up to 2000 RK4 steps stays at rounding level."""
    w = scenes.scaled(scenes.config_local_lattice(K=8), 48, 27)
    g = _run(rg, w, rg.RGEO_FLAG_ENERGY_DIAG)
    assert np.abs(g["drift"]).max() < 1e-4, np.abs(g["drift"]).max()


def test_local_batch_equals_separate_traces(rg):
    ws = [scenes.scaled(scenes.config_local_lattice(K=k, seed=s), 40, 24) for k, s in ((2, 3), (5, 4))]
    handles = [(rg.Metric(w.metric), rg.Scene(w.scene)) for w in ws]
    outs = [rg.alloc_outputs(w.n_pixels) for w in ws]
    rg.Batch([rg.instance(w, m, s, o) for w, (m, s), o in zip(ws, handles, outs)]).launch()
    rg.rgeo_sync()
    for w, (m, s), o in zip(ws, handles, outs):
        ref = rg.trace(w, m, s)
        rg.rgeo_sync()
        st = compare(gpu_arrays(o), dict(gpu_arrays(ref), hit=gpu_arrays(ref)["hit"].astype(np.float64)),
                     w.scene.n_spheres)
        assert st["agree"] >= 0.999, st
