"""Tracing with surrogate jumps (rgeo_trace_surrogate) on the GPU.

* With tau = 0 no jump is taken: rays are suspended and resumed between rounds,
  and the image must equal the plain tracer's bit for bit (the saved state is the
  whole ray state).
* Far-field training segments lie within the oracle's FP64 certificate and carry
  the oracle's residuals divided by the bound.
* A trained network takes jumps that replace RK4 work while the image stays within
  1e-3 scene units of the FP64 oracle on >= 99.9 % of pixels.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2005_05386_gb300 import scenes
from parity import gpu_arrays, objects

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rg():
    import torch
    import paper_2005_05386_gb300 as rg
    torch.cuda.set_device(0)
    return rg


def _work(W=160, H=90):
    return scenes.scaled(scenes.config_1080p_64(), W, H)


def _arrays(out):
    return {k: out[k].cpu().numpy() for k in ("id", "hit", "steps", "rgba")}


def test_tau_zero_equals_plain_trace(rg):
    w = _work()
    dm, ds = rg.Metric(w.metric), rg.Scene(w.scene)
    plain = rg.trace(w, dm, ds)
    rg.rgeo_sync()
    x = rg.Expmap(max_batch=4096, seed=1)
    out, st = rg.trace_surrogate(w, x, 0.0, metric=dm, scene=ds)
    rg.rgeo_sync()
    assert st["accepted"] == 0 and st["rejected"] > 0 and st["rounds"] > 1, st
    a, b = _arrays(out), _arrays(plain)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_far_field_generator_matches_oracle(rg):
    m = _work().metric
    eps, box, s_max, h = 0.01, 4.0, 0.5, 0.005
    X, T = rg.Expmap.generate(rg.Metric(m), 128, seed=5, box=box, s_max=s_max, h=h, accel_bound=eps)
    rg.rgeo_sync()
    X, T = X.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64)
    k = np.round(X[:, 6] * s_max / h)
    bounds = np.array([mlp.far_field_bound(m.center, m.amplitude, m.sigma, m.cutoff, row[:3] * box, kk * h)
                       for row, kk in zip(X, k)])
    assert (bounds <= eps * 1.001).all(), bounds.max()
    assert np.abs(T[:, :3]).max() <= 0.5 + 1e-6 and np.abs(T[:, 3:]).max() <= 1.0 + 1e-6
    R = mlp.segment_residuals(oracle.Metric.from_desc(m), X, box, s_max, h) / eps
    s = k * h
    Ug = np.concatenate([T[:, :3] * s[:, None] ** 2, T[:, 3:] * s[:, None]], axis=1)
    Ur = np.concatenate([R[:, :3] * s[:, None] ** 2, R[:, 3:] * s[:, None]], axis=1)
    # unscaled residual error in units of the bound: FP32 integration error / eps
    assert np.abs(Ug - Ur).max() * eps < 2e-6, np.abs(Ug - Ur).max() * eps


def test_trained_surrogate_removes_rk4_work_within_1e3_of_oracle(rg):
    """What the learned map does on this field: its jumps replace RK4 bump-term work while the
    image stays within 1e-3 of the FP64 oracle.  The certified far field is small here, so the
    work removed is small (about 1-2 % of the bump terms); the benchmark reports it with the
    wall-clock cost, and plain RK4 at its own largest step meeting the same bar is faster
    than the surrogate frame."""
    import torch
    w = _work(240, 135)
    dm, ds = rg.Metric(w.metric), rg.Scene(w.scene)
    eps = 0.01
    X, T = rg.Expmap.generate(dm, 1 << 21, seed=11, accel_bound=eps)
    x = rg.Expmap(max_batch=1 << 16, seed=7)
    g = torch.Generator(device="cuda").manual_seed(0)
    steps = 3000
    for it in range(steps):
        lr = 1e-4 + 0.5 * (2e-3 - 1e-4) * (1 + math.cos(math.pi * it / steps))
        idx = torch.randint(0, X.shape[0], (8192,), generator=g, device="cuda")
        x.train_step(X[idx], T[idx], lr)
    plain = rg.alloc_outputs(w.n_pixels, count=True)
    rg.trace(w, dm, ds, out=plain)
    out, st = rg.trace_surrogate(w, x, 0.1, accel_bound=eps, metric=dm, scene=ds,
                                 out=rg.alloc_outputs(w.n_pixels, count=True))
    rg.rgeo_sync()
    assert st["accepted"] > 0, st
    assert out["bump_evals"].item() < 0.998 * plain["bump_evals"].item(), (out["bump_evals"].item(),
                                                                         plain["bump_evals"].item())
    ref = oracle.trace(w)
    g = gpu_arrays(out)
    S = w.scene.n_spheres
    go, ro = objects(g["id"], S), objects(ref["id"], S)
    same = go == ro
    hit = same & (go >= 0)
    d = np.zeros(len(go))
    d[hit] = np.abs(g["hit"][hit] - ref["hit"][hit]).max(axis=1)
    ok = same & (d <= 1e-3)
    assert ok.mean() >= 0.999 and hit.sum() > 1000, (ok.mean(), hit.sum(), st)
    assert (out["steps"].cpu().numpy() <= w.max_steps).all()


def test_surrogate_rejects_bad_arguments(rg):
    w = _work(16, 16)
    dm, ds = rg.Metric(w.metric), rg.Scene(w.scene)
    x = rg.Expmap(max_batch=128, seed=1)
    bad = [dict(tau=-1.0), dict(tau=float("nan")), dict(tau=0.1, k_min=0), dict(tau=0.1, cool_check=0),
           dict(tau=0.1, box=0.0), dict(tau=0.1, s_max=0.001), dict(tau=0.1, accel_bound=-1.0)]
    for kw in bad:
        tau = kw.pop("tau")
        with pytest.raises(rg.RgeoError):
            rg.trace_surrogate(w, x, tau, metric=dm, scene=ds, **kw)
    tw = scenes.config_1080p_twist(width=16, height=16)
    with pytest.raises(rg.RgeoError):
        rg.trace_surrogate(tw, x, 0.1, scene=ds)
    aniso = scenes.Metric(center=w.metric.center, amplitude=w.metric.amplitude,
                          sigma=np.repeat(w.metric.sigma[:, :1], 3, axis=1) * np.array([1.0, 1.2, 0.9], np.float32))
    with pytest.raises(rg.RgeoError):
        rg.trace_surrogate(w, x, 0.1, accel_bound=0.01, metric=rg.Metric(aniso), scene=ds)
    with pytest.raises(rg.RgeoError):
        rg.Expmap.generate(rg.Metric(aniso), 128, seed=1, accel_bound=0.01)


def test_surrogate_full_1080p_sample_within_1e3_of_oracle(rg):
    """The benchmark's surrogate frame (1920x1080, far-field bound 0.03, tau 0.03, the network
    trained in one call exactly as the benchmark trains it) against the oracle on a seeded
    pixel sample at the 1e-3 bar, and the work its jumps remove against the plain frame.  The
    training step sums its gradients in a fixed order, so this network is the benchmark's, bit
    for bit, on a device with the same SM count.  The sample is 1 % of the frame (about 20,700
    pixels), so that the 0.999 bar tolerates about 20 misses; silhouette pixels miss at a rate
    of a few 1e-4, and a 0.2 % sample (4 tolerated misses) left the outcome to chance."""
    w = scenes.config_1080p_64()
    dm, ds = rg.Metric(w.metric), rg.Scene(w.scene)
    net = rg.Expmap(max_batch=1 << 18, seed=7)
    net.train(dm, n_segments=1 << 22, steps=8000, batch=8192, lr_max=2e-3, lr_min=1e-4, seed=11, accel_bound=0.03)
    plain = rg.alloc_outputs(w.n_pixels, count=True)
    rg.trace(w, dm, ds, out=plain)
    out, st = rg.trace_surrogate(w, net, 0.03, accel_bound=0.03, metric=dm, scene=ds,
                                 out=rg.alloc_outputs(w.n_pixels, count=True))
    rg.rgeo_sync()
    # jumps replace RK4 work on many rays, and the bump terms they save are a measurable
    # share of the frame's (the certified far field of this field is small: about 1.6 %)
    ratio = out["bump_evals"].item() / plain["bump_evals"].item()
    assert st["accepted"] > 200_000 and ratio < 0.995, (st, ratio)
    px = scenes.pixel_sample(w.n_pixels, 1234, 0.01)
    ref = oracle.trace(w, px)
    g = gpu_arrays(out, px)
    S = w.scene.n_spheres
    go, ro = objects(g["id"], S), objects(ref["id"], S)
    same = go == ro
    hit = same & (go >= 0)
    d = np.zeros(len(go))
    d[hit] = np.abs(g["hit"][hit] - ref["hit"][hit]).max(axis=1)
    ok = same & (d <= 1e-3)
    assert ok.mean() >= 0.999 and hit.sum() > 2500, (ok.mean(), (~ok).sum(), len(ok), hit.sum())
