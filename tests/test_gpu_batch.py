"""Batched launches, animated metrics, CUDA-graph replay and the autotuner (GPU)."""
import math

import numpy as np
import pytest

from paper_2005_05386_gb300 import scenes
from parity import assert_parity, compare, gpu_arrays

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rg():
    import torch
    import paper_2005_05386_gb300 as rg
    torch.cuda.set_device(0)
    return rg


def _small_instances():
    a = scenes.config_parity_64()
    b = scenes.config_1080p_64(width=160, height=90)
    c, amp, s = scenes.random_bumps(77, 13)
    d = scenes.config_1080p_64(width=96, height=54)
    d.metric = scenes.Metric(center=c, amplitude=amp, sigma=s)
    return [a, b, d]


def _same(x, y):
    for k in ("id", "steps", "rgba", "hit"):
        assert np.array_equal(x[k], y[k]), k


def _close(x, y, S):
    """Different kernels may contract multiply-adds differently: parity tolerance."""
    st = compare(x, dict(y, hit=y["hit"].astype(np.float64)), S)
    assert st["agree"] >= 0.999, st


@pytest.mark.parametrize("batch_params", [0, 1])
def test_batch_equals_separate_traces(rg, batch_params):
    """A batch traces each instance as rgeo_trace does (launch shape aside), whether its warps
    read the instance table from the kernel's parameter space (0) or shared-memory copies (1)."""
    saved = rg.rgeo_get_tuning()
    rg.rgeo_set_tuning(saved["rays_per_thread"], batch_params)
    try:
        ws = _small_instances()
        handles = [(rg.Metric(w.metric), rg.Scene(w.scene)) for w in ws]
        outs = [rg.alloc_outputs(w.n_pixels) for w in ws]
        batch = rg.Batch([rg.instance(w, m, s, o) for w, (m, s), o in zip(ws, handles, outs)])
        for _ in range(2):   # the second launch reuses the counters
            batch.launch()
            rg.rgeo_sync()
            for w, (m, s), o in zip(ws, handles, outs):
                ref = rg.trace(w, m, s)
                rg.rgeo_sync()
                _close(gpu_arrays(o), gpu_arrays(ref), w.scene.n_spheres)
    finally:
        rg.rgeo_set_tuning(saved["rays_per_thread"], saved["batch_params"])


def test_batch_parameter_space_equals_shared_copies(rg):
    """The two instance-table sources run the same arithmetic: identical images."""
    ws = _small_instances()
    handles = [(rg.Metric(w.metric), rg.Scene(w.scene)) for w in ws]
    res = []
    saved = rg.rgeo_get_tuning()
    try:
        for mode in (0, 1):
            rg.rgeo_set_tuning(saved["rays_per_thread"], mode)
            outs = [rg.alloc_outputs(w.n_pixels) for w in ws]
            rg.Batch([rg.instance(w, m, s, o) for w, (m, s), o in zip(ws, handles, outs)]).launch()
            rg.rgeo_sync()
            res.append([gpu_arrays(o) for o in outs])
    finally:
        rg.rgeo_set_tuning(saved["rays_per_thread"], saved["batch_params"])
    for a, b, w in zip(res[0], res[1], ws):
        _close(a, b, w.scene.n_spheres)


def test_batch_rejects_mixed_integrators(rg):
    a, b = scenes.config_parity_64(), scenes.config_parity_64()
    b.integrator = scenes.INTEGRATOR_EULER
    ha, hb = (rg.Metric(a.metric), rg.Scene(a.scene)), (rg.Metric(b.metric), rg.Scene(b.scene))
    oa, ob = rg.alloc_outputs(a.n_pixels), rg.alloc_outputs(b.n_pixels)
    with pytest.raises(rg.RgeoError) as e:
        rg.Batch([rg.instance(a, *ha, oa), rg.instance(b, *hb, ob)])
    assert e.value.status == rg.RGEO_EINVAL


def test_motion_matches_centres_set_on_the_host(rg):
    w = scenes.config_1080p_64(width=160, height=90)
    A, f, ph = scenes.motion(5, w.metric.n_bumps)
    m = rg.Metric(w.metric)
    rg.rgeo_metric_set_motion(m.handle, A, f, ph)
    t0 = 1.7
    rg.rgeo_metric_set_time(m.handle, t0)
    rg.rgeo_metric_advance(m.handle, 1.0 / 30.0)   # moves the centres to c(t0), then t += dt
    got = rg.trace(w, metric=m)
    rg.rgeo_sync()
    c = w.metric.center.astype(np.float64) + A * np.sin(2 * math.pi * f * t0 + ph)[:, None]
    w.metric.center = c.astype(np.float32)
    ref = rg.trace(w)
    rg.rgeo_sync()
    st = compare(gpu_arrays(got), dict(gpu_arrays(ref)), w.scene.n_spheres)
    assert st["agree"] >= 0.999 and st["hits"] > 1000, st


def test_graph_replay_of_animation_and_batch(rg):
    """A captured graph of [advance, batch launch] replays frame after frame with no host input
    and gives the same frames as direct calls."""
    import torch
    ws = _small_instances()[1:]
    handles = [(rg.Metric(w.metric), rg.Scene(w.scene)) for w in ws]
    for w, (m, _) in zip(ws, handles):
        A, f, ph = scenes.motion(9, w.metric.n_bumps)
        rg.rgeo_metric_set_motion(m.handle, A, f, ph)
    outs = [rg.alloc_outputs(w.n_pixels) for w in ws]
    batch = rg.Batch([rg.instance(w, m, s, o) for w, (m, s), o in zip(ws, handles, outs)])
    dt = 1.0 / 30.0
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for m, _ in handles:
            rg.rgeo_metric_advance(m.handle, dt, stream.cuda_stream)
        batch.launch(stream.cuda_stream)
    frames = []
    for m, _ in handles:
        rg.rgeo_metric_set_time(m.handle, 0.0)
    torch.cuda.synchronize()
    for _ in range(3):
        g.replay()
        torch.cuda.synchronize()
        frames.append([gpu_arrays(o) for o in outs])
    rg.rgeo_sync()
    # direct calls from the same start time
    for m, _ in handles:
        rg.rgeo_metric_set_time(m.handle, 0.0)
    for k in range(3):
        for m, _ in handles:
            rg.rgeo_metric_advance(m.handle, dt)
        batch.launch()
        rg.rgeo_sync()
        for o, ref in zip(outs, frames[k]):
            _same(gpu_arrays(o), ref)
    # the frames really move
    assert not np.array_equal(frames[0][0]["hit"], frames[2][0]["hit"])


def test_autotuner_returns_a_candidate_and_caches(rg, tmp_path, monkeypatch):
    """The tuner times every schedule of its candidate set, caches the winner, and the winner
    (like every candidate: no knob changes a result bit) reproduces the default image exactly."""
    from paper_2005_05386_gb300 import autotune
    monkeypatch.setenv("RGEO_TUNING_CACHE", str(tmp_path / "tuning.json"))
    w = scenes.config_1080p_64(width=256, height=144)
    first = autotune.tune(w, repeats=1)
    assert not first["cached"] and first["ms"] > 0
    assert {k: first[k] for k in autotune.KNOBS} in autotune.candidates(w)
    assert len(first["candidates"]) == len(autotune.candidates(w))
    second = autotune.tune(w, repeats=1)
    assert second["cached"] and all(second[k] == first[k] for k in autotune.KNOBS)
    ref = rg.trace(w)
    rg.rgeo_sync()
    tuned = autotune.apply(w, second)
    try:
        out = rg.trace(tuned)
        rg.rgeo_sync()
    finally:
        rg.rgeo_set_tuning()
    for k in ("id", "steps", "rgba", "hit"):
        assert np.array_equal(gpu_arrays(out)[k], gpu_arrays(ref)[k]), k


def test_batch16_full_size_against_oracle(rg):
    """The 16-instance batch at its full sizes (resolutions up to 1920x1080, 8-256 bumps), in the
    launch the benchmark times (one persistent launch over all instances), against the oracle
    on a seeded sample of each instance."""
    import oracle
    ws = scenes.config_batch16()
    scene = rg.Scene(ws[0].scene)
    metrics = [rg.Metric(w.metric) for w in ws]
    outs = [rg.alloc_outputs(w.n_pixels) for w in ws]
    rg.Batch([rg.instance(w, m, scene, o) for w, m, o in zip(ws, metrics, outs)]).launch()
    rg.rgeo_sync()
    oscene = oracle.Scene.from_desc(ws[0].scene)
    total, agreed = 0, 0.0
    for w, o in zip(ws, outs):
        px = scenes.pixel_sample(w.n_pixels, w.seed + 7, min(1.0, 300.0 / w.n_pixels))
        ref = oracle.trace(w, px, scene=oscene)
        st = compare(gpu_arrays(o, px), ref, w.scene.n_spheres)
        assert st["same_object"] >= 0.99 and st["agree"] >= 0.99, (w.name, st)
        total += len(px)
        agreed += st["agree"] * len(px)
    # the bar over the whole batch: >= 99.9 % of the sampled pixels agree
    assert total > 3000 and agreed / total >= 0.999, (agreed / total, total)
