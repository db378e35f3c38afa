"""The allocation-free entry point rgeo_trace_noalloc against rgeo_trace and the oracle.

Callers that cannot allocate device memory (a plugin whose host application
owns the device memory budget, a real-time loop where cudaMalloc is not
allowed, code with its own fixed arena) pass their inputs as device arrays they
own; the library keeps its scratch in a fixed device array.  Here the inputs
are staged with torch (the test may allocate; the entry point does not), the
same scene is traced through rgeo_trace with metric and scene handles, and the
outputs must agree within the parity tolerance of the other GPU tests, on two
calls in a row (the second reuses the scratch left by the first); both are also
held to the FP64 oracle.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
from paper_2005_05386_gb300 import scenes
from parity import assert_parity, compare, gpu_arrays

pytestmark = pytest.mark.gpu


def _spheres_only(w):
    w.scene = scenes.Scene(w.scene.spheres, np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32),
                           w.scene.albedo)
    return w


def _inputs(torch, w):
    m = w.metric
    dev = "cuda"
    return dict(center=torch.tensor(np.ascontiguousarray(m.center, np.float32).reshape(-1), device=dev),
                amp=torch.tensor(np.ascontiguousarray(m.amplitude, np.float32), device=dev),
                sigma=torch.tensor(np.ascontiguousarray(np.asarray(m.sigma).reshape(-1, 3)[:, 0], np.float32),
                                   device=dev),
                sph=torch.tensor(np.ascontiguousarray(w.scene.spheres, np.float32), device=dev),
                alb=torch.tensor(np.ascontiguousarray(w.scene.albedo, np.float32), device=dev))


def _call(rg, w, t, out, sph_ptr=None):
    m = w.metric
    ptr = lambda x: x.data_ptr() if x.numel() else 0  # noqa: E731
    rg.rgeo_trace_noalloc(ptr(t["center"]), ptr(t["amp"]), ptr(t["sigma"]), m.n_bumps, m.cutoff,
                          sph_ptr if sph_ptr is not None else ptr(t["sph"]), w.scene.n_spheres, t["alb"].data_ptr(),
                          rg.camera_struct(w.camera), w.width, w.height, w.h, w.max_steps, w.integrator, w.shading,
                          rg.outputs_struct(out))


def _noalloc(rg, torch, w):
    t = _inputs(torch, w)
    out = rg.alloc_outputs(w.n_pixels)
    torch.cuda.synchronize()
    _call(rg, w, t, out)
    rg.rgeo_sync()
    return gpu_arrays(out)


def _reference(rg, w):
    out = rg.trace(w)
    rg.rgeo_sync()
    return gpu_arrays(out)


def _rg():
    import torch
    import paper_2005_05386_gb300 as rg
    torch.cuda.set_device(0)
    return rg, torch


def test_noalloc_matches_trace_and_oracle_on_two_calls_in_a_row():
    rg, torch = _rg()
    first = _spheres_only(scenes.config_1080p_64(width=320, height=180))
    second = _spheres_only(scenes.config_parity_64())
    for w, min_hits, px in ((first, 1000, scenes.pixel_sample(320 * 180, 3, 0.05)), (second, 60, None)):
        got = _noalloc(rg, torch, w)
        ref = _reference(rg, w)
        st = compare(got, dict(ref, hit=ref["hit"].astype(np.float64)), w.scene.n_spheres)
        assert_parity(st, min_hits=min_hits)
        o = oracle.trace(w, px)
        sel = (lambda a: a) if px is None else (lambda a: a[px])
        g = {k: sel(v) for k, v in got.items() if v is not None}
        assert_parity(compare(g, o, w.scene.n_spheres), min_hits=min_hits // 20)


def test_noalloc_allocates_nothing_after_its_first_call():
    """Once the library's module is loaded (first call), further calls leave the device's free
    memory unchanged."""
    rg, torch = _rg()
    w = _spheres_only(scenes.config_parity_64())
    t = _inputs(torch, w)
    out = rg.alloc_outputs(w.n_pixels)
    torch.cuda.synchronize()
    _call(rg, w, t, out)
    rg.rgeo_sync()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _call(rg, w, t, out)
    rg.rgeo_sync()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_inert_bumps_and_no_bumps():
    """A bump with a NaN value or a spread <= 0 is inert: the frame equals the one traced
    without it.  With no bumps every ray is a straight line (rgeo_trace of the empty metric)."""
    rg, torch = _rg()
    base = _spheres_only(scenes.config_1080p_64(width=160, height=90))
    K = base.metric.n_bumps
    for bad in ("nan", "sigma0"):
        w = _spheres_only(scenes.config_1080p_64(width=160, height=90))
        c = np.array(w.metric.center, np.float32)
        a = np.array(w.metric.amplitude, np.float32)
        s = np.array(w.metric.sigma, np.float32)
        if bad == "nan":
            c[5, 1] = np.nan
        else:
            s[5, :] = 0.0
        w.metric = scenes.Metric(center=c, amplitude=a, sigma=s, cutoff=w.metric.cutoff)
        got = _noalloc(rg, torch, w)
        keep = np.arange(K) != 5
        ref_w = _spheres_only(scenes.config_1080p_64(width=160, height=90))
        ref_w.metric = scenes.Metric(center=c[keep], amplitude=a[keep], sigma=np.array(base.metric.sigma)[keep],
                                     cutoff=base.metric.cutoff)
        ref = _reference(rg, ref_w)
        st = compare(got, dict(ref, hit=ref["hit"].astype(np.float64)), w.scene.n_spheres)
        assert_parity(st, min_hits=500)
    w = _spheres_only(scenes.config_parity_64())
    w.metric = scenes.Metric(cutoff=w.metric.cutoff)
    got = _noalloc(rg, torch, w)
    ref = _reference(rg, w)
    for k in ("id", "steps", "rgba", "hit"):
        assert np.array_equal(got[k], ref[k]), k
    assert (got["id"] >= 0).sum() > 60 and (got["steps"] == 0).all()


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import paper_2005_05386_gb300 as rg
    cam = rg.camera_struct(scenes.Camera())
    out = rg.rgeo_outputs(1, 1, 1, 1, None)
    with pytest.raises(rg.RgeoError) as e:
        rg.rgeo_trace_noalloc(1, 1, 1, rg.RGEO_NOALLOC_MAX_BUMPS + 1, 4.0, 1, 1, 1, cam, 8, 8, 0.01, 10, 0, 0,
                              out, stream=0)
    assert e.value.status == rg.RGEO_EINVAL and "n_bumps" in str(e.value)
    with pytest.raises(rg.RgeoError) as e:
        rg.rgeo_trace_noalloc(1, 1, 1, 1, 4.0, 1, rg.RGEO_NOALLOC_MAX_SPHERES + 1, 1, cam, 8, 8, 0.01, 10, 0, 0,
                              out, stream=0)
    assert e.value.status == rg.RGEO_EINVAL and "n_spheres" in str(e.value)


def test_noalloc_rejects_misaligned_and_host_arrays():
    """Both checks run on the host before anything is enqueued: the kernels never see the
    rejected pointers."""
    rg, torch = _rg()
    w = _spheres_only(scenes.config_parity_64())
    t = _inputs(torch, w)
    out = rg.alloc_outputs(w.n_pixels)
    torch.cuda.synchronize()
    with pytest.raises(rg.RgeoError) as e:
        _call(rg, w, t, out, sph_ptr=t["sph"].data_ptr() + 4)
    assert e.value.status == rg.RGEO_EINVAL and "aligned" in str(e.value)
    host = np.ascontiguousarray(w.scene.spheres, np.float32)
    with pytest.raises(rg.RgeoError) as e:
        _call(rg, w, t, out, sph_ptr=host.ctypes.data)
    assert e.value.status == rg.RGEO_EINVAL and "device" in str(e.value)
    _call(rg, w, t, out)  # the valid call still works
    rg.rgeo_sync()
