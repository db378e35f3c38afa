"""The allocation-free entry point rgeo_trace_noalloc against rgeo_trace.

Callers that cannot allocate device memory (a plugin whose host application
owns the device memory budget, a real-time loop where cudaMalloc is not
allowed, code with its own fixed arena) pass their inputs as device arrays they
own; the library keeps its scratch in a fixed device array.  Here the inputs
are staged with torch (the test may allocate; the entry point does not), the
same scene is traced through rgeo_trace with metric and scene handles, and the
outputs must agree within the parity tolerance of the other GPU tests, on two
calls in a row (the second reuses the scratch left by the first).

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2005_05386_gb300 import scenes
from parity import assert_parity, compare, gpu_arrays

pytestmark = pytest.mark.gpu


def _spheres_only(w):
    w.scene = scenes.Scene(w.scene.spheres, np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32),
                           w.scene.albedo)
    return w


def _noalloc(rg, torch, w):
    m = w.metric
    dev = "cuda"
    center = torch.tensor(np.ascontiguousarray(m.center, np.float32), device=dev)
    amp = torch.tensor(np.ascontiguousarray(m.amplitude, np.float32), device=dev)
    sigma = torch.tensor(np.ascontiguousarray(m.sigma[:, 0], np.float32), device=dev)
    sph = torch.tensor(np.ascontiguousarray(w.scene.spheres, np.float32), device=dev)
    alb = torch.tensor(np.ascontiguousarray(w.scene.albedo, np.float32), device=dev)
    out = rg.alloc_outputs(w.n_pixels)
    torch.cuda.synchronize()
    rg.rgeo_trace_noalloc(center.data_ptr(), amp.data_ptr(), sigma.data_ptr(), m.n_bumps, m.cutoff,
                          sph.data_ptr(), w.scene.n_spheres, alb.data_ptr(), rg.camera_struct(w.camera),
                          w.width, w.height, w.h, w.max_steps, w.integrator, w.shading, rg.outputs_struct(out))
    rg.rgeo_sync()
    return gpu_arrays(out)


def _reference(rg, w):
    out = rg.trace(w)
    rg.rgeo_sync()
    return gpu_arrays(out)


def test_noalloc_matches_trace_on_two_calls_in_a_row():
    import torch
    import paper_2005_05386_gb300 as rg
    torch.cuda.set_device(0)
    first = _spheres_only(scenes.config_1080p_64(width=320, height=180))
    second = _spheres_only(scenes.config_parity_64())
    for w, min_hits in ((first, 1000), (second, 60)):
        got = _noalloc(rg, torch, w)
        ref = _reference(rg, w)
        st = compare(got, dict(ref, hit=ref["hit"].astype(np.float64)), w.scene.n_spheres)
        assert_parity(st, min_hits=min_hits)


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
