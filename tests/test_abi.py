"""The C-ABI library: loads, exports every declared symbol, and rejects invalid
arguments before touching the device.  CPU only (no compute calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rg():
    from paper_2005_05386_gb300 import _build
    _build.build()
    import paper_2005_05386_gb300 as rg
    rg.library()
    return rg


def _declared_functions():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            src = open(os.path.join(ROOT, "include", hdr)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(rgeo_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol(rg):
    declared = _declared_functions()
    assert len(declared) >= 10
    assert set(declared) == set(rg.EXPORTS)
    lib = ctypes.CDLL(rg.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name


def test_abi_version(rg):
    assert rg.rgeo_abi_version() == rg.RGEO_ABI_VERSION == 4


def _desc(rg, **kw):
    from paper_2005_05386_gb300 import scenes
    m = scenes.Metric(center=np.zeros((1, 3), np.float32), amplitude=np.ones(1, np.float32),
                      sigma=np.full((1, 3), 0.5, np.float32))
    for k, v in kw.items():
        setattr(m, k, v)
    return rg.metric_desc(m)


@pytest.mark.parametrize("bad", ["sigma", "amplitude", "kind", "quad", "reserved", "count"])
def test_metric_validation(rg, bad):
    d, keep = _desc(rg)
    if bad == "sigma":
        keep[2][0] = 0.0
    elif bad == "amplitude":
        keep[1][0] = np.nan
    elif bad == "kind":
        d.kind = 7
    elif bad == "quad":
        d.quad_A[1] = 0.5
    elif bad == "reserved":
        d.reserved[0] = 1
    elif bad == "count":
        d.n_bumps = rg.RGEO_MAX_BUMPS + 1
    with pytest.raises(rg.RgeoError) as e:
        rg.rgeo_metric_create(d)
    assert e.value.status == rg.RGEO_EINVAL
    assert rg.rgeo_last_error()


def _local_desc(rg, **kw):
    from paper_2005_05386_gb300 import scenes
    m = scenes.local_maps(1, 3)
    for k, v in kw.items():
        setattr(m, k, v)
    return rg.metric_desc(m)


@pytest.mark.parametrize("bad", ["not_diffeo", "count_zero", "count_max", "aniso", "quad", "affine", "direction",
                                 "nan_field", "reserved"])
def test_local_metric_validation(rg, bad):
    """Compositions of local maps: rejected before any device work (no GPU needed)."""
    from paper_2005_05386_gb300 import scenes
    if bad == "not_diffeo":   # |a| |v| e^-1/2 / sigma >= 1 on a map without a field
        m = scenes.local_maps(1, 3, with_field=False)
        m.amplitude = m.amplitude * np.float32(2.0)
        d, keep = rg.metric_desc(m)
    else:
        d, keep = _local_desc(rg)
    if bad == "count_zero":
        d.n_bumps = 0
    elif bad == "count_max":
        d.n_bumps = rg.RGEO_MAX_LOCAL_MAPS + 1
    elif bad == "aniso":
        keep[2][1] = keep[2][0] * 2
    elif bad == "quad":
        d.quad_A[0] = 1.0
    elif bad == "affine":
        d.affine_b[2] = 1.0
    elif bad == "direction":
        d.direction = None
    elif bad == "nan_field":
        keep[4][3] = np.nan
    elif bad == "reserved":
        d.reserved[2] = 1
    with pytest.raises(rg.RgeoError) as e:
        rg.rgeo_metric_create(d)
    assert e.value.status == rg.RGEO_EINVAL
    assert rg.rgeo_last_error()


def test_scene_validation(rg):
    alb = np.ones((2, 3), np.float32)
    with pytest.raises(rg.RgeoError) as e:
        rg.rgeo_scene_create(np.array([[0, 0, 0, -1.0]]), np.zeros((0, 3)), np.zeros((0, 3)), alb)
    assert e.value.status == rg.RGEO_EINVAL
    with pytest.raises(rg.RgeoError) as e:
        rg.rgeo_scene_create(np.zeros((0, 4)), np.zeros((3, 3)), np.array([[0, 1, 3]]), np.ones((1, 3)))
    assert "index" in str(e.value)
    with pytest.raises(rg.RgeoError):
        rg.rgeo_scene_create(np.zeros((0, 4)), np.zeros((0, 3)), np.zeros((0, 3)), np.full((1, 3), 2.0))


def test_trace_validation(rg):
    cam = rg.camera_struct(__import__("paper_2005_05386_gb300").scenes.Camera())
    out = rg.rgeo_outputs(1, 1, 1, 1, None)
    for args in [(None, None, cam, 4, 4, 0.01, 10, 0, 0, 0, out),]:
        with pytest.raises(rg.RgeoError) as e:
            rg.rgeo_trace(*args, stream=0)
        assert e.value.status == rg.RGEO_EINVAL
    # all remaining checks fail before the handles are dereferenced
    fake = 1
    for W, H, h, steps, integ, shade, flags, o in [
            (0, 4, 0.01, 10, 0, 0, 0, out), (4, 4, -1.0, 10, 0, 0, 0, out), (4, 4, float("nan"), 10, 0, 0, 0, out),
            (4, 4, 0.01, 0, 0, 0, 0, out), (4, 4, 0.01, 10, 5, 0, 0, out), (4, 4, 0.01, 10, 0, 9, 0, out),
            (4, 4, 0.01, 10, 0, 0, 64, out), (4, 4, 0.01, 10, 0, 0, 1, out),
            (65536, 65536, 0.01, 10, 0, 0, 0, out)]:
        with pytest.raises(rg.RgeoError) as e:
            rg.rgeo_trace(fake, fake, cam, W, H, h, steps, integ, shade, flags, o, stream=0)
        assert e.value.status == rg.RGEO_EINVAL
    bad_cam = rg.camera_struct(__import__("paper_2005_05386_gb300").scenes.Camera(up=(0.0, 0.0, 2.0)))
    with pytest.raises(rg.RgeoError) as e:
        rg.rgeo_trace(fake, fake, bad_cam, 4, 4, 0.01, 10, 0, 0, 0, out, stream=0)
    assert "parallel" in str(e.value)


def test_trace_lit_validation(rg):
    """rgeo_trace_lit checks the light before touching the device (fake handles are never used)."""
    from paper_2005_05386_gb300 import scenes
    cam = rg.camera_struct(scenes.Camera())
    out = rg.rgeo_outputs(1, 1, 1, 1, None)
    fake = 1
    st = rg.library().rgeo_trace_lit(fake, fake, ctypes.byref(cam), 4, 4, 0.01, 10, 0, None, ctypes.byref(out),
                                     None, None)
    assert st == rg.RGEO_EINVAL and "light" in rg.rgeo_last_error()
    good = scenes.Light()
    bad = [dict(h=0.0), dict(h=float("nan")), dict(pos=(0.0, float("inf"), 0.0)), dict(max_steps=0),
           dict(iters=-1), dict(tol=0.0), dict(delta=-1e-3), dict(schedule=2), dict(schedule=-1)]
    for kw in bad:
        import dataclasses
        lt = rg.light_struct(dataclasses.replace(good, **kw))
        with pytest.raises(rg.RgeoError) as e:
            rg.rgeo_trace_lit(fake, fake, cam, 4, 4, 0.01, 10, 0, lt, out, 0, stream=0)
        assert e.value.status == rg.RGEO_EINVAL, kw
    lt = rg.light_struct(good)
    lt.reserved[2] = 7
    with pytest.raises(rg.RgeoError) as e:
        rg.rgeo_trace_lit(fake, fake, cam, 4, 4, 0.01, 10, 0, lt, out, 0, stream=0)
    assert "reserved" in str(e.value)


def test_tuning_round_trip_and_validation(rg):
    """The launch tuning is host state: set and read back, defaults restored, bad values and
    nonzero reserved fields rejected (no device call)."""
    try:
        rg.rgeo_set_tuning(refill=1, tile_shape=1, sum_lists=2)
        t = rg.rgeo_get_tuning()
        assert (t["refill"], t["tile_shape"], t["sum_lists"]) == (1, 1, 2)
        rg.rgeo_set_tuning()
        t = rg.rgeo_get_tuning()
        assert (t["refill"], t["tile_shape"], t["sum_lists"], t["rays_per_thread"]) == (0, 2, 0, 1)
        for kw in (dict(refill=2), dict(refill=-1), dict(sum_lists=3), dict(tile_shape=4), dict(ctas_per_sm=33),
                   dict(wait_limit=-2), dict(rays_per_thread=3), dict(batch_order=2)):
            with pytest.raises(rg.RgeoError) as e:
                rg.rgeo_set_tuning(**kw)
            assert e.value.status == rg.RGEO_EINVAL, kw
        bad = rg.rgeo_tuning()
        bad.reserved[0] = 1
        assert rg.library().rgeo_set_tuning(ctypes.byref(bad)) == rg.RGEO_EINVAL
        assert "reserved" in rg.rgeo_last_error()
    finally:
        rg.rgeo_set_tuning()
