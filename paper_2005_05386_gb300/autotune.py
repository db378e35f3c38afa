"""Autotuner for the launch schedule of the geodesic tracer.

Candidates are timed on the GPU, through the C ABI, on a proxy of the workload:
the same metric, scene, camera and stepping at a reduced resolution (about a
quarter of a million rays).  The tuned knobs change the schedule only, never the
result beyond float32 summation order:

  cull_grid        G of the bump-support cull grid (-1: dense sums over all bumps)
  rays_per_thread  1, or 2 (two rays share each bump pair; dense sums only)

The winner is cached per (device name, workload signature) in a JSON file
(``$RGEO_TUNING_CACHE``, default ``~/.cache/rgeo/tuning.json``).
"""
from __future__ import annotations

import dataclasses
import json
import math
import os

from . import scenes

CANDIDATE_GRIDS = (-1, 32, 48, 64, 96, 128)


def cache_path() -> str:
    return os.environ.get("RGEO_TUNING_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "rgeo", "tuning.json"))


def signature(work: scenes.Workload) -> str:
    m, s = work.metric, work.scene
    aniso = bool(m.n_bumps) and bool((m.sigma != m.sigma[:, :1]).any())
    px = work.width * work.height
    return (f"k{m.kind}-K{m.n_bumps}-a{int(aniso)}-c{m.cutoff:g}-S{s.n_spheres}-T{s.n_tris}-"
            f"px{2 ** round(math.log2(max(px, 1)))}-h{work.h:g}-n{work.max_steps}-i{work.integrator}")


def _load():
    try:
        return json.load(open(cache_path()))
    except Exception:
        return {}


def _store(db):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    json.dump(db, open(tmp, "w"), indent=1, sort_keys=True)
    os.replace(tmp, p)


def proxy(work: scenes.Workload, rays: int = 1 << 18) -> scenes.Workload:
    px = work.width * work.height
    if px <= rays:
        return work
    f = math.sqrt(rays / px)
    return scenes.scaled(work, max(8, int(work.width * f)), max(4, int(work.height * f)))


def candidates(work: scenes.Workload):
    m = work.metric
    iso = m.kind == scenes.METRIC_GRAPH_BUMPS and m.n_bumps > 0 and not (m.sigma != m.sigma[:, :1]).any()
    if not iso or m.cutoff <= 0:
        return [dict(cull_grid=-1, rays_per_thread=1)]
    out = [dict(cull_grid=g, rays_per_thread=1) for g in CANDIDATE_GRIDS]
    out.append(dict(cull_grid=-1, rays_per_thread=2))
    return out


def tune(work: scenes.Workload, repeats: int = 2, use_cache: bool = True, verbose: bool = False) -> dict:
    """Best schedule for ``work`` on the current device: {'cull_grid', 'rays_per_thread', 'ms'}."""
    import torch

    from . import Metric, Scene, alloc_outputs, rgeo_get_tuning, rgeo_set_tuning, rgeo_sync, trace

    dev = torch.cuda.get_device_name(torch.cuda.current_device())
    key = f"{dev}|{signature(work)}"
    db = _load() if use_cache else {}
    if use_cache and key in db:
        return dict(db[key], cached=True)
    pw = proxy(work)
    scene = Scene(pw.scene)
    out = alloc_outputs(pw.n_pixels)
    saved = rgeo_get_tuning()
    results = []
    try:
        for cand in candidates(pw):
            metric = Metric(dataclasses.replace(pw.metric, cull_grid=cand["cull_grid"]))
            rgeo_set_tuning(cand["rays_per_thread"], saved["batch_params"])
            trace(pw, metric, scene, out)           # warm-up
            rgeo_sync()
            best = float("inf")
            for _ in range(repeats):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                trace(pw, metric, scene, out)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            rgeo_sync()
            results.append(dict(cand, ms=best))
            if verbose:
                print(f"autotune {signature(pw)} {cand} {best:.2f} ms", flush=True)
    finally:
        rgeo_set_tuning(saved["rays_per_thread"], saved["batch_params"])
    win = min(results, key=lambda r: r["ms"])
    if use_cache:
        db[key] = win
        _store(db)
    return dict(win, cached=False, candidates=results)


def apply(work: scenes.Workload, choice: dict) -> scenes.Workload:
    """The workload with the tuned cull grid; sets the process-wide rays-per-thread."""
    from . import rgeo_get_tuning, rgeo_set_tuning
    rgeo_set_tuning(int(choice["rays_per_thread"]), rgeo_get_tuning()["batch_params"])
    return dataclasses.replace(work, metric=dataclasses.replace(work.metric, cull_grid=int(choice["cull_grid"])))
