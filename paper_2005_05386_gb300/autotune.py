"""Autotuner for the launch schedule of the geodesic tracer.

Candidates are timed on the GPU, through the C ABI, on a proxy of the workload:
the same metric, scene, camera and stepping at a reduced resolution (about a
million rays).  The proxy's best few are then timed again at full size, which
picks the winner: on the proxy alone, the winner for the 1080p animation was up to
1.4 % slower at full size than the default schedule.  Every knob changes the
schedule only: each lane sums its own bumps in the same order whatever shares its
warp, so every candidate gives the same image bit for bit.

  cull_grid        G of the bump-support cull grid (-1: dense sums over all bumps)
  rays_per_thread  1, or 2 (two rays share each bump pair; dense sums only)
  ctas_per_sm      persistent CTAs per SM (0: as many as fit, seven for the isotropic
                   graph metric; 5 or fewer take the 96-register build of the kernel)
  tile_shape       the refill tile a warp takes from the queue: 1 (8 x 4) or 2 (4 x 8, the default)
                   pixels (16 x 2 was measured slower at 1080p and is left out)
  sum_lists        culled bump sums from one list for as many RK4 steps as its reach
                   covers (0) or from one per right-hand side (1)
  batch_order      batches: instances by decreasing cost (0) or as given (1)
  refill           a warp takes new rays in generations of 32, once all of its rays have
                   finished (0, the default), or each lane as soon as its ray has finished (1);
                   the second is timed with the default CTAs per SM only

The candidate set is the product of the knobs that apply to the workload's metric
(the grid, list and thread knobs only to isotropic truncated bumps).  The winner is
cached per (device name, workload signature) in a JSON file (``$RGEO_TUNING_CACHE``,
default ``~/.cache/rgeo/tuning.json``).
"""
from __future__ import annotations

import dataclasses
import itertools
import json
import math
import os

from . import scenes

CANDIDATE_GRIDS = (-1, 96, 128, 192)
CANDIDATE_CTAS = (0, 6, 5)
CANDIDATE_TILES = (1, 2)
CANDIDATE_LISTS = (0, 1)
CANDIDATE_REFILL = (0, 1)
KNOBS = ("cull_grid", "rays_per_thread", "ctas_per_sm", "tile_shape", "sum_lists", "batch_order", "refill")


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


def proxy(work: scenes.Workload, rays: int = 1 << 20) -> scenes.Workload:
    px = work.width * work.height
    if px <= rays:
        return work
    f = math.sqrt(rays / px)
    return scenes.scaled(work, max(8, int(work.width * f)), max(4, int(work.height * f)))


def candidates(work: scenes.Workload, batch: bool = False):
    """Every schedule to time for ``work``: dicts over KNOBS."""
    m = work.metric
    iso = m.kind == scenes.METRIC_GRAPH_BUMPS and m.n_bumps > 0 and not (m.sigma != m.sigma[:, :1]).any()
    culled = iso and m.cutoff > 0
    orders = (0, 1) if batch else (0,)
    out = []
    if culled:
        for g, c, t, s, b, f in itertools.product(CANDIDATE_GRIDS, CANDIDATE_CTAS, CANDIDATE_TILES, CANDIDATE_LISTS,
                                                  orders, CANDIDATE_REFILL):
            if (g == -1 and s == 1) or (f == 1 and c != 0):
                continue  # dense sums take no lists; per-lane refill with the default CTAs only
            out.append(dict(cull_grid=g, rays_per_thread=1, ctas_per_sm=c, tile_shape=t, sum_lists=s,
                            batch_order=b, refill=f))
        out += [dict(cull_grid=-1, rays_per_thread=2, ctas_per_sm=0, tile_shape=t, sum_lists=0, batch_order=b,
                     refill=0) for t, b in itertools.product(CANDIDATE_TILES, orders)]
    else:
        for c, t, b, f in itertools.product(CANDIDATE_CTAS, CANDIDATE_TILES, orders, CANDIDATE_REFILL):
            if f == 1 and c != 0:
                continue
            out.append(dict(cull_grid=-1, rays_per_thread=1, ctas_per_sm=c, tile_shape=t, sum_lists=0,
                            batch_order=b, refill=f))
    return out


def set_schedule(choice: dict, batch_params: int = 0):
    """Sets the process-wide launch tuning of a schedule (its cull grid belongs to the metric)."""
    from . import rgeo_set_tuning
    rgeo_set_tuning(rays_per_thread=int(choice["rays_per_thread"]), batch_params=batch_params,
                    ctas_per_sm=int(choice["ctas_per_sm"]), tile_shape=int(choice["tile_shape"]),
                    batch_order=int(choice.get("batch_order", 0)), sum_lists=int(choice["sum_lists"]),
                    refill=int(choice.get("refill", 0)))


def tune(work: scenes.Workload, repeats: int = 2, use_cache: bool = True, verbose: bool = False,
         refine: int = 3) -> dict:
    """Best schedule for ``work`` on the current device: the KNOBS and its proxy time 'ms'.
    The ``refine`` fastest on the proxy are timed once more at full size ('full_ms'), and the
    fastest there wins."""
    import torch

    from . import Metric, Scene, alloc_outputs, rgeo_get_tuning, rgeo_set_tuning, rgeo_sync, trace

    dev = torch.cuda.get_device_name(torch.cuda.current_device())
    key = f"{dev}|{signature(work)}"
    db = _load() if use_cache else {}
    if use_cache and key in db and all(k in db[key] for k in KNOBS):
        return dict(db[key], cached=True)
    pw = proxy(work)
    saved = rgeo_get_tuning()

    def timed(w, cands, reps):
        scene = Scene(w.scene)
        out = alloc_outputs(w.n_pixels)
        metrics = {}
        res = []
        for cand in cands:
            g = cand["cull_grid"]
            if g not in metrics:
                metrics[g] = Metric(dataclasses.replace(w.metric, cull_grid=g))
            metric = metrics[g]
            set_schedule(cand, saved["batch_params"])
            trace(w, metric, scene, out)           # warm-up
            rgeo_sync()
            best = float("inf")
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                trace(w, metric, scene, out)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            rgeo_sync()
            res.append(best)
            if verbose:
                print(f"autotune {signature(w)} {cand} {best:.2f} ms", flush=True)
        return res

    try:
        cands = candidates(pw)
        results = [dict(c, ms=ms) for c, ms in zip(cands, timed(pw, cands, repeats))]
        results.sort(key=lambda r: r["ms"])
        top = [dict(r) for r in results[:max(1, refine)]]
        if pw is not work and len(top) > 1:
            for r, ms in zip(top, timed(work, [{k: r[k] for k in KNOBS} for r in top], 1)):
                r["full_ms"] = ms
            win = min(top, key=lambda r: r["full_ms"])
        else:
            win = top[0]
    finally:
        rgeo_set_tuning(**saved)
    if use_cache:
        db[key] = win
        _store(db)
    return dict(win, cached=False, candidates=results, refined=top)


def apply(work: scenes.Workload, choice: dict) -> scenes.Workload:
    """The workload with the tuned cull grid; sets the process-wide launch tuning."""
    from . import rgeo_get_tuning
    set_schedule(choice, rgeo_get_tuning()["batch_params"])
    return dataclasses.replace(work, metric=dataclasses.replace(work.metric, cull_grid=int(choice["cull_grid"])))
