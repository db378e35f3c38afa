"""Shared comparison of GPU traces against the FP64 oracle.

Bar: at least 99.9 % of the compared pixels agree, where a pixel agrees when
both sides report the same object (sphere index, the mesh as one object, MISS
or BUDGET) and, for hits, the hit points differ by at most 1e-4 scene units in
every coordinate and the RGBA8 colours by at most 2 in every channel.
"""
import numpy as np

HIT_TOL = 1e-4
COLOUR_TOL = 2
AGREE_MIN = 0.999


def objects(ids, S):
    ids = np.asarray(ids)
    return np.where(ids >= S, S, ids)


def gpu_arrays(out, pixels=None):
    gid = out["id"].cpu().numpy()
    ghit = out["hit"].cpu().numpy().T
    gsteps = out["steps"].cpu().numpy()
    grgba = out["rgba"].cpu().numpy()
    gdrift = out["drift"].cpu().numpy() if out.get("drift") is not None else None
    if pixels is not None:
        gid, ghit, gsteps, grgba = gid[pixels], ghit[pixels], gsteps[pixels], grgba[pixels]
        gdrift = gdrift[pixels] if gdrift is not None else None
    return dict(id=gid, hit=ghit, steps=gsteps, rgba=grgba, drift=gdrift)


def agree_mask(g, ref, S):
    """Per pixel: same object and, for hits, hit points within HIT_TOL and colours within
    COLOUR_TOL."""
    go, ro = objects(g["id"], S), objects(ref["id"], S)
    same = go == ro
    hit = same & (go >= 0)
    herr = np.zeros(len(go))
    cerr = np.zeros(len(go), dtype=np.int64)
    herr[hit] = np.abs(g["hit"][hit] - ref["hit"][hit]).max(axis=1)
    cerr[hit] = np.abs(g["rgba"][hit].astype(np.int64) - ref["rgba"][hit].astype(np.int64)).max(axis=1)
    return same & (herr <= HIT_TOL) & (cerr <= COLOUR_TOL)


def compare(g, ref, S):
    go, ro = objects(g["id"], S), objects(ref["id"], S)
    same = go == ro
    hit = same & (go >= 0)
    herr = np.zeros(len(go))
    cerr = np.zeros(len(go), dtype=np.int64)
    herr[hit] = np.abs(g["hit"][hit] - ref["hit"][hit]).max(axis=1)
    cerr[hit] = np.abs(g["rgba"][hit].astype(np.int64) - ref["rgba"][hit].astype(np.int64)).max(axis=1)
    agree = same & (herr <= HIT_TOL) & (cerr <= COLOUR_TOL)
    stats = dict(n=len(go), agree=float(agree.mean()), same_object=float(same.mean()),
                 hits=int(hit.sum()), hit_err_max=float(herr[hit].max()) if hit.any() else 0.0,
                 hit_err_p999=float(np.quantile(herr[hit], 0.999)) if hit.any() else 0.0,
                 colour_err_max=int(cerr[hit].max()) if hit.any() else 0,
                 same_steps=float((g["steps"][same] == ref["steps"][same]).mean()) if same.any() else 1.0,
                 budget_frac=float((ro == -2).mean()), miss_frac=float((ro == -1).mean()))
    return stats


def assert_parity(stats, min_hits=1):
    assert stats["hits"] >= min_hits, stats
    assert stats["agree"] >= AGREE_MIN, stats
