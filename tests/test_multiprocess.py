"""The benchmark's multi-rank path on CPU (gloo, world size 2).

Rays shard with no data-path collective: each rank traces its own frame and the
only collectives are the timing barrier and the max over ranks.  These tests run
that host logic with two processes on the gloo backend, and the reference arm
(the FP64 oracle) under torchrun, where rank 0 alone works and prints.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank), RGEO_BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    w, r, local = bench.dist_setup(world)
    try:
        bench.barrier(w)
        q.put((r, w, local, bench.reduce_max(0.5 + r, w)))
    finally:
        dist.destroy_process_group()


def test_timing_collectives_take_the_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 2, 0, 1.5), (1, 2, 1, 1.5)]


def test_reference_arm_under_torchrun_prints_once():
    env = dict(os.environ, RGEO_BENCH_BACKEND="gloo")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--workload", "parity_64", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"


def _split_main(rank, world, port, q, W, H):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank), RGEO_BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist
    import bench
    import paper_2005_05386_gb300 as rg
    w, r, _ = bench.dist_setup(world)
    try:
        N = W * H
        px = rg.part_pixels(W, H, r, w)
        # stub outputs of this rank's part (what the kernels would write), zero elsewhere
        bufs = dict(id=torch.zeros(N, dtype=torch.int32), hit=torch.zeros(3, N, dtype=torch.float32),
                    steps=torch.zeros(N, dtype=torch.int32), rgba=torch.zeros(N, 4, dtype=torch.uint8))
        t = torch.from_numpy(px.astype(np.int64))
        bufs["id"][t] = t.to(torch.int32) - 2            # -2 .. N - 3: misses and budgets too
        bufs["hit"][:, t] = torch.stack([t * 0.5, -t * 0.25, t + 0.125]).to(torch.float32)
        bufs["steps"][t] = (t % 2000).to(torch.int32)
        bufs["rgba"][t] = torch.stack([t % 251 + 1, t % 7, t % 256, torch.full_like(t, 255)], 1).to(torch.uint8)
        bench.assemble_frame(bufs, w)
        q.put((r, px.tolist(), {k: v.numpy().copy() for k, v in bufs.items()} if r == 0 else None))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,W,H", [(2, 67, 29), (3, 64, 64), (2, 8, 4)])
def test_split_frame_covers_every_pixel_once_and_reassembles(world, W, H):
    """One frame over `world` ranks: the interleaved tile parts are disjoint and cover the frame
    (the kernels' own pixel mapping, through the library's host helper), and summing the ranks'
    zero-padded outputs onto rank 0 rebuilds every pixel's value exactly."""
    import numpy as np
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_main, args=(r, world, port, q, W, H)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=120) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    N = W * H
    parts = [set(g[1]) for g in got]
    assert sum(len(p) for p in parts) == N and set().union(*parts) == set(range(N))
    frame = got[0][2]
    t = np.arange(N)
    assert np.array_equal(frame["id"], (t - 2).astype(np.int32))
    assert np.array_equal(frame["hit"], np.stack([t * 0.5, -t * 0.25, t + 0.125]).astype(np.float32))
    assert np.array_equal(frame["steps"], (t % 2000).astype(np.int32))
    assert np.array_equal(frame["rgba"][:, 0], (t % 251 + 1).astype(np.uint8))
    assert (frame["rgba"][:, 3] == 255).all()
