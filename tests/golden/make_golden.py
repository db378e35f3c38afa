"""Writes the golden fixtures of this folder from the FP64 oracle (and nothing else).

Each fixture is the oracle's answer on seeded synthetic inputs of
``paper_2005_05386_gb300.scenes`` (the paper prints no worked example or
number, so no fixture holds a value printed in the paper).  They freeze the
oracle: ``tests/test_golden.py`` checks that the oracle still reproduces them
(on the CPU) and that the GPU path matches them at the parity bar (on a GPU).

Run from the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2005_05386_gb300 import scenes  # noqa: E402


def fixtures():
    """(name, citation, workload, pixel indices, light or None) of every fixture."""
    w0 = scenes.config_parity_64()
    ij = [(i, j) for j in range(0, w0.height, 2) for i in range(0, w0.width, 2)]
    px0 = np.array([j * w0.width + i for i, j in ij], dtype=np.int64)
    w1 = scenes.config_1080p_twist(width=24, height=16)
    px1 = np.arange(w1.width * w1.height, dtype=np.int64)
    w2 = scenes.config_1080p_64()
    px2 = scenes.pixel_sample(w2.n_pixels, 11, 200.0 / w2.n_pixels)
    return [
        ("graph_one_bump_64x64",
         "graph metric of one Gaussian bump (Eq. 5.2, Eq. 5.4, Eq. 6.1), RK4 (Eq. 3.3), segment tests "
         "(Section 4.1); 64x64 frame, every other pixel in each direction", w0, px0, None),
        ("twist_24x16",
         "pull-back metric of the twist map (Section 5.2, Eq. 5.6-5.8) through the 32-sphere / 10k-triangle "
         "scene; 24x16 frame, every pixel", w1, px1, None),
        ("graph_64_bumps_1080p_sample",
         "graph metric of 64 seeded bumps (Eq. 5.4, Eq. 6.1) at 1920x1080, h = 0.005, <= 2000 steps; "
         "seeded pixel sample (seed 11)", w2, px2, None),
        ("lit_one_bump_64x64",
         "Riemannian illumination (Section 4) of the one-bump 64x64 frame by a point light at (1, 4, -3): "
         "light geodesics by Gauss-Newton shooting, Riemannian Lambert cosine, shadows; every other pixel",
         w0, px0, scenes.Light(pos=(1.0, 4.0, -3.0))),
    ]


def trace(work, pixels, light):
    """The oracle's answer for a fixture (lit by ``light`` when it is not None)."""
    return oracle.trace(work, pixels) if light is None else oracle.trace_lit(work, light, pixels)


def write(name, cite, work, pixels, light):
    ref = trace(work, pixels, light)
    path = os.path.join(HERE, name + ".txt")
    with open(path, "w") as f:
        f.write(f"# {name}: FP64 oracle output ({cite}).\n")
        f.write("# Written by tests/golden/make_golden.py from the oracle alone.\n")
        f.write("# columns: pixel id steps hit_x hit_y hit_z r g b a (hit = end point for MISS/BUDGET)"
                + (" lit\n" if light is not None else "\n"))
        for k, p in enumerate(pixels):
            h = ref["hit"][k]
            c = ref["rgba"][k]
            f.write(f"{int(p)} {int(ref['id'][k])} {int(ref['steps'][k])} {h[0]:.17g} {h[1]:.17g} {h[2]:.17g} "
                    f"{int(c[0])} {int(c[1])} {int(c[2])} {int(c[3])}"
                    + (f" {int(ref['lit'][k])}\n" if light is not None else "\n"))
    return path


def read(name):
    """Returns (pixels, dict of id, steps, hit [n,3], rgba [n,4] and, for a lit fixture, lit) of a fixture."""
    rows = np.loadtxt(os.path.join(HERE, name + ".txt"), comments="#", ndmin=2)
    out = dict(id=rows[:, 1].astype(np.int32), steps=rows[:, 2].astype(np.int32), hit=rows[:, 3:6],
               rgba=rows[:, 6:10].astype(np.uint8))
    if rows.shape[1] > 10:
        out["lit"] = rows[:, 10].astype(np.int32)
    return rows[:, 0].astype(np.int64), out


if __name__ == "__main__":
    for name, cite, work, pixels, light in fixtures():
        print(write(name, cite, work, pixels, light))
