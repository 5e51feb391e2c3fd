"""Autotuner of the lattice kernel's build-time shape.

The tile height (VLB_TILE_Y: CTAs of 32 x TILE_Y threads, one per tile of as
many cells), the bound on resident CTAs per SM that sets the register
budget (VLB_LATTICE_MIN_BLOCKS) and, for batches, the form of the batched
step (VLB_BATCH_PERSISTENT: a persistent launch per step replayed from a
CUDA graph, or a CTA per tile plus a particle kernel per step) are
compile-time constants of the kernels.
The tuner builds the library once per candidate shape (each into a file of
its own), times a workload with each build in a fresh process on the GPU,
and records every result and the fastest shape in tuned.json, which
``build.build()`` then uses by default.

    python -m paper_2410_23802_gb300.autotune --workload cavity [--steps 200]
    python -m paper_2410_23802_gb300.autotune --workload channels --no-use

Workloads: ``cavity`` (2048^2, 2048 disks, FP32: the throughput case) and
``channels`` (256 channels of widths 64..256 stepped with vlb_step_batch).
The entry ``use`` names the workload whose winner the build takes.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys

from . import build as B

# (tile height, CTAs per SM the registers are budgeted for (None: 1024 threads
# per SM), default form of the batched step (None: the build's default, one
# CTA per tile; 1: persistent))
CANDIDATES = [(4, None, None), (2, None, None), (8, None, None), (4, 6, None), (4, None, 1), (8, None, 1)]


def candidates(workload: str) -> list[tuple]:
    """The shapes timed for a workload: the batched-step form matters only
    for batches."""
    return [c for c in CANDIDATES if workload == "channels" or c[2] is None]


def candidate_defines(tile_y: int, min_blocks: int | None, persistent: int | None = None) -> list[str]:
    d = [f"VLB_TILE_Y={tile_y}"]
    if min_blocks is not None:
        d.append(f"VLB_LATTICE_MIN_BLOCKS={min_blocks}")
    if persistent is not None:
        d.append(f"VLB_BATCH_PERSISTENT={persistent}")
    return d


_SHORT = {"VLB_TILE_Y": "y", "VLB_LATTICE_MIN_BLOCKS": "b", "VLB_BATCH_PERSISTENT": "p"}


def candidate_tag(defines: list[str]) -> str:
    """File name of a candidate build, e.g. tune_y4 or tune_y4_b6."""
    return "tune_" + "_".join(_SHORT[x.split("=")[0]] + x.split("=")[1] for x in defines)


_TIMER = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from paper_2410_23802_gb300 import vlb as V, workloads as W

def params(c):
    prm = {{k: v for k, v in c.params.items() if k != "precision"}}
    return V.vlb_params_default(precision=V.VLB_FP32, max_particles=max(len(c.x), 1), **prm)

cases = [W.cavity()] if {workload!r} == "cavity" else W.channels()
lats = []
for c in cases:
    lat = V.Lattice(params(c))
    lat.add_particles(np.column_stack([c.x, c.y]), c.radius, c.T0, k_ratio=c.k_ratio)
    lats.append(lat)
hs = [l.h for l in lats]
def run(n):
    if len(hs) == 1:
        V.vlb_step(hs[0], n)
    else:
        V.vlb_step_batch(hs, n)
    for h in hs:
        V.vlb_synchronize(h)
run(20)
best = None
for _ in range(3):
    t = time.perf_counter()
    run({steps})
    ms = 1e3 * (time.perf_counter() - t) / {steps}
    best = ms if best is None else min(best, ms)
print(json.dumps({{"ms_per_step": best, "cells": sum(c.cells for c in cases)}}))
"""


def time_candidate(lib: str, workload: str, steps: int) -> dict:
    """ms per step (best of three runs of `steps`, wall clock around a
    synchronised run) of the workload with the library `lib`."""
    code = _TIMER.format(root=B.ROOT, workload=workload, steps=steps)
    env = dict(os.environ, VLB_LIBRARY=lib)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def tune(workload: str, steps: int = 200, path: str = B.TUNED, use: bool = True, build=None, timer=None) -> dict:
    """Build and time every candidate, record the results for `workload` in
    tuned.json (kept entries of other workloads), and make this workload's
    winner the build's choice when `use`."""
    build = build or (lambda defines, out: B.build(defines=defines, out=out))
    timer = timer or time_candidate
    results = []
    for tile_y, mb, pers in candidates(workload):
        defines = candidate_defines(tile_y, mb, pers)
        lib = os.path.join(B.BUILD, candidate_tag(defines) + ".so")
        build(defines, lib)
        r = timer(lib, workload, steps)
        results.append({"defines": defines, "ms_per_step": r["ms_per_step"],
                        "mlups": r["cells"] / (r["ms_per_step"] * 1e-3) / 1e6})
    best = min(results, key=lambda r: r["ms_per_step"])
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        rec = {}
    rec[workload] = {"steps": steps, "results": results, "defines": best["defines"]}
    if use or "use" not in rec:
        rec["use"] = workload
    with open(path, "w") as fh:
        json.dump(rec, fh, indent=1)
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cavity", choices=["cavity", "channels"])
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--no-use", action="store_true", help="record only; the build keeps its choice")
    a = ap.parse_args()
    rec = tune(a.workload, a.steps, use=not a.no_use)
    print(json.dumps(rec[a.workload]))


if __name__ == "__main__":
    main()
