"""The CUDA path's raster functions (csrc/vlb_raster.cuh), compiled for the
host with nvcc, against the oracle's solid fraction on random and degenerate
cells: circles through cell corners, centres on corners and edges, tangent
edges.  Classes must agree exactly; fractions within 2e-7 (R + 1) in FP32
(the FP32 rounding of the disk centre relative to the cell, about 6e-8 R per
coordinate) and 1e-14 (R + 1)^2 in FP64 (the rounding of the oracle's
inclusion-exclusion of quadrant areas of size pi R^2)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import vlbref as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("raster") / "raster_host")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-x", "cu", "-I", os.path.join(ROOT, "paper_2410_23802_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "harness", "raster_host.cu"), "-o", exe], check=True)
    return exe


def _cases():
    rng = np.random.default_rng(21)
    rows = []
    # circles through cell corners: integer centre, integer radius with Pythagorean corners
    for (X, Y, R) in [(50.0, 300.0, 10.0), (20.0, 20.0, 5.0), (13.0, 17.0, 13.0), (8.5, 8.5, 4.0),
                      (10.0, 10.5, 4.0), (12.25, 9.75, 6.5)]:
        for j in range(int(Y - R) - 1, int(Y + R) + 2):
            for i in range(int(X - R) - 1, int(X + R) + 2):
                rows.append((X, Y, R, i, j))
    for _ in range(3000):
        R = rng.uniform(1.0, 32.0)
        X, Y = rng.uniform(40, 60, 2)
        ang = rng.uniform(0, 2 * np.pi)
        rr = R + rng.uniform(-1.5, 1.5)
        i, j = int(np.floor(X + rr * np.cos(ang))), int(np.floor(Y + rr * np.sin(ang)))
        rows.append((X, Y, R, i, j))
    return rows


def test_host_compiled_raster_matches_oracle(harness):
    rows = _cases()
    inp = "\n".join(f"{float(X)!r} {float(Y)!r} {float(R)!r} {i} {j}" for X, Y, R, i, j in rows) + "\n"
    out = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    worst32 = worst64 = 0.0
    for (X, Y, R, i, j), line in zip(rows, out):
        c32, f32, c64, f64 = line.split()
        ras = O.cell_flags(np.array([i]), np.array([j]), O.quantise(X), O.quantise(Y), O.quantise(R))[0]
        assert int(c32) == ras and int(c64) == ras, (X, Y, R, i, j)
        if ras == O.SOLID:
            ref = 1.0
        elif ras == O.FLUID:
            ref = 0.0
        else:
            ref = float(np.clip(O.cell_disk_area(float(i), i + 1.0, float(j), j + 1.0, X, Y, R), 0, 1))
        worst32 = max(worst32, abs(float(f32) - ref) / (R + 1.0))
        worst64 = max(worst64, abs(float(f64) - ref) / (R + 1.0) ** 2)
    assert worst32 < 2e-7, worst32
    assert worst64 < 1e-14, worst64
