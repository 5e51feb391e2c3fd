"""Pins of the oracle's solid-fraction field (Sec. 2: f_s is the volume
fraction of solid in each cell, fixed by the particle position).

* the quadrant area against adaptive quadrature of the chord length;
* the per-cell area against brute-force subsampling (error <= 4/N at N^2
  samples per cell);
* the sum over cells of an interior disk against pi R^2;
* the integer cell classes against a direct corner-by-corner test in exact
  Python integers, and against the areas they imply;
* several owners of one cell: ascending ids, fractions scaled to sum 1."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import vlbref as V


def _chord_length(u, b, R):
    if abs(u) >= R:
        return 0.0
    s = math.sqrt(R * R - u * u)
    return max(0.0, min(b, s) + s)


@pytest.mark.parametrize("R", [3.0, 8.0, 10.0])
def test_quadrant_area_against_quadrature(R):
    rng = np.random.default_rng(5)
    for a, b in rng.uniform(-1.3 * R, 1.3 * R, size=(40, 2)):
        hi = min(a, R)
        ref = 0.0 if hi <= -R else integrate.quad(lambda u: _chord_length(u, b, R), -R, hi,
                                                  epsabs=1e-13, epsrel=1e-13, limit=200,
                                                  points=[p for p in (-math.sqrt(max(R*R-b*b, 0)), math.sqrt(max(R*R-b*b, 0))) if -R < p < hi])[0]
        assert abs(float(V.quadrant_area(a, b, R)) - ref) < 1e-10


@pytest.mark.parametrize("X,Y,R", [(10.3, 11.7, 8.0), (16.0, 16.0, 10.0), (12.51, 9.25, 4.5)])
def test_area_sum_is_disk_area(X, Y, R):
    ras = V.rasterise(32, 32, [X], [Y], [R])
    assert abs(ras.fs.sum() - math.pi * R * R) < 1e-11


def test_area_against_subsampling():
    N = 1024
    X, Y, R = 6.37, 5.81, 3.9
    ras = V.rasterise(13, 12, [X], [Y], [R])
    t = (np.arange(N) + 0.5) / N
    worst = 0.0
    for j in range(12):
        for i in range(13):
            xs = i + t
            ys = j + t
            inside = ((xs[None, :] - X) ** 2 + (ys[:, None] - Y) ** 2) <= R * R
            frac = inside.mean()
            worst = max(worst, abs(frac - ras.fs[j, i]))
    assert worst <= 4.0 / N


def _brute_flag(i, j, Xq, Yq, Rq):
    Q = 1 << V.QBITS
    corners = [(i * Q, j * Q), ((i + 1) * Q, j * Q), (i * Q, (j + 1) * Q), ((i + 1) * Q, (j + 1) * Q)]
    if all((cx - Xq) ** 2 + (cy - Yq) ** 2 <= Rq * Rq for cx, cy in corners):
        return V.SOLID
    px = min(max(Xq, i * Q), (i + 1) * Q)
    py = min(max(Yq, j * Q), (j + 1) * Q)
    if (px - Xq) ** 2 + (py - Yq) ** 2 >= Rq * Rq:
        return V.FLUID
    return V.INTERFACE


def test_flags_against_exact_integer_corner_test():
    rng = np.random.default_rng(6)
    # include centres on cell corners, edges and centres, plus random ones
    cases = [(8.0, 8.0, 4.0), (8.5, 8.5, 4.0), (8.0, 8.5, 3.5), (8.25, 7.75, 5.0)]
    cases += [tuple(v) for v in np.column_stack([rng.uniform(6, 10, 12), rng.uniform(6, 10, 12), rng.uniform(2, 5, 12)])]
    for X, Y, R in cases:
        ras = V.rasterise(17, 17, [X], [Y], [R])
        Xq, Yq, Rq = int(V.quantise(X)), int(V.quantise(Y)), int(V.quantise(R))
        for j in range(17):
            for i in range(17):
                fl = _brute_flag(i, j, Xq, Yq, Rq)
                got = int(ras.flag[j, i, 0]) if ras.count[j, i] else V.FLUID
                assert got == fl, (X, Y, R, i, j)
                a = float(V.cell_disk_area(i, i + 1.0, j, j + 1.0, X, Y, R))
                if fl == V.SOLID:
                    assert ras.fs[j, i] == 1.0 and abs(a - 1) < 1e-9
                elif fl == V.FLUID:
                    assert ras.fs[j, i] == 0.0 and a < 1e-9
                else:
                    assert 0.0 <= ras.fs[j, i] <= 1.0


def test_two_owners_scaled_and_ordered():
    # two overlapping disks: cells in the lens have two owners
    ras = V.rasterise(30, 20, [16.0, 10.0], [10.0, 10.0], [5.0, 5.0])
    two = ras.count == 2
    assert two.any()
    assert (ras.owner[two][:, 0] == 0).all() and (ras.owner[two][:, 1] == 1).all()
    assert (ras.fs <= 1.0 + 1e-15).all()
    # cells solid for both have each fraction scaled to 1/2
    both_solid = two & (ras.flag[:, :, 0] == V.SOLID) & (ras.flag[:, :, 1] == V.SOLID)
    assert both_solid.any()
    np.testing.assert_allclose(ras.fsp[both_solid][:, :2], 0.5, atol=1e-15)


def test_bounding_box_clipped_at_walls():
    ras = V.rasterise(20, 20, [4.5], [3.0], [4.0])
    # the disk sticks out of the domain: only the inside area is counted
    ref = sum(float(V.cell_disk_area(i, i + 1.0, j, j + 1.0, 4.5, 3.0, 4.0)) for i in range(20) for j in range(20))
    assert abs(ras.fs.sum() - ref) < 1e-12
    assert ras.fs.sum() < math.pi * 16
