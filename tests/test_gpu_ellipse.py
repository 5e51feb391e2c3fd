"""Elliptical particles (Sec. 3.2, reading R13) and the fully developed
outflow boundary (reading R14) on the GPU against the FP64 oracle.

* Raster: ellipses of several shapes and angles, with disks beside them,
  vlb_get_solid_fraction against the oracle's raster: counts, owners and
  classes equal except where the oracle's own FP64 decision sits within
  1e-12 of the threshold (the two sides evaluate cos and sin of the angle
  separately and may differ in the last bit there); fractions within FP32
  rounding.
* The paper's elliptical-particle channel (Sec. 3.2: width 104 cells, a = 13,
  b = 6.5, released at 45 degrees, open bottom), shortened to 6 widths, over
  500 steps: FP32 rho, u within 1e-5 relative L2 over the stacked snapshots,
  particle position and angle within 1e-4; FP64 within 1e-9.
* The mirror image of the release (x -> W - x, theta -> -theta) stays its
  mirror image on the GPU, to FP32 rounding."""
import math

import numpy as np
import pytest

from helpers import gpu_lattice, oracle_sim, rel_l2
from oracle import vlbref as O
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _near_tie(i, j, X, Y, a, b, th, tol=1e-12):
    """Whether the oracle's class decision for cell (i, j) is within tol of
    its threshold (a corner's or an edge minimum's quadratic form near 1)."""
    c, s = math.cos(th), math.sin(th)
    corners = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
    uv = [O.ellipse_frame(float(x), float(y), X, Y, a, b, c, s) for x, y in corners]
    qs = [u * u + v * v for u, v in uv]
    for k in range(4):
        (u0, v0), (u1, v1) = uv[k], uv[(k + 1) % 4]
        du, dv = u1 - u0, v1 - v0
        t = min(max(-(u0 * du + v0 * dv) / (du * du + dv * dv), 0.0), 1.0)
        qs.append((u0 + t * du) ** 2 + (v0 + t * dv) ** 2)
    return min(abs(q - 1.0) for q in qs) < tol


@pytest.mark.parametrize("prec,tol", [("fp32", 3e-6), ("fp64", 1e-12)])
def test_ellipse_raster_matches_oracle(prec, tol):
    from paper_2410_23802_gb300 import vlb as V
    nx, ny = 120, 90
    xs = [25.3, 62.0, 95.7, 30.0, 80.25]
    ys = [30.6, 45.2, 28.0, 70.5, 72.0]
    a = [13.0, 9.5, 7.0, 6.0, 5.5]
    b = [6.5, 2.5, 7.0, 3.0, 5.5]   # two disks among them
    th = [math.pi / 4, -1.1, 0.0, 2.7, 0.0]
    case = W.Case("ellipses", dict(nx=nx, ny=ny, tau_f=0.8, prandtl=0.7, rho_ratio=1.5, cv_ratio=2.0,
                                   k_ratio_default=3.0, gravity=(0.0, -1e-5), beta=0.0, T_ref=1.0, T_fluid_init=1.0),
                  xs, ys, a, [0.0] * 5, semi_minor=b, theta0=th)
    with gpu_lattice(case, precision=prec) as lat:
        count, owner, flag, fsp = V.vlb_get_solid_fraction(lat.h, nx, ny)
    ras = O.rasterise_shapes(nx, ny, xs, ys, a, b, th)
    bad = np.argwhere((count != ras.count) | (owner != ras.owner).any(axis=2) | (flag != ras.flag).any(axis=2))
    for j, i in bad:
        assert any(_near_tie(i, j, xs[p], ys[p], a[p], b[p], th[p]) for p in range(5) if a[p] != b[p]), (i, j)
    assert len(bad) <= 2
    ok = np.ones((ny, nx), dtype=bool)
    ok[tuple(bad.T)] = False
    np.testing.assert_allclose(fsp[ok], ras.fsp[ok], rtol=0, atol=tol)
    assert abs(fsp.sum() - sum(math.pi * p * q for p, q in zip(a, b))) < 1e-3


SNAP, NSNAP = 100, 5


@pytest.fixture(scope="module")
def channel_ref():
    sim = oracle_sim(W.ellipse_sedimentation(length_w=6.0))
    out = []
    for _ in range(NSNAP):
        sim.step(SNAP)
        out.append(({k: v.copy() for k, v in sim.fields().items()}, sim.particle_state()))
    return out


@pytest.mark.parametrize("prec,tol,ptol", [("fp32", 1e-5, 1e-4), ("fp64", 1e-9, 1e-9)])
def test_ellipse_channel_with_open_bottom_matches_oracle(channel_ref, prec, tol, ptol):
    got = []
    with gpu_lattice(W.ellipse_sedimentation(length_w=6.0, precision=prec), precision=prec) as lat:
        for _ in range(NSNAP):
            lat.step(SNAP)
            got.append((lat.fields(), lat.particles()))
    st = lambda runs, k: np.stack([r[0][k] for r in runs])  # noqa: E731
    e_rho = rel_l2(st(got, "rho"), st(channel_ref, "rho"))
    e_u = rel_l2(np.stack([st(got, "ux"), st(got, "uy")]), np.stack([st(channel_ref, "ux"), st(channel_ref, "uy")]))
    print(f"ellipse channel {prec}: rho {e_rho:.2e} u {e_u:.2e}")
    assert e_rho < tol and e_u < tol
    for (gf, gp), (rf, rp) in zip(got, channel_ref):
        for k in ("x", "y", "theta"):
            assert abs(gp[k][0] - rp[k][0]) < ptol, (k, gp[k][0], rp[k][0])
    assert abs(channel_ref[-1][1]["theta"][0] - math.pi / 4) > 1e-4  # it turns
    assert abs(got[-1][1]["uy"][0]) > 1e-3  # and settles


def test_ellipse_mirror_release_stays_mirrored():
    W_ = 104
    runs = []
    for sign in (1.0, -1.0):
        c = W.ellipse_sedimentation(length_w=6.0, theta0=sign * math.pi / 4, x_offset=sign * 3.0)
        with gpu_lattice(c, precision="fp32") as lat:
            lat.step(400)
            runs.append(lat.particles())
    p1, p2 = runs
    assert abs(p1["x"][0] - (W_ - p2["x"][0])) < 1e-4 and abs(p1["y"][0] - p2["y"][0]) < 1e-4
    assert abs(p1["theta"][0] + p2["theta"][0]) < 1e-5
