"""GPU vs oracle on the integer work of the hot path, bit for bit: cell
classes (fluid / interface / solid), ownership lists and contact pairs, on
identical particle inputs fed to both.  Per-owner fractions agree within the
arithmetic's rounding."""
import math

import numpy as np
import pytest

from helpers import gpu_lattice
from oracle import vlbref as O
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _random_disks(nx, ny, n, rmin, rmax, gap_min, seed):
    rng = W.SplitMix64(seed)
    xs, ys, rs = [], [], []
    tries = 0
    while len(xs) < n and tries < 200000:
        tries += 1
        r = rng.uniform(rmin, rmax)
        x = rng.uniform(r + 0.0, nx - r)
        y = rng.uniform(r + 0.0, ny - r)
        if all(math.hypot(x - a, y - b) >= r + c + gap_min for a, b, c in zip(xs, ys, rs)):
            xs.append(x); ys.append(y); rs.append(r)
    return xs, ys, rs


def _special_disks():
    # centres on corners, edges, quarter points; touching walls; a 4-owner cell
    xs = [10.0, 20.5, 30.25, 4.0, 60.0, 42.0, 39.0, 42.0, 39.0]
    ys = [10.0, 10.0, 11.75, 30.0, 4.5, 42.0, 42.0, 39.0, 39.0]
    rs = [4.0, 3.5, 2.75, 4.0, 4.5, 1.5, 1.5, 1.5, 1.5]
    return xs, ys, rs


def _case(nx, ny, xs, ys, rs):
    params = dict(nx=nx, ny=ny, tau_f=0.8, prandtl=0.7, rho_ratio=1.5, cv_ratio=2.0, k_ratio_default=3.0,
                  gravity=(0.0, -1e-5), beta=0.0, T_ref=1.0, T_fluid_init=1.0)
    return W.Case("raster", params, xs, ys, rs, [0.0] * len(xs))


@pytest.mark.parametrize("prec,tol", [("fp32", 3e-6), ("fp64", 1e-12)])
@pytest.mark.parametrize("which", ["special", "random"])
def test_cell_classes_and_owners_bit_exact(prec, tol, which):
    nx, ny = 97, 61
    if which == "special":
        xs, ys, rs = _special_disks()
    else:
        xs, ys, rs = _random_disks(nx, ny, 40, 1.2, 7.0, 0.05, seed=11)
    case = _case(nx, ny, xs, ys, rs)
    from paper_2410_23802_gb300 import vlb as V
    with gpu_lattice(case, precision=prec) as lat:
        count, owner, flag, fsp = V.vlb_get_solid_fraction(lat.h, nx, ny)
    ras = O.rasterise(nx, ny, xs, ys, rs)
    np.testing.assert_array_equal(count, ras.count)
    np.testing.assert_array_equal(owner, ras.owner)
    np.testing.assert_array_equal(flag, ras.flag)
    np.testing.assert_allclose(fsp, ras.fsp, rtol=0, atol=tol)
    if which == "special":
        assert count.max() == 4
    else:
        assert count.max() >= 2


def test_contact_pairs_bit_exact():
    nx, ny = 160, 120
    xs, ys, rs = _random_disks(nx, ny, 120, 2.0, 5.0, 0.01, seed=12)
    case = _case(nx, ny, xs, ys, rs)
    from paper_2410_23802_gb300 import vlb as V
    with gpu_lattice(case, precision="fp32") as lat:
        lat.step(0)
        pairs = V.vlb_get_contact_pairs(lat.h)
    ref = O.contact_pairs(np.array(xs), np.array(ys), np.array(rs), 2.0)
    assert len(ref) > 20
    assert [tuple(p) for p in pairs.tolist()] == ref
