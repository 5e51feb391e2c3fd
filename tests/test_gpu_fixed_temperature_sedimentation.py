"""The held-temperature reading (R11) against the paper's Table 4: the cold
disk held at T_c settling in a channel of width 4D drifts to an equilibrium
distance from the wall.  For Gr = 1000 the time-averaged x* over
t* = 120..200 must lie within 0.1 of the paper's 2.91 (the five methods in
Table 4 spread over 2.76..2.91) and the particle must have stopped drifting.
(Measured: 2.855.  Gr = 2000 gives 2.850 against 2.74, and Gr = 4500 settles
on the centreline instead of oscillating with amplitude 1.27: the paper does
not say how it holds the temperature, and those two regimes do not come out
of this reading; they are reported, not asserted.)"""
import json
import os

import numpy as np
import pytest

from helpers import gpu_lattice
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fixed_temperature_sedimentation_table4.json")


def test_gr1000_equilibrium_position():
    ref = json.load(open(GOLDEN))["x_eq"]["1000"]["present"]
    case = W.fixed_temperature_sedimentation(1000.0, length_d=150.0)
    D = 2.0 * case.radius[0]
    u_ref = 40.5 * (0.53 - 0.5) / 3.0 / D
    chunk = 1000
    xs, ts = [], []
    with gpu_lattice(case, precision="fp32") as lat:
        while True:
            lat.step(chunk)
            t = (len(ts) + 1) * chunk * u_ref / D
            ps = lat.particles()
            xs.append(ps["x"][0] / D)
            ts.append(t)
            if t >= 200.0:
                break
    xs, ts = np.array(xs), np.array(ts)
    window = xs[ts >= 120.0]
    print(f"x* over t* 120..200: mean {window.mean():.3f}, range {window.min():.3f}..{window.max():.3f}; paper {ref}")
    assert abs(window.mean() - ref) < 0.1
    assert window.max() - window.min() < 0.1
