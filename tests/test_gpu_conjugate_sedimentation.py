"""The CUDA path against numbers the paper prints: the cold disk settling
with conjugate heat transfer (Sec. 3.4; tests/golden/
conjugate_sedimentation_min_temperature.json).  After t* = U_ref t / D =
2.625 (10,000 steps at U_ref = 0.00525 lu, D = 20 lu) the minimal temperature
of the cells inside the disk (f_s = 1) must match the printed values for
R_cv = 1, 2, 4 and 8 within 0.02: the paper gives three digits, and it leaves
the channel length and the end walls open (the run is the same for channels
of 40 D and 60 D to four digits, so they do not matter by t*)."""
import json
import os

import numpy as np
import pytest

from helpers import gpu_lattice
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "conjugate_sedimentation_min_temperature.json")


@pytest.mark.parametrize("r_cv", [1, 2, 4, 8])
def test_min_particle_temperature_matches_paper(r_cv):
    ref = json.load(open(GOLDEN))
    case = W.conjugate_sedimentation(r_cv)
    d = 2.0 * case.radius[0]
    u_ref = 10.5 * (0.53 - 0.5) / 3.0 / d
    steps = int(round(ref["t_star"] * d / u_ref))
    assert steps == 10000
    with gpu_lattice(case, precision="fp32") as lat:
        lat.step(steps)
        f = lat.fields()
        ps = lat.particles()
    inside = f["fs"] > 0.999
    assert inside.sum() > 250  # the disk's interior cells (pi R^2 = 314 minus the rim)
    t_min = float(f["T"][inside].min())
    print(f"R_cv={r_cv}: min T inside {t_min:.4f}, paper {ref['min_T_inside'][str(r_cv)]}")
    assert abs(t_min - ref["min_T_inside"][str(r_cv)]) < 0.02
    # it settles downwards and stays on the centreline (FP32 rounding breaks the
    # left-right symmetry only at the 1e-6 lu level over these steps: 1.3e-6
    # measured; a real asymmetry of the method would move it much further)
    assert ps["uy"][0] < 0.0
    assert abs(ps["x"][0] - 40.0) < 1e-5
