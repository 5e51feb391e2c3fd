"""Particles held at their temperature (readings R11 and R11b of the
held-temperature sedimentation case of Sec. 3.3): the CUDA path against the
FP64 oracle on a small cavity where some disks are held (over the covered
part of each cell, or over every owned cell whole) and the others conduct,
in FP32 and FP64."""
import dataclasses

import pytest

from test_gpu_parity import _compare, _gpu_snapshots, _oracle_snapshots
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _case(mode=1):
    base = W.cavity(side=128, n=12, seed=7)
    held = [mode if k % 2 == 0 else 0 for k in range(len(base.x))]
    return dataclasses.replace(base, fixed_T=held)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp64", 1e-9)])
def test_held_particles_match_oracle(precision, tol, mode):
    case = _case(mode)
    ref = _oracle_snapshots(case, 3)
    gpu = _gpu_snapshots(case, 3, precision)
    _compare(gpu, ref, tol, 1e-4, 1e-4)


def test_held_particle_keeps_its_temperature_inside():
    """Cells that one held disk covers completely stay at its temperature."""
    import numpy as np
    from helpers import gpu_lattice
    from paper_2410_23802_gb300 import vlb as V
    case = _case()
    with gpu_lattice(case, precision="fp32") as lat:
        lat.step(150)
        f = lat.fields()
        count, owner, flag, fsp = V.vlb_get_solid_fraction(lat.h, case.params["nx"], case.params["ny"])
    held_solid = (count == 1) & (flag[:, :, 0] == 2) & (owner[:, :, 0] % 2 == 0)
    assert held_solid.sum() > 100
    assert np.abs(f["T"][held_solid] - 0.0).max() < 1e-6
