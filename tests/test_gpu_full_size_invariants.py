"""Properties that hold at any size, checked at the full bench size (2048^2
cavity, 2048 moving disks, per-particle conductivities 10^U[-1,1]) over the
first 1000 steps, where the oracle would need hours.

* Uniform temperature stays uniform (the Appendix A invariant for beta_1 =
  -4 and sigma_0 = 1, which holds for any particle motion, conductivity and
  heat-capacity ratio): fluid, disks and walls all at T0, the disks settling
  ten times faster than in the bench case (g = 1e-4, rho_s/rho_f = 1.5) so
  that they cross cells; |T - T0| <= 5e-6 in FP32 (both thermal-rate modes;
  measured 2.5e-7).
* Closed-box mass: the walls are closed and the volumetric correction keeps
  every cell's mass, so the FP64 audit of sum f stays put (measured drift
  7e-11 over 1000 steps of the bench case; bound 1e-8)."""
import dataclasses

import numpy as np
import pytest

from helpers import gpu_lattice
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

T0 = 0.7


def _isothermal_cavity(side, n, mode):
    c = W.cavity(side=side, n=n, k_log_uniform=True)
    prm = dict(c.params, T_ref=T0, T_fluid_init=T0, wall_T=(0.0, 0.0, T0, T0), thermal_rates_mode=mode,
               gravity=(0.0, -1e-4), rho_ratio=1.5)
    return dataclasses.replace(c, params=prm, T0=[T0] * len(c.x))


@pytest.mark.parametrize("side,n,mode", [(2048, 2048, 1), (1024, 512, 0)])
def test_uniform_temperature_stays_uniform(side, n, mode):
    case = _isothermal_cavity(side, n, mode)
    worst = 0.0
    with gpu_lattice(case) as lat:
        m0 = lat.audit()[0]
        p0 = lat.particles()
        for _ in range(4):
            lat.step(250)
            f = lat.fields()
            worst = max(worst, float(np.abs(f["T"] - T0).max()))
        p1 = lat.particles()
        m1 = lat.audit()[0]
    moved = float(np.hypot(p1["x"] - p0["x"], p1["y"] - p0["y"]).max())
    print(f"max |T - T0| {worst:.2e}, largest displacement {moved:.2f} lu, mass drift {abs(m1 / m0 - 1):.2e}")
    assert moved > 1.0  # the disks really moved across cells: the source terms were active
    assert worst <= 5e-6
    assert abs(m1 / m0 - 1) < 1e-8


def test_closed_box_mass_of_the_bench_case():
    case = W.cavity()
    with gpu_lattice(case) as lat:
        lat.step(0)
        m0 = lat.audit()[0]
        lat.step(1000)
        m1 = lat.audit()[0]
    print(f"mass {m0:.10e} -> {m1:.10e}, relative drift {abs(m1 / m0 - 1):.2e}")
    assert abs(m1 / m0 - 1) < 1e-8


def test_bench_cavity_runs_its_20000_steps():
    """The 2048^2 cavity with 2048 disks for the configuration's 20,000 steps
    (beta from Gr = 100 on the cavity height, reading R9): no device flag
    (no NaN, no disk faster than 0.5 lu per step, none out of the domain),
    the disks settled lower, mass kept."""
    case = W.cavity(side=2048, n=2048)
    with gpu_lattice(case, precision="fp32") as lat:
        m0 = lat.audit()[0]
        y0 = np.array(case.y)
        for _ in range(20):
            lat.step(1000)  # raises on a device flag
        ps = lat.particles()
        m1 = lat.audit()[0]
    speed = np.hypot(ps["ux"], ps["uy"])
    print(f"20000 steps: largest disk speed {speed.max():.3e}, mean settling {np.mean(y0 - ps['y']):.1f} lu")
    assert speed.max() < 0.5 and np.mean(y0 - ps["y"]) > 0.5
    assert abs(m1 - m0) / m0 < 1e-7
