"""Pins of the oracle's thermal half (Sec. 2.2, Appendix A).

* Sec. 3.1, stationary: the conjugate erfc solution (Eq. 31) for
  R_lambda in {1, 4}, R_cv in {1/4, 1, 4}, lambda_f = 0.1, t = 2000.
* Sec. 3.1, moving (U = 0.05): the same closed form with X_i = U t; the
  error of the source-term convection falls as U^2.
* Steady conduction through a fluid-solid composite slab between walls held
  at T = 1 and 0: series conductances, linear T in each layer, continuous T
  and flux -- exact to rounding for a face-aligned interface.
* Appendix A, generalised to 2-D coupled runs: an initially isothermal
  system stays at T0 under any particle motion with beta1 = -4 and the
  df_s/dt recursion of Eq. 24; planting beta1 = 0 or a backward difference
  breaks it.
* Energy bookkeeping: with sigma_0 = 1 and adiabatic walls,
  sum g^{n+1} = sum g^n + sum q_c^n exactly; at R_cv = 1 with the fluid at
  rest, sum eps is conserved and the field relaxes to T_eq = sum c_v T /
  sum c_v (the energy balance of Sec. 3.5)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import vlbref as V

HERE = os.path.dirname(os.path.abspath(__file__))


def _erfc_case(Rl, Rc, U, x0, nx, steps):
    sim = V.PrescribedFlowThermal(nx, 1, 0.1, Rl, Rc, lambda t: V.slab_fraction(nx, 1, x0 + U * t), 1.0, 0.0,
                                  velocity=(U, 0.0), thermal_wall=(1, 1, 0, 0), wall_T=(1.0, 0.0, 0.0, 0.0),
                                  periodic=(False, True))
    sim.step(steps)
    xc = np.arange(nx) + 0.5
    Tex = V.conjugate_erfc(xc, steps, x0 + U * steps, 1.0, 0.0, 0.1, Rl, Rc)
    return np.abs(sim.T[0] - Tex).max()


@pytest.mark.parametrize("Rl", [1.0, 4.0])
@pytest.mark.parametrize("Rc", [0.25, 1.0, 4.0])
def test_stationary_conjugate_erfc(Rl, Rc):
    assert _erfc_case(Rl, Rc, 0.0, 400.0, 800, 2000) < 3e-4


@pytest.mark.parametrize("Rl,Rc", [(1.0, 1.0), (1.0, 4.0)])
def test_moving_conjugate_erfc_converges_as_U_squared(Rl, Rc):
    errs = [_erfc_case(Rl, Rc, U, 250.0, 600, int(round(100 / U))) for U in (0.05, 0.025)]
    assert errs[0] < 2e-2
    assert 3.0 < errs[0] / errs[1] < 5.5, errs


@pytest.mark.parametrize("Rl,Rc,mode", [(5.0, 2.0, 0), (5.0, 2.0, 1), (0.5, 0.5, 0)])
def test_composite_slab_series_conduction(Rl, Rc, mode):
    L, Lf, lamf = 32, 16, 0.4
    fs = np.where(np.arange(L) >= Lf, 1.0, 0.0)[None, :]
    sim = V.PrescribedFlowThermal(L, 1, lamf, Rl, Rc, lambda t: fs, 0.5, 0.5, thermal_wall=(1, 1, 0, 0),
                                  wall_T=(1.0, 0.0, 0.0, 0.0), mode=mode)
    prev = sim.T.copy()
    for _ in range(60):
        sim.step(1000)
        if np.abs(sim.T - prev).max() < 1e-15:
            break
        prev = sim.T.copy()
    lams = Rl * lamf
    q = 1.0 / (Lf / lamf + (L - Lf) / lams)
    xc = np.arange(L) + 0.5
    Tex = np.where(xc < Lf, 1 - q * xc / lamf, 1 - q * Lf / lamf - q * (xc - Lf) / lams)
    assert np.abs(sim.T[0] - Tex).max() < 1e-12
    gx, _ = V.temperature_gradient(sim.g, sim.cref, sim.tau_g)
    flux = -np.where(fs[0] > 0.5, lams, lamf) * gx[0]
    assert np.abs(flux / q - 1).max() < 1e-11


def _isothermal(mode, T0=0.7, steps=150, beta=3.0):
    prm = V.Params(nx=36, ny=44, tau_f=0.8, rho_ratio=1.8, cv_ratio=3.0, k_ratio_default=7.0,
                   gravity=(5e-5, -3e-4), beta=beta, T_ref=T0, T_fluid_init=T0, thermal_rates_mode=mode,
                   thermal_wall=(0, 1, 0, 1), wall_T=(0.0, T0, 0.0, T0))
    sim = V.Simulation(prm, [17.3, 9.0, 26.0], [28.2, 12.6, 12.0], [6.0, 4.5, 4.0], [T0, T0, T0],
                       k_ratio=[7.0, 0.3, 2.0], ux=[0.0, 0.03, -0.02], uy=[0.0, 0.01, 0.0],
                       omega=[0.0, 0.003, -0.002])
    worst = 0.0
    source = 0.0
    for _ in range(steps):
        sim.step()
        worst = max(worst, np.abs(sim.T - T0).max())
        source = max(source, np.abs(sim.dfs).max())
    return worst, source


@pytest.mark.parametrize("mode", [0, 1])
def test_appendix_a_isothermal_invariant(mode):
    worst, source = _isothermal(mode)
    assert source > 1e-2  # interface cells really changed: the source term is active
    assert worst < 1e-13


def test_appendix_a_invariant_detects_wrong_beta1(monkeypatch):
    monkeypatch.setattr(V, "BETA1", 0.0)
    worst, _ = _isothermal(0, steps=60)
    assert worst > 1e-6


def test_appendix_a_invariant_detects_backward_difference(monkeypatch):
    monkeypatch.setattr(V, "dfs_dt_update", lambda new, old, d: new - old)
    worst, _ = _isothermal(0, steps=60)
    assert worst > 1e-6


def test_energy_bookkeeping_identity():
    prm = V.Params(nx=30, ny=40, tau_f=0.8, rho_ratio=1.6, cv_ratio=2.5, k_ratio_default=4.0,
                   gravity=(0.0, -3e-5), beta=2.0, T_ref=1.0, T_fluid_init=1.0)
    sim = V.Simulation(prm, [15.2, 8.0], [26.0, 12.3], [5.0, 3.5], [0.0, 0.3], ux=[0.0, 0.01])
    for _ in range(80):
        before = sim.g.sum() + sim.qc.sum()
        sim.step()
        assert abs(sim.g.sum() - before) < 1e-11 * abs(before)


def test_energy_conserved_and_relaxes_to_balance_temperature():
    # R_cv = 1 with the fluid at rest: q_c vanishes, so sum eps is conserved
    prm = V.Params(nx=24, ny=24, tau_f=0.8, prandtl=0.2, rho_ratio=1.0, cv_ratio=1.0, k_ratio_default=2.0,
                   gravity=(0.0, 0.0), beta=0.0, T_fluid_init=1.0)
    sim = V.Simulation(prm, [8.0, 16.5], [9.0, 15.5], [4.0, 5.0], [0.0, 0.25])
    e0 = sim.eps.sum()
    teq = e0 / sim.cv.sum()
    sim.step(3000)
    assert abs(sim.eps.sum() - e0) < 1e-11 * e0
    assert np.abs(sim.T - teq).max() < 1e-6


def test_paper_cavity_balance_temperature():
    """T_eq of the 2048-particle cavity of Sec. 3.5, from its setup."""
    with open(os.path.join(HERE, "golden", "cavity_balance_temperature.json")) as fh:
        gold = json.load(fh)
    phi = gold["n_particles"] * math.pi * (gold["diameter"] / 2) ** 2 / gold["side"] ** 2
    cvs = gold["R_cv"]
    teq = ((1 - phi) * 1.0 * gold["T_h"] + phi * cvs * gold["T_c"]) / ((1 - phi) + phi * cvs)
    assert abs(teq - gold["T_eq"]) < 5e-5


def _fixed_T_sim(ux=0.0, T_p=0.0, beta=0.0, walls=(1, 1, 1, 1), wall_T=1.0, mode=1):
    p = V.Params(nx=48, ny=48, tau_f=0.8, prandtl=0.7, rho_ratio=1.0, cv_ratio=1.0, k_ratio_default=1.0,
                 gravity=(0.0, -1e-5), beta=beta, T_ref=1.0, T_fluid_init=1.0, thermal_wall=walls,
                 wall_T=(wall_T,) * 4)
    return V.Simulation(p, [20.3], [24.6], [7.0], [T_p], ux=[ux], fixed_T=[mode])


def test_fixed_temperature_particle_interior_stays_at_its_temperature():
    """Reading R11: cells a held particle covers completely carry the
    equilibrium at its temperature, so their T is exactly T_p (the gradient
    of an equilibrium vanishes and c_vs = c_vf leaves no source term)."""
    sim = _fixed_T_sim(T_p=0.25)
    sim.step(40)
    inside = sim.ras.fs == 1.0
    assert inside.sum() > 100
    assert np.abs(sim.T[inside] - 0.25).max() < 1e-13
    # the fluid around it cools towards it, between T_p and the walls
    assert sim.T.min() >= 0.25 - 1e-12 and sim.T.max() <= 1.0 + 1e-12
    assert (sim.T[~inside] < 1.0 - 1e-6).any()


def test_fixed_temperature_particle_at_fluid_temperature_changes_nothing():
    """A held particle at the fluid and wall temperature, moving through the
    fluid, leaves T uniform to rounding (nothing in the correction acts on
    a uniform temperature field)."""
    sim = _fixed_T_sim(ux=0.02, T_p=1.0)
    sim.step(60)
    assert np.abs(sim.T - 1.0).max() < 1e-12


def test_whole_cell_hold_sets_every_owned_cell():
    """Reading R11b: every cell the held particle owns, interface cells
    included, takes the equilibrium at T_p whole, so with R_cv = 1 its T is
    T_p exactly there; under reading R11 the interface cells keep part of
    the warmer fluid and lie strictly between T_p and the walls."""
    T = {}
    for mode in (1, 2):
        sim = _fixed_T_sim(T_p=0.25, mode=mode)
        sim.step(30)
        T[mode] = sim.T.copy()
        owned, partial = sim.ras.count > 0, (sim.ras.count > 0) & (sim.ras.fs < 1.0)
    assert partial.sum() > 20
    assert np.abs(T[2][owned] - 0.25).max() < 1e-13
    assert (T[1][partial] > 0.25 + 1e-6).all()
    assert np.abs(T[1][owned & ~partial] - 0.25).max() < 1e-13


def test_whole_cell_holds_of_two_owners_share_the_cell():
    """Reading R11b where two held particles own one cell: the cell takes
    their mean equilibrium (weights summing above 1 are scaled to 1), so
    with R_cv = 1 it sits at the mean of their temperatures; a cell owned by
    one of them only is at that particle's temperature."""
    p = V.Params(nx=40, ny=30, tau_f=0.8, prandtl=0.7, rho_ratio=1.0, cv_ratio=1.0, k_ratio_default=1.0,
                 gravity=(0.0, 0.0), beta=0.0, T_ref=1.0, T_fluid_init=1.0)
    sim = V.Simulation(p, [13.6, 26.0], [15.2, 15.2], [6.1, 6.1], [0.0, 1.0], fixed_T=[2, 2])
    sim.step(1)
    shared = sim.ras.count == 2
    only = [(sim.ras.count == 1) & (sim.ras.owner[:, :, 0] == k) for k in (0, 1)]
    assert shared.sum() >= 2
    assert np.abs(sim.T[shared] - 0.5).max() < 1e-13
    assert np.abs(sim.T[only[0]]).max() < 1e-13 and np.abs(sim.T[only[1]] - 1.0).max() < 1e-13
