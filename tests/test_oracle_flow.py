"""Pins of the oracle's flow half (Sec. 2.1).

* Plane Poiseuille flow between halfway bounce-back walls: with
  (1/s_p - 1/2)(1/s_q - 1/2) = 3/16 the MRT steady state is the parabola of
  walls on the cell faces to rounding; with the paper's 1/12 the error falls
  by 4 per doubling of the channel (second order).
* Periodic stepping with f_s = 0 and equal rates against BGK + Guo force and
  np.roll streaming written separately (the reduction of Sec. 2.1).
* The volumetric correction (Eq. 8) keeps the mass of every cell and makes
  u = u_s in solid cells; total mass is conserved in a closed box.
* A disk and its fluid in uniform translation feel no MES force (Eq. 28)."""
import math

import numpy as np
import pytest

from oracle import vlbref as V


def _poiseuille(H, lam, tau=0.8, Fx=1e-5, steps=None):
    S = V.flow_rates(tau, lam, 1.25)
    nu = (tau - 0.5) / 3
    y = np.arange(H) + 0.5
    uex = Fx * y * (H - y) / (2 * nu)
    FX = np.full((H, 1), Fx)
    FY = np.zeros((H, 1))
    f = V.feq(np.ones((H, 1)), uex[:, None].copy(), np.zeros((H, 1)))
    rho, ux, uy = V.flow_macroscopics(f, FX, FY)
    for _ in range(steps or 30 * H * H):
        f = V.stream_flow(V.collide_flow(f, rho, ux, uy, FX, FY, S), (True, False))
        rho, ux, uy = V.flow_macroscopics(f, FX, FY)
    return ux[:, 0], uex


@pytest.mark.parametrize("H", [8, 16])
def test_poiseuille_exact_with_magic_3_16(H):
    u, uex = _poiseuille(H, 3.0 / 16.0)
    assert np.abs(u - uex).max() / uex.max() < 1e-10


def test_poiseuille_second_order_with_paper_rates():
    errs = []
    for H in (8, 16, 32):
        u, uex = _poiseuille(H, 1.0 / 12.0)
        errs.append(np.sqrt(((u - uex) ** 2).sum() / (uex ** 2).sum()))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.8 < r1 < 4.2 and 3.8 < r2 < 4.2, errs


def _bgk_guo_periodic(f, Fx, Fy, tau, steps):
    W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    for _ in range(steps):
        rho = f.sum(0)
        ux = ((ex[:, None, None] * f).sum(0) + 0.5 * Fx) / rho
        uy = ((ey[:, None, None] * f).sum(0) + 0.5 * Fy) / rho
        out = np.empty_like(f)
        for i in range(9):
            eu = ex[i] * ux + ey[i] * uy
            fe = W[i] * rho * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * (ux * ux + uy * uy))
            Fi = W[i] * (1 - 0.5 / tau) * (3 * ((ex[i] - ux) * Fx + (ey[i] - uy) * Fy) + 9 * eu * (ex[i] * Fx + ey[i] * Fy))
            post = f[i] - (f[i] - fe) / tau + Fi
            out[i] = np.roll(np.roll(post, ey[i], axis=0), ex[i], axis=1)
        f = out
    return f


def test_no_solid_periodic_equals_bgk_guo():
    rng = np.random.default_rng(7)
    ny, nx, tau = 12, 10, 0.9
    f0 = V.feq(1 + 0.01 * rng.standard_normal((ny, nx)), 0.01 * rng.standard_normal((ny, nx)),
               0.01 * rng.standard_normal((ny, nx)))
    Fx = 1e-4 * rng.standard_normal((ny, nx))
    Fy = 1e-4 * rng.standard_normal((ny, nx))
    S = np.full(9, 1 / tau)
    f = f0.copy()
    for _ in range(20):
        rho, ux, uy = V.flow_macroscopics(f, Fx, Fy)
        f = V.stream_flow(V.collide_flow(f, rho, ux, uy, Fx, Fy, S), (True, True))
    ref = _bgk_guo_periodic(f0.copy(), Fx, Fy, tau, 20)
    np.testing.assert_allclose(f, ref, rtol=0, atol=1e-14)


def test_correction_keeps_cell_mass():
    rng = np.random.default_rng(8)
    ras = V.rasterise(24, 24, [8.0, 15.5], [9.0, 15.2], [4.0, 3.3])
    fstar = V.feq(1 + 0.02 * rng.standard_normal((24, 24)), 0.02 * rng.standard_normal((24, 24)),
                  0.02 * rng.standard_normal((24, 24)))
    part = {"x": np.array([8.0, 15.5]), "y": np.array([9.0, 15.2]), "ux": np.array([0.01, -0.02]),
            "uy": np.array([0.003, 0.0]), "omega": np.array([0.001, -0.002])}
    f, F, T = V.correct_and_exchange(fstar, ras, part)
    np.testing.assert_allclose(f.sum(0), fstar.sum(0), rtol=0, atol=2e-15)


def _coupled(periodic=(False, False), gravity=(0.0, -2e-5), beta=0.0):
    prm = V.Params(nx=40, ny=48, tau_f=0.8, rho_ratio=1.5, cv_ratio=2.0, k_ratio_default=3.0,
                   gravity=gravity, beta=beta, T_ref=1.0, T_fluid_init=1.0, periodic=periodic)
    return V.Simulation(prm, [20.3, 11.0], [30.2, 14.7], [6.0, 4.5], [0.0, 0.5],
                        ux=[0.0, 0.004], uy=[0.0, 0.001], omega=[0.0, 0.002])


def test_solid_cells_move_with_the_particle_and_mass_is_conserved():
    sim = _coupled(beta=5.0)
    m0 = sim.audit()[0]
    for _ in range(60):
        sim.step()
        ras = sim.ras
        P = sim.part
        for p in range(2):
            sel = (ras.count == 1) & (ras.owner[:, :, 0] == p) & (ras.flag[:, :, 0] == V.SOLID)
            jj, ii = np.nonzero(sel)
            assert jj.size > 0
            usx, usy = V.solid_velocity(ii + 0.5, jj + 0.5, P["ux"][p], P["uy"][p], P["omega"][p], P["x"][p], P["y"][p])
            assert np.abs(sim.ux[sel] - usx).max() < 1e-14
            assert np.abs(sim.uy[sel] - usy).max() < 1e-14
    assert abs(sim.audit()[0] - m0) / m0 < 1e-13


def test_uniform_translation_feels_no_force():
    prm = V.Params(nx=40, ny=40, tau_f=0.8, rho_ratio=1.5, gravity=(0.0, 0.0), beta=0.0, periodic=(True, True))
    U = (0.02, -0.01)
    sim = V.Simulation(prm, [20.0], [20.0], [6.0], [1.0], ux=[U[0]], uy=[U[1]])
    one = np.ones((40, 40))
    sim.f = V.feq(one, U[0] * one, U[1] * one)
    sim.rho, sim.ux, sim.uy = V.flow_macroscopics(sim.f, 0 * one, 0 * one)
    sim.F_mes[:] = 0.0
    sim.T_mes[:] = 0.0
    for _ in range(40):
        sim.step()
        assert np.abs(sim.F_mes).max() < 1e-13 and np.abs(sim.T_mes).max() < 1e-12
    ps = sim.particle_state()
    assert abs(ps["ux"][0] - U[0]) < 1e-13 and abs(ps["x"][0] - (20 + 40 * U[0])) < 1e-11
