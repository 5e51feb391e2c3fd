"""Pins of the oracle's lattice, moment matrix and equilibria.

The moment matrix of Eq. 4 is checked against the polynomial basis it is
built from (Lallemand & Luo 2000), the equilibria of Eqs. 6 and 19 against
the textbook D2Q9 forms, and the MRT collision of Eq. 3a against BGK with
Guo forcing (Guo, Zheng & Shi 2002) when all rates are equal -- the
reduction stated in Sec. 2.1 ("precisely degenerate into the standard LB
method")."""
import numpy as np
import pytest

from oracle import vlbref as V

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def test_velocity_set_and_opposites():
    e = V.E
    assert e[0].tolist() == [0, 0]
    assert sorted(map(tuple, e[1:5].tolist())) == [(-1, 0), (0, -1), (0, 1), (1, 0)]
    assert all(abs(a) == 1 and abs(b) == 1 for a, b in e[5:].tolist())
    for i in range(9):
        assert (e[V.OPP[i]] == -e[i]).all()


def test_moment_matrix_is_the_polynomial_basis():
    ex, ey = V.EX, V.EY
    e2 = ex * ex + ey * ey
    basis = np.stack([
        np.ones(9),
        -4 + 3 * e2,
        4 - 10.5 * e2 + 4.5 * e2 * e2,
        ex,
        (-5 + 3 * e2) * ex,
        ey,
        (-5 + 3 * e2) * ey,
        ex * ex - ey * ey,
        ex * ey,
    ])
    np.testing.assert_array_equal(V.M, basis)
    G = V.M @ V.M.T
    assert np.count_nonzero(G - np.diag(np.diag(G))) == 0


def test_flow_equilibrium_is_textbook_polynomial():
    rng = np.random.default_rng(1)
    rho = 1 + 0.1 * rng.standard_normal(50)
    ux = 0.1 * rng.standard_normal(50)
    uy = 0.1 * rng.standard_normal(50)
    f = V.feq(rho, ux, uy)
    eu = V.EX[:, None] * ux + V.EY[:, None] * uy
    ref = W[:, None] * rho * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * (ux * ux + uy * uy))
    np.testing.assert_allclose(f, ref, rtol=0, atol=1e-15)


def test_thermal_equilibrium_components():
    rng = np.random.default_rng(2)
    eps = rng.uniform(0.2, 3.0, 40)
    T = rng.uniform(0.0, 1.0, 40)
    cref = 1.2
    g = V.geq(eps, T, cref)
    np.testing.assert_allclose(g.sum(axis=0), eps, atol=1e-15)
    np.testing.assert_allclose(np.tensordot(V.EX, g, axes=(0, 0)), 0, atol=1e-15)
    np.testing.assert_allclose(np.tensordot(V.EY, g, axes=(0, 0)), 0, atol=1e-15)
    # moving populations are w_i c_ref T (the D2Q9 weights), the rest carries eps
    np.testing.assert_allclose(g[1:], W[1:, None] * cref * T, atol=1e-15)
    np.testing.assert_allclose(g[0], eps - 5 / 9 * cref * T, atol=1e-15)


def _guo_bgk(f, rho, ux, uy, Fx, Fy, tau):
    """BGK collision with Guo's forcing term, written in velocity space."""
    fe = V.feq(rho, ux, uy)
    out = np.empty_like(f)
    for i in range(9):
        ex, ey = V.EX[i], V.EY[i]
        eu = ex * ux + ey * uy
        Fi = W[i] * (1 - 0.5 / tau) * (3 * ((ex - ux) * Fx + (ey - uy) * Fy) + 9 * eu * (ex * Fx + ey * Fy))
        out[i] = f[i] - (f[i] - fe[i]) / tau + Fi
    return out


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.3])
def test_mrt_with_equal_rates_is_bgk_with_guo_force(tau):
    rng = np.random.default_rng(3)
    n = 64
    rho = 1 + 0.05 * rng.standard_normal(n)
    ux = 0.05 * rng.standard_normal(n)
    uy = 0.05 * rng.standard_normal(n)
    f = V.feq(rho, ux, uy) + 1e-3 * rng.standard_normal((9, n))
    # keep the conserved moments consistent with rho, u (Eq. 9)
    Fx = 1e-3 * rng.standard_normal(n)
    Fy = 1e-3 * rng.standard_normal(n)
    rho, ux, uy = V.flow_macroscopics(f, Fx, Fy)
    S = np.full(9, 1.0 / tau)
    a = V.collide_flow(f, rho, ux, uy, Fx, Fy, S)
    b = _guo_bgk(f, rho, ux, uy, Fx, Fy, tau)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)


def test_collision_conserves_mass_and_adds_force():
    rng = np.random.default_rng(4)
    n = 32
    f = V.feq(np.ones(n), 0.02 * rng.standard_normal(n), 0.02 * rng.standard_normal(n))
    f += 1e-3 * rng.standard_normal((9, n))
    Fx, Fy = 1e-4 * rng.standard_normal(n), 1e-4 * rng.standard_normal(n)
    rho, ux, uy = V.flow_macroscopics(f, Fx, Fy)
    fb = V.collide_flow(f, rho, ux, uy, Fx, Fy, V.flow_rates(0.8))
    np.testing.assert_allclose(fb.sum(0), f.sum(0), atol=1e-15)
    jx0 = np.tensordot(V.EX, f, axes=(0, 0))
    jx1 = np.tensordot(V.EX, fb, axes=(0, 0))
    np.testing.assert_allclose(jx1 - jx0, Fx, atol=1e-16)


def test_flow_rates_rules():
    S = V.flow_rates(0.8, 1.0 / 12.0, 1.25)
    assert S[0] == 1 and S[3] == 1 and S[5] == 1
    assert S[1] == 1.25 and S[2] == 1.25
    assert abs(S[7] - 1 / 0.8) < 1e-15 and S[7] == S[8]
    assert abs((1 / S[7] - 0.5) * (1 / S[4] - 0.5) - 1 / 12) < 1e-15
    assert abs(S[4] - 9 / 7) < 1e-14  # tau_f = 0.8 gives s_q = 9/7


def test_thermal_rates_rules():
    tg = np.array([0.7, 6 / 7, 17 / 14, 2.0])
    R = V.thermal_rates(tg, 0)
    assert (R[0] == 1).all()
    np.testing.assert_allclose(R[3], 1 / tg)
    np.testing.assert_allclose(R[4], R[3])
    np.testing.assert_allclose((1 / R[3] - 0.5) * (1 / R[1] - 0.5), 0.25)
    np.testing.assert_array_equal(R[1], R[2])
    np.testing.assert_array_equal(R[7], R[1])
    R1 = V.thermal_rates(tg, 1)
    assert (R1[[0, 1, 2, 7, 8]] == 1).all()


def test_conductivity_relation():
    # Eq. 22 with alpha1 = -2: lambda = (1/3) c_ref (tau_g - 1/2)
    for lam, cref in [(0.1, 1.0), (1 / 7, 1.2), (0.4, 0.4)]:
        tg = V.tau_g_of(lam, cref)
        assert abs(cref * (tg - 0.5) / 3 - lam) < 1e-15
