"""Pins of the oracle's momentum-exchange force and torque (Eq. 28) and of
its buoyancy branch (Sec. 3.3 with reading R4: the force
(1 - f_s) b (T - T_ref) and the joint solve of Eq. 25 with Eq. 9).

Momentum exchange, checked against conservation laws and Stokes flow rather
than against its own formula:

* Linear momentum.  Streaming conserves sum_x sum_i e_i f_i on a periodic
  lattice, the collision adds exactly the body force F (Eq. 3a with
  rho u = j + F/2, Eq. 9), and the correction changes the momentum of the
  fluid by -F_MES.  So, at every step and whatever the flow,
      sum j^{n+1} - sum j^n = sum F^n - F_MES^{n+1}.
* Angular momentum about a fixed point X0.  Streaming moves e_i f_i from x
  to x + e_i, and (x + e_i - X0) x e_i = (x - X0) x e_i, so it conserves
  sum (x - X0) x j as long as no population crosses a boundary carrying
  momentum; the correction changes it by -(T_MES + (X_p - X0) x F_MES).
* Stokes flow past a square array of fixed cylinders (Hasimoto 1959,
  extended by Sangani & Acrivos 1982): F / (mu U) =
  4 pi / (-ln(c)/2 - 0.738 + c - 0.887 c^2 + 2.039 c^3), c the solid
  fraction and U the mean velocity over the cell.  The diffuse interface
  of the volumetric method makes the disk act as a slightly smaller one
  (about R - 0.35 lu at R = 8 and tau_f = 0.8), so the pin is loose; its
  sign and size fail for any plausible slip in Eq. 28.
* A cylinder spinning at Omega in a periodic square array: the steady
  torque is -4 pi mu Omega R^2 / (1 - c) + O(c^2) (a rotlet with the
  uniform counter-vorticity that periodicity demands).

Buoyancy, with exact discrete answers (the MRT rates with
(1/s_p - 1/2)(1/s_q - 1/2) = 3/16 make halfway bounce-back exact for
quadratic and, as measured here, cubic profiles):

* A uniform fluid at T0 != T_ref between adiabatic walls with gravity along
  the channel: T stays T0 and the flow is the Poiseuille parabola of the
  force rho_f beta |g| (T0 - T_ref), hot fluid moving against gravity.
* A vertical slot between walls held at T_h and T_c, periodic along
  gravity, T_ref the mean: T is linear and u the cubic
  (beta |g| dT W^2 / (12 nu)) xi (2 xi - 1)(xi - 1) (Batchelor 1954).
* A stably stratified layer (hot top, cold bottom): T is exactly linear
  only if the u in Eq. 25 is the one of Eq. 9 with the buoyancy of the same
  level; a lagged T/u coupling or a dropped F/2 leaves a visible error.

Each pin is shown to fail on a planted mistake."""
import math

import numpy as np
import pytest

from oracle import vlbref as V

G_SMALL = 1e-5


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------


def _momentum(f):
    return float(np.tensordot(V.EX, f, axes=(0, 0)).sum()), float(np.tensordot(V.EY, f, axes=(0, 0)).sum())


def _angular_momentum(f, X0, Y0):
    ny, nx = f.shape[1:]
    yy, xx = np.meshgrid(np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    jx = np.tensordot(V.EX, f, axes=(0, 0))
    jy = np.tensordot(V.EY, f, axes=(0, 0))
    return float(((xx - X0) * jy - (yy - Y0) * jx).sum())


def _hold(sim, X, Y, U=(0.0, 0.0), Om=0.0):
    """Replace the particle update of `sim` by a disk held at (X, Y) moving
    at U and spinning at Om (the correction then uses exactly these)."""
    def held():
        P = sim.part
        P["x"][0], P["y"][0] = X, Y
        P["ux"][0], P["uy"][0], P["omega"][0] = U[0], U[1], Om
        P["ux_prev"][0], P["uy_prev"][0], P["omega_prev"][0] = U[0], U[1], Om
    sim._particle_update = held


def _flip_force(orig):
    def f(fstar, ras, part):
        ff, F, T = orig(fstar, ras, part)
        return ff, -F, T
    return f


def _flip_torque(orig):
    def f(fstar, ras, part):
        ff, F, T = orig(fstar, ras, part)
        return ff, F, -T
    return f


def _corner_arm(orig):
    # arm from the cell's lower-left corner instead of its centre:
    # (x - 1/2 - X) x dF = (x - X) x dF - (1/2, 1/2) x dF, summed
    def f(fstar, ras, part):
        ff, F, T = orig(fstar, ras, part)
        return ff, F, T - 0.5 * (F[:, 1] - F[:, 0])
    return f


# ---------------------------------------------------------------------------
# exact balances of the exchange terms (every step)
# ---------------------------------------------------------------------------


def _falling_disk_residuals(steps=12):
    """Linear-momentum balance of a free, falling, spinning disk in a
    periodic box with a buoyant body force: one residual per step."""
    prm = V.Params(nx=40, ny=44, tau_f=0.8, rho_ratio=1.5, cv_ratio=2.0, k_ratio_default=3.0,
                   gravity=(0.3e-4, -1e-4), beta=2.0, T_ref=0.6, T_fluid_init=1.0, periodic=(True, True))
    sim = V.Simulation(prm, [19.7], [22.4], [6.5], [0.2], ux=[0.004], uy=[-0.006], omega=[0.003])
    res, scale = [], []
    for _ in range(steps):
        j0 = _momentum(sim.f)
        F0 = (float(sim.Fx.sum()), float(sim.Fy.sum()))
        sim.step()
        j1 = _momentum(sim.f)
        Fm = sim.F_mes[0]
        res.append(max(abs(j1[k] - j0[k] - F0[k] + Fm[k]) for k in range(2)))
        scale.append(max(abs(F0[0]), abs(F0[1]), abs(Fm[0]), abs(Fm[1])))
    return np.array(res), np.array(scale)


def test_exchange_force_balances_the_fluid_momentum_every_step():
    res, scale = _falling_disk_residuals()
    assert scale.min() > 1e-4  # the terms are far from zero
    assert (res < 1e-11 * scale).all(), res / scale


@pytest.mark.parametrize("plant", [_flip_force, lambda o: (lambda a, b, c: (lambda r: (r[0], 2.0 * r[1], r[2]))(o(a, b, c)))])
def test_exchange_force_balance_detects_a_wrong_sign_or_factor(monkeypatch, plant):
    monkeypatch.setattr(V, "correct_and_exchange", plant(V.correct_and_exchange))
    res, scale = _falling_disk_residuals(steps=3)
    assert (res > 1e-3 * scale).any()


def _moving_disk_torque_residuals(steps=10):
    """Angular-momentum balance about a fixed point for a translating,
    spinning disk (held at its motion so that it moves on): one residual per
    step, while the disturbance is still far from the periodic boundary."""
    X0, Y0 = 30.0, 29.0
    prm = V.Params(nx=60, ny=60, tau_f=0.8, rho_ratio=1.5, gravity=(0.0, 0.0), beta=0.0, periodic=(True, True))
    U, Om = (0.012, -0.007), 0.004
    sim = V.Simulation(prm, [30.4], [28.7], [7.0], [1.0], ux=[U[0]], uy=[U[1]], omega=[Om])
    pos = [30.4, 28.7]

    def moving():
        P = sim.part
        pos[0] += U[0]
        pos[1] += U[1]
        P["x"][0], P["y"][0] = pos
        P["ux"][0], P["uy"][0], P["omega"][0] = U[0], U[1], Om
        P["ux_prev"][0], P["uy_prev"][0], P["omega_prev"][0] = U[0], U[1], Om
    sim._particle_update = moving
    res, scale = [], []
    for _ in range(steps):
        L0 = _angular_momentum(sim.f, X0, Y0)
        sim.step()
        L1 = _angular_momentum(sim.f, X0, Y0)
        Fm, Tm = sim.F_mes[0], sim.T_mes[0]
        arm = (pos[0] - X0) * Fm[1] - (pos[1] - Y0) * Fm[0]
        res.append(abs(L1 - L0 + Tm + arm))
        scale.append(max(abs(Tm), abs(arm), 1e-300))
    return np.array(res), np.array(scale)


def test_exchange_torque_balances_the_fluid_angular_momentum_every_step():
    res, scale = _moving_disk_torque_residuals()
    assert scale.min() > 1e-3
    assert (res < 1e-11 * scale).all(), res / scale


@pytest.mark.parametrize("plant", [_flip_torque, _corner_arm])
def test_exchange_torque_balance_detects_a_wrong_sign_or_arm(monkeypatch, plant):
    monkeypatch.setattr(V, "correct_and_exchange", plant(V.correct_and_exchange))
    res, scale = _moving_disk_torque_residuals(steps=3)
    assert (res > 1e-3 * scale).any()


# ---------------------------------------------------------------------------
# Stokes magnitudes
# ---------------------------------------------------------------------------


def _array_drag(L=64, R=8.0, tau=0.8, U0=2e-3, steps=2500):
    """A disk held at rest in a periodic box, the fluid driven past it at a
    fixed mean velocity U0: each step the body force is set so that the
    momentum lost to the disk in the last step is replaced and the mean
    momentum returns to U0 L^2 (flow-rate control, which leaves only the fast
    transients).  Returns the steady drag, the body force that holds the flow
    and the mean velocity."""
    X, Y = L / 2 + 0.3, L / 2 - 0.2
    c = math.pi * R * R / (L * L)
    prm = V.Params(nx=L, ny=L, tau_f=tau, gravity=(-1.0, 0.0), beta=0.0, T_ref=0.0, T_fluid_init=1.0,
                   periodic=(True, True))
    sim = V.Simulation(prm, [X], [Y], [R], [1.0])
    _hold(sim, X, Y)
    ux0 = np.where(sim.ras.fs < 1.0, U0 / (1.0 - c), 0.0)
    f0 = V.feq(np.ones((L, L)), ux0, 0.0 * ux0)
    sim.f, _, _ = V.correct_and_exchange(f0, sim.ras, sim.part)
    sim.rho, sim.ux, sim.uy = V.flow_macroscopics(sim.f, sim.Fx, sim.Fy)
    fluid = float((1.0 - sim.ras.fs).sum())
    G = 0.0
    for _ in range(steps):
        jx, _ = _momentum(sim.f)
        G = (U0 * L * L - jx + sim.F_mes[0, 0]) / fluid
        sim.b = (G, 0.0)  # buoyancy b (T - T_ref) with T - T_ref = 1: a uniform force G on the fluid
        sim.Fx = (1.0 - sim.ras.fs) * G
        sim.step()
    jx, _ = _momentum(sim.f)
    return float(sim.F_mes[0, 0]), G * fluid, jx / (L * L), c, (tau - 0.5) / 3.0


def test_drag_on_a_periodic_array_matches_hasimoto():
    F, Fbody, U, c, nu = _array_drag()
    assert abs(F - Fbody) < 1e-3 * Fbody  # steady: the disk takes what the body force gives
    hasimoto = 4.0 * math.pi / (-0.5 * math.log(c) - 0.738 + c - 0.887 * c * c + 2.039 * c ** 3)
    ratio = (F / (nu * U)) / hasimoto
    # measured 0.951 (effective radius about R - 0.35 lu)
    assert 0.92 < ratio < 1.02, ratio


def test_torque_on_a_spinning_disk_opposes_the_spin_with_the_rotlet_value():
    L, R, tau, Om = 64, 8.0, 0.8, 1e-3
    X, Y = L / 2 + 0.3, L / 2 - 0.2
    prm = V.Params(nx=L, ny=L, tau_f=tau, gravity=(0.0, 0.0), beta=0.0, periodic=(True, True))
    sim = V.Simulation(prm, [X], [Y], [R], [1.0], omega=[Om])
    _hold(sim, X, Y, Om=Om)
    sim.step(3000)
    c = math.pi * R * R / (L * L)
    nu = (tau - 0.5) / 3.0
    expect = -4.0 * math.pi * nu * Om * R * R / (1.0 - c)
    # measured 1.0069 x expected after 3000 steps, still falling slowly
    assert 0.99 < sim.T_mes[0] / expect < 1.03, sim.T_mes[0] / expect


# ---------------------------------------------------------------------------
# buoyancy
# ---------------------------------------------------------------------------


def _poiseuille_by_buoyancy(H=8, beta=0.5, T0=1.3, T_ref=1.0):
    prm = V.Params(nx=2, ny=H, tau_f=0.8, lambda_q_flow=3.0 / 16.0, gravity=(-G_SMALL, 0.0), beta=beta,
                   T_ref=T_ref, T_fluid_init=T0, periodic=(True, False))
    sim = V.Simulation(prm, [], [], [], [])
    sim.step(30 * H * H)
    nu = (0.8 - 0.5) / 3.0
    F = 1.0 * beta * G_SMALL * (T0 - T_ref)  # rho_f beta |g| (T - T_ref), along -g
    y = np.arange(H) + 0.5
    return sim, F * y * (H - y) / (2.0 * nu)


def test_buoyant_fluid_flows_against_gravity_as_the_exact_parabola():
    sim, uex = _poiseuille_by_buoyancy()
    assert np.abs(sim.T - 1.3).max() < 1e-13  # a uniform temperature stays uniform
    assert (uex > 0).all()  # hot fluid moves against gravity (gravity along -x)
    assert np.abs(sim.ux[:, 0] - uex).max() < 1e-9 * uex.max()
    assert np.abs(sim.uy).max() < 1e-14


def test_buoyant_parabola_fails_on_a_flipped_or_doubled_force(monkeypatch):
    orig = V.temperature_and_velocity

    def flipped(G, cv, cv_f, cv_s, dfs, rho, jx, jy, fs, bx, by, T_ref, gTx, gTy):
        return orig(G, cv, cv_f, cv_s, dfs, rho, jx, jy, fs, -bx, -by, T_ref, gTx, gTy)

    def doubled(G, cv, cv_f, cv_s, dfs, rho, jx, jy, fs, bx, by, T_ref, gTx, gTy):
        return orig(G, cv, cv_f, cv_s, dfs, rho, jx, jy, fs, 2 * bx, 2 * by, T_ref, gTx, gTy)

    def no_half_force(G, cv, cv_f, cv_s, dfs, rho, jx, jy, fs, bx, by, T_ref, gTx, gTy):
        T, ux, uy, Fx, Fy = orig(G, cv, cv_f, cv_s, dfs, rho, jx, jy, fs, bx, by, T_ref, gTx, gTy)
        return T, jx / rho, jy / rho, Fx, Fy

    for plant in (flipped, doubled, no_half_force):
        monkeypatch.setattr(V, "temperature_and_velocity", plant)
        sim, uex = _poiseuille_by_buoyancy()
        assert np.abs(sim.ux[:, 0] - uex).max() > 1e-3 * uex.max(), plant.__name__


def _slot(W=16, steps=7000):
    Th, Tc = 1.0, 0.0
    beta = 0.5
    prm = V.Params(nx=W, ny=2, tau_f=0.8, lambda_q_flow=3.0 / 16.0, gravity=(0.0, -G_SMALL), beta=beta,
                   T_ref=0.5 * (Th + Tc), T_fluid_init=0.5 * (Th + Tc), thermal_wall=(1, 1, 0, 0),
                   wall_T=(Th, Tc, 0.0, 0.0), periodic=(False, True))
    sim = V.Simulation(prm, [], [], [], [])
    sim.step(steps)
    nu = (0.8 - 0.5) / 3.0
    xi = (np.arange(W) + 0.5) / W
    T = Th + (Tc - Th) * xi
    u = beta * G_SMALL * (Th - Tc) * W * W / (12.0 * nu) * xi * (2 * xi - 1) * (xi - 1)
    return sim, T, u


def test_vertical_slot_conduction_regime_is_linear_in_T_and_cubic_in_u():
    sim, T, u = _slot()
    assert np.abs(sim.T[0] - T).max() < 1e-12
    assert u[0] > 0 > u[-1]  # rising at the hot wall, sinking at the cold one
    assert np.abs(sim.uy[0] - u).max() < 1e-8 * np.abs(u).max()
    assert np.abs(sim.ux).max() < 1e-14


def _stratified(steps=6000):
    Hs = 16
    prm = V.Params(nx=2, ny=Hs, tau_f=0.8, lambda_q_flow=3.0 / 16.0, gravity=(0.0, -G_SMALL), beta=20.0,
                   T_ref=0.0, T_fluid_init=0.5, thermal_wall=(0, 0, 1, 1), wall_T=(0.0, 0.0, 0.0, 1.0),
                   periodic=(True, False))
    sim = V.Simulation(prm, [], [], [], [])
    sim.step(steps)
    return sim, (np.arange(Hs) + 0.5) / Hs


def test_stably_stratified_layer_conducts_with_an_exactly_linear_temperature():
    sim, T = _stratified()
    assert np.abs(sim.T[:, 0] - T).max() < 1e-12
    assert sim.rho[-1, 0] > sim.rho[0, 0]  # hydrostatic: the buoyancy of the hot top is held by a density gradient


def test_stratified_layer_detects_a_lagged_temperature_velocity_coupling(monkeypatch):
    def lagged(G, cv, cv_f, cv_s, dfs, rho, jx, jy, fs, bx, by, T_ref, gTx, gTy):
        # Eq. 25 with u = j / rho, the buoyancy of the level left out of the T solve
        D = cv - 0.5 * (cv_s - cv_f) * dfs
        T = (G - 0.5 * cv * ((jx / rho) * gTx + (jy / rho) * gTy)) / D
        ax, ay = (1 - fs) * bx / (2 * rho), (1 - fs) * by / (2 * rho)
        return (T, jx / rho + ax * (T - T_ref), jy / rho + ay * (T - T_ref), (1 - fs) * bx * (T - T_ref),
                (1 - fs) * by * (T - T_ref))

    monkeypatch.setattr(V, "temperature_and_velocity", lagged)
    sim, T = _stratified(steps=3000)
    assert np.abs(sim.T[:, 0] - T).max() > 1e-5
