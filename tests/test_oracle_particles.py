"""Pins of the oracle's particle dynamics (Sec. 2.3) and contact model.

* With the hydrodynamic MES force switched off, Eqs. 26, 29, 30 by forward
  Euler with the backward-differenced inside-fluid force give the linear
  recursion a_n = (M_in/M) a_{n-1} + B/M for the velocity increments, whose
  closed form a_n = (B/M)(1 - r^{n+1})/(1 - r), r = 1/rho_r, tends to the
  acceleration g of the rigid body with its added inside fluid.
* Contact pairs of a chain of disks placed at known gaps; Newton's third law
  holds bitwise; the wall force of a disk at a known distance."""
import math

import numpy as np
import pytest

from oracle import vlbref as V


def test_free_fall_closed_form():
    rho_r, g = 1.5, -2e-5
    prm = V.Params(nx=40, ny=200, rho_ratio=rho_r, gravity=(0.0, g))
    sim = V.Simulation(prm, [20.0], [150.0], [6.0], [1.0])
    M = sim.mass[0]
    B = (rho_r - 1.0) * math.pi * 36.0 * g
    r = 1.0 / rho_r
    U, Y = 0.0, 150.0
    for n in range(200):
        sim.F_mes[:] = 0.0
        sim.T_mes[:] = 0.0
        sim._particle_update()
        Y += U
        U += (B / M) * (1 - r ** (n + 1)) / (1 - r)
        assert abs(sim.part["uy"][0] - U) < 1e-17 + 1e-12 * abs(U)
        assert abs(sim.part["y"][0] - Y) < 1e-12
    assert abs((sim.part["uy"][0] - sim.part["uy_prev"][0]) - g) < 1e-9 * abs(g)


def test_contact_pairs_of_a_chain():
    zeta = 2.0
    R = np.array([4.0, 4.0, 4.0, 4.0, 4.0])
    gaps = [1.0, 2.0, 1.999, 3.0]  # surface gaps between neighbours
    X = [10.0]
    for gp in gaps:
        X.append(X[-1] + 8.0 + gp)
    X = np.array(X)
    Y = np.full(5, 20.0)
    pairs = V.contact_pairs(X, Y, R, zeta)
    assert pairs == [(0, 1), (2, 3)]


def test_contact_third_law_and_wall_force():
    rng = np.random.default_rng(9)
    prm = V.Params(nx=60, ny=60, rho_ratio=1.3, gravity=(0.0, -1e-4), contact_eps_p=0.01, contact_eps_w=0.005)
    X = np.array([20.0, 28.9, 24.0, 55.5])
    Y = np.array([20.0, 21.0, 27.5, 30.0])
    R = np.array([4.0, 4.5, 3.0, 4.0])
    pairs = V.contact_pairs(X, Y, R, prm.contact_range)
    F = V.contact_forces(X, Y, R, prm, pairs)
    # particle 3 only touches the x+ wall at distance 4.5 (image gap 2R + zeta - 2d = 1)
    c = 0.3 * 1.0 * 1e-4 * math.pi * 16.0
    ref = -(c / 0.005) * (1.0 / 2.0) ** 2
    assert abs(F[3, 0] - ref) < 1e-13 * abs(ref)
    assert F[3, 1] == 0.0
    # pairwise forces are equal and opposite, bit for bit
    for i, j in pairs:
        fij = V.contact_forces(X[[i, j]], Y[[i, j]], R[[i, j]],
                               V.Params(nx=10 ** 6, ny=10 ** 6, rho_ratio=1.3, gravity=(0.0, -1e-4),
                                        periodic=(True, True)), [(0, 1)])
        assert fij[0, 0] == -fij[1, 0] and fij[0, 1] == -fij[1, 1]
        assert fij[0, 0] * (X[i] - X[j]) > 0  # repulsive


def test_insertion_into_a_rest_state_keeps_it_at_rest():
    """Mid-run insertion (reading R12) pinned by what must not change: disks
    of the fluid's density inserted at rest into a fluid at rest at one
    temperature, without gravity, leave the flow at rest, the temperature
    uniform and the mass of the closed box unchanged, whatever R_cv and
    R_lambda (only f_s and c_v change)."""
    import numpy as np
    from oracle import vlbref as O
    prm = O.Params(nx=48, ny=40, tau_f=0.8, rho_ratio=1.0, cv_ratio=2.5, k_ratio_default=4.0, T_fluid_init=0.6,
                   T_ref=0.6)
    sim = O.Simulation(prm, [14.0], [12.0], [5.0], [0.6])
    sim.step(5)
    m0 = sim.audit()[0]
    sim.insert_particles([31.3, 20.2], [25.6, 30.1], [6.0, 4.5], [0.6, 0.6], k_ratio=[0.3, 8.0])
    sim.step(20)
    assert np.abs(sim.ux).max() < 1e-14 and np.abs(sim.uy).max() < 1e-14
    assert np.abs(sim.T - 0.6).max() < 1e-13
    assert abs(sim.audit()[0] / m0 - 1) < 1e-14
    assert (sim.ras.fs > 0).sum() > 200  # the new disks are in the raster


def test_insertion_before_the_first_step_equals_construction():
    import numpy as np
    from oracle import vlbref as O
    prm = O.Params(nx=40, ny=40, rho_ratio=1.4, gravity=(0.0, -1e-4), beta=2.0, T_ref=1.0)
    a = O.Simulation(prm, [12.0, 28.0], [26.0, 20.0], [5.0, 4.0], [0.0, 0.5])
    st, h = O.vlbref_create(prm)
    O.vlbref_add_particles(h, 1, [12.0, 26.0], [5.0], [0.0])
    O.vlbref_insert_particles(h, 1, [28.0, 20.0], [4.0], [0.5])
    O.vlbref_step(h, 6)
    a.step(6)
    assert np.array_equal(h.sim.fields()["T"], a.fields()["T"])
    assert np.array_equal(h.sim.particle_state()["y"], a.particle_state()["y"])
