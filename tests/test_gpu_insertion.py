"""Mid-run particle insertion (vlb_insert_particles, reading R12) against
the oracle doing the same: a cavity stepped 20 times, two disks inserted in
its lower part (one moving), 30 more steps; fields and particle state
element by element (FP32 bar 1e-5 relative L2 and 1e-4 on the particles;
FP64 1e-9).  Refusals: a disk larger than the band tables hold, one
overlapping a disk where that disk is now, one beyond max_particles."""
import numpy as np
import pytest

from helpers import gpu_lattice, oracle_sim, rel_l2
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NEW_XY = [[40.0, 25.0], [90.0, 30.0]]
NEW_R = [5.0, 6.5]
NEW_T = [0.0, 0.3]
NEW_UV = [[0.0, 0.0], [0.004, -0.002]]


def _case():
    return W.cavity(side=128, n=8, seed=11, k_log_uniform=True)


@pytest.mark.parametrize("precision,tol,ptol", [("fp32", 1e-5, 1e-4), ("fp64", 1e-9, 1e-9)])
def test_insertion_matches_oracle(precision, tol, ptol):
    case = _case()
    with gpu_lattice(case, precision=precision, max_particles=12) as lat:
        lat.step(20)
        lat.insert_particles(NEW_XY, NEW_R, NEW_T, k_ratio=[2.0, 0.5], uv=NEW_UV)
        lat.step(30)
        f, p = lat.fields(), lat.particles()
    sim = oracle_sim(case)
    sim.step(20)
    xy = np.array(NEW_XY)
    uv = np.array(NEW_UV)
    sim.insert_particles(xy[:, 0], xy[:, 1], NEW_R, NEW_T, k_ratio=[2.0, 0.5], ux=uv[:, 0], uy=uv[:, 1])
    sim.step(30)
    ref, rp = sim.fields(), sim.particle_state()
    assert len(p["x"]) == 10
    assert rel_l2(f["rho"], ref["rho"]) < tol
    assert rel_l2(np.stack([f["ux"], f["uy"]]), np.stack([ref["ux"], ref["uy"]])) < tol
    assert rel_l2(f["T"], ref["T"]) < tol
    assert np.abs(f["fs"] - ref["fs"]).max() < 1e-4
    assert max(np.abs(p["x"] - rp["x"]).max(), np.abs(p["y"] - rp["y"]).max()) < ptol
    umax = np.hypot(rp["ux"], rp["uy"]).max()
    assert np.abs(p["uy"] - rp["uy"]).max() / umax < ptol


def test_insertion_refusals():
    from paper_2410_23802_gb300 import vlb as V
    case = _case()
    with gpu_lattice(case, max_particles=9) as lat:
        lat.step(5)
        with pytest.raises(V.VlbError, match="EINVAL"):   # larger than the band tables hold (R <= 8)
            lat.insert_particles([[40.0, 25.0]], [9.0], [0.0])
        with pytest.raises(V.VlbError, match="EINVAL"):   # overlaps a disk where it is now
            p = lat.particles()
            lat.insert_particles([[p["x"][0] + 3.0, p["y"][0]]], [4.0], [0.0])
        with pytest.raises(V.VlbError, match="EOVERFLOW"):  # beyond max_particles
            lat.insert_particles(NEW_XY, NEW_R, NEW_T)
        lat.insert_particles(NEW_XY[:1], NEW_R[:1], NEW_T[:1])
        lat.step(5)
        assert len(lat.particles()["x"]) == 9


def test_no_disk_reaches_across_a_periodic_boundary():
    """On a periodic axis a disk must keep R + 1 from the boundary (reading
    R7), so two disks on opposite sides stay at least R1 + R2 + 2 apart
    through it and can neither overlap nor touch there; a disk placed closer
    to the boundary, which would touch one on the other side, is refused on
    adding and on insertion, like the oracle's twin of the call."""
    from oracle import vlbref as O
    from paper_2410_23802_gb300 import vlb as V
    params = dict(nx=96, ny=64, tau_f=0.8, prandtl=0.7, rho_ratio=1.5, cv_ratio=1.5, k_ratio_default=2.0,
                  gravity=(0.0, -1e-5), beta=0.0, T_ref=1.0, T_fluid_init=1.0, periodic=(1, 0))
    case = W.Case("periodic channel", params, [7.0], [30.0], [6.0], [0.0])
    across = [[96.0 - 4.0, 30.0]]  # 9 lu from the first disk through the boundary, R1 + R2 = 11
    with gpu_lattice(case, max_particles=3) as lat:
        with pytest.raises(V.VlbError, match="EINVAL"):
            lat.add_particles(across, [5.0], [0.0])
        lat.add_particles([[90.0, 30.0]], [5.0], [0.0])  # R + 1 from the boundary, 13 lu through it: accepted
        lat.step(3)
        with pytest.raises(V.VlbError, match="EINVAL"):
            lat.insert_particles(across, [5.0], [0.0])
    st, h = O.vlbref_create(O.Params(**{**params, "periodic": (True, False)}))
    assert O.vlbref_add_particles(h, 1, [7.0, 30.0], [6.0], [0.0]) == O.VLBREF_OK
    assert O.vlbref_add_particles(h, 1, across[0], [5.0], [0.0]) == O.VLBREF_EINVAL
