"""GPU vs oracle parity of the whole hot path, element by element on the
same seeded inputs: macroscopic rho, u, T over stacked snapshots (relative
L2), particle position (absolute) and velocity (relative to max |U|).

FP32 tolerances: 1e-5 relative L2 on rho, u, T; 1e-4 on particle position
and velocity over the first 1000 steps.  FP64: 1e-9."""
import numpy as np
import pytest

from helpers import gpu_lattice, oracle_sim, rel_l2
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SNAP = 100


def _oracle_snapshots(case, nsnap, **over):
    sim = oracle_sim(case, **over)
    out = []
    for _ in range(nsnap):
        sim.step(SNAP)
        out.append(({k: v.copy() for k, v in sim.fields().items()},
                    sim.particle_state(), sim.audit()))
    return out


def _gpu_snapshots(case, nsnap, precision, **over):
    out = []
    with gpu_lattice(case, precision=precision, **over) as lat:
        for _ in range(nsnap):
            lat.step(SNAP)
            out.append((lat.fields(), lat.particles(), lat.audit()))
    return out


def _compare(gpu, ref, tol_field, tol_pos, tol_vel):
    stack = lambda snaps, k: np.stack([s[0][k] for s in snaps])  # noqa: E731
    e_rho = rel_l2(stack(gpu, "rho"), stack(ref, "rho"))
    u_g = np.stack([stack(gpu, "ux"), stack(gpu, "uy")])
    u_r = np.stack([stack(ref, "ux"), stack(ref, "uy")])
    e_u = rel_l2(u_g, u_r)
    e_T = rel_l2(stack(gpu, "T"), stack(ref, "T"))
    e_fs = np.abs(stack(gpu, "fs") - stack(ref, "fs")).max()
    assert e_rho < tol_field, e_rho
    assert e_u < tol_field, e_u
    assert e_T < tol_field, e_T
    assert e_fs < 1e-4, e_fs
    if len(ref[0][1]["x"]):
        pos = max(max(np.abs(g[1]["x"] - r[1]["x"]).max(), np.abs(g[1]["y"] - r[1]["y"]).max())
                  for g, r in zip(gpu, ref))
        umax = max(np.hypot(r[1]["ux"], r[1]["uy"]).max() for r in ref)
        vel = max(max(np.abs(g[1]["ux"] - r[1]["ux"]).max(), np.abs(g[1]["uy"] - r[1]["uy"]).max())
                  for g, r in zip(gpu, ref)) / max(umax, 1e-30)
        assert pos < tol_pos, pos
        assert vel < tol_vel, vel
    return e_rho, e_u, e_T


@pytest.fixture(scope="module")
def channel_ref():
    return _oracle_snapshots(W.channel(), 10)


def test_channel_fp64(channel_ref):
    gpu = _gpu_snapshots(W.channel(), 4, "fp64")
    _compare(gpu, channel_ref[:4], 1e-9, 1e-9, 1e-9)


def test_channel_fp32(channel_ref):
    gpu = _gpu_snapshots(W.channel(), 10, "fp32")
    _compare(gpu, channel_ref, 1e-5, 1e-4, 1e-4)
    # mass audit of the GPU state against the oracle's
    for g, r in zip(gpu, channel_ref):
        assert abs(g[2][0] - r[2][0]) / r[2][0] < 1e-6
        assert abs(g[2][1] - r[2][1]) / abs(r[2][1]) < 1e-5
        assert abs(g[2][2] - r[2][2]) / abs(r[2][2]) < 1e-5


def test_small_cavity_fp32():
    case = W.cavity(side=160, n=24, seed=3)
    ref = _oracle_snapshots(case, 3)
    gpu = _gpu_snapshots(case, 3, "fp32")
    _compare(gpu, ref, 1e-5, 1e-4, 1e-4)


def test_small_cavity_per_particle_conductivity_fp32():
    case = W.cavity(side=128, n=16, seed=5, k_log_uniform=True)
    ref = _oracle_snapshots(case, 2)
    gpu = _gpu_snapshots(case, 2, "fp32")
    _compare(gpu, ref, 1e-5, 1e-4, 1e-4)


def test_ragged_periodic_no_particles():
    # natural convection in a vertical slot, periodic in y: hot wall x-, cold wall x+
    params = dict(nx=37, ny=29, tau_f=0.7, prandtl=0.7, rho_ratio=1.5, cv_ratio=1.0, k_ratio_default=1.0,
                  gravity=(0.0, -1e-5), beta=50.0, T_ref=0.5, T_fluid_init=0.5, thermal_wall=(1, 1, 0, 0),
                  wall_T=(1.0, 0.0, 0.0, 0.0), periodic=(0, 1))
    case = W.Case("ragged periodic", params, [], [], [], [])
    ref = _oracle_snapshots(case, 2)
    for prec, tol in (("fp32", 1e-5), ("fp64", 1e-11)):
        gpu = _gpu_snapshots(case, 2, prec)
        _compare(gpu, ref, tol, 0, 0)


def test_particle_against_wall_with_contact():
    params = dict(nx=64, ny=80, tau_f=0.8, prandtl=0.7, rho_ratio=2.0, cv_ratio=1.5, k_ratio_default=2.0,
                  gravity=(0.0, -2e-4), beta=5.0, T_ref=1.0, T_fluid_init=1.0)
    # the lower disk starts within the contact range of the bottom wall
    case = W.Case("wall contact", params, [32.0, 30.0], [6.5, 24.0], [5.0, 5.0], [0.0, 0.5])
    ref = _oracle_snapshots(case, 3)
    gpu = _gpu_snapshots(case, 3, "fp32")
    _compare(gpu, ref, 1e-5, 1e-4, 1e-4)
    assert ref[-1][1]["y"][0] > 5.0  # the wall force held the disk up


def test_rest_state_stays_at_rest():
    params = dict(nx=33, ny=17, tau_f=0.9, prandtl=0.7, rho_ratio=1.5, cv_ratio=1.0, k_ratio_default=1.0,
                  gravity=(0.0, 0.0), beta=0.0, T_ref=1.0, T_fluid_init=0.3)
    case = W.Case("rest", params, [], [], [], [])
    with gpu_lattice(case, precision="fp32") as lat:
        lat.step(0)
        lat.step(50)
        f = lat.fields()
    assert np.abs(f["rho"] - 1).max() < 1e-6 and np.abs(f["ux"]).max() < 1e-7
    assert np.abs(f["T"] - 0.3).max() < 1e-6


def test_state_errors():
    from paper_2410_23802_gb300 import vlb as V
    case = W.channel()
    with gpu_lattice(case, precision="fp32", max_particles=4) as lat:
        with pytest.raises(V.VlbError) as e:
            lat.add_particles([[20.0, 20.0], [27.0, 20.0]], [4.0, 4.0], [0.0, 0.0])  # overlap
        assert e.value.status == V.VLB_EINVAL
        with pytest.raises(V.VlbError) as e:
            lat.add_particles([[2.0, 20.0]], [4.0], [0.0])  # outside the walls
        assert e.value.status == V.VLB_EINVAL
        lat.step(1)
        with pytest.raises(V.VlbError) as e:
            lat.add_particles([[70.0, 100.0]], [4.0], [0.0])
        assert e.value.status == V.VLB_ESTATE


def test_full_size_cavity_first_steps():
    """The bench workload at full size (2048^2, 2048 disks): all fields after
    3 steps, element by element."""
    case = W.cavity()
    sim = oracle_sim(case)
    sim.step(3)
    ref = sim.fields()
    with gpu_lattice(case, precision="fp32") as lat:
        lat.step(3)
        got = lat.fields()
        ps = lat.particles()
    assert rel_l2(got["rho"], ref["rho"]) < 1e-6
    assert rel_l2(np.stack([got["ux"], got["uy"]]), np.stack([ref["ux"], ref["uy"]])) < 1e-5
    assert rel_l2(got["T"], ref["T"]) < 1e-6
    assert np.abs(got["fs"] - ref["fs"]).max() < 1e-5
    rp = sim.particle_state()
    assert np.abs(ps["y"] - rp["y"]).max() < 1e-9


def test_partial_particle_state_read():
    """vlb_get_particle_state for the first n of N particles returns exactly
    their part of the full read (one strided copy of n elements per array)."""
    from paper_2410_23802_gb300 import vlb as V
    case = W.cavity(side=128, n=16, seed=11)
    with gpu_lattice(case, max_particles=24) as lat:
        lat.step(12)
        full = V.vlb_get_particle_state(lat.h)
        part = V.vlb_get_particle_state(lat.h, 5)
        none = V.vlb_get_particle_state(lat.h, 0)
    for k in full:
        assert np.array_equal(part[k], full[k][:5]), k
        assert none[k].shape == (0,)


def test_async_particle_state_reads_every_step():
    """Copies queued after each step and collected one step later equal the
    synchronous reads of the same levels; the ring holds two copies."""
    from paper_2410_23802_gb300 import vlb as V
    case = W.cavity(side=128, n=16, seed=11)
    sync = []
    with gpu_lattice(case) as a:
        for _ in range(6):
            a.step(1)
            sync.append(V.vlb_get_particle_state(a.h))
    got = []
    with gpu_lattice(case) as b:
        with pytest.raises(V.VlbError, match="ESTATE"):
            V.vlb_particle_state_wait(b.h, 16)
        b.step(1)
        V.vlb_particle_state_async(b.h, 16)
        for k in range(1, 6):
            b.step(1)
            V.vlb_particle_state_async(b.h, 16)
            with pytest.raises(V.VlbError, match="ESTATE"):  # a third copy
                V.vlb_particle_state_async(b.h, 16)
            got.append(V.vlb_particle_state_wait(b.h, 16))
        got.append(V.vlb_particle_state_wait(b.h, 16))
    for k, ((st, step), ref) in enumerate(zip(got, sync)):
        assert step == k + 1
        assert np.array_equal(st["xy"][:, 0], ref["x"]) and np.array_equal(st["xy"][:, 1], ref["y"])
        assert np.array_equal(st["uv"][:, 1], ref["uy"]) and np.array_equal(st["omega"], ref["omega"])
        assert np.array_equal(st["force"][:, 1], ref["fy"]) and np.array_equal(st["torque"], ref["torque"])
