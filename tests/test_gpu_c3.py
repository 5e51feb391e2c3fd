"""The largest configuration: a 4096 x 4096 cavity with 8192 disks (D = 16)
and per-particle conductivity ratios 10^U[-1, 1].

* FP32 against the FP64 oracle after 2 steps, every cell (the oracle needs
  about a minute and a half for them).
* FP16 and BF16 population storage (stochastic rounding) against the FP32
  GPU run over 200 steps (snapshots every 50): the reduced-precision bar u,
  T <= 1e-3 relative L2 and settling velocities within 1 %; regression
  bounds at about twice the measured errors.  The 16-bit storages are
  compared with the oracle itself over 1000 steps on a dense 512^2 window of
  this configuration's shape (tests/test_gpu_dense_window.py)."""
import numpy as np
import pytest

from helpers import gpu_lattice, oracle_sim, rel_l2
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _case():
    return W.cavity(side=4096, n=8192, k_log_uniform=True)


def test_c3_first_steps_against_oracle():
    case = _case()
    sim = oracle_sim(case)
    sim.step(2)
    ref = sim.fields()
    rp = sim.particle_state()
    with gpu_lattice(case, precision="fp32") as lat:
        lat.step(2)
        got = lat.fields()
        ps = lat.particles()
    assert rel_l2(got["rho"], ref["rho"]) < 1e-6
    assert rel_l2(np.stack([got["ux"], got["uy"]]), np.stack([ref["ux"], ref["uy"]])) < 1e-5
    assert rel_l2(got["T"], ref["T"]) < 1e-6
    assert np.abs(got["fs"] - ref["fs"]).max() < 1e-5
    assert np.abs(ps["y"] - rp["y"]).max() < 1e-9


_runs = {}


def _run(name):
    if name in _runs:
        return _runs[name]
    from paper_2410_23802_gb300 import vlb as V
    case = _case()
    prm = {k: v for k, v in case.params.items() if k != "precision"}
    code = {"fp32": V.VLB_FP32, "fp16": V.VLB_FP16_STORE, "bf16": V.VLB_BF16_STORE}[name]
    p = V.vlb_params_default(precision=code, max_particles=len(case.x), **prm)
    snaps = []
    with V.Lattice(p) as lat:
        lat.add_particles(np.column_stack([case.x, case.y]), case.radius, case.T0, k_ratio=case.k_ratio)
        for _ in range(4):
            lat.step(50)
            f = lat.fields()
            snaps.append((np.stack([f["ux"], f["uy"]]), f["T"], lat.particles()["uy"].copy()))
    _runs[name] = snaps
    return snaps


def _errors(name):
    a, b = _run(name), _run("fp32")
    return {
        "u": rel_l2(np.stack([s[0] for s in a]), np.stack([s[0] for s in b])),
        "T": rel_l2(np.stack([s[1] for s in a]), np.stack([s[1] for s in b])),
        "v": float(np.abs(a[-1][2] - b[-1][2]).max() / np.abs(b[-1][2]).max()),
    }


BAR = {"u": 1e-3, "T": 1e-3, "v": 1e-2}
# measured (stochastic rounding): fp16 u 2.27e-4, T 4.8e-5, v 1.4e-4; bf16 u 1.8e-3 (misses), T 3.9e-4, v 1.0e-3
REGRESSION = {"fp16": {"u": 5e-4, "T": 1e-4, "v": 5e-4}, "bf16": {"u": 4e-3, "T": 8e-4, "v": 2e-3}}


def _cases():
    for name in ("fp16", "bf16"):
        for q in ("u", "T", "v"):
            marks = [pytest.mark.xfail(strict=True, reason="BF16 significand noise")] if (name, q) == ("bf16", "u") else []
            yield pytest.param(name, q, marks=marks, id=f"{name}-{q}")


@pytest.mark.parametrize("name,quantity", list(_cases()))
def test_c3_reduced_precision_bar(name, quantity):
    e = _errors(name)
    print(name, {k: f"{v:.3e}" for k, v in e.items()})
    assert e[quantity] < BAR[quantity], e[quantity]


@pytest.mark.parametrize("name", ["fp16", "bf16"])
def test_c3_reduced_precision_regression(name):
    e = _errors(name)
    for q, bound in REGRESSION[name].items():
        assert e[q] < bound, (q, e[q])
