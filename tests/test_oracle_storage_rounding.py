"""What 16-bit population storage costs, measured on the oracle alone.

The FP64 oracle is run twice on the settling-disk channel: once as it is, once
with every post-collision population rounded to FP16 or BF16 (as the deviation
from the rest equilibrium that the CUDA path stores) before streaming.  The
u error of that rounding alone, over stacked snapshots of 1000 steps, already
exceeds the 1e-3 bar of the reduced-precision parity check, so a CUDA path
with 16-bit population storage cannot meet it whatever its arithmetic.  CPU
only; about a minute and a half."""
import numpy as np
import pytest

from helpers import oracle_sim, rel_l2
from oracle import vlbref as O
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.slow

SNAP, NSNAP = 100, 10


def _bf16(x):
    """Round to BF16 (nearest even), returned as float64."""
    b = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _fp16(x):
    return x.astype(np.float32).astype(np.float16).astype(np.float64)


def _snapshots(sim):
    out = []
    for _ in range(NSNAP):
        sim.step(SNAP)
        f = sim.fields()
        out.append((np.stack([f["ux"], f["uy"]]), f["T"].copy()))
    return out


@pytest.fixture(scope="module")
def exact():
    return _snapshots(oracle_sim(W.channel()))


@pytest.mark.parametrize("name,rnd,u_min", [("fp16", _fp16, 1e-3), ("bf16", _bf16, 1e-2)])
def test_storage_rounding_alone_misses_the_bar(exact, monkeypatch, name, rnd, u_min):
    case = W.channel()
    sim = oracle_sim(case)
    p = sim.prm
    w = O.feq(np.ones((1, 1)), np.zeros((1, 1)), np.zeros((1, 1)))
    g_rest = O.geq(np.full((1, 1), p.T_fluid_init * 1.0), np.full((1, 1), p.T_fluid_init), p.cref)
    collide_f, collide_g = O.collide_flow, O.collide_thermal
    monkeypatch.setattr(O, "collide_flow", lambda *a: w + rnd(collide_f(*a) - w))
    monkeypatch.setattr(O, "collide_thermal", lambda *a: g_rest + rnd(collide_g(*a) - g_rest))
    rounded = _snapshots(sim)
    e_u = rel_l2(np.stack([r[0] for r in rounded]), np.stack([e[0] for e in exact]))
    e_T = rel_l2(np.stack([r[1] for r in rounded]), np.stack([e[1] for e in exact]))
    print(f"{name}: u {e_u:.3e}  T {e_T:.3e}")
    assert u_min < e_u < 10 * u_min, e_u
    assert e_T < e_u
