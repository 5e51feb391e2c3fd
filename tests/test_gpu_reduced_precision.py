"""FP16 and BF16 storage of the populations (FP32 arithmetic, FP64 particle
sums and integration) against the FP64 oracle on the settling-disk channel.

The bar: u and T within 1e-3 relative L2 over stacked snapshots of the first
1000 steps, the settling velocity within 1 %.  The stored deviations are
rounded stochastically (unbiased, decorrelated from step to step).  With
round-to-nearest the same rounding error repeated every step wherever the
flow is steady and added up coherently in the exchange force, which took
FP16 to u 1.2e-3 and BF16 to u 2.9e-2 (the same numbers as the oracle with
its populations rounded the same way on the CPU).  Stochastic rounding leaves
only the noise: FP16 meets the whole bar; BF16 meets it for T and the
settling velocity, and its 8-bit significand keeps u near 2.5e-3 (the CPU
emulation gives the same), a strict expected failure (a pass means the
storage changed and the mark must go).  Regression bounds at about twice the
measured errors keep both from getting worse unnoticed."""
import numpy as np
import pytest

from helpers import oracle_sim, rel_l2
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SNAP, NSNAP = 100, 10
BAR = {"u": 1e-3, "T": 1e-3, "v": 1e-2}
# CPU emulation of the rounding alone: fp16 u 3.5e-4, T 1.1e-5, v 1.6e-4; bf16 u 2.5e-3, T 8.3e-5, v 6.6e-4
REGRESSION = {"fp16": {"u": 8e-4, "T": 5e-5, "v": 1e-3}, "bf16": {"u": 6e-3, "T": 3e-4, "v": 3e-3}}
MISSES = {("bf16", "u")}


@pytest.fixture(scope="module")
def channel_ref():
    sim = oracle_sim(W.channel())
    out = []
    for _ in range(NSNAP):
        sim.step(SNAP)
        out.append(({k: v.copy() for k, v in sim.fields().items()}, sim.particle_state()))
    return out


_cache = {}


def _errors(channel_ref, precision):
    if precision in _cache:
        return _cache[precision]
    from paper_2410_23802_gb300 import vlb as V
    prm = {k: v for k, v in W.channel().params.items() if k != "precision"}
    code = {"fp16": V.VLB_FP16_STORE, "bf16": V.VLB_BF16_STORE}[precision]
    p = V.vlb_params_default(precision=code, max_particles=1, **prm)
    case = W.channel()
    gpu = []
    with V.Lattice(p) as lat:
        lat.add_particles(np.column_stack([case.x, case.y]), case.radius, case.T0)
        for _ in range(NSNAP):
            lat.step(SNAP)
            gpu.append((lat.fields(), lat.particles()))
    st = lambda s, k: np.stack([x[0][k] for x in s])  # noqa: E731
    e = {
        "u": rel_l2(np.stack([st(gpu, "ux"), st(gpu, "uy")]), np.stack([st(channel_ref, "ux"), st(channel_ref, "uy")])),
        "T": rel_l2(st(gpu, "T"), st(channel_ref, "T")),
        "v": abs(gpu[-1][1]["uy"][0] - channel_ref[-1][1]["uy"][0]) / abs(channel_ref[-1][1]["uy"][0]),
    }
    print(f"{precision}: u {e['u']:.3e}  T {e['T']:.3e}  settling velocity {e['v']:.3e}")
    _cache[precision] = e
    return e


def _cases():
    for precision in ("fp16", "bf16"):
        for q in ("u", "T", "v"):
            marks = [pytest.mark.xfail(strict=True, reason="BF16 significand noise")] if (precision, q) in MISSES else []
            yield pytest.param(precision, q, marks=marks, id=f"{precision}-{q}")


@pytest.mark.parametrize("precision,quantity", list(_cases()))
def test_reduced_precision_bar(channel_ref, precision, quantity):
    e = _errors(channel_ref, precision)
    assert e[quantity] < BAR[quantity], e[quantity]


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_reduced_precision_regression(channel_ref, precision):
    e = _errors(channel_ref, precision)
    for q, bound in REGRESSION[precision].items():
        assert e[q] < bound, (q, e[q])
