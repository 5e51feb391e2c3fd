"""FP16 and BF16 storage of the populations (FP32 arithmetic, FP64 particle
sums and integration) against the FP64 oracle on the settling-disk channel.

The bar: u and T within 1e-3 relative L2 over stacked snapshots of the first
1000 steps, the settling velocity within 1 %.  Rounding the stored
populations to 16 bits misses part of it: the same rounding applied to the
oracle's own populations on the CPU gives the same errors to two digits
(FP16: u 1.18e-3; BF16: u 2.87e-2, T 4.12e-3, settling velocity 5e-2), so those checks are
expected failures (strict: a pass means the storage changed and the mark must
go).  Separate regression bounds at about twice the measured errors keep the
16-bit paths from getting worse unnoticed."""
import numpy as np
import pytest

from helpers import oracle_sim, rel_l2
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SNAP, NSNAP = 100, 10
BAR = {"u": 1e-3, "T": 1e-3, "v": 1e-2}
# measured: fp16 u 1.17e-3, T 1.2e-4, v 1.6e-3; bf16 u 2.9e-2, T 4.1e-3, v 5.2e-2
REGRESSION = {"fp16": {"u": 2.5e-3, "T": 3e-4, "v": 5e-3}, "bf16": {"u": 6e-2, "T": 1e-2, "v": 1e-1}}
MISSES = {("fp16", "u"), ("bf16", "u"), ("bf16", "T"), ("bf16", "v")}


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
            marks = [pytest.mark.xfail(strict=True, reason="16-bit population rounding")] if (precision, q) in MISSES else []
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
