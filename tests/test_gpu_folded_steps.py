"""vlb_step of two or more steps folds each level's particle steps into the
lattice launch of the level before (lattice_folded_kernel: the CTA that
finishes the last tile of a particle's range runs its step).  Single steps
use the two-kernel form.  Both must give the same bits: a case stepped N
times by vlb_step(h, 1) equals the case stepped by one vlb_step(h, N), and
calls of both forms may alternate (fields, particle state, contact pairs,
step count), in FP32, FP64, FP16 and BF16 storage, with a held particle,
and on a dense cavity whose disks touch."""
import dataclasses

import numpy as np
import pytest

from helpers import gpu_lattice
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _state(lat):
    from paper_2410_23802_gb300 import vlb as V
    return lat.fields(), lat.particles(), V.vlb_get_step(lat.h), V.vlb_get_contact_pairs(lat.h)


def _same(a, b):
    fa, pa, sa, ca = a
    fb, pb, sb, cb = b
    assert sa == sb
    for k in fa:
        assert np.array_equal(fa[k], fb[k], equal_nan=True), k
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k
    assert np.array_equal(ca, cb)


def _cases():
    cav = W.cavity(side=192, n=40, seed=3, gap=0.5)
    held = dataclasses.replace(W.cavity(side=128, n=10, seed=5), fixed_T=[1, 0, 2, 0, 1, 0, 0, 0, 0, 0])
    return [(cav, "fp32"), (cav, "fp64"), (cav, "fp16"), (cav, "bf16"), (held, "fp32"),
            (W.channels(n=1, seed=2)[0], "fp32")]


@pytest.mark.parametrize("idx", range(6))
def test_folded_steps_equal_single_steps(idx):
    case, prec = _cases()[idx]
    with gpu_lattice(case, precision=prec) as a, gpu_lattice(case, precision=prec) as b:
        for _ in range(40):
            a.step(1)
        b.step(40)
        _same(_state(a), _state(b))
        # mixed calls continue the same levels
        a.step(7)
        a.step(1)
        a.step(2)
        for _ in range(10):
            b.step(1)
        _same(_state(a), _state(b))
