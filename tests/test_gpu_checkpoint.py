"""Checkpoint and resume (vlb_state_size / vlb_save_state / vlb_load_state).

A run that is saved after n steps and restored into a fresh handle continues
bit for bit: after m more steps on both, fields, particle state and step
count are identical to the uninterrupted run.  Images of other handles are
rejected."""
import numpy as np
import pytest

from helpers import gpu_lattice
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N_BEFORE, N_AFTER = 40, 25


def _snapshot(lat):
    from paper_2410_23802_gb300 import vlb as V
    return lat.fields(), lat.particles(), V.vlb_get_step(lat.h)


def _assert_same(a, b):
    fa, pa, sa = a
    fb, pb, sb = b
    assert sa == sb
    for k in fa:
        assert np.array_equal(fa[k], fb[k], equal_nan=True), k
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k


@pytest.mark.parametrize("precision,held", [("fp32", False), ("fp64", False), ("fp32", True)])
def test_resume_continues_bit_for_bit(tmp_path, precision, held):
    import dataclasses
    case = W.cavity(side=128, n=16, seed=11, k_log_uniform=True)
    if held:  # the held flags travel with the image (the fresh handle does not set them)
        case = dataclasses.replace(case, fixed_T=[k % 3 == 0 for k in range(16)])
    with gpu_lattice(case, precision=precision) as a:
        a.step(N_BEFORE)
        path = tmp_path / "state.bin"
        img = a.save_state(path)
        a.step(N_AFTER)
        ref = _snapshot(a)
    # from the in-memory image and from the file, each into a fresh handle
    fresh = dataclasses.replace(case, fixed_T=None)
    for source in (img, str(path)):
        with gpu_lattice(fresh, precision=precision) as b:
            b.load_state(source)
            b.step(N_AFTER)
            _assert_same(_snapshot(b), ref)


def test_resume_reads_fields_of_the_saved_level():
    case = W.cavity(side=96, n=6, seed=2)
    with gpu_lattice(case) as a:
        a.step(30)
        img = a.save_state()
        ref = _snapshot(a)
    with gpu_lattice(case) as b:
        b.load_state(img)
        _assert_same(_snapshot(b), ref)


def test_foreign_image_is_rejected():
    from paper_2410_23802_gb300 import vlb as V
    case = W.cavity(side=96, n=6, seed=2)
    with gpu_lattice(case) as a:
        a.step(3)
        img = a.save_state()
    other = W.cavity(side=128, n=6, seed=2)
    with gpu_lattice(other) as b:
        with pytest.raises(V.VlbError, match="EINVAL"):
            b.load_state(img)
    with gpu_lattice(case) as b:
        bad = img.copy()
        bad[:8] = 0
        with pytest.raises(V.VlbError, match="EINVAL"):
            b.load_state(bad)
        with pytest.raises(V.VlbError, match="EINVAL"):
            b.load_state(img[: len(img) // 2])
