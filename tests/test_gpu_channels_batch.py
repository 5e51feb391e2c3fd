"""Many independent channels stepped together (vlb_step_batch): 256 seeded
single-disk channels, widths 64..256, each 4 widths long.

* Batching changes nothing: every case stepped in the batch is bit for bit
  the case stepped alone with vlb_step (fields, particle state, step count),
  also in a batch that mixes FP32, FP64, FP16 and BF16 storage, held
  particles, many disks in contact range, an ellipse in a channel with an
  open bottom and none (one persistent launch of each lattice kernel variant
  per step), and with single steps between calls.
* The batch against the FP64 oracle: the narrowest, the widest and one
  middle channel of the 256-case batch, element by element (FP32 bar: 1e-5
  relative L2 on rho, u, T; 1e-4 on the particle).
* Argument errors: a repeated or NULL handle, negative counts."""
import numpy as np
import pytest

from helpers import gpu_lattice, oracle_sim, rel_l2
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _state(lat):
    from paper_2410_23802_gb300 import vlb as V
    return lat.fields(), lat.particles(), V.vlb_get_step(lat.h)


def _same(a, b):
    fa, pa, sa = a
    fb, pb, sb = b
    assert sa == sb
    for k in fa:
        assert np.array_equal(fa[k], fb[k], equal_nan=True), k
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k


def _mixed_cases():
    """Cases whose batch needs several lattice kernels (FP32, FP64, FP16 and
    BF16 storage, the held-temperature path), many particles with contacts,
    and none."""
    import dataclasses
    ch = W.channels(n=6, seed=7)
    cav = W.cavity(side=96, n=6, seed=2)
    empty = dataclasses.replace(W.channels(n=1, seed=9)[0], x=[], y=[], radius=[], T0=[])
    held = dataclasses.replace(ch[5], fixed_T=[1])
    ell = W.ellipse_sedimentation(length_w=5.0)
    return [(ch[0], "fp32"), (ch[1], "fp32"), (ch[2], "fp64"), (ch[3], "fp16"), (ch[4], "bf16"),
            (held, "fp32"), (cav, "fp32"), (empty, "fp32"), (cav, "fp64"), (ell, "fp32")]


@pytest.fixture(params=[0, 1], ids=["tiles", "persistent"])
def batch_form(request):
    from paper_2410_23802_gb300 import vlb as V
    old = V.vlb_get_batch_form()
    V.vlb_set_batch_form(request.param)
    yield request.param
    V.vlb_set_batch_form(old)


def test_batch_equals_alone(batch_form):
    from paper_2410_23802_gb300 import vlb as V
    cases = _mixed_cases()
    chunks = (1, 17, 30, 0, 2)  # uneven calls, both parities; 50 steps in all
    lats = [gpu_lattice(c, precision=p) for c, p in cases]
    try:
        for k in chunks:
            V.vlb_step_batch([l.h for l in lats], k)
        got = [_state(l) for l in lats]
    finally:
        for l in lats:
            l.close()
    for (c, p), g in zip(cases, got):
        with gpu_lattice(c, precision=p) as lat:
            lat.step(sum(chunks))
            _same(g, _state(lat))


def test_batch_then_single_steps_continue(batch_form):
    """vlb_step after vlb_step_batch (and the other way round) continues the
    same levels: buffer and list parities and band stamps carry over."""
    from paper_2410_23802_gb300 import vlb as V
    cases = _mixed_cases()[:3] + _mixed_cases()[6:7]
    lats = [gpu_lattice(c, precision=p) for c, p in cases]
    try:
        V.vlb_step_batch([l.h for l in lats], 3)
        for l in lats:
            l.step(2)
        V.vlb_step_batch([l.h for l in lats[::-1]], 5)
        got = [_state(l) for l in lats]
    finally:
        for l in lats:
            l.close()
    for (c, p), g in zip(cases, got):
        with gpu_lattice(c, precision=p) as lat:
            lat.step(10)
            _same(g, _state(lat))


def test_batch_of_256_against_oracle():
    from paper_2410_23802_gb300 import vlb as V
    cases = W.channels()
    widths = [c.params["nx"] for c in cases]
    pick = sorted({int(np.argmin(widths)), int(np.argmax(widths)), len(cases) // 2})
    steps = 100
    lats = [gpu_lattice(c) for c in cases]
    try:
        V.vlb_step_batch([l.h for l in lats], steps)
        got = {i: (lats[i].fields(), lats[i].particles()) for i in pick}
        # every case advanced and stayed healthy
        for l in lats:
            assert V.vlb_get_step(l.h) == steps
            V.vlb_synchronize(l.h)
    finally:
        for l in lats:
            l.close()
    for i in pick:
        sim = oracle_sim(cases[i])
        sim.step(steps)
        ref, rp = sim.fields(), sim.particle_state()
        f, p = got[i]
        assert rel_l2(f["rho"], ref["rho"]) < 1e-5
        assert rel_l2(np.stack([f["ux"], f["uy"]]), np.stack([ref["ux"], ref["uy"]])) < 1e-5, i
        assert rel_l2(f["T"], ref["T"]) < 1e-5, i
        assert np.abs(f["fs"] - ref["fs"]).max() < 1e-4
        assert np.abs(p["y"] - rp["y"]).max() < 1e-4
        umax = max(np.hypot(rp["ux"], rp["uy"]).max(), 1e-30)
        assert np.abs(p["uy"] - rp["uy"]).max() / umax < 1e-4


def test_batch_argument_errors():
    from paper_2410_23802_gb300 import vlb as V
    cases = W.channels(n=2, seed=3)
    with gpu_lattice(cases[0]) as a, gpu_lattice(cases[1]) as b:
        with pytest.raises(V.VlbError, match="EINVAL"):
            V.vlb_step_batch([a.h, b.h, a.h], 1)
        with pytest.raises(V.VlbError, match="EINVAL"):
            V.vlb_step_batch([a.h, None], 1)
        with pytest.raises(V.VlbError, match="EINVAL"):
            V.vlb_step_batch([a.h, b.h], -1)
        V.vlb_step_batch([], 5)            # nothing to do
        V.vlb_step_batch([a.h, b.h], 0)    # initialises only
        assert V.vlb_get_step(a.h) == 0
        V.vlb_step_batch([b.h, a.h], 2)
        assert V.vlb_get_step(a.h) == V.vlb_get_step(b.h) == 2


def test_channels_for_5000_steps():
    """The whole configuration: 256 channels, 5000 steps each, batched.  No
    case raises a device flag, every disk has settled (more than 1 lu down,
    slower than 0.5 lu per step; a disk that reached the bottom may rebound
    through the wall contact force), and the narrowest channel still matches
    the oracle element by element after its first 500 steps (FP32 bar)."""
    from paper_2410_23802_gb300 import vlb as V
    cases = W.channels()
    narrow = int(np.argmin([c.params["nx"] for c in cases]))
    lats = [gpu_lattice(c) for c in cases]
    try:
        hs = [l.h for l in lats]
        V.vlb_step_batch(hs, 500)
        f500, p500 = lats[narrow].fields(), lats[narrow].particles()
        V.vlb_step_batch(hs, 4500)
        ps = []
        for l in lats:
            V.vlb_synchronize(l.h)  # raises on any device flag
            assert V.vlb_get_step(l.h) == 5000
            ps.append(l.particles())
    finally:
        for l in lats:
            l.close()
    for c, p in zip(cases, ps):
        assert p["y"][0] < c.y[0] - 1.0
        assert np.hypot(p["ux"][0], p["uy"][0]) < 0.5
    sim = oracle_sim(cases[narrow])
    sim.step(500)
    ref, rp = sim.fields(), sim.particle_state()
    assert rel_l2(np.stack([f500["ux"], f500["uy"]]), np.stack([ref["ux"], ref["uy"]])) < 1e-5
    assert rel_l2(f500["T"], ref["T"]) < 1e-5
    assert np.abs(p500["y"] - rp["y"]).max() < 1e-4
