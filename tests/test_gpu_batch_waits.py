"""The persistent form of the batched step (vlb_step_batch, form 1): its
bounded waits and its plain-launch form, and both forms on short calls.

* A wait made to run out: with the test hook, the particle steps of the
  first case of a two-case batch wait for a tile count that is never
  reached (limit 20 ms).  The call returns, that handle's next call reports
  VLB_ETIMEOUT, the other case of the same launches equals its solo run bit
  for bit, and a new batch afterwards equals its solo runs (the context stays
  usable).  Nothing faults or hangs: every wait ends by its time limit.
* On the legacy default stream, which cannot be captured into a CUDA graph,
  the same launches go out one by one; the cases still equal their solo runs.
* One-step and two-step calls (no graph replay) equal their solo runs."""
import numpy as np
import pytest

from helpers import gpu_lattice
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture
def form():
    """Sets the batched-step form for one test and restores the default."""
    from paper_2410_23802_gb300 import vlb as V
    old = V.vlb_get_batch_form()
    yield V.vlb_set_batch_form
    V.vlb_set_batch_form(old)


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


def _solo(case, steps, precision="fp32"):
    with gpu_lattice(case, precision=precision) as lat:
        lat.step(steps)
        return _state(lat)


def _cases():
    ch = W.channels(n=3, seed=11)
    return [ch[0], ch[1], W.cavity(side=96, n=5, seed=4)]


def test_wait_that_runs_out_reports_etimeout_and_leaves_the_context_usable(form):
    from paper_2410_23802_gb300 import vlb as V
    form(V.VLB_BATCH_PERSISTENT)
    stuck, other = _cases()[:2]
    lats = [gpu_lattice(stuck), gpu_lattice(other)]
    try:
        V.vlb_debug_batch_wait(20_000_000, 0)  # 20 ms; handle position 0 never gets its tiles
        try:
            V.vlb_step_batch([l.h for l in lats], 4)
            V.vlb_synchronize(lats[1].h)
        finally:
            V.vlb_debug_batch_wait(0, -1)
        with pytest.raises(V.VlbError, match="ETIMEOUT"):
            V.vlb_synchronize(lats[0].h)
        got_other = _state(lats[1])
    finally:
        for l in lats:
            l.close()
    _same(got_other, _solo(other, 4))
    # the context and the persistent path work as before
    cases = _cases()
    lats = [gpu_lattice(c) for c in cases]
    try:
        V.vlb_step_batch([l.h for l in lats], 6)
        got = [_state(l) for l in lats]
    finally:
        for l in lats:
            l.close()
    for c, g in zip(cases, got):
        _same(g, _solo(c, 6))


def test_bad_hook_position_and_form_are_refused():
    from paper_2410_23802_gb300 import vlb as V
    with pytest.raises(V.VlbError, match="EINVAL"):
        V.vlb_debug_batch_wait(0, -2)
    with pytest.raises(V.VlbError, match="EINVAL"):
        V.vlb_set_batch_form(2)


@pytest.mark.parametrize("which", [0, 1])
def test_batch_on_the_legacy_default_stream(form, which):
    from paper_2410_23802_gb300 import vlb as V
    form(which)
    cases = _cases()
    lats = [gpu_lattice(c) for c in cases]
    try:
        for l in lats:
            V.vlb_set_stream(l.h, 0)
        V.vlb_step_batch([l.h for l in lats], 7)
        got = [_state(l) for l in lats]
    finally:
        for l in lats:
            l.close()
    for c, g in zip(cases, got):
        _same(g, _solo(c, 7))


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("chunks", [(1,), (2,), (1, 1, 2, 1)])
def test_short_calls_without_graph_replay(form, which, chunks):
    from paper_2410_23802_gb300 import vlb as V
    form(which)
    cases = _cases()
    lats = [gpu_lattice(c) for c in cases]
    try:
        for k in chunks:
            V.vlb_step_batch([l.h for l in lats], k)
        got = [_state(l) for l in lats]
    finally:
        for l in lats:
            l.close()
    for c, g in zip(cases, got):
        _same(g, _solo(c, sum(chunks)))
