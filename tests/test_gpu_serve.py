"""Served mode (vlb_serve_*): cases of several sizes, particle counts and
storage types arrive while others run, wait for the HBM budget, and advance
together in rounds.

* Each result is the one the case gives alone (vlb_step on its own handle),
  bit for bit, although it was admitted mid-run, queued behind the budget and
  stepped in rounds shared with other cases.
* Admission respects the budget and max_active; a case that cannot be placed
  fails alone; unknown, unfinished and oversized cases are refused.
* vlb_device_bytes agrees with the device memory a handle takes."""
import dataclasses

import numpy as np
import pytest

from helpers import gpu_lattice
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _params(case, V):
    prm = {k: v for k, v in case.params.items() if k != "precision"}
    code = {"fp64": V.VLB_FP64, "fp32": V.VLB_FP32, "fp16": V.VLB_FP16_STORE,
            "bf16": V.VLB_BF16_STORE}[case.params["precision"]]
    return V.vlb_params_default(precision=code, max_particles=max(len(case.x), 1), **prm)


def _stream():
    """Eight small cases with 23..79 steps each."""
    out = []
    for k, (_, c, _) in enumerate(W.served_cases(n=8, seed=31, side_log2=(6.0, 8.0), max_particles_log2=5.0)):
        out.append((c, 23 + 8 * k))
    return out


def _submit(srv, V, case, steps):
    return srv.submit(_params(case, V), np.column_stack([case.x, case.y]), case.radius, case.T0, steps,
                      k_ratio=case.k_ratio)


def test_served_results_equal_alone():
    from paper_2410_23802_gb300 import vlb as V
    cases = _stream()
    sizes = [V.vlb_device_bytes(_params(c, V), c.radius) for c, _ in cases]
    budget = sum(sorted(sizes)[-3:])  # about three cases resident at a time
    ids, results = {}, {}
    with V.Server(hbm_budget=budget, steps_per_round=16) as srv:
        for k in range(4):
            ids[k] = _submit(srv, V, *cases[k])
        rounds = 0
        while len(results) < len(cases):
            q, a, d = srv.poll()
            rounds += 1
            assert rounds < 1000
            if rounds == 2:  # the rest arrive while the first run
                for k in range(4, len(cases)):
                    ids[k] = _submit(srv, V, *cases[k])
            for k, cid in ids.items():
                if k not in results and srv.info(cid)["state"] == V.VLB_CASE_DONE:
                    results[k] = srv.take(cid)
    for k, (c, steps) in enumerate(cases):
        with gpu_lattice(c) as lat:
            lat.step(steps)
            f, p = lat.fields(), lat.particles()
        fs, ps = results[k]
        for name in f:
            assert np.array_equal(f[name], fs[name], equal_nan=True), (k, name)
        for name in ps:
            assert np.array_equal(p[name], ps[name]), (k, name)


def test_served_admission_and_failures():
    from paper_2410_23802_gb300 import vlb as V
    cases = _stream()[:4]
    sizes = [V.vlb_device_bytes(_params(c, V), c.radius) for c, _ in cases]
    with V.Server(hbm_budget=max(sizes) + (1 << 20), steps_per_round=10, max_active=1) as srv:
        ids = [_submit(srv, V, c, s) for c, s in cases]
        # overlapping disks: accepted, then fails at admission on its own
        c0 = cases[0][0]
        bad = dataclasses.replace(c0, x=[30.0, 31.0], y=[40.0, 40.0], radius=[4.0, 4.0], T0=[0.0, 0.0],
                                  k_ratio=None)
        bad_id = _submit(srv, V, bad, 5)
        with pytest.raises(V.VlbError, match="ENOMEM"):  # larger than the whole budget
            _submit(srv, V, W.cavity(side=1024, n=8), 5)
        with pytest.raises(V.VlbError, match="ESTATE"):
            srv.take(ids[0])
        with pytest.raises(V.VlbError, match="EINVAL"):
            srv.info(10 ** 9)
        seen_active = 0
        for _ in range(1000):
            q, a, d = srv.poll()
            seen_active = max(seen_active, a)
            if d == len(ids) + 1:
                break
        assert seen_active == 1
        times = [srv.info(i) for i in ids]
        for t in times:
            assert t["state"] == V.VLB_CASE_DONE
            assert t["t_submit"] <= t["t_admit"] <= t["t_done"]
        # one at a time, first come first served
        for a, b in zip(times, times[1:]):
            assert a["t_done"] <= b["t_admit"]
        assert srv.info(bad_id)["state"] == V.VLB_CASE_FAILED
        with pytest.raises(V.VlbError, match="EINVAL"):
            srv.take(bad_id)
        for i in ids:
            f, p = srv.take(i)
            assert np.isfinite(f["T"]).all()


def test_device_bytes_match_the_allocation():
    import torch
    from paper_2410_23802_gb300 import vlb as V
    case = W.cavity(side=1024, n=256, seed=5)
    est = V.vlb_device_bytes(_params(case, V), case.radius)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    with gpu_lattice(case) as lat:
        lat.step(0)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1
    # allocations are rounded up to 2 MiB pages (about 15 of them)
    assert est <= used + (4 << 20) and used <= est + (40 << 20), (est, used)


def test_unstable_case_fails_alone():
    """A case whose disk is driven past 0.5 lu per step (strong gravity: the
    device sets its too-fast flag, no fault) ends as a failed case with
    VLB_EUNSTABLE; the cases stepped in the same rounds finish and equal
    their solo runs."""
    from paper_2410_23802_gb300 import vlb as V
    good = _stream()[:3]
    c0 = W.channels(n=1, seed=5)[0]
    prm = dict(c0.params, gravity=(0.0, -0.05), rho_ratio=3.0)
    fast = dataclasses.replace(c0, params=prm)
    with V.Server(steps_per_round=16) as srv:
        ids = [_submit(srv, V, c, s) for c, s in good[:1]]
        bad_id = _submit(srv, V, fast, 200)
        ids += [_submit(srv, V, c, s) for c, s in good[1:]]
        for _ in range(1000):
            q, a, d = srv.poll()
            if d == len(ids) + 1:
                break
        assert srv.info(bad_id)["state"] == V.VLB_CASE_FAILED
        with pytest.raises(V.VlbError, match="EUNSTABLE"):
            srv.take(bad_id)
        results = [srv.take(i) for i in ids]
    for (c, steps), (fs, ps) in zip(good, results):
        with gpu_lattice(c) as lat:
            lat.step(steps)
            f, p = lat.fields(), lat.particles()
        for name in f:
            assert np.array_equal(f[name], fs[name], equal_nan=True), name
        for name in ps:
            assert np.array_equal(p[name], ps[name]), name


def test_served_results_against_the_oracle():
    """Served cases against the FP64 oracle, not only against their solo runs:
    two small cavities (FP32 and FP16 storage) admitted together with a third
    case and stepped in shared rounds of uneven length.  FP32: rho, u, T
    within 1e-5 relative L2, particles within 1e-4; FP16 storage: u and T
    within 1e-3, particles within 1e-3."""
    from helpers import oracle_sim, rel_l2
    from paper_2410_23802_gb300 import vlb as V
    a = W.cavity(side=96, n=4, seed=41, precision="fp32")
    b = W.cavity(side=112, n=6, seed=43, precision="fp16")
    c = W.cavity(side=128, n=8, seed=47, precision="fp32")
    steps = {0: 60, 1: 50, 2: 37}
    with V.Server(hbm_budget=1 << 30, steps_per_round=13) as srv:
        ids = [_submit(srv, V, case, steps[k]) for k, case in enumerate((a, b, c))]
        for _ in range(1000):
            q, act, d = srv.poll()
            if d == 3:
                break
        got = [srv.take(i) for i in ids[:2]]
    for (case, n, tol, ptol), (f, p) in zip([(a, 60, 1e-5, 1e-4), (b, 50, 1e-3, 1e-3)], got):
        sim = oracle_sim(case)
        sim.step(n)
        ref = sim.fields()
        e_rho = rel_l2(f["rho"], ref["rho"])
        e_u = rel_l2(np.stack([f["ux"], f["uy"]]), np.stack([ref["ux"], ref["uy"]]))
        e_T = rel_l2(f["T"], ref["T"])
        print(f"served {case.params['precision']}: rho {e_rho:.2e} u {e_u:.2e} T {e_T:.2e}")
        assert e_u < tol and e_T < tol and (case.params["precision"] != "fp32" or e_rho < tol)
        rp = sim.particle_state()
        for k in ("x", "y", "ux", "uy"):
            assert np.abs(p[k] - rp[k]).max() < ptol, k
