"""Throughput of the coupled flow + thermal + particle step on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload cavity|channels]

Workload (default): 2048 cold disks (D = 16 lu) in a 2048 x 2048 cavity, FP32
(the seeded synthetic case of paper_2410_23802_gb300.workloads.cavity).  One
step is one full pass of the hot path: particle update and contacts, solid
fraction, f and g collide/stream with the volumetric correction, MES partial
sums.  Metric: coupled MLUPS (one lattice update = f and g at one cell).
Under torchrun each rank runs its own replica of the case on its GPU (weak
scaling, no collective on the data path); rank 0 prints one JSON line.

On one GPU the same line also carries the other forms, each timed on its own
(CUDA events, nvidia-smi clocks): `forms` (the same cavity with FP16 and BF16
population storage), `batched` (256 channels stepped together with
vlb_step_batch against the same cases one after the other) and `served` (a
shortened seeded stream through the vlb_serve_* request loop against the
plain path: cases/s, p50/p99 time to result).  --no-forms leaves them out.

--workload channels: 256 independent single-disk channels (widths 64..256,
4 widths long; workloads.channels), all resident, stepped together with
vlb_step_batch (one launch of each kernel per step for all cases), against
the same cases on their own streams and one after the other with vlb_step.
One JSON line, 1 GPU.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# f and g read + write (18 populations each way) plus S read + write (FP32, or FP64)
BYTES_PER_CELL = {"fp32": 152, "fp64": 304, "fp16": 80, "bf16": 80}
METRIC = "coupled flow+thermal MLUPS"
UNIT = "MLUPS"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _max_over_ranks(x: float) -> float:
    """The largest value of x over all ranks (the job's time is its slowest
    rank's); x itself without a process group or with one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_mlups(world: int, cells: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: every rank advances its own replica of `cells`
    by `steps` steps (weak scaling); the job takes the slowest rank's time."""
    return world * cells * steps / seconds / 1e6


L2_BYTES = 129e6  # GB300 L2


def _l2_note(bytes_per_step: float) -> str:
    """Whether the lattice state read and written per step exceeds L2 (so
    that consecutive steps cannot be served from it)."""
    mb = bytes_per_step / 1e6
    if bytes_per_step > L2_BYTES:
        return f"inputs larger than L2: {mb:.0f} MB of lattice state read and written per step (L2 129 MB)"
    return f"lattice state of {mb:.0f} MB read and written per step fits in L2 (129 MB): not a DRAM-bound measurement"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the files the lattice kernel is compiled from
LATTICE_SOURCES = ["vlb_common.cuh", "vlb_kernels.h", "vlb_lattice.cu", "vlb_lattice_body.cuh", "vlb_raster.cuh"]


def _source_hash():
    """Hash of the lattice kernel's sources (a recorded DRAM traffic stands
    only while they are unchanged)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2410_23802_gb300", "csrc")
    for f in LATTICE_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(workload_key):
    """DRAM bytes per lattice launch from the committed ncu summary, if it
    was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "lattice_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        ent = rec.get(workload_key)
        if ent and ent.get("source_hash") == _source_hash():
            return float(ent["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        rows = []
        with open(self.out.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.out.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _make_case(args, precision=None):
    from paper_2410_23802_gb300 import workloads as W
    return W.cavity(side=args.side, n=args.particles, precision=precision or args.precision)


def _params(case, V):
    prm = {k: v for k, v in case.params.items() if k != "precision"}
    prec = {"fp64": V.VLB_FP64, "fp32": V.VLB_FP32, "fp16": V.VLB_FP16_STORE,
            "bf16": V.VLB_BF16_STORE}[case.params["precision"]]
    return V.vlb_params_default(precision=prec, max_particles=len(case.x), **prm)


def _time_cavity(case, V, stream, warmup, steps, local, world):
    """K device-resident steps of one cavity case after W untimed ones, timed
    with CUDA events on the library's stream (a torch stream passed through
    vlb_set_stream), with the lattice kernel's own launches timed by the
    library's profiling events and nvidia-smi sampled meanwhile."""
    import numpy as np
    import torch
    lat = V.Lattice(_params(case, V))
    V.vlb_set_stream(lat.h, stream.cuda_stream)
    lat.add_particles(np.column_stack([case.x, case.y]), case.radius, case.T0, k_ratio=case.k_ratio)
    with torch.cuda.stream(stream):
        lat.step(warmup)
        V.vlb_synchronize(lat.h)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.3)
        V.vlb_profile_begin(lat.h, steps)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        lat.step(steps)
        t1.record(stream)
        V.vlb_synchronize(lat.h)
        torch.cuda.synchronize()
        clocks = sampler.stop()
    elapsed_ms = t0.elapsed_time(t1)
    lattice_ms, lattice_launches, launches_per_step = V.vlb_profile_end(lat.h)
    lat.close()
    return elapsed_ms, lattice_ms, lattice_launches, launches_per_step, clocks


def _roofline(precision, cells, lattice_ms, lattice_launches, key):
    peak, peak_kind = _peaks()
    lattice_avg_s = lattice_ms * 1e-3 / max(lattice_launches, 1)
    bpc = BYTES_PER_CELL[precision]
    achieved = bpc * cells / lattice_avg_s / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": _ncu_traffic(key),
            "kernel": "lattice_kernel<STEP>", "bytes_per_cell": bpc, "peak_kind": peak_kind,
            "avg_launch_us": round(lattice_avg_s * 1e6, 2)}


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2410_23802_gb300 import vlb as V
    if args.batch_form is not None:
        V.vlb_set_batch_form(args.batch_form)

    case = _make_case(args)
    cells = case.cells
    stream = torch.cuda.Stream()
    xy = np.column_stack([case.x, case.y])

    # ---- device-resident throughput ------------------------------------------
    elapsed_ms, lattice_ms, lattice_launches, launches_per_step, clocks = _time_cavity(
        case, V, stream, args.warmup, args.steps, local, world)
    elapsed_ms = _max_over_ranks(elapsed_ms)
    if world > 1:
        torch.distributed.barrier()

    # ---- end to end through the public API with host buffers -------------------
    e2e_steps = args.steps
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    npart = len(case.x)
    w0 = time.perf_counter()
    lat2 = V.Lattice(_params(case, V))
    lat2.add_particles(xy, case.radius, case.T0, k_ratio=case.k_ratio)
    # each step's result, the particle state, to host: queued after the step
    # and collected after the next one is queued, so the GPU does not wait
    buf = None
    for k in range(e2e_steps):
        lat2.step(1)
        V.vlb_particle_state_async(lat2.h, npart)
        if k > 0:
            buf, _ = V.vlb_particle_state_wait(lat2.h, npart, buf)
    buf, _ = V.vlb_particle_state_wait(lat2.h, npart, buf)
    fields = lat2.fields()
    V.vlb_synchronize(lat2.h)
    e2e_s = time.perf_counter() - w0
    lat2.close()
    assert np.isfinite(fields["T"]).all() and np.isfinite(buf["xy"]).all()
    e2e_s = _max_over_ranks(e2e_s)
    h2d = len(case.x) * (2 * 8 + 3 * 8)                         # centres, radius, T0, k_ratio (once)
    d2h = cells * 5 * 8 + e2e_steps * len(case.x) * 12 * 8     # five fields once; 12 state arrays every step

    # ---- the other graded forms (1 GPU only: rank 0 of a one-rank job) ---------
    forms = batched = served = None
    if world == 1 and not args.no_forms:
        forms = {}
        for prec in ("fp16", "bf16"):
            c2 = _make_case(args, precision=prec)
            ms, lms, ll, lps, ck = _time_cavity(c2, V, stream, args.warmup, args.steps, local, world)
            forms[prec] = {"value": round(cells * args.steps / (ms * 1e-3) / 1e6, 1), "unit": UNIT,
                           "ms_per_step": round(ms / args.steps, 5),
                           "vs_fp32": round(elapsed_ms / ms, 4),
                           "roofline": _roofline(prec, cells, lms, ll, f"cavity{args.side}_{args.particles}_{prec}"),
                           "gpu_launches": lps * args.steps, "clocks": ck,
                           "storage": f"populations as {prec.upper()} deviations from the rest equilibrium, "
                                      "FP32 arithmetic, FP64 particles"}
        batched = measure_batched(V, local, n_cases=256, steps=args.steps, warmup=args.warmup)
        served = measure_served(V, local, n_cases=args.serve_cases, steps=args.serve_case_steps)

    if rank != 0:
        return
    value = _job_mlups(world, cells, args.steps, elapsed_ms * 1e-3)
    key = f"cavity{args.side}_{args.particles}_{args.precision}"
    bpc = BYTES_PER_CELL[args.precision]
    line = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(elapsed_ms / args.steps, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp16": "f16 storage / f32", "bf16": "bf16 storage / f32"}[
            args.precision],
        "data": "synthetic (seeded SplitMix64 placement)",
        "config": {"workload": case.name, "cells": cells, "particles": len(case.x),
                   "storage": args.precision, "parallelism": f"replicas x{world}",
                   "l2": _l2_note(cells * bpc)},
        "roofline": _roofline(args.precision, cells, lattice_ms, lattice_launches, key),
        "e2e": {"value": round(_job_mlups(world, cells, e2e_steps, e2e_s), 1), "unit": UNIT,
                "h2d_bytes_per_step": round(h2d / e2e_steps, 1), "d2h_bytes_per_step": round(d2h / e2e_steps, 1),
                "note": "create + host particle upload + steps, each step's particle state to host "
                        "(vlb_particle_state_async / _wait), + the five fields to host at the end; wall clock"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    if forms is not None:
        line["forms"] = forms
        line["batched"] = batched
        line["served"] = served
    if not args.no_cpu_baseline and world == 1:  # the host cores are timed at N = 1 only
        line["cpu_baseline"] = cpu_baseline(args, budget_s=15.0)
    print(json.dumps(line), flush=True)


def _channel_lattices(V, cases, streams):
    import numpy as np
    lats = []
    for c, st in zip(cases, streams):
        lat = V.Lattice(_params(c, V))
        V.vlb_set_stream(lat.h, st.cuda_stream)
        lat.add_particles(np.column_stack([c.x, c.y]), c.radius, c.T0, k_ratio=c.k_ratio)
        lats.append(lat)
    return lats


def _persistent_batches() -> bool:
    from paper_2410_23802_gb300 import vlb as V
    return V.vlb_get_batch_form() == V.VLB_BATCH_PERSISTENT


def _batch_form() -> str:
    if _persistent_batches():
        return "one persistent launch per step (tiles, then the next level's particle steps), CUDA-graph replay"
    return "a CTA per tile and a particle kernel per step"


def _batch_launches(steps: int) -> int:
    """Kernels of one vlb_step_batch call of `steps` steps over one kernel
    variant without ellipses: the level-0 particle step, steps - 1 persistent
    launches and the last level's tiles; or two per step."""
    return steps + 1 if _persistent_batches() else 2 * steps


def measure_batched(V, local, n_cases, steps, warmup, precision="fp32"):
    """The 256-channel configuration resident at once: K steps of all cases
    with vlb_step_batch (one launch of each kernel per step for every case),
    against the plain path (each case stepped with vlb_step, one after the
    other on one stream).  Device time from CUDA events on a stream joined
    with every case's stream."""
    import torch
    from paper_2410_23802_gb300 import workloads as W
    cases = W.channels(n=n_cases, precision=precision)
    cells = sum(c.cells for c in cases)
    main_stream = torch.cuda.Stream()
    streams = [torch.cuda.Stream() for _ in cases]
    lats = _channel_lattices(V, cases, streams)
    hs = [l.h for l in lats]

    def timed(run, sts):
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(main_stream)
        for st in sts:
            st.wait_event(t0)
        run()
        for st in sts:
            ev = torch.cuda.Event()
            ev.record(st)
            main_stream.wait_event(ev)
        t1.record(main_stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1)

    V.vlb_step_batch(hs, warmup)
    for l in lats:
        V.vlb_synchronize(l.h)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.2)
    batched_ms = timed(lambda: V.vlb_step_batch(hs, steps), streams)
    clocks = sampler.stop()
    for l in lats:  # the plain path: one stream, one case after the other
        V.vlb_set_stream(l.h, streams[0].cuda_stream)
    plain_ms = timed(lambda: [l.step(steps) for l in lats], streams[:1])
    for l in lats:
        l.close()
    mlups = lambda ms: cells * steps / (ms * 1e-3) / 1e6  # noqa: E731
    return {"value": round(mlups(batched_ms), 1), "unit": UNIT, "ms_per_step": round(batched_ms / steps, 5),
            "cases_per_s": round(len(cases) * steps / (batched_ms * 1e-3) / 5000.0, 2),
            "cases_per_s_note": "cases of 5000 steps each",
            "plain": {"value": round(mlups(plain_ms), 1), "unit": UNIT,
                      "cases_per_s": round(len(cases) * steps / (plain_ms * 1e-3) / 5000.0, 2),
                      "note": "one stream, one case after the other with vlb_step"},
            "vs_plain": round(plain_ms / batched_ms, 3),
            "workload": f"{len(cases)} channels W~U{{64..256}} x 4W, 1 disk each, {cells} cells, {precision}",
            "steps": steps, "warmup": warmup, "gpu_launches": _batch_launches(steps), "form": _batch_form(),
            "clocks": clocks}


def _serve_stream(n_cases, steps):
    from paper_2410_23802_gb300 import workloads as W
    items = W.served_cases(n=n_cases, steps=steps)
    import numpy as np
    gaps = np.array([g for g, _, _ in items])
    return gaps, [(c, n) for _, c, n in items]


def _plain_alone(V, stream_ptr, c, n):
    """The plain path: one case on its own, FP32 populations, created,
    stepped, read back to host memory and freed."""
    import dataclasses

    import numpy as np
    lat = V.Lattice(_params(dataclasses.replace(c, params=dict(c.params, precision="fp32")), V))
    V.vlb_set_stream(lat.h, stream_ptr)
    lat.add_particles(np.column_stack([c.x, c.y]), c.radius, c.T0, k_ratio=c.k_ratio)
    lat.step(n)
    f, p = lat.fields(), lat.particles()
    lat.close()
    return f, p


def _plain_run(V, stream_ptr, gaps, cases, rate):
    """Arrivals at `rate` (None: all at once) served one after the other by
    the plain path; time to result per case and the makespan."""
    import numpy as np
    arrive = np.cumsum(gaps) / rate if rate else np.zeros(len(cases))
    start = time.perf_counter()
    lat_s = []
    for (c, n), ta in zip(cases, arrive):
        now = time.perf_counter() - start
        if now < ta:
            time.sleep(ta - now)
        _plain_alone(V, stream_ptr, c, n)
        lat_s.append(time.perf_counter() - start - ta)
    return np.array(lat_s), time.perf_counter() - start - arrive[0]


def _served_run(V, gaps, cases, rate, budget_gb, round_steps):
    """The same arrivals through the server (vlb_serve_*)."""
    import numpy as np
    arrive = np.cumsum(gaps) / rate if rate else np.zeros(len(cases))
    # the server's clock starts a little after `start`: times to result
    # below count from the arrival and may be overstated by that much
    start = time.perf_counter()
    srv = V.Server(hbm_budget=int(budget_gb * 1e9), steps_per_round=round_steps)
    pending, lat_s = {}, {}
    k = 0
    while len(lat_s) < len(cases):
        now = time.perf_counter() - start
        while k < len(cases) and arrive[k] <= now:
            c, n = cases[k]
            pending[k] = srv.submit(_params(c, V), np.column_stack([c.x, c.y]), c.radius, c.T0, n,
                                    k_ratio=c.k_ratio)
            k += 1
        q, a, d = srv.poll()
        for j, cid in (list(pending.items()) if d else []):
            inf = srv.info(cid)
            if inf["state"] in (V.VLB_CASE_DONE, V.VLB_CASE_FAILED):
                srv.take(cid)
                lat_s[j] = inf["t_done"] - arrive[j]
                del pending[j]
        if q == 0 and a == 0 and k < len(cases):
            wait = arrive[k] - (time.perf_counter() - start)
            if wait > 0:
                time.sleep(wait)
    srv.close()
    return np.array([lat_s[j] for j in range(len(cases))]), time.perf_counter() - start - arrive[0]


def _latency_summary(lat_s, span, n, work):
    import numpy as np
    return {"p50_ms": round(1e3 * float(np.percentile(lat_s, 50)), 2),
            "p99_ms": round(1e3 * float(np.percentile(lat_s, 99)), 2),
            "cases_per_s": round(n / span, 2), "mlups": round(work / span / 1e6, 1)}


def measure_served(V, local, n_cases, steps, budget_gb=2.0, round_steps=100, loads=(None, 0.8, 1.2)):
    """A shortened seeded stream of the served configuration (cavities of
    side 2^U[6,10], 1-512 disks, half FP16 storage) through the server and
    through the plain path (one case after the other, FP32): all arriving at
    once (saturation), and Poisson arrivals at 0.8 and 1.2 x the plain path's
    measured service rate.  Time to result = arrival to fields and particle
    state in host memory."""
    import torch
    stream = torch.cuda.Stream()
    gaps, cases = _serve_stream(n_cases, steps)
    work = sum(c.cells * n for c, n in cases)
    for c, n in cases[:3]:
        _plain_alone(V, stream.cuda_stream, c, 20)
    res = {}
    sampler = ClockSampler(local)
    sampler.start()
    lp, span_p = _plain_run(V, stream.cuda_stream, gaps, cases, None)
    rate_plain = len(cases) / span_p
    res["all_at_once"] = {"plain": _latency_summary(lp, span_p, len(cases), work)}
    ls, span = _served_run(V, gaps, cases, None, budget_gb, round_steps)
    res["all_at_once"]["served"] = _latency_summary(ls, span, len(cases), work)
    for load in loads:
        if load is None:
            continue
        rate = load * rate_plain
        ls, span = _served_run(V, gaps, cases, rate, budget_gb, round_steps)
        lp, span_p = _plain_run(V, stream.cuda_stream, gaps, cases, rate)
        res[f"poisson_{load}x"] = {"offered_cases_per_s": round(rate, 2),
                                   "served": _latency_summary(ls, span, len(cases), work),
                                   "plain": _latency_summary(lp, span_p, len(cases), work)}
    clocks = sampler.stop()
    sat = res["all_at_once"]
    return {"value": sat["served"]["mlups"], "unit": UNIT,
            "cases_per_s": sat["served"]["cases_per_s"],
            "vs_plain_cases_per_s": round(sat["served"]["cases_per_s"] / sat["plain"]["cases_per_s"], 3),
            "workload": f"{len(cases)} seeded cavity cases, side 2^U[6,10], 1-512 disks of D~U[8,24], "
                        f"half FP16 storage, {steps} steps each; HBM budget {budget_gb} GB, "
                        f"{round_steps} steps per round",
            "plain_service_rate": round(rate_plain, 2), "loads": res, "clocks": clocks,
            "note": "value and cases_per_s: the server with every case arriving at once (saturation); "
                    "plain: one case after the other with FP32 populations; wall clock from arrival to "
                    "results in host memory"}


def run_channels(args):
    """Many small cases at once: one launch of each kernel per step for all
    cases (vlb_step_batch), against the same cases on their own streams with
    vlb_step, and one after the other on one stream (the plain path)."""
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")  # hardware queues for the streams leg
    import torch
    from paper_2410_23802_gb300 import vlb as V
    from paper_2410_23802_gb300 import workloads as W

    rank, world, local = _dist()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    if args.batch_form is not None:
        V.vlb_set_batch_form(args.batch_form)
    cases = W.channels(n=args.cases, precision=args.precision)
    cells = sum(c.cells for c in cases)
    main_stream = torch.cuda.Stream()
    streams = [torch.cuda.Stream() for _ in cases]
    lats = _channel_lattices(V, cases, streams)
    hs = [l.h for l in lats]

    def timed(run):
        """Device time from an event on main_stream that every case stream
        waits for to one main_stream records after waiting for all of them."""
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(main_stream)
        for st in streams:
            st.wait_event(t0)
        run()
        for st in streams:
            ev = torch.cuda.Event()
            ev.record(st)
            main_stream.wait_event(ev)
        t1.record(main_stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1)

    mlups = lambda ms: cells * args.steps / (ms * 1e-3) / 1e6  # noqa: E731
    V.vlb_step_batch(hs, args.warmup)
    for l in lats:
        V.vlb_synchronize(l.h)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    batched_ms = timed(lambda: V.vlb_step_batch(hs, args.steps))
    clocks = sampler.stop()
    wall0 = time.perf_counter()
    V.vlb_step_batch(hs, args.steps)
    for l in lats:
        V.vlb_synchronize(l.h)
    host_s = time.perf_counter() - wall0
    streams_ms = timed(lambda: [l.step(args.steps) for l in lats])
    for l in lats:  # the plain path: one stream, one case after the other
        V.vlb_set_stream(l.h, streams[0].cuda_stream)
    plain_ms = timed(lambda: [l.step(args.steps) for l in lats])
    for l in lats:
        l.close()
    value = mlups(batched_ms)
    line = {
        "metric": METRIC + " (batched independent cases)",
        "value": round(value, 1),
        "unit": UNIT,
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(batched_ms / args.steps, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp16": "f16 storage / f32", "bf16": "bf16 storage / f32"}[
            args.precision],
        "data": "synthetic (seeded SplitMix64 widths and parameters)",
        "config": {"workload": f"{len(cases)} channels W~U{{64..256}} x 4W, 1 disk each", "cells": cells,
                   "storage": args.precision, "l2": _l2_note(cells * BYTES_PER_CELL[args.precision])},
        "streams": {"value": round(mlups(streams_ms), 1), "unit": UNIT,
                    "note": "each case on its own stream with vlb_step, issued one after another"},
        "plain": {"value": round(mlups(plain_ms), 1), "unit": UNIT,
                  "note": "one stream, one case after the other with vlb_step"},
        "cases_per_s": round(len(cases) * args.steps / (batched_ms * 1e-3) / 5000.0, 2),
        "cases_per_s_note": "cases of 5000 steps each",
        "host_wall_mlups": round(cells * args.steps / host_s / 1e6, 1),
        "gpu_launches": _batch_launches(args.steps),
        "form": _batch_form(),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Served mode (FP32 and FP16 storage, half each) against the plain
    path (one case after the other, FP32) under the same seeded arrivals:
    all at once, and Poisson arrivals at 0.8 and 1.2 times the plain path's
    measured service rate; time to result (arrival to fields and particle
    state in host memory) per case, aggregate MLUPS and cases/s over the
    makespan."""
    import torch
    from paper_2410_23802_gb300 import vlb as V

    rank, world, local = _dist()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    if args.batch_form is not None:
        from paper_2410_23802_gb300 import vlb as _V
        _V.vlb_set_batch_form(args.batch_form)
    r = measure_served(V, local, args.cases, args.serve_steps, budget_gb=args.budget_gb,
                       round_steps=args.round_steps, loads=(None, 0.8, 1.2))
    line = {
        "metric": "served p50/p99 time to result (ms) and aggregate MLUPS",
        "value": r["value"],
        "unit": "MLUPS",
        "n_gpus": 1,
        "steps": args.serve_steps,
        "warmup": 3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 / f16 storage (half each)",
        "data": "synthetic (seeded SplitMix64 arrivals, sizes and placements)",
        "config": {"workload": r["workload"]},
        **{k: v for k, v in r.items() if k not in ("value", "unit", "workload")},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# CPU oracle legs
# ---------------------------------------------------------------------------

def _crop_case(args, side):
    """The cavity workload restricted to a side x side window at its top
    centre (same parameters, the disks lying inside the window)."""
    from paper_2410_23802_gb300 import workloads as W
    full = _make_case(args)
    x0 = (args.side - side) // 2
    y0 = args.side - side
    xs, ys, rs, ts = [], [], [], []
    for x, y, r, t in zip(full.x, full.y, full.radius, full.T0):
        if x - r - 2 >= x0 and x + r + 2 <= x0 + side and y - r - 2 >= y0 and y + r + 2 <= y0 + side:
            xs.append(x - x0); ys.append(y - y0); rs.append(r); ts.append(t)
    prm = dict(full.params)
    prm["nx"] = prm["ny"] = side
    return W.Case(f"{side}x{side} window of {full.name}", prm, xs, ys, rs, ts)


_CPU_CHILD = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from oracle import vlbref as O
from paper_2410_23802_gb300 import workloads as W
spec = json.loads({spec!r})
case = W.Case(**spec["case"])
prm = {{k: v for k, v in case.params.items() if k != "precision"}}
sim = O.Simulation(O.Params(**prm), case.x, case.y, case.radius, case.T0)
for _ in range(spec["warmup"]):
    sim.step()
times = []
t_start = time.perf_counter()
for _ in range(spec["steps"]):
    t = time.perf_counter()
    sim.step()
    times.append(time.perf_counter() - t)
    if spec["budget"] > 0 and time.perf_counter() - t_start > spec["budget"]:
        break
print(json.dumps({{"times": times}}))
"""


def _oracle_cmd(case, steps, warmup, budget):
    import dataclasses
    spec = {"case": dataclasses.asdict(case), "steps": steps, "warmup": warmup, "budget": budget}
    spec["case"]["params"] = {k: (list(v) if isinstance(v, tuple) else v) for k, v in case.params.items()}
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    return [sys.executable, "-c", _CPU_CHILD.format(root=ROOT, spec=json.dumps(spec))], env


def _run_oracle(case, steps, warmup, budget):
    cmd, env = _oracle_cmd(case, steps, warmup, budget)
    out = subprocess.run(cmd, capture_output=True, text=True, env=env, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])["times"]


def _run_oracle_all_cores(case, budget, nproc):
    """nproc oracle processes (one thread each) on copies of the case at the
    same time: aggregate cell updates per second over the slowest's wall time."""
    cmd, env = _oracle_cmd(case, steps=1000, warmup=1, budget=budget)
    t0 = time.perf_counter()
    procs = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, env=env)
             for _ in range(nproc)]
    steps = 0
    busy = 0.0
    for p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("oracle process failed")
        t = json.loads(out.strip().splitlines()[-1])["times"]
        steps += len(t)
        busy = max(busy, sum(t))
    return case.cells * steps / busy / 1e6, steps, time.perf_counter() - t0


def cpu_baseline(args, budget_s):
    """The oracle on a window of the workload: on all host cores (one process
    per core, aggregate throughput) and on one core."""
    side = min(512, args.side)
    case = _crop_case(args, side)
    times = _run_oracle(case, steps=1000, warmup=1, budget=budget_s)
    one = case.cells / (sum(times) / len(times)) / 1e6
    nproc = os.cpu_count() or 1
    agg, steps, _ = _run_oracle_all_cores(case, budget_s, nproc)
    return {"value": round(agg, 4), "unit": UNIT, "cores": nproc, "kind": "oracle",
            "single_core_value": round(one, 4),
            "sample": f"{steps} steps in all of the FP64 numpy oracle on the {case.name} "
                      f"({len(case.x)} disks), {nproc} processes of 1 thread at once, about {budget_s:.0f} s each "
                      f"after 1 untimed step; single_core_value: {len(times)} steps in 1 process alone"}


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    # size the window so that the K timed steps take about 60 s of CPU time
    probe = _crop_case(args, 256)
    t_probe = statistics.median(_run_oracle(probe, steps=3, warmup=1, budget=0))
    per_cell = 1.5 * t_probe / probe.cells  # per-cell cost grows with the window
    side = int((60.0 / max(args.steps, 1) / per_cell) ** 0.5)
    side = max(64, min(args.side, side - side % 32))
    case = _crop_case(args, side)
    times = _run_oracle(case, steps=args.steps, warmup=min(args.warmup, 3), budget=0)
    total = sum(times)
    value = case.cells * len(times) / total / 1e6
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 4),
        "unit": UNIT,
        "n_gpus": world,
        "steps": len(times),
        "warmup": min(args.warmup, 3),
        "ms_per_step": round(1e3 * total / len(times), 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded SplitMix64 placement)",
        "config": {"workload": _make_case(args).name, "sample": case.name, "particles": len(case.x),
                   "storage": "fp64"},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{len(times)} steps on the {case.name}"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=2048)
    ap.add_argument("--particles", type=int, default=2048)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp16", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="cavity", choices=["cavity", "channels", "serve"])
    ap.add_argument("--cases", type=int, default=None, help="channels: 256; serve: 200")
    ap.add_argument("--serve-steps", type=int, default=2000)
    ap.add_argument("--budget-gb", type=float, default=2.0)
    ap.add_argument("--round-steps", type=int, default=100)
    ap.add_argument("--no-forms", action="store_true", help="skip the FP16/BF16, batched and served sub-records")
    ap.add_argument("--serve-cases", type=int, default=48, help="served sub-record: cases in the stream")
    ap.add_argument("--serve-case-steps", type=int, default=400, help="served sub-record: steps per case")
    ap.add_argument("--batch-form", type=int, default=None, choices=[0, 1],
                    help="form of vlb_step_batch (0 a CTA per tile, 1 persistent; default: the build's)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "channels":
        args.cases = args.cases or 256
        run_channels(args)
    elif args.workload == "serve":
        args.cases = args.cases or 200
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
