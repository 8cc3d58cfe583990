#!/usr/bin/env python
"""Benchmark of the block-selection + NCC block-matching path on GB300.

One step = the whole hot path on one synthetic volume pair already resident
in device memory: variance block selection (keys, radix select, compaction),
box sums of the reference volume, and exhaustive NCC block matching of every
selected block.  Metric: NCC evaluations per second, one evaluation being
one (block, shift) pair of the search (nominal count: selected blocks x
(2R+1)^3).

Default workload: the clinical-size single registration, 256x256x124 uint16
phantom pair (40 Gaussians, smooth field max 8 voxels, noise sigma 30),
ellipsoidal mask, blocks 7^3 on a stride-2 grid, top 5% by variance
(~19.4k blocks), search radius 5 (1331 shifts).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torchrun) every rank runs an independent replica of
the workload on its own GPU (the path has no exchange step); the reported
value is all ranks' evaluations over the slowest rank's time.
``--impl reference`` times the CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "NCC evals/s (block x shift)"
UNIT = "evals/s"
FP32_LANES_PER_SM = 128  # FFMA lanes per Blackwell SM


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="clinical")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--batched-reps", type=int, default=5)
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-highres", action="store_true")
    p.add_argument("--no-aniso", action="store_true")
    p.add_argument("--no-spacing", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-small", action="store_true")
    p.add_argument("--no-fem", action="store_true")
    p.add_argument("--fem-only", action="store_true",
                   help="select and match the workload once, then run only the FEM leg (for profiling)")
    p.add_argument("--fem-grids", default="8,4", help="vertex spacings of the FEM leg")
    p.add_argument("--serve-open-requests", type=int, default=1000)  # 50 s at 20 req/s
    p.add_argument("--serve-sweep-requests", type=int, default=300)
    p.add_argument("--serve-closed-requests", type=int, default=1000)
    return p.parse_args()


def aggregate_replicas(local_s: float, world: int, units_per_rank: int, pg=None):
    """Replicas only: every rank processed `units_per_rank` independently;
    the job's time is the slowest rank's.  Returns (max seconds, whole-job
    units per second)."""
    import torch

    t = local_s
    if pg is not None and world > 1:
        dev = torch.device("cuda", torch.cuda.current_device()) if pg.get_backend() == "nccl" else torch.device("cpu")
        x = torch.tensor([local_s], dtype=torch.float64, device=dev)
        pg.all_reduce(x, op=pg.ReduceOp.MAX)
        t = float(x.item())
    return t, world * units_per_rank / t


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _config(w, n_blocks=None, extra=None):
    c = {"workload": w.name, "volume": "x".join(map(str, w.dims)) + " uint16", "block": w.block,
         "stride": w.stride, "frac": w.frac, "radius": w.radius, "shifts": (2 * w.radius + 1) ** 3,
         "phantom": f"40 Gaussians, field max {w.umax:g} vox, noise sigma {w.noise:g}, seed-fixed",
         "l2": "flushed between timed steps (256 MiB write, twice the 126.5 MB L2)"}
    if n_blocks is not None:
        c["n_blocks"] = int(n_blocks)
    if extra:
        c.update(extra)
    return c


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "50"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t_start: float, t_end: float):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9 and f[1].replace(".", "").isdigit():
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------------------
# recorded ncu traffic of the match kernel (valid only for the same source)
# --------------------------------------------------------------------------
def _kernel_source_hash(csrc=None):
    """First 16 hex digits of sha256 over the match kernel's sources with
    their // comments and blank lines removed (an edit of a comment does not
    change the kernel the counters were taken on)."""
    csrc = csrc or os.path.join(ROOT, "paper_2308_10868_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("nrr_match.cuh", "nrr_ptx.cuh"):
        text = open(os.path.join(csrc, f), encoding="utf-8").read()
        code = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in code if ln).encode())
    return h.hexdigest()[:16]


def _recorded_traffic():
    path = os.path.join(ROOT, "profiles", "match_kernel_clinical.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m1 = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    m2 = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not (m1 and m2) or m1.group(1) != _kernel_source_hash():
        return None
    return float(m2.group(1))


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return json.load(open(path))
        except ValueError:
            pass
    return {}


# --------------------------------------------------------------------------
# CPU oracle timings (baseline only)
# --------------------------------------------------------------------------
def _oracle_step(w, pre, intra, mask, sample_every=1):
    import oracle

    t0 = time.perf_counter()
    centers, _ = oracle.select_blocks(pre, mask, w.block, w.stride, w.frac)
    sub = centers[::sample_every]
    oracle.match(pre, intra, sub, w.block, w.radius)
    dt = time.perf_counter() - t0
    return len(sub) * (2 * w.radius + 1) ** 3, dt, len(centers)


def _cpu_baseline(w, pre, intra, mask):
    import oracle

    oracle.build()
    ev, dt, n = _oracle_step(w, pre, intra, mask)
    return {"value": ev / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"whole workload: selection of {n} blocks + matching all of them ({ev} evals), "
                      f"{dt:.2f} s, FP64 C oracle, OpenMP over blocks"}


def _cpu_baseline_fem(d_mask, centers, n_sel, out):
    """The FEM oracle (scipy sparse direct solves, FP64) on the bench's FEM
    leg inputs at vertex spacing 8, timed once on the host."""
    from oracle import fem as ofem

    n = int(n_sel.item())
    args = [t.cpu().numpy() for t in (d_mask, centers[:n], out[0][:n], out[1][:n], out[2][:n])]
    t0 = time.perf_counter()
    ofem.update(*args, 8, 1.0, 0.45, 2, 1, 0.05)
    return {"kind": "oracle", "grid": 8, "update_s": time.perf_counter() - t0,
            "sample": "the whole update (2 approximation steps + 1 interpolation step), numpy/scipy, one process"}


def run_reference(a):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_2308_10868_gb300 import synth

    oracle.build()
    w = synth.WORKLOADS[a.workload]
    pre, intra, mask = synth.workload_pair(a.workload)
    for _ in range(a.warmup):
        _oracle_step(w, pre, intra, mask, sample_every=4)
    evs, tot, n = 0, 0.0, 0
    for _ in range(a.steps):
        ev, dt, n = _oracle_step(w, pre, intra, mask, sample_every=4)
        evs += ev
        tot += dt
    v = evs / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": _config(w, n, {"sample": "selection of all blocks + matching every 4th selected block",
                                     "l2": "not applicable (host CPU run)"}),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "per step: full selection + matching every 4th selected block"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# the GPU path
# --------------------------------------------------------------------------
def _events_time(fn, flush, stream, fill):
    """Seconds between CUDA events recorded on ``stream`` around ``fn()``
    (host gaps inside ``fn`` included), L2 flushed before; returns (s, fn())."""
    import torch

    flush.fill_(fill)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3, out


def _plan_counts(plan, n):
    return [int(plan.view(i)[0].item()) for i in range(n)]


def _batched_search(a, nrr, synth, d_pre, d_intra, d_mask, w, flush):
    """The batched parameter search: 64 settings on the clinical pair, one
    graph-captured plan (autotuned; and the same plan with the sharing off)
    against 64 sequential plain calls; then settings spread over four pairs
    of different sizes in one plan against their plain calls."""
    import torch

    settings = synth.parameter_settings(64)
    stream = torch.cuda.current_stream()
    reps = max(2, a.batched_reps)

    def evals_of(counts, sets):
        return sum(n * (2 * r + 1) ** 3 for n, (b, r, f) in zip(counts, sets))

    # plain: one select (host count) + one match (own box sums) per setting
    def plain(jobs):
        counts = []
        for (p, i, m), (b, r, f) in jobs:
            c = nrr.select_blocks(p, m, b, 2, f)
            nrr.block_match(p, i, c, b, r)
            counts.append(c.shape[0])
        return counts

    def best(fn, fill):
        fn()
        torch.cuda.synchronize()
        ts, out = [], None
        for _ in range(reps):
            t, out = _events_time(fn, flush, stream, fill)
            ts.append(t)
        return min(ts), out

    one = [((d_pre, d_intra, d_mask), s) for s in settings]
    tp, counts = best(lambda: plain(one), 3)
    t0 = time.perf_counter()
    plan = nrr.BatchPlan(d_pre, d_intra, d_mask, [(b, 2, r, f) for b, r, f in settings], graph=True, autotune=True)
    t_create = time.perf_counter() - t0
    tb, _ = best(plan.run, 5)
    nrr.device_status()
    assert _plan_counts(plan, len(settings)) == counts, "batched and plain selections differ"
    plan.close()
    nod = nrr.BatchPlan(d_pre, d_intra, d_mask, [(b, 2, r, f) for b, r, f in settings], graph=True, dedup=False)
    tn, _ = best(nod.run, 6)
    nrr.device_status()
    assert _plan_counts(nod, len(settings)) == counts, "no-dedup plan and plain selections differ"
    nod.close()
    ev = evals_of(counts, settings)
    # work the plan actually computes: settings that differ only in the
    # fraction share the largest one's matched blocks, and a unit whose box
    # nests in a matched unit's box with no larger fraction is reported by
    # that unit's search (up to 4 extra radii per job)
    unit = {}
    for n, (b, r, f) in zip(counts, settings):
        if (b, r) not in unit or unit[(b, r)][1] < f:
            unit[(b, r)] = (n, f)
    launched = []
    for (b, r), (n, f) in sorted(unit.items(), key=lambda kv: (-kv[0][1], -kv[1][1])):
        host = [u for u in launched if u[0] == b and u[1] >= r and u[3] >= f and u[4] < 4]
        if host:
            host[0][4] += 1
        else:
            launched.append([b, r, n, f, 0])
    ev_computed = sum(n * (2 * r + 1) ** 3 for b, r, n, f, _ in launched)
    out = {"workload": "clinical pair x 64 settings (block 5/7/9, radius 3..7, fraction 2..10%, stride 2)",
           "settings": len(settings), "evals": ev, "evals_computed_by_plan": ev_computed,
           "dedup": "settings sharing (block, stride, radius) match the largest fraction's blocks once; a "
                    "smaller search box nested in a matched one (no larger fraction) is reported by that "
                    "search; the others' results are gathered (nested selections)",
           "plain_ms": 1e3 * tp, "batched_ms": 1e3 * tb, "batched_no_dedup_ms": 1e3 * tn,
           "plan_create_s": t_create,
           "plain_registrations_per_s": len(settings) / tp, "batched_registrations_per_s": len(settings) / tb,
           "batched_no_dedup_registrations_per_s": len(settings) / tn,
           "plain_evals_per_s": ev / tp, "batched_evals_per_s": ev / tb, "speedup": tp / tb,
           "speedup_no_dedup": tp / tn,
           "timing": "every arm: CUDA events on the launching stream around the whole arm (the plain arm's "
                     "host gaps and per-setting count reads included); best of repeats, L2 flushed before each"}
    # several registrations of different sizes in one plan: the clinical pair
    # and the three served sizes, 16 settings each
    pairs = [(d_pre, d_intra, d_mask)]
    for k in range(len(synth.SERVE_SIZES)):
        p_, i_, m_ = synth.serve_pair(k, 0)
        pairs.append((nrr.to_device_u16(p_), nrr.to_device_u16(i_), torch.from_numpy(m_).to(d_pre.device)))
    msets, pof = [], []
    for k in range(len(pairs)):
        for s_ in synth.parameter_settings(16, seed=synth.SEED_BASE + 40 + k):
            msets.append(s_)
            pof.append(k)
    jobs = [(pairs[k], s_) for k, s_ in zip(pof, msets)]
    tpm, mcounts = best(lambda: plain(jobs), 7)
    mplan = nrr.BatchPlan(settings=[(b, 2, r, f) for b, r, f in msets], pairs=pairs, pair_of=pof, graph=True,
                          autotune=True)
    tbm, _ = best(mplan.run, 8)
    nrr.device_status()
    assert _plan_counts(mplan, len(msets)) == mcounts, "multi-pair plan and plain selections differ"
    # the same plan with plain match launches (one CTA per block, no queue)
    pplan = nrr.BatchPlan(settings=[(b, 2, r, f) for b, r, f in msets], pairs=pairs, pair_of=pof, graph=True,
                          plain_launch=True)
    tpl, _ = best(pplan.run, 9)
    nrr.device_status()
    same = all(all(torch.equal(x.view(torch.uint8), y.view(torch.uint8))
                   for x, y in zip(mplan.result(i), pplan.result(i))) for i in range(len(msets)))
    mplan.close()
    pplan.close()
    out["multi_pair"] = {
        "workload": "4 pairs (256x256x124 clinical, 128x128x64, 192x192x96, 256x256x160) x 16 settings each",
        "settings": len(msets), "evals": evals_of(mcounts, msets), "plain_ms": 1e3 * tpm, "batched_ms": 1e3 * tbm,
        "plain_registrations_per_s": len(msets) / tpm, "batched_registrations_per_s": len(msets) / tbm,
        "speedup": tpm / tbm,
        "plain_launch_batched_ms": 1e3 * tpl, "persistent_speedup_over_plain_launch": tpl / tbm,
        "plain_launch_same_results": same}
    return out


def _serving(a, nrr, synth, dev):
    """The served stream: Poisson arrivals (mean 20 requests/s) of
    registrations of three volume sizes with random (block, radius,
    fraction); volumes resident on the device.  Reports p50/p99 latency
    (scheduled arrival to completion on the device) and registrations/s, the
    same for arrival rates from 50 to 1600 requests/s, and a saturation run (all
    requests queued at once) served with 8 slots (same-variant requests
    grouped into one match launch, and without grouping) against
    one-at-a-time FIFO service (1 slot, no grouping)."""
    import numpy as np
    import torch

    pool = []
    for si in range(len(synth.SERVE_SIZES)):
        pre, intra, mask = synth.serve_pair(si, 0)
        pool.append((nrr.to_device_u16(pre, dev), nrr.to_device_u16(intra, dev), torch.from_numpy(mask).to(dev)))
    torch.cuda.synchronize()

    def run(reqs, slots, open_loop, lone=False, arrays=None, max_group=16):
        srv = nrr.Server(slots=slots, reserve_bytes=2 << 30, max_group=max_group)
        try:
            # warm the kernels of every variant used, outside the measurement
            t0 = time.perf_counter()
            tickets, late = [], []
            for t_arr, si, b, r, f in reqs:
                if open_loop:
                    # sleep to within a millisecond of the arrival, then spin
                    # (sleep alone can wake late by several milliseconds)
                    dt = t_arr - (time.perf_counter() - t0)
                    if dt > 2e-3:
                        time.sleep(dt - 1e-3)
                    while time.perf_counter() - t0 < t_arr:
                        pass
                p, i, m = pool[si]
                # how long after its scheduled arrival the request was submitted
                late.append(max(0.0, (time.perf_counter() - t0) - t_arr) if open_loop else 0.0)
                tickets.append(srv.submit(p, i, m, b, 2, r, f))
                if lone:  # each request alone on the device: its service time
                    while srv.poll(tickets[-1]) is None:
                        pass
            done = {}
            while len(done) < len(tickets):
                for t in tickets:
                    if t not in done:
                        res = srv.poll(t)
                        if res is not None:
                            done[t] = (res["latency_s"], res["n"])
                            srv.release(t)
            wall = time.perf_counter() - t0
        finally:
            srv.stop()
        lat = np.array([done[t][0] for t in tickets])
        sched = lat + np.array(late)  # from the scheduled arrival
        if arrays is not None:
            arrays.append(sched)
        p50, p99 = float(np.percentile(sched, 50)), float(np.percentile(sched, 99))
        return {"requests": len(tickets), "slots": slots, "wall_s": wall, "registrations_per_s": len(tickets) / wall,
                "p50_ms": 1e3 * p50, "p99_ms": 1e3 * p99, "p99_over_p50": p99 / p50,
                "mean_ms": 1e3 * float(sched.mean()),
                "from_submission_p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "from_submission_p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "submission_late_max_ms": 1e3 * max(late)}

    reqs_open = synth.poisson_arrivals(a.serve_open_requests, 20.0)
    warm = [(0.0, si, b, r, f) for (si, b, r, f) in {(q[1], q[2], q[3], q[4]) for q in reqs_open}]
    run(warm, 8, False)
    out = {"workload": "Poisson 20 req/s, volumes 128x128x64 / 192x192x96 / 256x256x160 uint16, block 5/7/9, "
                       "radius 3..7, fraction 2..10%, stride 2, volumes resident on the device",
           "latency": "scheduled arrival to completion on the device (host callback timestamp); the "
                      "from_submission figures leave out how late the client submitted"}
    arr = []
    out["open_loop_20rps"] = run(reqs_open, 8, True, arrays=arr)
    # every request of the stream again, alone on the device: its service
    # time.  The stream's latency spread is mostly the spread of the work
    # (volume size x blocks x block size x search box spans two orders of
    # magnitude); the slowdown (latency / lone service time) isolates what
    # the serving adds
    out["lone_service"] = run(reqs_open, 1, False, lone=True, arrays=arr)
    slow = arr[0] / arr[1]
    out["open_loop_20rps"].update({
        "slowdown_p50": float(np.percentile(slow, 50)), "slowdown_p99": float(np.percentile(slow, 99)),
        "slowdown_p99_over_p50": float(np.percentile(slow, 99) / np.percentile(slow, 50)),
        "lone_service_p50_ms": 1e3 * float(np.percentile(arr[1], 50)),
        "lone_service_p99_ms": 1e3 * float(np.percentile(arr[1], 99))})
    # arrival-rate sweep up to saturation (same request mix, fresh arrivals)
    sweep = {}
    for rate in (50.0, 100.0, 200.0, 400.0, 800.0, 1600.0):
        reqs = synth.poisson_arrivals(a.serve_sweep_requests, rate, seed=synth.SEED_BASE + 20 + int(rate))
        sweep[f"{rate:g}rps"] = run(reqs, 8, True)
    out["open_loop_rate_sweep"] = sweep
    reqs_closed = [(0.0, si, b, r, f) for (_, si, b, r, f) in synth.poisson_arrivals(a.serve_closed_requests, 20.0,
                                                                                      seed=synth.SEED_BASE + 11)]
    # each saturated configuration twice, the second timed: the first maps
    # the request pool's memory for that many requests in flight
    for name, slots, mg in (("saturated_served_8_slots", 8, 16), ("saturated_8_slots_no_grouping", 8, 1),
                            ("saturated_fifo_1_slot", 1, 1)):
        run(reqs_closed, slots, False, max_group=mg)
        out[name] = run(reqs_closed, slots, False, max_group=mg)
    out["saturated_speedup"] = (out["saturated_served_8_slots"]["registrations_per_s"] /
                                out["saturated_fifo_1_slot"]["registrations_per_s"])
    return out


def _highres(a, nrr, synth, dev, flush):
    """The high-resolution variant: 512x512x256, block 9^3, stride 3, top 5%,
    radius 7 (3375 shifts), as uint16 (exact path) and as float32 u/65535
    (FP32 search, FP64 rescoring), and as float32 on an offset of 100.  Their agreement with the oracle is checked by
    tests/test_gpu_highres.py and tests/test_gpu_parity.py, not here."""
    import numpy as np
    import torch

    w = synth.WORKLOADS["highres"]
    pre, intra, mask = synth.workload_pair("highres")
    dpre, dintra = nrr.to_device_u16(pre, dev), nrr.to_device_u16(intra, dev)
    dmask = torch.from_numpy(mask).to(dev)
    p32, i32 = synth.as_f32(pre), synth.as_f32(intra)
    fpre, fintra = torch.from_numpy(p32).to(dev), torch.from_numpy(i32).to(dev)
    stream = torch.cuda.current_stream()
    centers = nrr.select_blocks(dpre, dmask, w.block, w.stride, w.frac)
    n = centers.shape[0]
    evals = n * (2 * w.radius + 1) ** 3
    out = {"workload": w.name, "n_blocks": n, "shifts": (2 * w.radius + 1) ** 3, "evals": evals}
    # float32 on a large offset: 100 + u/65535 (a block's spread is 10^-2 to
    # 10^-4 of the intensity range, so the offset is 10^4 to 10^6 times it),
    # which the centred float box sums keep boundable; the float spacing at
    # 100 (2^-17) still resolves every uint16 step (about 2^-16)
    opre = torch.from_numpy((np.float32(100.0) + p32).astype(np.float32)).to(dev)
    ointra = torch.from_numpy((np.float32(100.0) + i32).astype(np.float32)).to(dev)
    # the same with the reference volume's centre voxel set to 0: c = 0, so
    # the box sums are the plain sums of J and J^2 (what centring removes)
    zintra = ointra.clone()
    zintra[zintra.shape[0] // 2, zintra.shape[1] // 2, zintra.shape[2] // 2] = 0.0
    for name, (p, i) in (("u16", (dpre, dintra)), ("f32", (fpre, fintra)), ("f32_offset", (opre, ointra)),
                         ("f32_offset_sums_uncentred", (opre, zintra))):
        box = nrr.boxsums(i, w.block)
        res = nrr.block_match(p, i, centers, w.block, w.radius, box=box)
        ts = []
        for _ in range(3):
            flush.fill_(7)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nrr.block_match(p, i, centers, w.block, w.radius, box=box, out=res)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        nrr.device_status()
        t = min(ts)
        out[name] = {"match_ms": 1e3 * t, "evals_per_s": evals / t,
                     "roofline_frac": 2.0 * evals * w.block ** 3 / t / 1e12 / (
                         torch.cuda.get_device_properties(dev).multi_processor_count * FP32_LANES_PER_SM * 2 *
                         float(_peaks().get("sm_max_mhz", 2070.0)) * 1e6 / 1e12)}
    return out


ANISO_BLOCK = (9, 9, 5)   # edges along x, y, z: thick slices along z
ANISO_RADIUS = (5, 5, 3)


def _aniso(a, nrr, synth, d_pre, d_intra, d_mask, w, flush):
    """Blocks with a different edge per axis on the step's clinical pair:
    block 9x9x5, radius 5x5x3 (847 shifts), stride 2, top 5%: selection, box
    sums (three separable passes) and matching, each timed on its own with
    CUDA events (best of 3, L2 flushed before each).  Agreement with the
    oracle is checked by tests/test_gpu_aniso.py."""
    import torch

    stream = torch.cuda.current_stream()
    bl, r = ANISO_BLOCK, ANISO_RADIUS
    shifts = (2 * r[0] + 1) * (2 * r[1] + 1) * (2 * r[2] + 1)
    nblk = bl[0] * bl[1] * bl[2]

    def timed(fn):
        ts = []
        for _ in range(3):
            flush.fill_(7)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return min(ts)

    centers = nrr.select_blocks(d_pre, d_mask, bl, w.stride, w.frac)
    n = centers.shape[0]
    cbuf, cnt = nrr.select_blocks(d_pre, d_mask, bl, w.stride, w.frac, sync=False)
    t_sel = timed(lambda: nrr.select_blocks(d_pre, d_mask, bl, w.stride, w.frac, centers=cbuf, n_selected=cnt,
                                            sync=False))
    box = nrr.boxsums(d_intra, bl)
    t_box = timed(lambda: nrr.boxsums(d_intra, bl, out=box))
    box = nrr.boxsums(d_intra, bl)
    res = nrr.block_match(d_pre, d_intra, centers, bl, r, box=box)
    t_match = timed(lambda: nrr.block_match(d_pre, d_intra, centers, bl, r, box=box, out=res))
    nrr.device_status()
    evals = n * shifts
    peak = (torch.cuda.get_device_properties(d_pre.device).multi_processor_count * FP32_LANES_PER_SM * 2 *
            float(_peaks().get("sm_max_mhz", 2070.0)) * 1e6)
    return {"workload": f"clinical pair, block {bl[0]}x{bl[1]}x{bl[2]}, radius {r[0]}x{r[1]}x{r[2]}, "
                        f"stride {w.stride}, top {w.frac:.0%}",
            "n_blocks": n, "shifts": shifts, "evals": evals,
            "select_ms": 1e3 * t_sel, "box_sums_ms": 1e3 * t_box, "match_ms": 1e3 * t_match,
            "evals_per_s": evals / (t_sel + t_box + t_match), "match_evals_per_s": evals / t_match,
            "match_roofline_frac": 2.0 * evals * nblk / t_match / peak}


def _same_results(out, n_sel, ref):
    """Whether the outputs (disp, ncc, valid) and the device count equal the
    reference copies bit for bit, over the blocks the count covers (entries
    past it are never written)."""
    import torch

    n = int(ref[3].item())
    if not torch.equal(n_sel.view(torch.uint8), ref[3].view(torch.uint8)):
        return False
    return all(torch.equal(x[:n].contiguous().view(torch.uint8), y[:n].contiguous().view(torch.uint8))
               for x, y in zip(out, ref[:3]))


def _small(a, nrr, synth, dev, flush):
    """The small single registration (64x64x48 uint16, blocks 7^3 on a
    stride-2 grid, top 10%, radius 4: about 940 blocks x 729 shifts), a
    latency-bound case: selection, box sums and matching of one registration
    on the launching stream, CUDA events around each (median of 20, L2 flushed
    before each), as eager calls and as a replayed CUDA graph of the calls."""
    import torch

    stream = torch.cuda.current_stream()
    w = synth.WORKLOADS["small"]
    pre, intra, mask = synth.workload_pair("small")
    d_pre, d_intra = nrr.to_device_u16(pre, dev), nrr.to_device_u16(intra, dev)
    d_mask = torch.from_numpy(mask).to(dev)
    cap = nrr.max_selected(w.dims, w.stride, w.frac)
    centers = torch.empty((cap, 3), dtype=torch.int32, device=dev)
    n_sel = torch.zeros(1, dtype=torch.int32, device=dev)
    out = (torch.empty((cap, 3), dtype=torch.int32, device=dev), torch.empty(cap, dtype=torch.float64, device=dev),
           torch.empty(cap, dtype=torch.uint8, device=dev))
    box_raw = torch.empty(nrr.boxsum_bytes(d_intra) + 256, dtype=torch.uint8, device=dev)
    step_ms, match_ms = [], []
    for k in range(23):
        flush.fill_(k & 0xFF)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        nrr.select_blocks(d_pre, d_mask, w.block, w.stride, w.frac, max_blocks=cap, centers=centers, n_selected=n_sel,
                          sync=False)
        box = nrr.boxsums(d_intra, w.block, out=box_raw)
        e[1].record(stream)
        nrr.block_match(d_pre, d_intra, centers, w.block, w.radius, n_blocks=n_sel, box=box, out=out)
        e[2].record(stream)
        e[2].synchronize()
        if k >= 3:
            step_ms.append(e[0].elapsed_time(e[2]))
            match_ms.append(e[1].elapsed_time(e[2]))
    nrr.device_status()
    n = int(n_sel.item())
    evals = n * (2 * w.radius + 1) ** 3
    st, mt = sorted(step_ms)[len(step_ms) // 2], sorted(match_ms)[len(match_ms) // 2]
    res = {"workload": w.name, "n_blocks": n, "shifts": (2 * w.radius + 1) ** 3, "evals": evals,
           "eager_step_ms": st, "match_ms": mt, "valid_blocks": int(out[2][:n].sum().item())}
    # the same registration replayed from a CUDA graph of the three calls:
    # the eager calls' launch latency dominates a registration this small.
    # Every buffer it writes is cleared first and the replay must reproduce
    # the eager results bit for bit.
    ref = [t.clone() for t in out] + [n_sel.clone()]
    timing = "eager calls"
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="thread_local"):
            nrr.select_blocks(d_pre, d_mask, w.block, w.stride, w.frac, max_blocks=cap, centers=centers,
                              n_selected=n_sel, sync=False)
            box = nrr.boxsums(d_intra, w.block, out=box_raw)
            nrr.block_match(d_pre, d_intra, centers, w.block, w.radius, n_blocks=n_sel, box=box, out=out)
        for t in list(out) + [centers, n_sel, box_raw]:
            t.zero_()
        g.replay()
        torch.cuda.synchronize()
        nrr.device_status()
        if _same_results(out, n_sel, ref):
            gms = []
            for k in range(23):
                flush.fill_(k & 0xFF)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.replay()
                e1.record(stream)
                e1.synchronize()
                if k >= 3:
                    gms.append(e0.elapsed_time(e1))
            st = sorted(gms)[len(gms) // 2]
            timing = "CUDA graph of the three calls, replayed"
    except Exception as ex:
        torch.cuda.synchronize()
        timing = f"eager calls (graph capture failed: {type(ex).__name__})"
    res.update({"step_ms": st, "step_timing": timing, "evals_per_s": evals / (st / 1e3),
                "registrations_per_s": 1e3 / st})
    return res


def _spacing(a, nrr, synth, d_pre, d_mask, w, flush):
    """Selection with the face / edge / vertex connectivity patterns (6 / 18 /
    26 neighbours on the candidate grid) on the step's volume, against the
    plain selection: device time per selection (CUDA events, L2 flushed
    before each) and the number selected."""
    import torch

    stream = torch.cuda.current_stream()
    out = {"workload": w.name, "timing": "CUDA events around one selection, best of 5, L2 flushed before each"}
    for conn in (0, 6, 18, 26):
        ts = []
        for _ in range(6):
            flush.fill_(3)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c, n = nrr.select_blocks(d_pre, d_mask, w.block, w.stride, w.frac, connectivity=conn, sync=False)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        nrr.device_status()
        out[f"conn{conn}"] = {"select_ms": min(ts[1:]), "n_selected": int(n.item())}
    return out


def _fem(a, nrr, d_mask, centers, n_sel, out, w, flush):
    """The robust finite-element update (nrr_fem_update) on the step's block
    matches: device time per update (CUDA events, best of 3, L2 flushed
    before each) at vertex spacings 8 and 4 voxels, with each solve's
    conjugate-gradient iterations; E = 1, nu = 0.45, two approximation steps
    rejecting 5 % each and one interpolation step, tolerance 1e-10 on the
    warm start's residual.  (The oracle's time for the same update is part
    of the CPU-baseline leg.)"""
    import torch

    stream = torch.cuda.current_stream()
    n = int(n_sel.item())
    c, disp, ncc, valid = centers[:n], out[0][:n], out[1][:n], out[2][:n]
    kw = dict(young=1.0, poisson=0.45, n_rej=2, n_int=1, reject_frac=0.05, cg_tol=1e-10)
    res = {"workload": w.name + " block matches", "n_blocks": n, "params": kw,
           "timing": "CUDA events around one nrr_fem_update call (which waits once for its stream), best of 3"}
    for g in (int(v) for v in a.fem_grids.split(",")):
        ts, iters = [], None
        for _ in range(4):
            flush.fill_(5)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            U, sk, step, iters = nrr.fem_update(d_mask, c, disp, ncc, valid, grid=g, **kw)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        nrr.device_status()
        nv = U.shape[0] * U.shape[1] * U.shape[2]
        res[f"grid{g}"] = {"update_ms": min(ts[1:]), "vertices": nv, "cg_iterations": iters,
                           "ms_per_cg_iteration": min(ts[1:]) / max(1, sum(iters)),
                           "rejected": int((step >= 0).sum().item()), "max_abs_U": float(U.abs().max().item())}
    return res


def _phases(w, select_ms, box_ms, match_ms, peaks):
    """Device time of the three phases of a step (CUDA events on the launching
    stream, averaged over the timed steps) and, for the two HBM-type phases,
    algorithmic bytes over time against the measured copy bandwidth:
    selection reads the volume (2 B/voxel) and the mask (1 B/voxel) and
    writes one 8-byte key per grid point (plus passes over the keys, not
    counted); box sums read 2 B and write 8 B per voxel."""
    nv = w.dims[0] * w.dims[1] * w.dims[2]
    ng = 1
    for d in w.dims:
        ng *= -(-d // w.stride)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    sel_s = sum(select_ms) / len(select_ms) / 1e3
    box_s = sum(box_ms) / len(box_ms) / 1e3
    sel_b, box_b = 3 * nv + 8 * ng, 10 * nv
    return {"selection_ms": 1e3 * sel_s, "box_sums_ms": 1e3 * box_s,
            "match_ms": sum(match_ms) / len(match_ms),
            "selection_hbm": {"algorithmic_bytes": sel_b, "achieved_gbs": sel_b / sel_s / 1e9,
                              "frac_of_measured_hbm": sel_b / sel_s / 1e9 / hbm},
            "box_sums_hbm": {"algorithmic_bytes": box_b, "achieved_gbs": box_b / box_s / 1e9,
                             "frac_of_measured_hbm": box_b / box_s / 1e9 / hbm}}


def _plain_vs_persistent(a, nrr, d_pre, d_intra, centers, n_sel, box_raw, w, flush, cap, dev):
    """Matching alone on the clinical blocks, in the plain launch form (one CTA
    per block, nrr_block_match_plain) and in the persistent form the step
    uses; CUDA events on the launching stream, L2 flushed before each launch,
    results compared bit for bit."""
    import torch

    stream = torch.cuda.current_stream()
    box = nrr.boxsums(d_intra, w.block, out=box_raw)
    outs = {}
    times = {}
    reps = max(10, min(a.steps, 50))
    for plain in (False, True):
        out = (torch.empty((cap, 3), dtype=torch.int32, device=dev), torch.empty(cap, dtype=torch.float64, device=dev),
               torch.empty(cap, dtype=torch.uint8, device=dev))
        ms = []
        for k in range(reps + 3):
            flush.fill_(k & 0xFF)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            nrr.block_match(d_pre, d_intra, centers, w.block, w.radius, n_blocks=n_sel, box=box, out=out, plain=plain)
            s1.record(stream)
            s1.synchronize()
            if k >= 3:
                ms.append(s0.elapsed_time(s1))
        nrr.device_status()
        outs[plain] = out
        times[plain] = sum(ms) / len(ms)
    same = all(torch.equal(x.view(torch.uint8), y.view(torch.uint8)) for x, y in zip(outs[False], outs[True]))
    return {"workload": "clinical blocks, matching only, L2 flushed before each launch",
            "persistent_match_ms": times[False], "plain_match_ms": times[True],
            "persistent_speedup": times[True] / times[False], "launches_timed": reps, "same_results": same}


def run_ours(a):
    import numpy as np
    import torch

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    from paper_2308_10868_gb300 import build as nbuild

    nbuild.build()
    from paper_2308_10868_gb300 import nrr, synth

    w = synth.WORKLOADS[a.workload]
    pre, intra, mask = synth.workload_pair(a.workload)
    d_pre, d_intra = nrr.to_device_u16(pre, dev), nrr.to_device_u16(intra, dev)
    d_mask = torch.from_numpy(mask).to(dev)
    cap = nrr.max_selected(w.dims, w.stride, w.frac)
    centers = torch.empty((cap, 3), dtype=torch.int32, device=dev)
    n_sel = torch.zeros(1, dtype=torch.int32, device=dev)
    out = (torch.empty((cap, 3), dtype=torch.int32, device=dev), torch.empty(cap, dtype=torch.float64, device=dev),
           torch.empty(cap, dtype=torch.uint8, device=dev))
    box_raw = torch.empty(nrr.boxsum_bytes(d_intra) + 256, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # twice the L2
    stream = torch.cuda.current_stream()

    side = torch.cuda.Stream(device=dev)

    def registration(p, i, m, c_, n_, b_, o_):
        # the box sums of the reference volume do not depend on the selection:
        # they run on a second stream beside it (the selection's radix passes
        # leave most of the GPU idle) and matching waits for both.  The fork
        # and join are taken from the current stream, so that a graph capture
        # (which runs on a capture stream of its own) records both branches.
        cur = torch.cuda.current_stream()
        side.wait_stream(cur)
        with torch.cuda.stream(side):
            bx = nrr.boxsums(i, w.block, out=b_)
        nrr.select_blocks(p, m, w.block, w.stride, w.frac, max_blocks=cap, centers=c_, n_selected=n_, sync=False)
        cur.wait_stream(side)
        nrr.block_match(p, i, c_, w.block, w.radius, n_blocks=n_, box=bx, out=o_)

    def step(p, i, m, ev_phase=None):
        # ev_phase: events after selection, after box sums, after matching
        # (the phases in sequence on one stream, to time each)
        if ev_phase is None:
            registration(p, i, m, centers, n_sel, box_raw, out)
            return
        nrr.select_blocks(p, m, w.block, w.stride, w.frac, max_blocks=cap, centers=centers, n_selected=n_sel,
                          sync=False)
        ev_phase[0].record(stream)
        box = nrr.boxsums(i, w.block, out=box_raw)
        ev_phase[1].record(stream)
        nrr.block_match(p, i, centers, w.block, w.radius, n_blocks=n_sel, box=box, out=out)
        ev_phase[2].record(stream)

    if a.fem_only:
        step(d_pre, d_intra, d_mask)
        nrr.device_status()
        if rank == 0:
            print(json.dumps({"fem": _fem(a, nrr, d_mask, centers, n_sel, out, w, flush)}), flush=True)
        return 0
    for _ in range(max(3, a.warmup)):
        flush.fill_(1)
        step(d_pre, d_intra, d_mask)
    nrr.device_status()
    n_blocks = int(n_sel.item())
    evals = n_blocks * (2 * w.radius + 1) ** 3
    valid_count = int(out[2][:n_blocks].sum().item())

    # one step captured as a CUDA graph (the step's launches are short and
    # many: replaying them from a graph keeps host launch latency out of the
    # device timeline); the graph's results are checked against the eager step
    graph, graph_note = None, ("one step captured as a CUDA graph and replayed; its box sums run on a second stream "
                                "beside the selection")
    ref = [t.clone() for t in out] + [n_sel.clone()]
    try:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, capture_error_mode="thread_local"):
            step(d_pre, d_intra, d_mask)
        # everything the step computes is cleared first, so that a graph that
        # skipped any of it fails the comparison below
        for t in list(out) + [centers, n_sel, box_raw]:
            t.zero_()
        for _ in range(max(3, a.warmup)):
            flush.fill_(1)
            graph.replay()
        torch.cuda.synchronize()
        nrr.device_status()
        same = _same_results(out, n_sel, ref)
        if not same:
            graph, graph_note = None, "graph replay differed from the eager step; eager steps timed"
    except Exception as ex:  # capture not available: time the eager steps
        graph, graph_note = None, f"graph capture failed ({type(ex).__name__}); eager steps timed"
        torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    evm = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(a.steps)]
    evg = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    l0 = nrr.kernel_launches()
    with ClockSampler(local) as clk:
        t_start = time.time()
        # eager steps through the public calls, with per-phase events
        for k in range(a.steps):
            flush.fill_(k & 0xFF)
            evs[k][0].record(stream)
            step(d_pre, d_intra, d_mask, evm[k])
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        launches = nrr.kernel_launches() - l0
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        # the timed steps of the headline: graph replays of the same step
        if graph is not None:
            for k in range(a.steps):
                flush.fill_(k & 0xFF)
                evg[k][0].record(stream)
                graph.replay()
                evg[k][1].record(stream)
            torch.cuda.synchronize()
        t_end = time.time()
    nrr.device_status()
    if pg:
        pg.barrier()
    eager_ms = [s.elapsed_time(e) for s, e in evs]
    step_ms = [s.elapsed_time(e) for s, e in evg] if graph is not None else eager_ms
    # the graph replays launch the same kernels per step as the eager steps
    select_ms = [s.elapsed_time(p[0]) for (s, _), p in zip(evs, evm)]
    box_ms = [p[0].elapsed_time(p[1]) for p in evm]
    match_ms = [p[1].elapsed_time(p[2]) for p in evm]
    total_s, value = aggregate_replicas(sum(step_ms) / 1e3, world, a.steps * evals, pg)

    # ---- end to end through the public API with host buffers --------------
    h_pre = torch.from_numpy(np.ascontiguousarray(pre).view(np.int16)).pin_memory()
    h_intra = torch.from_numpy(np.ascontiguousarray(intra).view(np.int16)).pin_memory()
    h_mask = torch.from_numpy(np.ascontiguousarray(mask)).pin_memory()
    e_pre, e_intra, e_mask = torch.empty_like(d_pre), torch.empty_like(d_intra), torch.empty_like(d_mask)
    h_out = (torch.empty((cap, 3), dtype=torch.int32).pin_memory(), torch.empty(cap, dtype=torch.float64).pin_memory(),
             torch.empty(cap, dtype=torch.uint8).pin_memory(), torch.empty(1, dtype=torch.int32).pin_memory())
    bi = h_pre.numel() * 2 + h_intra.numel() * 2 + h_mask.numel()
    bo = sum(t.numel() * t.element_size() for t in h_out)
    ke = max(10, min(a.steps, 100))
    e2e_ms = []
    for k in range(ke + 3):
        flush.fill_(k & 0xFF)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        e_pre.copy_(h_pre, non_blocking=True)
        e_intra.copy_(h_intra, non_blocking=True)
        e_mask.copy_(h_mask, non_blocking=True)
        step(e_pre, e_intra, e_mask)
        for h, d in zip(h_out, out + (n_sel,)):
            h.copy_(d, non_blocking=True)
        s1.record(stream)
        s1.synchronize()
        if k >= 3:
            e2e_ms.append(s0.elapsed_time(s1))
    assert int(h_out[3].item()) == n_blocks
    e2e_serial = world * evals / (sum(e2e_ms) / len(e2e_ms) / 1e3)

    # ---- the same, as a stream of registrations: the next step's inputs are
    # copied in and the previous step's results copied out while a step
    # computes (three streams, double-buffered device inputs and outputs)
    h2d_s, d2h_s = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    din = [(torch.empty_like(d_pre), torch.empty_like(d_intra), torch.empty_like(d_mask)) for _ in range(2)]
    dout = [(torch.empty((cap, 3), dtype=torch.int32, device=dev), torch.zeros(1, dtype=torch.int32, device=dev),
             (torch.empty((cap, 3), dtype=torch.int32, device=dev), torch.empty(cap, dtype=torch.float64, device=dev),
              torch.empty(cap, dtype=torch.uint8, device=dev)),
             torch.empty(nrr.boxsum_bytes(d_intra) + 256, dtype=torch.uint8, device=dev)) for _ in range(2)]

    # each registration's compute (L2 flush, selection, box sums, matching)
    # replayed from a CUDA graph captured from the same public calls, one per
    # double-buffer parity: one launch per registration from the host instead
    # of the calls' dozen (eager calls if capture is not available)
    cgraphs = []
    try:
        for par in range(2):
            g = torch.cuda.CUDAGraph()
            p_, i_, m_ = din[par]
            c_, n_, o_, b_ = dout[par]
            with torch.cuda.graph(g, capture_error_mode="thread_local"):
                flush.fill_(par + 1)
                registration(p_, i_, m_, c_, n_, b_, o_)
            cgraphs.append(g)
    except Exception:
        cgraphs = []
        torch.cuda.synchronize()

    def pipelined(kk):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev_in = [torch.cuda.Event() for _ in range(kk)]
        ev_done = [torch.cuda.Event() for _ in range(kk)]
        ev_out = [torch.cuda.Event() for _ in range(kk)]
        t0.record(stream)
        h2d_s.wait_event(t0)

        def copy_in(k):
            with torch.cuda.stream(h2d_s):
                if k >= 2:
                    h2d_s.wait_event(ev_done[k - 2])  # buffer k % 2 was read by step k - 2
                for d, h in zip(din[k % 2], (h_pre, h_intra, h_mask)):
                    d.copy_(h, non_blocking=True)
                ev_in[k].record(h2d_s)

        copy_in(0)
        for k in range(kk):
            stream.wait_event(ev_in[k])
            if k >= 2:
                stream.wait_event(ev_out[k - 2])  # outputs k % 2 were read back
            p_, i_, m_ = din[k % 2]
            c_, n_, o_, b_ = dout[k % 2]
            if cgraphs:
                cgraphs[k % 2].replay()
            else:
                flush.fill_(k & 0xFF)
                registration(p_, i_, m_, c_, n_, b_, o_)
            ev_done[k].record(stream)
            with torch.cuda.stream(d2h_s):
                d2h_s.wait_event(ev_done[k])
                for h, d in zip(h_out, o_ + (n_,)):
                    h.copy_(d, non_blocking=True)
                ev_out[k].record(d2h_s)
            if k + 1 < kk:
                copy_in(k + 1)
        stream.wait_event(ev_out[kk - 1])
        t1.record(stream)
        t1.synchronize()
        return t0.elapsed_time(t1) / kk

    pipelined(3)
    e2e_value = world * evals / (pipelined(ke) / 1e3)
    assert int(h_out[3].item()) == n_blocks
    # the last pipelined registration's results, read back to the host, are
    # the device-resident step's results bit for bit
    for h, d in zip(h_out[:3], ref[:3]):
        if not torch.equal(h[:n_blocks].view(torch.uint8), d[:n_blocks].cpu().view(torch.uint8)):
            raise RuntimeError("pipelined end-to-end results differ from the device-resident step")

    if rank != 0:
        return 0

    # ---- roofline of the dominant kernel (the match kernel) ---------------
    peaks = _peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    match_s = sum(match_ms) / len(match_ms) / 1e3
    flops = 2.0 * evals * w.block ** 3
    achieved = flops / match_s / 1e12
    traffic = _recorded_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * total_s / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u16", "data": "synthetic", "config": _config(w, n_blocks, {"parallelism": f"replicas x{world}"}),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": traffic,
                     "kernel": "match_kernel (FP32 FFMA search + exact rescoring)",
                     "peak_basis": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                                   f"{sm_max:.0f} MHz (max SM clock)",
                     "match_ms": 1e3 * match_s},
        "phases": _phases(w, select_ms, box_ms, match_ms, peaks),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                "pipelining": "each step's inputs copied from pinned host memory and results copied back inside "
                              "the timed region, overlapped with the neighbouring steps' compute (3 streams); "
                              + ("each step's compute replayed from a CUDA graph captured from the public calls"
                                 if cgraphs else "each step's compute launched by the public calls"),
                "serial_value": e2e_serial},
        "gpu_launches": launches,
        "gpu_launches_per_step": launches / a.steps,
        "step_timing": graph_note,
        "eager_ms_per_step": sum(eager_ms) / len(eager_ms),
        "registrations_per_s": world * a.steps / total_s,
        "valid_blocks": valid_count,
        "clocks": clk.summary(t_start, t_end),
    }
    if not a.no_plain:
        line["plain_vs_persistent"] = _plain_vs_persistent(a, nrr, d_pre, d_intra, centers, n_sel, box_raw, w, flush,
                                                           cap, dev)
    if not a.no_small:
        line["small"] = _small(a, nrr, synth, dev, flush)
    if not a.no_batched:
        line["batched"] = _batched_search(a, nrr, synth, d_pre, d_intra, d_mask, w, flush)
    if not a.no_serving:
        line["serving"] = _serving(a, nrr, synth, dev)
    if not a.no_highres:
        line["highres"] = _highres(a, nrr, synth, dev, flush)
    if not a.no_spacing:
        line["spacing"] = _spacing(a, nrr, synth, d_pre, d_mask, w, flush)
    if not a.no_aniso:
        line["aniso"] = _aniso(a, nrr, synth, d_pre, d_intra, d_mask, w, flush)
    if not a.no_fem:
        line["fem"] = _fem(a, nrr, d_mask, centers, n_sel, out, w, flush)
    if world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(w, pre, intra, mask)
        if not a.no_fem:
            line["cpu_baseline"]["fem"] = _cpu_baseline_fem(d_mask, centers, n_sel, out)
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def main():
    a = _args()
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
