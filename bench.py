#!/usr/bin/env python
"""Benchmark of the contention-aware partition/allocation path on GB300.

Headline workload (the schedulability-ratio sweep): 1 000 000 synthetic task
sets of 4..64 tasks (uniform) on a 148-SM GPU, U = 0.1 .. 6.0 in steps of 0.1
(equal sets per step), memory intensity Beta(2, 5), D = 0.75 T.  One step
decides every set twice, as the sweep compares them: by the paper's
partition-and-allocate heuristic (Alg. 1-3, SMS order, no ACT pre-pass) and
by the 1G baseline (the GPU as one partition), each one gpa_allocate call
replayed from a CUDA graph with launch shapes picked by the library's
autotuner; end to end from pinned host buffers, one gpa_allocate_multi call
per step copies the batch in once and decides it under both.  Metric: task sets decided per second (whole job, all ranks);
candidate allocations tested per second beside it (the heuristic's merge
candidates plus one 1G candidate per set).

The line also carries one record per other workload under "configs": the
single instance (every explicit SM split x map of 8 tasks on 8 SMs, enumerated
and tested on the device), the batching workload (100 000 sets on 80 SMs, the
plain one-launch-per-set form beside it), the exhaustive optimum (20 000 sets
of 12 tasks on 20 TPC units), the paper's §7 setting (3 400 sets of 50 tasks on
68 SMs, the merge-heavy case) and serving (Poisson admission queries against
device-resident tenants, p50 / p99 latency, continuous batching against one
request per launch).  Each record has its own roofline, CPU oracle baseline
and end-to-end figure.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload sweep|sweep1g|batch|exhaustive|single|paper50|paper200] [--no-configs]

Under torchrun each rank decides its own batch (seed offset by rank: weak
scaling, no data-path collective); the timed region is bracketed by a barrier
and a device synchronize, and the step time is the max over ranks.  The L2
(129 MB) is flushed before every timed step by writing a 512 MB buffer and
then reading a second 256 MB one (so the L2 holds clean lines, none of the
inputs).  ``--impl reference`` times the CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2105_10312_gb300 import shard  # noqa: E402
from paper_2105_10312_gb300 import workloads as W  # noqa: E402

METRIC = "candidate allocations tested/sec, tasksets decided/sec (1 GB300); serve p50/p99 ms"

DESCR = {
    "sweep": "sweep: 1000000 task sets x U{4..64} tasks, 148 SMs, U=0.1..6.0 step 0.1, Beta(2,5) intensity, "
             "D=0.75T; every set decided by the heuristic (SMS/INA) and by the 1G baseline",
    "sweep1g": "sweep: 1000000 task sets x U{4..64} tasks, 148 SMs, U=0.1..6.0 step 0.1, Beta(2,5) intensity; "
               "1G baseline only",
    "batch": "batching: 100000 task sets x U{16..32} tasks, 80 SMs, U~U[0.5,3.0], D=0.75T; heuristic SMS/INA per set",
    "exhaustive": "exhaustive: 20000 task sets x 12 tasks, 20 TPC units, 1..4 partitions; exact optimum per set",
    "single": "single instance: 8 tasks, U=0.8, 8 SMs in exactly 2 partitions; all 7 x 2^8 = 1792 explicit "
              "candidates enumerated and tested on the device",
    "paper50": "paper setting: 3400 task sets x 50 tasks, 68 SMs, U=2..68 step 2, D=0.75T; heuristic SMS/INA",
    "paper200": "paper setting: 3400 task sets x 200 tasks, 68 SMs, U=2..68 step 2, D=0.75T; heuristic SMS/INA",
}
# the calls of one step of each workload (policy of each gpa_allocate call, or the search entry point)
CALLS = {"sweep": ("SMS", "ONE_GPU"), "sweep1g": ("ONE_GPU",), "batch": ("SMS",), "paper50": ("SMS",),
         "paper200": ("SMS",), "exhaustive": ("SEARCH",), "single": ("EXPLICIT",)}
DEFAULT_STEPS = {"sweep": 50, "sweep1g": 50, "batch": 1000, "paper50": 100, "paper200": 3, "exhaustive": 10,
                 "single": 500}
SUBRECORDS = ("single", "batch", "exhaustive", "paper50")


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the sources each profiled kernel is compiled from
KERNEL_SOURCES = {
    "alloc": ("k_alloc.cu", "alloc_dev.cuh", "gpa_device.cuh", "bulk_pipe.cuh", "gpa_ns.h", "gpa_internal.h"),
    "search": ("k_search.cu", "gpa_device.cuh", "gpa_ns.h", "gpa_internal.h"),
}


def kernel_source_hash(kernel="alloc_fast"):
    """Hash of the sources `kernel` is compiled from."""
    d = os.path.join(ROOT, "paper_2105_10312_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES["search" if kernel.startswith("search") else "alloc"]:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# the committed ncu summary of each workload's kernels
PROFILES = {("alloc_fast", "batch"): "alloc_fast_batch.md", ("alloc_merge", "paper50"): "alloc_merge_paper50.md",
            ("one_gpu", "sweep"): "one_gpu_sweep.md", ("one_gpu_fast", "sweep"): "one_gpu_fast_sweep.md",
            ("search_sets", "exhaustive"): "search_sets_exhaustive.md",
            ("alloc_fast", "sweep"): "alloc_fast_sweep.md"}


def recorded_profile(kernel, workload):
    """Figures of the committed ncu summary of `kernel` on `workload` (DRAM
    bytes per launch, ALU pipe, issue and warps-active percentages), if it
    was taken on the current kernel sources; else None."""
    name = PROFILES.get((kernel, workload))
    path = os.path.join(ROOT, "profiles", name) if name else None
    if not path or not os.path.exists(path):
        return None
    text = open(path).read()
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    if not h or h.group(1) != kernel_source_hash(kernel):
        return None
    out = {"source": "profiles/" + name}
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.]+)", text)
    out["traffic"] = float(m.group(1)) if m else None
    m = re.search(r"captured_tasks:\s*([0-9]+)", text)
    out["captured_tasks"] = int(m.group(1)) if m else None
    for key, metric in (("alu_pipe_pct", "sm__pipe_alu_cycles_active.avg.pct_of_peak_sustained_active"),
                        ("issue_active_pct", "smsp__issue_active.avg.pct_of_peak_sustained_active"),
                        ("warps_active_pct", "sm__warps_active.avg.pct_of_peak_sustained_active")):
        m = re.search(r"\| " + re.escape(metric) + r" \| ([0-9.]+)", text)
        out[key] = float(m.group(1)) if m else None
    return out


def scaled_traffic(prof, ntasks):
    """DRAM bytes per launch from a committed capture, scaled from the
    captured case's task count to this launch's (the kernels' traffic grows
    with the tasks they read), with its source; None without a capture on
    the current sources."""
    if not prof or prof.get("traffic") is None:
        return None
    cap = prof.get("captured_tasks")
    if not cap:
        return None
    return {"bytes": prof["traffic"] * ntasks / cap, "captured_bytes": prof["traffic"], "captured_tasks": cap,
            "launch_tasks": ntasks, "source": prof["source"],
            "note": "dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of a smaller case of the same "
                    "kernel, scaled by tasks"}


def e2e_bytes(calls, nsets, ntasks, kmax, multi):
    """Bytes one end-to-end step copies in and out.  In: the task columns
    (set_off as int64 per set and one more; T, D, A, B, u_ppm as int64 and
    type as a byte per task), once per call, or once for every policy of a
    multi-policy call.  Out, per call: an allocation's verdict and reason
    (bytes), n_parts, Pi and n_tests (int32) and W (int64) per set, and
    part_of_task (byte) and size_of_part (int16) per task; a search's
    feasible (byte), W (int64), sum_minm, n_blocks and spare (int32) per
    set, rgs (byte) per task and minm_block (int16) per set and block."""
    h2d = (8 * (nsets + 1) + 41 * ntasks) * (1 if multi else len(calls))
    d2h = sum((22 * nsets + 3 * ntasks) if c not in ("SEARCH", "EXPLICIT") else
              (21 * nsets + ntasks + 2 * kmax * nsets) for c in calls)
    return h2d, d2h


def gpu_id_for_smi(local):
    """nvidia-smi id of the CUDA device `local` (UUID when torch exposes it)."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(local).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            ids = [x.strip() for x in vis.split(",") if x.strip()]
            if local < len(ids):
                return ids[local]
        return str(local)


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self, wait_s=3.0):
        """Starts sampling and waits (up to wait_s) for the first sample."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
            return
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < wait_s and self.proc.poll() is None:
            time.sleep(0.02)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def head_sets(sets, n):
    """The first n sets of a host batch (a view sharing the columns)."""
    off = sets["set_off"][: n + 1]
    t = int(off[-1])
    out = {k: sets[k][:t] for k in ("T", "D", "A", "B", "u_ppm", "type")}
    out["set_off"] = off
    out["n_max"] = sets["n_max"]
    return out


def oracle_step(sets, md, workload, threads):
    """One pass of the oracle, as it stands, over `sets`: the calls of one
    step of the workload."""
    import oracle
    wp = W.WORKLOADS["exhaustive" if workload == "exhaustive" else "single" if workload == "single" else "batch"]
    for call in CALLS[workload]:
        if call == "SEARCH":
            oracle.search_best(sets, md["M"], md["g"], md["k_c_pm"], md["k_m_pm"], wp["kmin"], wp["kmax"],
                               nthreads=threads, sched=md.get("sched", "DM"), sizes=md.get("sizes"))
        elif call == "EXPLICIT":
            oracle.search_best(sets, md["M"], md["g"], md["k_c_pm"], md["k_m_pm"], wp["kmin"], wp["kmax"],
                               explicit=True, nthreads=threads, sched=md.get("sched", "DM"))
        else:
            oracle.allocate(sets, md["M"], md["g"], md["k_c_pm"], md["k_m_pm"], policy=call, act=False,
                            nthreads=threads, sched=md.get("sched", "DM"), sizes=md.get("sizes"))


def oracle_sample(sets, md, workload, threads, target_s):
    """A prefix of the batch that one oracle pass finishes in about target_s
    seconds: timed on a small prefix (grown until it takes 50 ms), then
    scaled linearly (the sets are independent).  For the 200-task workload
    the prefix is taken from its U = 2 sets only (every 34th set): one such
    set takes the oracle about a second, one at U = 34 minutes, so a plain
    prefix cannot be bounded."""
    if workload == "paper200":
        import paper_2105_10312_gb300.gen as G
        steps = W.WORKLOADS["paper200"]["gen"]["U_steps"]
        sets = G.subset(sets, np.arange(0, len(sets["set_off"]) - 1, steps))
    nsets = len(sets["set_off"]) - 1
    n = min(nsets, 1 if workload == "paper200" else 64)
    while True:
        t0 = time.perf_counter()
        oracle_step(head_sets(sets, n), md, workload, threads)
        el = time.perf_counter() - t0
        if el >= 0.05 or n == nsets:
            break
        n = min(nsets, n * 4)
    n = int(max(1, min(nsets, n * target_s / max(el, 1e-9))))
    return (sets if n == nsets else head_sets(sets, n)), n


def sample_words(workload, n, nsets):
    if workload == "paper200":
        return f"{n} of the batch's U = 2 sets (the oracle's time per 200-task set grows to minutes at high U)"
    return f"the {nsets}-set batch" if n == nsets else f"the first {n} of the {nsets} sets"


def cpu_baseline_oracle(sets, md, workload, target_wall=2.0, max_wall=20.0):
    """The CPU oracle as it stands, on the host cores, over repeated passes
    of the same workload (bounded: a prefix of the batch when a full pass
    would take more than a second)."""
    threads = os.cpu_count() or 1
    sub, n = oracle_sample(sets, md, workload, threads, 1.0)
    t0 = time.perf_counter()
    passes = 0
    while True:
        oracle_step(sub, md, workload, threads)
        passes += 1
        el = time.perf_counter() - t0
        if el >= target_wall or el >= max_wall:
            break
    nsets = len(sets["set_off"]) - 1
    # the same oracle on one thread, on a sample of about half a second
    sub1, n1 = oracle_sample(sets, md, workload, 1, 0.5)
    t1 = time.perf_counter()
    oracle_step(sub1, md, workload, 1)
    el1 = time.perf_counter() - t1
    return {"value": passes * n / el, "unit": "tasksets/s", "cores": threads, "kind": "oracle",
            "sample": f"{passes} pass(es) over {sample_words(workload, n, nsets)}, {threads} threads, "
                      f"{el:.2f} s wall",
            "single_thread": {"value": n1 / el1, "unit": "tasksets/s",
                              "sample": f"one pass over {n1} sets, 1 thread, {el1:.2f} s wall"}}


def serve_bench(local, rates=(2000, 5000, 10000, 20000, 50000), duration=0.5, plain=False, population=512,
                seed=5, warm_s=0.3):
    """Open-loop Poisson stream of admission queries (10 % ADMIT of a new
    tenant, 45 % ADD of one task, 45 % REMOVE) against a live population;
    latency = submit to completion.  plain=True: one request per launch, one
    stream (the per-request form).  An untimed warm-up stream of warm_s
    seconds at the lowest rate precedes the measured rates.  Completed
    requests per second = requests / (last completion - first submission),
    completion = submission + the request's own latency."""
    import ctypes

    import paper_2105_10312_gb300 as gpa
    rng = np.random.default_rng(seed)
    ctx = gpa.Context(local)
    srv = gpa.Server(ctx, M=148, max_batch=1 if plain else 512, nstreams=1 if plain else 4,
                     max_tenants=1 << 16, slots_per_chunk=1024)
    L = gpa.lib()
    nmax_new = 200000
    sets = gpa.gen_tasksets(**W.gen_params("serve", nsets=population + nmax_new // 10 + 10, seed=seed))
    pool = gpa.gen_tasksets(**W.gen_params("serve", nsets=nmax_new, seed=seed + 1, n_min=1, n_max=1,
                                           U_lo_ppm=20000, U_hi_ppm=1000000))
    keep = []

    def req_for(op, tenant, k=None, j=None, index=0):
        if op == "ADMIT":
            o, e = sets["set_off"][k], sets["set_off"][k + 1]
            cols = [np.ascontiguousarray(sets[c][o:e]) for c in ("T", "D", "A", "B", "u_ppm", "type")]
            n = e - o
        elif op == "ADD":
            cols = [np.ascontiguousarray(pool[c][j:j + 1]) for c in ("T", "D", "A", "B", "u_ppm", "type")]
            n = 1
        else:
            cols, n = [None] * 6, 0
        keep.append(cols)
        ptrs = [c.ctypes.data if c is not None else None for c in cols]
        return gpa.Request(gpa.SERVE_OP[op], int(n), int(tenant), int(index), 0, *ptrs)

    # population (not timed)
    ids = [srv.submit("ADMIT", t, tasks={c: sets[c][sets["set_off"][t]:sets["set_off"][t + 1]]
                                         for c in ("T", "D", "A", "B", "u_ppm", "type")}) for t in range(population)]
    live = [t for t, i in zip(range(population), ids) if srv.poll(i)["verdict"]]
    sizes = {t: int(sets["set_off"][t + 1] - sets["set_off"][t]) for t in live}
    state = {"tenant": population, "set": population, "task": 0}
    rid = ctypes.c_uint64()

    def stream_of(rate, seconds):
        nreq = max(1, int(rate * seconds))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, nreq))
        reqs = []
        for _ in range(nreq):
            x = rng.random()
            if x < 0.10 or not live:
                reqs.append(req_for("ADMIT", state["tenant"], k=state["set"]))
                live.append(state["tenant"])
                sizes[state["tenant"]] = int(sets["set_off"][state["set"] + 1] - sets["set_off"][state["set"]])
                state["tenant"] += 1
                state["set"] += 1
            else:
                t = live[int(rng.integers(len(live)))]
                if x < 0.55 and sizes[t] < 128:
                    reqs.append(req_for("ADD", t, j=state["task"]))
                    state["task"] += 1
                    sizes[t] += 1
                elif sizes[t] > 1:
                    reqs.append(req_for("REMOVE", t, index=0))
                    sizes[t] -= 1
                else:
                    reqs.append(req_for("ADD", t, j=state["task"]))
                    state["task"] += 1
                    sizes[t] += 1
        return arrivals, reqs

    def run(arrivals, reqs):
        sent, sub_t = [], []
        t0 = time.perf_counter()
        for k in range(len(reqs)):
            while time.perf_counter() - t0 < arrivals[k]:
                pass
            ts = time.perf_counter() - t0
            L.gpa_serve_submit(ctx.handle, ctypes.byref(reqs[k]), ctypes.byref(rid))
            sent.append(rid.value)
            sub_t.append(ts)
        t_sub = time.perf_counter() - t0
        lat, errors, notfound = [], 0, 0
        for i in sent:
            r = srv.poll(i)
            lat.append(r["latency_us"])
            # the stream is generated up front, so it also sends ADD / REMOVE
            # to tenants whose ADMIT was rejected: those answer NOTFOUND
            notfound += r["status"] == gpa.ERR_NOTFOUND
            errors += r["status"] not in (0, gpa.ERR_NOTFOUND)
        lat = np.array(lat, dtype=np.float64)
        done = np.array(sub_t) + lat * 1e-6
        span = float(done.max() - sub_t[0]) if len(sent) else 0.0
        return {"p50_ms": float(np.percentile(lat, 50)) / 1000, "p99_ms": float(np.percentile(lat, 99)) / 1000,
                "offered_req_s": len(reqs) / max(t_sub, 1e-9), "completed_req_s": len(reqs) / max(span, 1e-9),
                "requests": len(reqs), "errors": int(errors), "to_rejected_tenants": int(notfound)}

    run(*stream_of(rates[0], warm_s))  # warm-up: kernels loaded, slots and streams in use
    out = {str(rate): run(*stream_of(rate, duration)) for rate in rates}
    st = srv.stats()
    srv.stop()
    ctx.close()
    return {"rates": out, "batches": st["batches"], "max_batch": st["max_batch"], "overlapped_batches": st["overlapped"],
            "form": "one request per launch, 1 stream" if plain else "continuous batching, up to 512 per batch, 4 streams"}


def build_workload(name, rank, nsets_override=None):
    import paper_2105_10312_gb300 as gpa
    base = "sweep" if name == "sweep1g" else name
    p = W.gen_params(base)
    p["seed"] = shard.rank_seed(p["seed"], rank)
    if nsets_override:
        p["nsets"] = nsets_override
    s = gpa.gen_tasksets(**p)
    return s, W.model(base)


def run_reference(args):
    rank, world, _ = shard.dist_env()
    if rank != 0:
        return 0
    sets, md = build_workload(args.workload, 0, args.nsets)
    md["sched"] = args.sched.upper()
    if args.sizes:
        md["sizes"] = [int(x) for x in args.sizes.split(",")]
    threads = os.cpu_count() or 1
    nsets_all = len(sets["set_off"]) - 1
    # each step: one pass over a prefix of the workload sized so that the
    # K steps take about a minute at most
    sub, nsets = oracle_sample(sets, md, args.workload, threads, max(0.005, 60.0 / max(args.steps, 1)))
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_step(sub, md, args.workload, threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(sub, md, args.workload, threads)
    el = time.perf_counter() - t0
    v = args.steps * nsets / el
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "tasksets/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": DESCR.get(args.workload, args.workload), "nsets": nsets, "M": md["M"],
                   "calls": list(CALLS[args.workload]), "sched": md["sched"]},
        "cpu_baseline": {"value": v, "unit": "tasksets/s", "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} pass(es) over " + sample_words(args.workload, nsets, nsets_all)},
        "e2e": {"value": v, "unit": "tasksets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


class Bench:
    """The device, stream, flush buffers and measured peaks shared by the records."""

    def __init__(self, args, local):
        import torch

        import paper_2105_10312_gb300 as gpa
        self.args = args
        self.local = local
        self.dev = torch.device("cuda", local)
        self.stream = torch.cuda.Stream(self.dev)
        self.flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=self.dev)
        self.flush_rd = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.int32, device=self.dev)
        self.hbm_peak, self.hbm_src = read_peaks()
        c = gpa.Context(local, stream=self.stream)
        with torch.cuda.stream(self.stream):
            for i in range(3):
                self.flush_l2(i)  # the flush's own kernels load lazily on first use
            self.alu = c.measure_alu_peak()
        c.close()

    def flush_l2(self, i):
        self.flush.fill_(i)
        return self.flush_rd.sum()

    def read_floor(self, nbytes, kernel_ms, reps=20):
        """The same-size reference for the roofline: one streaming read of
        the kernel's read bytes (torch's int64 sum over a buffer of that
        size, L2 flushed first, CUDA events on the same stream).  The peak
        above is a large copy; a ~100 MB launch also pays the launch, the
        ramp to full DRAM throughput and the tail."""
        import torch
        buf = torch.ones(max(1, nbytes // 8), dtype=torch.int64, device=self.dev)
        ts = []
        with torch.cuda.stream(self.stream):
            for i in range(reps + 3):
                self.flush_l2(i)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(self.stream)
                buf.sum()
                e1.record(self.stream)
                e1.synchronize()
                if i >= 3:
                    ts.append(e0.elapsed_time(e1))
        f = float(np.median(ts))
        del buf
        return {"what": "torch int64 sum over a buffer of the kernel's read bytes (one streaming read), "
                        "L2 flushed first, CUDA events on the same stream; median of %d" % reps,
                "bytes": nbytes, "ms": f, "gbs": nbytes / (f / 1000.0) / 1e9, "kernel_ms_over_floor_ms": kernel_ms / f}


def measure(bench, name, rank, world, steps, warmup, with_cpu=True, e2e_steps=5, plain_sample=0):
    """One workload's record: step time over K flushed steps, per-kernel
    times and rooflines, candidates, terms, the end-to-end figure on host
    buffers and the CPU oracle baseline."""
    import torch

    import paper_2105_10312_gb300 as gpa
    args = bench.args
    dev, stream = bench.dev, bench.stream
    sets, md = build_workload(name, rank, args.nsets if name == args.workload else None)
    md["sched"] = args.sched.upper()
    if args.sizes and name == args.workload:
        md["sizes"] = [int(x) for x in args.sizes.split(",")]
    nsets = len(sets["set_off"]) - 1
    ntasks = int(sets["set_off"][-1])
    calls = CALLS[name]
    d = gpa.to_device(sets, dev)
    torch.cuda.synchronize(dev)
    ctx = gpa.Context(bench.local, stream=stream)
    autotune = not args.no_autotune
    ctx.set_option("AUTOTUNE", 1 if autotune else 0)
    ctx.set_option("GRAPH", 1)
    wp = W.WORKLOADS.get(name, W.WORKLOADS["batch"])
    outs = []
    for call in calls:
        outs.append(ctx.best_result(d, wp["kmax"]) if call in ("SEARCH", "EXPLICIT") else ctx.alloc_result(d))

    def n_undecided(os_):
        """Sets the outputs mark undecided (a per-partition test hit its step
        limit: reason UNDECIDED, or feasible == 2 for the searches)."""
        n = 0
        for o in os_:
            if "reason" in o:
                n += int((o["reason"] == gpa.REASON["UNDECIDED"]).sum())
            else:
                n += int((o["feasible"] == 2).sum())
        return n

    undecided = [0]

    def tolerant(fn, os_):
        """fn(), with undecided sets counted rather than fatal: the library
        reports them as GPA_ERR_TIMEOUT, which also covers a pipeline wait
        that gave up, so the outputs must show them."""
        try:
            fn()
        except gpa.GpaError as e:
            k = n_undecided(os_) if e.code == gpa.ERR_TIMEOUT else 0
            if k == 0:
                raise
            undecided[0] = max(undecided[0], k)

    def do_call(i, call, target=None, o=None):
        target = d if target is None else target
        o = outs[i] if o is None else o
        if call == "SEARCH":
            ctx.search_best(target, **md, kmin=wp["kmin"], kmax=wp["kmax"], out=o)
        elif call == "EXPLICIT":
            ctx.search_explicit(target, **md, kmin=wp["kmin"], kmax=wp["kmax"], out=o)
        else:
            ctx.allocate(target, **md, policy=call, act=False, linear=args.merge == "linear", out=o)

    def step():
        for i, call in enumerate(calls):
            do_call(i, call)

    with torch.cuda.stream(stream):
        for i in range(max(warmup, 0)):
            bench.flush_l2(i)
            step()
        torch.cuda.synchronize(dev)
        tolerant(ctx.sync, outs)
        shard.barrier()
        torch.cuda.synchronize(dev)
        sampler = ClockSampler(gpu_id_for_smi(bench.local))
        sampler.start()
        # K steps, each after an L2 flush, queued back to back (so a stall
        # of this host thread cannot leave the GPU idle inside a step),
        # timed by CUDA events on the context stream
        launches0 = ctx.launch_count()
        events = []
        t_wall0 = time.perf_counter()
        for i in range(steps):
            bench.flush_l2(i)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            events.append((e0, e1))
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t_wall0
        launches = ctx.launch_count() - launches0
        step_ms = [a.elapsed_time(b) for a, b in events]
        # a second pass of the same K steps with the library's in-graph
        # kernel events (they add graph nodes, so they stay out of the step
        # time); each call's kernel times are read after it
        ctx.set_option("PROFILE", 1)
        for i, call in enumerate(calls):
            do_call(i, call)  # the profiled graphs are captured outside the timed steps
        torch.cuda.synchronize(dev)
        kern = [[] for _ in calls]
        for i in range(steps):
            bench.flush_l2(i)
            for j, call in enumerate(calls):
                do_call(j, call)
                kern[j].append(ctx.last_timing())
        ctx.set_option("PROFILE", 0)
        clocks = sampler.stop()
        # interference terms of each call (the counter holds the last call's)
        terms = []
        for j, call in enumerate(calls):
            do_call(j, call)
            terms.append(ctx.last_terms())
        tolerant(ctx.sync, outs)
    shard.barrier()

    mean_ms = float(np.mean(step_ms))
    max_ms = shard.max_over_ranks(mean_ms)
    total_sets = shard.sum_over_ranks(nsets)
    value = total_sets / (max_ms / 1000.0)

    # candidate allocations tested per step
    cand = 0.0
    cand_parts = {}
    for j, call in enumerate(calls):
        if call == "ONE_GPU":
            c = float(nsets)
        elif call == "SEARCH":
            c = float((4095 + 700075) * nsets)  # subset size searches + RGS keys per 12-task set
        elif call == "EXPLICIT":
            c = float(ctx.explicit_count(d, md["M"], md["g"], wp["kmin"], wp["kmax"]) * nsets)
        else:
            c = float(outs[j]["n_tests"].sum().item())
        cand_parts[call] = c
        cand += c
    cand_total = shard.sum_over_ranks(cand)

    # per-kernel times and rooflines
    names = {"SMS": ("alloc_fast", "alloc_merge"), "ONE_GPU": ("one_gpu_fast", "one_gpu"), "SEARCH": ("search_sets",),
             "EXPLICIT": ("search_explicit",)}
    kernels = []
    for j, call in enumerate(calls):
        ks = names[call]
        for q, kname in enumerate(ks):
            ts = [t[q] for t in kern[j] if len(t) > q]
            if not ts:
                continue
            kms = float(np.mean(ts))
            rec = {"kernel": kname, "kernel_ms": kms}
            if kname in ("alloc_fast", "one_gpu_fast"):
                # both stream every set once (the heuristic's Lemma 2 pass, the 1G pre-pass)
                # per task: T, D, A, B, u (5 x 8 B) + type (1 B) read; part (1 B) + size (2 B) written;
                # per set: offset (8 B) read; verdict, reason, n_parts, Pi, W, n_tests (22 B) written
                alg = 44 * ntasks + 30 * nsets
                ach = alg / (kms / 1000.0) / 1e9
                prof = recorded_profile(kname, name)
                tr = scaled_traffic(prof, ntasks)
                rec.update({"bound": "hbm", "achieved": ach, "peak": bench.hbm_peak, "unit": "GB/s",
                            "frac": ach / bench.hbm_peak, "traffic": tr["bytes"] if tr else None, "traffic_detail": tr,
                            "algorithmic_bytes": alg, "peak_source": bench.hbm_src + " hbm_gbs (MEASURED_PEAKS.json)",
                            "ncu": prof})
            else:
                t = terms[j]
                ach = t / (kms / 1000.0)
                prof = recorded_profile(kname, name)
                tr = scaled_traffic(prof, ntasks)
                rec.update({"bound": "alu", "achieved": ach, "peak": bench.alu["terms_per_s"],
                            "unit": "interference terms/s", "frac": ach / bench.alu["terms_per_s"],
                            "traffic": tr["bytes"] if tr else None, "traffic_detail": tr, "terms_per_launch": t,
                            "peak_source": "measured in this run by gpa_measure_alu_peak (the term's arithmetic, "
                                           "4 independent iterations per thread, every SM and warp slot)",
                            "ncu": prof})
            kernels.append(rec)
    dom = max(kernels, key=lambda r: r["kernel_ms"]) if kernels else None
    roof = dict(dom) if dom else None
    if roof:
        roof["kernel_timing"] = ("CUDA events recorded by the library around each kernel (inside its graphs), "
                                 "a second pass of the same K flushed steps")
        if roof["kernel"] in ("alloc_fast", "one_gpu_fast"):
            roof["size_floor"] = bench.read_floor(44 * ntasks + 8 * nsets, roof["kernel_ms"])

    # outcome summaries the configurations ask for (untimed)
    outcome = None
    if name == "exhaustive":
        with torch.cuda.stream(stream):
            h = ctx.allocate(d, **md, policy="SMS", act=False)
            tolerant(ctx.sync, [h])
        fo = outs[0]["feasible"].cpu().numpy() == 1
        fh = h["verdict"].cpu().numpy().astype(bool)
        wo, wh = outs[0]["W"].cpu().numpy(), h["W"].cpu().numpy()
        nph = h["n_parts"].cpu().numpy()
        comp = fo & fh & (nph >= wp["kmin"]) & (nph <= wp["kmax"])
        outcome = {"optimum_feasible": float(fo.mean()), "heuristic_feasible": float(fh.mean()),
                   "heuristic_partitions_mean": float(nph[fh].mean()) if fh.any() else None,
                   "heuristic_within_kmax": float(comp.sum() / max(1, (fo & fh).sum())),
                   "mean_W_heuristic_over_optimum_within_kmax":
                       float((wh[comp] / np.maximum(wo[comp], 1)).mean()) if comp.any() else None,
                   "optimum_partitions": f"{wp['kmin']}..{wp['kmax']}",
                   "note": "the heuristic stops as soon as its partitions fit (Pi <= M, Lemma 3), so it keeps up to "
                           "one partition per task; W is compared only where it ended within kmax partitions"}
    elif name in ("sweep", "sweep1g"):
        steps_u = W.WORKLOADS["sweep"]["gen"]["U_steps"]
        st = np.arange(nsets) % steps_u
        outcome = {"U": [round(0.1 * (j + 1), 1) for j in range(steps_u)]}
        for j, call in enumerate(calls):
            v = outs[j]["verdict"].cpu().numpy()
            outcome["heuristic" if call == "SMS" else "1G"] = [round(float(v[st == u].mean()), 4)
                                                               for u in range(steps_u)]
    elif name == "single":
        o = outs[0]
        outcome = {"feasible": int(o["feasible"][0].item()), "W": int(o["W"][0].item()),
                   "sum_minm": int(o["sum_minm"][0].item()), "n_blocks": int(o["n_blocks"][0].item())}

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    e2e = None
    if e2e_steps > 0:
        hs = {}
        for k in ("set_off", "T", "D", "A", "B", "u_ppm", "type"):
            hs[k] = torch.from_numpy(np.ascontiguousarray(sets[k])).pin_memory().numpy()
        hs["n_max"] = sets["n_max"]
        houts = []
        for call in calls:
            o = ctx.best_result(hs, wp["kmax"]) if call in ("SEARCH", "EXPLICIT") else ctx.alloc_result(hs)
            houts.append({k: (torch.from_numpy(v).pin_memory().numpy() if v is not None else None)
                          for k, v in o.items()})
        ctx_h = gpa.Context(bench.local, stream=stream)
        ctx_h.set_option("GRAPH", 1)
        ctx_h.set_option("HOST_SLICES", args.host_slices)
        ctx_h.set_option("AUTOTUNE", 1 if autotune else 0)
        saved = ctx
        ctx = ctx_h
        # several allocation policies over one batch: one gpa_allocate_multi
        # call, which copies the batch in once for all of them
        multi = len(calls) > 1 and all(c not in ("SEARCH", "EXPLICIT") for c in calls)

        def e2e_step():  # synchronous: H2D, kernels, D2H
            if multi:
                tolerant(lambda: ctx.allocate_multi(hs, **md, policies=list(calls), act=False,
                                                    linear=args.merge == "linear", outs=houts), houts)
            else:
                for j, call in enumerate(calls):
                    tolerant(lambda: do_call(j, call, hs, houts[j]), [houts[j]])

        with torch.cuda.stream(stream):
            for _ in range(2):  # warm-up: the autotuner and the graphs of every host slice
                e2e_step()
            times = []
            for i in range(e2e_steps):
                bench.flush_l2(i)
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                e2e_step()
                times.append(time.perf_counter() - t0)
        ctx = saved
        ctx_h.close()
        e2e_t = shard.max_over_ranks(float(np.mean(times)))
        h2d, d2h = e2e_bytes(calls, nsets, ntasks, wp.get("kmax", 0), multi)  # kmax: searches only
        ms = sorted(1000.0 * t for t in times)
        e2e = {"value": total_sets / e2e_t, "unit": "tasksets/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1000.0 * e2e_t,
               "step_ms": {"steps": len(ms), "min": ms[0], "median": float(np.median(ms)), "max": ms[-1],
                           "each": [round(1000.0 * t, 3) for t in times]},
               "path": (f"one gpa_allocate_multi call per step ({' + '.join(calls)}) on pinned host buffers, "
                        "synchronous (inputs copied in once for every policy, kernels, results copied out)"
                        if multi else
                        f"{len(calls)} C-ABI call(s) per step on pinned host buffers, each synchronous "
                        "(inputs copied in, kernels, results copied out)")}

    # the plain form: one launch sequence per task set, on a sample
    plain = None
    if plain_sample > 0 and calls == ("SMS",):
        import paper_2105_10312_gb300.gen as G
        sub = G.subset(sets, np.arange(min(plain_sample, nsets)))
        ds = gpa.to_device(sub, dev)
        c2 = gpa.Context(bench.local, stream=stream)
        c2.set_option("PER_SET_LAUNCH", 1)
        with torch.cuda.stream(stream):
            o2 = c2.alloc_result(ds)
            c2.allocate(ds, **md, policy="SMS", act=False, out=o2)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c2.allocate(ds, **md, policy="SMS", act=False, out=o2)
            e1.record(stream)
            e1.synchronize()
        c2.close()
        nsub = len(sub["set_off"]) - 1
        plain = {"tasksets_per_s": nsub / (e0.elapsed_time(e1) / 1000.0), "sample_sets": nsub,
                 "launches_per_set": 2}

    cpu = None
    if with_cpu and rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_oracle(sets, md, name)
    ctx.close()
    return {
        "metric": METRIC, "value": value, "unit": "tasksets/s", "ms_per_step": max_ms, "steps": steps,
        "warmup": warmup,
        "config": {"workload": DESCR.get(name, name), "nsets_per_gpu": nsets, "tasks_per_gpu": ntasks,
                   "M": md["M"], "g": md["g"], "calls": list(calls), "sched": md["sched"],
                   "merge_search": args.merge, "sizes": md.get("sizes"),
                   "l2": "flushed before every timed step (512 MB write, then 256 MB read); inputs %.0f MB"
                         % ((41 * ntasks + 8 * nsets) / 1e6),
                   "parallelism": f"{world} independent shard(s)",
                   "launch": "persistent kernels, CUDA graph per call" if calls[0] not in ("SEARCH", "EXPLICIT")
                   else "one persistent launch per call",
                   "launch_shape": "autotuned by the library on the first call" if autotune else "library default"},
        "candidates_tested_per_s": cand_total / (max_ms / 1000.0),
        "candidates_per_step": cand_parts,
        "roofline": roof, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clocks, "per_set_launch": plain, "wall_s_timed": wall, "outcome": outcome,
        "undecided_sets_per_step": undecided[0],
    }


def run_gpu(args):
    import torch

    rank, world, local = shard.dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(torch.device("cuda", local))
    bench = Bench(args, local)
    head = measure(bench, args.workload, rank, world, args.steps or DEFAULT_STEPS[args.workload], args.warmup,
                   e2e_steps=args.e2e_steps,
                   plain_sample=args.plain_sample)
    configs = None
    if not args.no_configs and args.workload == "sweep":
        configs = {}
        for name in SUBRECORDS:
            configs[name] = measure(bench, name, rank, world, DEFAULT_STEPS[name], args.warmup,
                                    e2e_steps=args.e2e_steps, plain_sample=args.plain_sample if name == "batch" else 0)
        if args.serve_duration > 0 and rank == 0:
            cont = serve_bench(local, duration=args.serve_duration)
            per = serve_bench(local, duration=args.serve_duration, plain=True)
            configs["serve"] = {
                "metric": "serve p50/p99 ms", "continuous": cont, "per_request": per,
                "config": {"workload": "serving: Poisson admission queries at 2k-50k req/s (10 % ADMIT of a "
                                       "4..128-task set, 45 % ADD, 45 % REMOVE of one task) against 512+ resident "
                                       "tenants on 148 SMs"},
                "continuous_p99_le_per_request_p99": {
                    r: cont["rates"][r]["p99_ms"] <= per["rates"][r]["p99_ms"] for r in cont["rates"]}}
    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": "tasksets/s", "n_gpus": world,
            "steps": head["steps"], "warmup": head["warmup"], "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded generator; the paper's evaluation is synthetic too)",
            "config": head["config"],
            "candidates_tested_per_s": head["candidates_tested_per_s"],
            "candidates_per_step": head["candidates_per_step"],
            "roofline": head["roofline"], "kernels": head["kernels"], "cpu_baseline": head["cpu_baseline"],
            "e2e": head["e2e"], "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
            "alu_peak": bench.alu, "wall_s_timed": head["wall_s_timed"], "outcome": head["outcome"],
            "per_set_launch": head["per_set_launch"], "undecided_sets_per_step": head["undecided_sets_per_step"],
            "configs": configs,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps of the headline workload (default: sweep 50, batch 1000, paper50 100, "
                         "exhaustive 10, single 500, paper200 3); the other records use their defaults")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gpa", "reference"], default="gpa")
    ap.add_argument("--workload", choices=sorted(DESCR), default="sweep")
    ap.add_argument("--no-configs", action="store_true", help="only the headline workload (no per-config records)")
    ap.add_argument("--nsets", type=int, default=0, help="override the headline workload's set count (profiling)")
    ap.add_argument("--sizes", default="",
                    help="comma-separated admissible partition sizes (default: every multiple of g)")
    ap.add_argument("--merge", choices=["linear", "binary"], default="linear",
                    help="Alg. 2 size search of a merge: upwards from the smallest size (default) or the binary "
                         "search of §5.2")
    ap.add_argument("--sched", choices=["dm", "edf"], default="dm",
                    help="per-partition policy: deadline-monotonic response-time test (default) or EDF demand test")
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--host-slices", type=int, default=0,
                    help="host-buffer path: 0 = library default (split batches over 48 MB), 1 = whole batch checked "
                         "before computing, n = n slices")
    ap.add_argument("--plain-sample", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default launch shapes")
    ap.add_argument("--serve-duration", type=float, default=0.5,
                    help="seconds of Poisson arrivals per offered rate in the serving measurement (0: skip)")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.steps is None:
            args.steps = 10
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
