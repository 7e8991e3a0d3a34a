"""gpa_allocate_noalloc against the oracle and gpa_allocate (GPU; collected last on purpose).

gpa_allocate_noalloc serves callers that may not allocate device memory (an
application that owns the allocator, a fixed memory budget, a real-time
process that must not allocate after start-up): it takes no context and keeps
its scratch in a static device array.  Its results must equal the oracle's
and the regular entry point's, bit for bit (the computation is integer), on
two calls in a row -- the second call reuses the scratch the first one left
behind -- under both per-partition policies, and the problems its kernels
find must reach the caller through gpa_allocate_noalloc_status.  This file
runs last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2105_10312_gb300 as gpa
from paper_2105_10312_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("verdict", "reason", "n_parts", "Pi", "W", "n_tests", "part_of_task", "size_of_part")


def _batches():
    merge_heavy = gpa.gen_tasksets(**W.gen_params("paper50", nsets=136))  # many sets go through the merge queue
    batch = gpa.gen_tasksets(**W.gen_params("batch", nsets=5000))          # mostly decided by the fast kernel
    return [("paper50", merge_heavy, W.model("paper50")), ("batch", batch, W.model("batch"))]


@pytest.mark.parametrize("policy,act,sched", [("SMS", False, "DM"), ("BF", True, "DM"), ("SMS", False, "EDF"),
                                              ("BF", True, "EDF")])
def test_noalloc_matches_oracle_and_allocate_on_two_calls(policy, act, sched):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = gpa.Context(0)
    try:
        gpa.allocate_noalloc_status()  # whatever an earlier test left recorded
        for name, s, md in _batches():
            d = gpa.to_device(s)
            want = oracle.allocate(s, md["M"], md["g"], md["k_c_pm"], md["k_m_pm"], policy=policy, act=act,
                                   nthreads=8, sched=sched)
            ref = ctx.allocate(d, **md, policy=policy, act=act, sched=sched)
            ctx.sync()
            for call in range(2):
                out = ctx.alloc_result(d)
                for v in out.values():
                    if v is not None:
                        v.fill_(7)  # stale values must be overwritten
                gpa.allocate_noalloc(d, out, **md, policy=policy, act=act, sched=sched)
                gpa.allocate_noalloc_status()  # nothing went wrong on the device
                for k in KEYS:
                    got = out[k].cpu().numpy()
                    assert np.array_equal(got, want[k]), f"{name} {sched} call {call}: {k} differs from the oracle"
                    assert torch.equal(out[k], ref[k]), f"{name} {sched} call {call}: {k} differs from gpa_allocate"
    finally:
        ctx.close()


def test_noalloc_reports_an_undecided_set():
    """Two tasks on one SM (M = 1), so the merge loop tests them together: the
    higher-priority task (T = D = C = 1) makes the other's iteration (C = 1,
    D = T = 2^21) climb by one per step, so it passes D only after about 2^21
    steps, beyond the 2^20 limit (the oracle's unbounded iteration finds the
    merge fails, so the set fails).  The GPU marks the set undecided, never
    failed, and the status call reports GPA_ERR_TIMEOUT, then, cleared,
    GPA_OK; the set before it is decided normally on both calls."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tasks = [[(1000, 1000, 10), (1000, 1000, 10)], [(1, 1, 1), (1 << 21, 1 << 21, 1)]]
    off, cols = [0], {k: [] for k in ("T", "D", "A", "B", "u_ppm", "type")}
    for ts in tasks:
        for j, (T, D, C) in enumerate(ts):
            for k, v in (("T", T), ("D", D), ("A", 1000 * C), ("B", 0), ("u_ppm", 10**6 * C // T), ("type", j % 2)):
                cols[k].append(v)
        off.append(off[-1] + len(ts))
    s = {k: np.array(v, np.uint8 if k == "type" else np.int64) for k, v in cols.items()}
    s["set_off"] = np.array(off, np.int64)
    s["n_max"] = 2
    d = gpa.to_device(s)
    want = oracle.allocate(s, 1, 1, 1000, 1000)
    assert list(want["verdict"]) == [1, 0] and want["n_parts"][0] == 1
    ctx = gpa.Context(0)
    try:
        for call in range(2):
            out = ctx.alloc_result(d)
            gpa.allocate_noalloc(d, out, M=1, k_c_pm=1000, k_m_pm=1000)
            with pytest.raises(gpa.GpaError) as ei:
                gpa.allocate_noalloc_status()
            assert ei.value.code == gpa.ERR_TIMEOUT
            gpa.allocate_noalloc_status()  # cleared
            v, r = out["verdict"].cpu().numpy(), out["reason"].cpu().numpy()
            assert v[0] == 1 and r[0] == 0 and out["n_parts"][0].item() == 1
            assert v[1] == 0 and r[1] == gpa.REASON["UNDECIDED"], (call, v, r)
    finally:
        ctx.close()


def test_noalloc_rejects_oversized_batches():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = gpa.NOALLOC_MAX_SETS + 1
    s = {"set_off": torch.zeros(n + 1, dtype=torch.int64, device="cuda"),
         "T": torch.zeros(0, dtype=torch.int64, device="cuda"), "D": torch.zeros(0, dtype=torch.int64, device="cuda"),
         "A": torch.zeros(0, dtype=torch.int64, device="cuda"), "B": torch.zeros(0, dtype=torch.int64, device="cuda"),
         "u_ppm": torch.zeros(0, dtype=torch.int64, device="cuda"),
         "type": torch.zeros(0, dtype=torch.uint8, device="cuda")}
    out = {"verdict": torch.zeros(n, dtype=torch.uint8, device="cuda"),
           "reason": torch.zeros(n, dtype=torch.uint8, device="cuda"),
           "n_parts": torch.zeros(n, dtype=torch.int32, device="cuda"),
           "Pi": torch.zeros(n, dtype=torch.int32, device="cuda"), "W": torch.zeros(n, dtype=torch.int64, device="cuda"),
           "n_tests": None, "part_of_task": torch.zeros(0, dtype=torch.uint8, device="cuda"),
           "size_of_part": torch.zeros(0, dtype=torch.int16, device="cuda")}
    with pytest.raises(gpa.GpaError) as ei:
        gpa.allocate_noalloc(s, out, M=80)
    assert ei.value.code == gpa.ERR_RANGE
