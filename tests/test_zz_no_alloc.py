"""gpa_allocate_noalloc against gpa_allocate (GPU; collected last on purpose).

gpa_allocate_noalloc serves callers that may not allocate device memory (an
application that owns the allocator, a fixed memory budget, a real-time
process that must not allocate after start-up): it takes no context and keeps
its scratch in a static device array.  Its results must equal the regular
entry point's, bit for bit (the computation is integer), on two calls in a
row -- the second call reuses the scratch the first one left behind.  This
file runs last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

import paper_2105_10312_gb300 as gpa
from paper_2105_10312_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("verdict", "reason", "n_parts", "Pi", "W", "n_tests", "part_of_task", "size_of_part")


def _batches():
    merge_heavy = gpa.gen_tasksets(**W.gen_params("paper50", nsets=136))  # many sets go through the merge queue
    batch = gpa.gen_tasksets(**W.gen_params("batch", nsets=5000))          # mostly decided by the fast kernel
    return [("paper50", merge_heavy, W.model("paper50")), ("batch", batch, W.model("batch"))]


@pytest.mark.parametrize("policy,act", [("SMS", False), ("BF", True)])
def test_noalloc_matches_allocate_on_two_calls(policy, act):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = gpa.Context(0)
    try:
        for name, s, md in _batches():
            d = gpa.to_device(s)
            ref = ctx.allocate(d, **md, policy=policy, act=act)
            ctx.sync()
            for call in range(2):
                out = ctx.alloc_result(d)
                for v in out.values():
                    if v is not None:
                        v.fill_(7)  # stale values must be overwritten
                gpa.allocate_noalloc(d, out, **md, policy=policy, act=act)
                torch.cuda.synchronize()
                for k in KEYS:
                    assert torch.equal(out[k], ref[k]), f"{name} call {call}: {k} differs"
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
