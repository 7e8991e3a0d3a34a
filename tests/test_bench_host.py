"""The bench's output contract on the host (no GPU): the reference arm (the
CPU oracle) prints one JSON line with the required keys, and under a
multi-rank launch only rank 0 prints."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def _run(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    p = subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, env=e, capture_output=True, text=True,
                       timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    return [ln for ln in p.stdout.splitlines() if ln.strip()]


@pytest.mark.parametrize("workload", ["batch", "exhaustive"])
def test_reference_arm_prints_one_contract_line(workload):
    lines = _run(["--impl", "reference", "--workload", workload, "--nsets", "400", "--steps", "2", "--warmup", "1"])
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in KEYS:
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "tasksets/s"
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_print_nothing():
    lines = _run(["--impl", "reference", "--nsets", "200", "--steps", "1", "--warmup", "1", "--gpus", "2"],
                 env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert lines == []


@pytest.mark.parametrize("calls,multi", [(("SMS", "ONE_GPU"), True), (("SMS", "ONE_GPU"), False), (("SMS",), False),
                                         (("SEARCH",), False), (("EXPLICIT",), False)])
def test_e2e_byte_counts_are_the_copied_arrays(calls, multi):
    """The end-to-end line's bytes per step equal the sizes of the arrays the
    calls copy: the input columns (once for a multi-policy call) and every
    call's result arrays, as the binding allocates them."""
    sys.path.insert(0, ROOT)
    import bench
    import paper_2105_10312_gb300 as gpa
    s = gpa.gen_tasksets(seed=5, nsets=300, n_min=0, n_max=12, U_lo_ppm=100000, U_hi_ppm=2000000, deadline_pm=750)
    nsets, ntasks, kmax = 300, int(s["set_off"][-1]), 4
    cols = sum(s[k].nbytes for k in ("set_off", "T", "D", "A", "B", "u_ppm", "type"))
    outs = 0
    for c in calls:
        o = gpa.Context.best_result(None, s, kmax) if c in ("SEARCH", "EXPLICIT") else gpa.Context.alloc_result(None, s)
        outs += sum(v.nbytes for v in o.values() if v is not None)
    assert bench.e2e_bytes(calls, nsets, ntasks, kmax, multi) == (cols * (1 if multi else len(calls)), outs)


def test_every_workload_with_a_search_call_has_its_block_limit():
    """Each bench workload whose step makes a search call names kmax (the
    end-to-end byte count and the search calls read it); the others need none."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2105_10312_gb300 import workloads as W
    for name, calls in bench.CALLS.items():
        wp = W.WORKLOADS.get(name, W.WORKLOADS["batch"])
        if any(c in ("SEARCH", "EXPLICIT") for c in calls):
            assert "kmax" in wp and "kmin" in wp, name
