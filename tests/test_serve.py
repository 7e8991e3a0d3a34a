"""The serving loop on the GPU: every response equals the CPU replay of its
tenant's request sequence, whether the tenant's requests run alone or mixed
with many other tenants' requests in shared micro-batches."""
import numpy as np
import pytest
import torch

import oracle
import paper_2105_10312_gb300 as gpa
import serve_seq
from paper_2105_10312_gb300 import workloads as W

pytestmark = pytest.mark.gpu
KC, KM = W.K_C, W.K_M
M = 148


def _replay(seq, sched="DM", sizes=None):
    """Oracle responses for one tenant's sequence, and the concrete ops."""
    t = oracle.Tenant(M, 1, KC, KM, sched=sched, sizes=sizes)
    out, concrete = [], []
    alive = False
    for op, arg in seq:
        if op == "ADMIT":
            r = t.admit(arg)
            alive = bool(r["verdict"])
            concrete.append(("ADMIT", arg, 0))
            out.append(r)
        elif not alive:
            break
        elif op == "ADD":
            if t.n >= 128:
                continue
            concrete.append(("ADD", arg, 0))
            out.append(t.add(arg))
        elif op == "REMOVE":
            if t.n == 0:
                continue
            idx = int(arg * t.n)
            concrete.append(("REMOVE", None, idx))
            out.append(t.remove(idx))
        elif op == "EVICT":
            concrete.append(("EVICT", None, 0))
            out.append({"verdict": 1, "n_tasks": 0, "n_parts": 0, "Pi": 0, "W": 0,
                        "part_of_task": np.zeros(0, np.uint8), "size_of_part": np.zeros(0, np.int16)})
            alive = False
    return concrete, out


def _task_cols(task):
    return {k: np.asarray([task[k]]) for k in serve_seq.COLS}


def _same(r, e, what):
    for k in ("verdict", "n_tasks", "n_parts", "Pi", "W"):
        assert r[k] == e[k], (what, k, r[k], e[k])
    assert np.array_equal(r["part_of_task"], e["part_of_task"]), what
    assert np.array_equal(r["size_of_part"], e["size_of_part"]), what
    if "path" in e:
        assert r["path"] == e["path"], (what, "path")


def _submit(srv, tenant, op, arg, idx):
    if op == "ADMIT":
        return srv.submit("ADMIT", tenant, tasks=arg)
    if op == "ADD":
        return srv.submit("ADD", tenant, tasks=_task_cols(arg))
    if op == "REMOVE":
        return srv.submit("REMOVE", tenant, index=idx)
    return srv.submit("EVICT", tenant)


@pytest.fixture(scope="module")
def workload():
    ops = serve_seq.make_ops(48, 30, seed=11, evict=True)
    return [_replay(seq) for seq in ops]


def test_serve_alone_matches_oracle(workload):
    ctx = gpa.Context(0)
    srv = gpa.Server(ctx, M=M, max_batch=64, nstreams=2)
    try:
        for k, (concrete, expect) in enumerate(workload[:8]):
            for (op, arg, idx), e in zip(concrete, expect):
                r = srv.poll(_submit(srv, k, op, arg, idx))
                assert r["status"] == 0
                _same(r, e, f"alone tenant {k} {op}")
    finally:
        srv.stop()
        ctx.close()


def test_serve_mix_matches_alone_and_oracle(workload):
    """All tenants' requests submitted at once: micro-batches mix tenants and
    overlap on the GPU, yet every response equals its tenant's replay."""
    ctx = gpa.Context(0)
    srv = gpa.Server(ctx, M=M, max_batch=16, nstreams=3, slots_per_chunk=256)
    try:
        ids = []
        # interleave: request j of every tenant before request j + 1 of any
        depth = max(len(c) for c, _ in workload)
        for j in range(depth):
            for k, (concrete, expect) in enumerate(workload):
                if j < len(concrete):
                    op, arg, idx = concrete[j]
                    ids.append((k, j, _submit(srv, 1000 + k, op, arg, idx)))
        for k, j, rid in ids:
            r = srv.poll(rid)
            assert r["status"] == 0
            _same(r, workload[k][1][j], f"mix tenant {k} request {j}")
        st = srv.stats()
        assert st["completed"] == len(ids)
        assert st["batches"] > 1 and st["max_batch"] > 1
    finally:
        srv.stop()
        ctx.close()


def test_serve_errors_and_poll_contract():
    ctx = gpa.Context(0)
    srv = gpa.Server(ctx, M=M, max_batch=8, nstreams=2)
    try:
        r = srv.poll(srv.submit("REMOVE", 7, index=0))
        assert r["status"] == gpa.ERR_NOTFOUND  # unknown tenant
        with pytest.raises(gpa.GpaError) as ei:
            srv.poll(123456789, timeout_us=0)
        assert ei.value.code == gpa.ERR_NOTFOUND
        bad = {k: np.asarray([v]) for k, v in zip(serve_seq.COLS, (100, 101, 1000, 0, 1, 0))}  # D > T
        with pytest.raises(gpa.GpaError) as ei:
            srv.submit("ADMIT", 8, tasks=bad)
        assert ei.value.code == gpa.ERR_RANGE
        s = serve_seq.tenant_sets(1, seed=5)
        ok = srv.poll(srv.submit("ADMIT", 9, tasks=serve_seq.set_of(s, 0)))
        again = srv.poll(srv.submit("ADMIT", 9, tasks=serve_seq.set_of(s, 0)))
        assert ok["status"] == 0 and again["status"] == gpa.ERR_ARG  # the tenant exists
        r = srv.poll(srv.submit("REMOVE", 9, index=500))
        assert r["status"] == gpa.ERR_RANGE
    finally:
        srv.stop()
        ctx.close()


@pytest.mark.parametrize("sched,sizes", [("EDF", None), ("DM", [4, 8, 12, 16, 24, 32, 48, 64, 96, 148]),
                                         ("EDF", [7, 14, 21, 28, 42, 74, 148])])
def test_serve_policy_and_sizes_match_oracle(sched, sizes):
    """The EDF policy and admissible size lists in the serving loop: mixed
    micro-batches, every response equal to its tenant's replay."""
    ops = serve_seq.make_ops(24, 25, seed=13, evict=True)
    work = [_replay(seq, sched=sched, sizes=sizes) for seq in ops]
    ctx = gpa.Context(0)
    srv = gpa.Server(ctx, M=M, max_batch=16, nstreams=3, sched=sched, sizes=sizes)
    try:
        ids = []
        depth = max(len(c) for c, _ in work)
        for j in range(depth):
            for k, (concrete, expect) in enumerate(work):
                if j < len(concrete):
                    op, arg, idx = concrete[j]
                    ids.append((k, j, _submit(srv, 2000 + k, op, arg, idx)))
        for k, j, rid in ids:
            r = srv.poll(rid)
            assert r["status"] == 0
            _same(r, work[k][1][j], f"{sched} {sizes is not None} tenant {k} request {j}")
        if sizes:
            used = set()
            for _, expect in work:
                for e in expect:
                    used |= set(e["size_of_part"].tolist())
            assert used and used <= set(sizes)
    finally:
        srv.stop()
        ctx.close()
