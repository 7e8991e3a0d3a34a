"""Parity at the workloads' full sizes, in the launch configuration the bench
times (default launch shape, CUDA graphs on, non-default stream): the GPU
computes every set of the batch, the oracle a seeded sample of them, and
the sampled sets' outputs must be equal element by element."""
import numpy as np
import pytest
import torch

import oracle
import paper_2105_10312_gb300 as gpa
from paper_2105_10312_gb300 import gen as G
from paper_2105_10312_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KC, KM = W.K_C, W.K_M
SET_KEYS = ("verdict", "reason", "n_parts", "Pi", "W", "n_tests")
TASK_KEYS = ("part_of_task", "size_of_part")
BEST_SET_KEYS = ("feasible", "W", "sum_minm", "n_blocks", "spare")


@pytest.fixture(scope="module")
def gctx():
    stream = torch.cuda.Stream()
    c = gpa.Context(0, stream=stream)
    c.set_option("GRAPH", 1)
    yield c
    c.close()


def _sample(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=min(k, n), replace=False))


def _task_index(off, idx):
    return np.concatenate([np.arange(off[i], off[i + 1]) for i in idx]) if len(idx) else np.zeros(0, np.int64)


def _check(got, ref, idx, tidx, set_keys, task_keys, what):
    for k in set_keys:
        g = got[k].cpu().numpy()[idx]
        if not np.array_equal(g, ref[k]):
            bad = np.nonzero(g != ref[k])[0]
            raise AssertionError(f"{what}: {k} differs at sampled sets {idx[bad[:8]]}")
    for k in task_keys:
        g = got[k].cpu().numpy()[tidx]
        if not np.array_equal(g, ref[k]):
            raise AssertionError(f"{what}: {k} differs at {np.count_nonzero(g != ref[k])} sampled tasks")


def _alloc_full(gctx, name, policy, act, k, seed, pick=None):
    s = gpa.gen_tasksets(**W.gen_params(name))
    md = W.model(name)
    out = gctx.allocate(gpa.to_device(s), **md, policy=policy, act=act)
    gctx.sync()
    nsets = len(s["set_off"]) - 1
    idx = _sample(nsets, k, seed) if pick is None else pick(nsets)
    ref = oracle.allocate(G.subset(s, idx), md["M"], md["g"], KC, KM, policy=policy, act=act, nthreads=8)
    _check(out, ref, idx, _task_index(s["set_off"], idx), SET_KEYS, TASK_KEYS, f"{name} {policy} act={act}")
    return ref


@pytest.mark.parametrize("policy", ["SMS", "ONE_GPU"])
def test_sweep_full_size_sampled(gctx, policy):
    """1 000 000 sets of 4-64 tasks on 148 SMs; 20 000 sampled."""
    ref = _alloc_full(gctx, "sweep", policy, False, 20000, 11)
    assert 0 < ref["verdict"].sum() < 20000


@pytest.mark.parametrize("policy,act", [("SMS", False), ("BF", True)])
def test_paper50_full_size_sampled(gctx, policy, act):
    """The §7 batch (3 400 sets of 50 tasks); 200 sampled."""
    ref = _alloc_full(gctx, "paper50", policy, act, 200, 12)
    assert ref["n_tests"].sum() > 10000


def test_paper200_full_size_sampled(gctx):
    """The 200-task batch (3 400 sets, the 256-task build); the oracle's
    sample is the first six sets at U = 2 (minutes per set at high U)."""
    ref = _alloc_full(gctx, "paper200", "SMS", False, 0, 0, pick=lambda n: np.arange(0, 6 * 34, 34))
    assert ref["verdict"].all() and ref["n_tests"].min() > 1000


def test_exhaustive_full_size_sampled(gctx):
    """20 000 sets of 12 tasks, 1-4 partitions of 20 TPC units; 150 sampled."""
    p = W.WORKLOADS["exhaustive"]
    s = gpa.gen_tasksets(**W.gen_params("exhaustive"))
    md = W.model("exhaustive")
    out = gctx.search_best(gpa.to_device(s), **md, kmin=p["kmin"], kmax=p["kmax"])
    gctx.sync()
    idx = _sample(len(s["set_off"]) - 1, 150, 13)
    ref = oracle.search_best(G.subset(s, idx), md["M"], md["g"], KC, KM, p["kmin"], p["kmax"], nthreads=8)
    _check(out, ref, idx, _task_index(s["set_off"], idx), BEST_SET_KEYS, ("rgs",), "exhaustive")
    mb = out["minm_block"].cpu().numpy().reshape(-1, p["kmax"])[idx]
    assert np.array_equal(mb, ref["minm_block"].reshape(-1, p["kmax"]))
    assert ref["feasible"].sum() > 0 and (ref["n_blocks"] > 1).any()
