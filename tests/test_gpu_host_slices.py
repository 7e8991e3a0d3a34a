"""gpa_allocate on host buffers: batches split into slices whose copies in,
kernels and copies out overlap, and page-locked arrays moved by the staging
kernel.  Results equal the oracle's for every slice count, policy, copy
route and array alignment, and a rejected batch still names its first
invalid set."""
import numpy as np
import pytest
import torch

import oracle
import paper_2105_10312_gb300 as gpa
from paper_2105_10312_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KC, KM = W.K_C, W.K_M
ALLOC_KEYS = ("verdict", "reason", "n_parts", "Pi", "W", "n_tests", "part_of_task", "size_of_part")


def _assert_equal(got, ref, keys, what):
    for k in keys:
        g, r = got[k], ref[k]
        if g is None:
            continue
        if not np.array_equal(g, r):
            bad = np.nonzero(g != r)[0]
            raise AssertionError(f"{what}: {k} differs at {len(bad)} positions, first {bad[:8]}: "
                                 f"gpu {g[bad[:8]]} oracle {r[bad[:8]]}")


@pytest.fixture(scope="module")
def sctx():
    stream = torch.cuda.Stream()
    c = gpa.Context(0, stream=stream)
    yield c
    c.close()


@pytest.mark.parametrize("slices", [0, 2, 3, 7, 64])
def test_sliced_batch_matches_oracle(sctx, slices):
    s = gpa.gen_tasksets(**W.gen_params("batch", nsets=6001))
    md = W.model("batch")
    ref = oracle.allocate(s, md["M"], md["g"], KC, KM, nthreads=8)
    sctx.set_option("HOST_SLICES", slices)
    try:
        for graph in (0, 1, 1):  # direct launches, then a captured graph per slice and its replay
            sctx.set_option("GRAPH", graph)
            out = sctx.allocate(s, **md)
            _assert_equal(out, ref, ALLOC_KEYS, f"{slices} slices graph={graph}")
        no_tests = sctx.alloc_result(s, with_tests=False)
        out = sctx.allocate(s, **md, out=no_tests)
        _assert_equal(out, ref, ALLOC_KEYS, f"{slices} slices without n_tests")
    finally:
        sctx.set_option("GRAPH", 0)
        sctx.set_option("HOST_SLICES", 0)


@pytest.mark.parametrize("policy,act,sched,sizes", [("SMS", True, "DM", None), ("BF", False, "EDF", None),
                                                    ("ONE_GPU", False, "DM", None),
                                                    ("BF", True, "DM", [4, 8, 12, 20, 40, 80])])
def test_sliced_policies_match_oracle(sctx, policy, act, sched, sizes):
    """Sets of 0..64 tasks at every load of the sweep, so that slices hold
    empty sets, sets the fast path decides and sets that merge."""
    s = gpa.gen_tasksets(seed=91, nsets=4000, n_min=0, n_max=64, U_lo_ppm=100000, U_hi_ppm=40000000,
                         deadline_pm=750, mu_dist="BETA25", T_lo=1000, T_hi=100000)
    M, g = 80, 2
    sctx.set_option("HOST_SLICES", 5)
    try:
        out = sctx.allocate(s, M, g=g, k_c_pm=KC, k_m_pm=KM, policy=policy, act=act, sched=sched, sizes=sizes)
    finally:
        sctx.set_option("HOST_SLICES", 0)
    ref = oracle.allocate(s, M, g, KC, KM, policy=policy, act=act, nthreads=8, sched=sched, sizes=sizes)
    _assert_equal(out, ref, ALLOC_KEYS, f"sliced {policy} act={act} {sched} sizes={sizes}")


def test_large_batch_is_split_and_matches_oracle(sctx):
    """300 000 sets of the batching workload (about 300 MB of task columns):
    the default splits it into 5 slices."""
    s = gpa.gen_tasksets(**W.gen_params("batch", nsets=300000))
    md = W.model("batch")
    out = sctx.allocate(s, **md)
    ref = oracle.allocate(s, md["M"], md["g"], KC, KM, nthreads=8)
    _assert_equal(out, ref, ALLOC_KEYS, "auto slices")


@pytest.mark.parametrize("bad_set", [0, 2999, 3777, 4999])
def test_sliced_rejection_names_first_invalid_set(sctx, bad_set):
    s = gpa.gen_tasksets(**W.gen_params("batch", nsets=5000))
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}
    bad["T"][int(bad["set_off"][bad_set])] = 0
    md = W.model("batch")
    sctx.set_option("HOST_SLICES", 4)
    try:
        with pytest.raises(gpa.GpaError) as ei:
            sctx.allocate(bad, **md)
        assert ei.value.code == gpa.ERR_RANGE and str(bad_set) in str(ei.value)
        out = sctx.allocate(s, **md)  # the context is clean afterwards
    finally:
        sctx.set_option("HOST_SLICES", 0)
    ref = oracle.allocate(s, md["M"], md["g"], KC, KM, nthreads=8)
    _assert_equal(out, ref, ALLOC_KEYS, "after a rejected sliced call")


def test_sliced_rejection_of_decreasing_offsets(sctx):
    """set_off that decreases: rejected whether or not the host can split the
    batch at the bad offset."""
    s = gpa.gen_tasksets(**W.gen_params("batch", nsets=4000))
    md = W.model("batch")
    for at in (1000, 2000, 3999):
        bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}
        bad["set_off"][at] = bad["set_off"][at - 1] - 1
        sctx.set_option("HOST_SLICES", 2)
        try:
            with pytest.raises(gpa.GpaError) as ei:
                sctx.allocate(bad, **md)
        finally:
            sctx.set_option("HOST_SLICES", 0)
        assert ei.value.code == gpa.ERR_RANGE


def _pinned(a, offset_bytes=0):
    """A page-locked copy of `a` starting `offset_bytes` past a page-locked
    allocation's start (a multiple of the element size)."""
    dt = torch.from_numpy(a[:0]).dtype
    k = offset_bytes // a.itemsize
    t = torch.empty(len(a) + k + 1, dtype=dt).pin_memory()
    v = t.numpy()[k:k + len(a)]
    v[:] = a
    return v


@pytest.mark.parametrize("slices,copy", [(0, 0), (0, 1), (1, 0), (4, 0), (4, 1), (1, 2), (3, 7)])
@pytest.mark.parametrize("aligned", [True, False])
def test_page_locked_buffers_match_oracle(sctx, slices, copy, aligned):
    """Inputs and outputs in page-locked memory at 16-byte aligned starts, or
    at starts that leave the staging kernel its 8-byte and byte paths; both
    copy routes, whole and sliced."""
    s = gpa.gen_tasksets(**W.gen_params("batch", nsets=6001))
    md = W.model("batch")
    ref = oracle.allocate(s, md["M"], md["g"], KC, KM, nthreads=8)
    off64, off8 = (0, 0) if aligned else (8, 3)
    hs = {k: (_pinned(v, off8 if v.dtype == np.uint8 else off64) if isinstance(v, np.ndarray) else v)
          for k, v in s.items()}
    out = {k: (_pinned(v, 0 if aligned else v.itemsize * (1 if v.itemsize > 1 else 5)) if v is not None else None)
           for k, v in sctx.alloc_result(s).items()}
    sctx.set_option("HOST_SLICES", slices)
    sctx.set_option("HOST_COPY", copy)
    try:
        got = sctx.allocate(hs, **md, out=out)
    finally:
        sctx.set_option("HOST_SLICES", 0)
        sctx.set_option("HOST_COPY", 0)
    _assert_equal(got, ref, ALLOC_KEYS, f"page-locked slices={slices} copy={copy} aligned={aligned}")


def test_mixed_page_locked_and_pageable_columns(sctx):
    s = gpa.gen_tasksets(**W.gen_params("batch", nsets=3000))
    md = W.model("batch")
    ref = oracle.allocate(s, md["M"], md["g"], KC, KM, nthreads=8)
    hs = dict(s)
    for k in ("T", "A", "type"):
        hs[k] = _pinned(s[k])
    out = sctx.alloc_result(s)
    out["W"] = _pinned(out["W"])
    out["part_of_task"] = _pinned(out["part_of_task"])
    for slices in (0, 1, 2):
        sctx.set_option("HOST_SLICES", slices)
        try:
            got = sctx.allocate(hs, **md, out=out)
        finally:
            sctx.set_option("HOST_SLICES", 0)
        _assert_equal(got, ref, ALLOC_KEYS, f"mixed slices={slices}")


def test_page_locked_inputs_for_the_other_entry_points(sctx):
    """The candidate test and the exhaustive search stage page-locked inputs
    through the same kernel."""
    s = gpa.gen_tasksets(seed=82, nsets=60, n_min=1, n_max=9, U_lo_ppm=500000, U_hi_ppm=3500000, deadline_pm=750,
                         T_lo=1000, T_hi=100000)
    hs = {k: (_pinned(v, 8 if v.dtype != np.uint8 else 1) if isinstance(v, np.ndarray) else v) for k, v in s.items()}
    out = sctx.search_best(hs, 40, g=2, k_c_pm=KC, k_m_pm=KM, kmin=1, kmax=4)
    ref = oracle.search_best(s, 40, 2, KC, KM, 1, 4, nthreads=8)
    for k in ("feasible", "W", "sum_minm", "n_blocks", "spare", "rgs", "minm_block"):
        assert np.array_equal(out[k], ref[k]), k


_MULTI_SETS = dict(seed=93, nsets=4000, n_min=0, n_max=64, U_lo_ppm=100000, U_hi_ppm=40000000, deadline_pm=750,
                   mu_dist="BETA25", T_lo=1000, T_hi=100000)
_MULTI_REF = {}


def _multi_ref(s, policy, act, sched):
    key = (policy, act, sched)
    if key not in _MULTI_REF:
        _MULTI_REF[key] = oracle.allocate(s, 80, 2, KC, KM, policy=policy, act=act, nthreads=8, sched=sched)
    return _MULTI_REF[key]


@pytest.mark.parametrize("slices", [1, 0, 5])
def test_multi_policy_call_matches_oracle(sctx, slices):
    """gpa_allocate_multi on host arrays: one copy of the batch, decided
    under four policies; each result equals the oracle's for its policy,
    with the batch whole, split by default and in 5 slices."""
    s = gpa.gen_tasksets(**_MULTI_SETS)
    pols = [("SMS", True), ("ONE_GPU", False), ("BF", False), ("SMS", False)]
    sctx.set_option("HOST_SLICES", slices)
    try:
        outs = sctx.allocate_multi(s, 80, g=2, k_c_pm=KC, k_m_pm=KM, policies=pols)
    finally:
        sctx.set_option("HOST_SLICES", 0)
    assert len(outs) == len(pols)
    for (pol, act), out in zip(pols, outs):
        _assert_equal(out, _multi_ref(s, pol, act, "DM"), ALLOC_KEYS, f"multi {pol} act={act} slices={slices}")


def test_multi_policy_call_on_device_arrays(sctx):
    s = gpa.gen_tasksets(**_MULTI_SETS)
    pols = [("BF", True), ("ONE_GPU", False)]
    outs = sctx.allocate_multi(gpa.to_device(s), 80, g=2, k_c_pm=KC, k_m_pm=KM, policies=pols, sched="EDF")
    sctx.sync()
    for (pol, act), out in zip(pols, outs):
        got = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
        _assert_equal(got, _multi_ref(s, pol, act, "EDF"), ALLOC_KEYS, f"multi device {pol} act={act} EDF")


def test_multi_policy_call_rejections(sctx):
    s = gpa.gen_tasksets(**_MULTI_SETS)
    for pols in ([], ["SMS"] * (gpa.MULTI_MAX_POLICIES + 1)):
        with pytest.raises(gpa.GpaError) as ei:
            sctx.allocate_multi(s, 80, g=2, k_c_pm=KC, k_m_pm=KM, policies=pols)
        assert ei.value.code == gpa.ERR_RANGE
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}
    bad["D"][int(bad["set_off"][3001])] = 0
    sctx.set_option("HOST_SLICES", 4)
    try:
        with pytest.raises(gpa.GpaError) as ei:
            sctx.allocate_multi(bad, 80, g=2, k_c_pm=KC, k_m_pm=KM, policies=["SMS", "ONE_GPU"])
        assert ei.value.code == gpa.ERR_RANGE and "3001" in str(ei.value)
        outs = sctx.allocate_multi(s, 80, g=2, k_c_pm=KC, k_m_pm=KM, policies=[("SMS", True), "ONE_GPU"])
    finally:
        sctx.set_option("HOST_SLICES", 0)
    _assert_equal(outs[0], _multi_ref(s, "SMS", True, "DM"), ALLOC_KEYS, "multi after a rejected call")
    _assert_equal(outs[1], _multi_ref(s, "ONE_GPU", False, "DM"), ALLOC_KEYS, "multi 1G after a rejected call")
