"""GPU parity with admissible partition-size lists (whole GPCs / MIG-style
slices): the heuristic, the candidate test and the exhaustive search
against the oracle, element by element."""
import numpy as np
import pytest
import torch

import oracle
import paper_2105_10312_gb300 as gpa
from paper_2105_10312_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KC, KM = W.K_C, W.K_M
ALLOC_KEYS = ("verdict", "reason", "n_parts", "Pi", "W", "n_tests", "part_of_task", "size_of_part")
BEST_KEYS = ("feasible", "W", "sum_minm", "n_blocks", "spare", "rgs", "minm_block")
GPC68 = [4, 8, 12, 16, 20, 24, 28, 32, 36, 40, 44, 48, 52, 56, 60, 64, 68]  # 17 clusters of 4 SMs
MIGLIKE = [7, 14, 21, 28, 42, 68]


def _np(x):
    return x.cpu().numpy() if torch.is_tensor(x) else x


def _assert_equal(got, ref, keys, what):
    for k in keys:
        g, r = _np(got[k]), ref[k]
        if not np.array_equal(g, r):
            bad = np.nonzero(g != r)[0]
            raise AssertionError(f"{what}: {k} differs at {len(bad)} positions, first {bad[:8]}: "
                                 f"gpu {g[bad[:8]]} oracle {r[bad[:8]]}")


@pytest.mark.parametrize("sizes", [GPC68, MIGLIKE])
@pytest.mark.parametrize("policy,act", [("SMS", False), ("BF", True)])
def test_sizes_allocate_paper_setting(ctx, sizes, policy, act):
    s = gpa.gen_tasksets(**W.gen_params("paper50", nsets=34 * 2))
    md = W.model("paper50")
    for linear in (True, False):
        out = ctx.allocate(gpa.to_device(s), **md, policy=policy, act=act, linear=linear, sizes=sizes)
        ctx.sync()
        ref = oracle.allocate(s, md["M"], md["g"], KC, KM, policy=policy, act=act, linear=linear, nthreads=8,
                              sizes=sizes)
        _assert_equal(out, ref, ALLOC_KEYS, f"sizes {policy} act={act} linear={linear}")
    used = set(ref["size_of_part"][ref["size_of_part"] > 0].tolist())
    assert used and used <= set(sizes)


def test_sizes_allocate_batch_tpc_and_every_multiple(ctx):
    b = gpa.gen_tasksets(**W.gen_params("batch", nsets=4000))
    md = W.model("batch")
    sizes = [2, 4, 6, 10, 16, 24, 40, 60, 80]
    out = ctx.allocate(gpa.to_device(b), **md, sizes=sizes)
    ctx.sync()
    ref = oracle.allocate(b, md["M"], md["g"], KC, KM, nthreads=8, sizes=sizes)
    _assert_equal(out, ref, ALLOC_KEYS, "batch sizes")
    s = gpa.gen_tasksets(seed=80, nsets=300, n_min=1, n_max=40, U_lo_ppm=500000, U_hi_ppm=20000000,
                         deadline_pm=750, T_lo=1000, T_hi=100000)
    md = dict(M=40, g=2, k_c_pm=KC, k_m_pm=KM)
    every = list(range(2, 41, 2))
    plain = ctx.allocate(gpa.to_device(s), **md)
    listed = ctx.allocate(gpa.to_device(s), **md, sizes=every)
    tpc = ctx.allocate(gpa.to_device(s), **md, sizes=[4, 8, 20, 40], sched="EDF")
    ctx.sync()
    for k in ALLOC_KEYS:
        assert np.array_equal(_np(plain[k]), _np(listed[k])), k
    ref = oracle.allocate(s, 40, 2, KC, KM, nthreads=8, sizes=[4, 8, 20, 40], sched="EDF")
    _assert_equal(tpc, ref, ALLOC_KEYS, "TPC sizes EDF")


def test_sizes_candidates_and_host_rejection(ctx):
    rng = np.random.default_rng(3)
    s = gpa.gen_tasksets(seed=81, nsets=64, n_min=0, n_max=64, U_lo_ppm=100000, U_hi_ppm=6000000,
                         deadline_pm=750, mu_dist="BETA25")
    M, sizes, k, stride = 68, MIGLIKE, 4, 64
    nc = 2000
    cset = rng.integers(0, 64, nc).astype(np.int64)
    cmap = rng.integers(0, k, nc * stride).astype(np.uint8)
    csize = np.array([0] + sizes, np.int32)[rng.integers(0, len(sizes) + 1, nc * k)]
    v, R = ctx.test_schedulable(gpa.to_device(s), M, torch.from_numpy(cset).cuda(), torch.from_numpy(cmap).cuda(),
                                torch.from_numpy(csize).cuda(), stride, k, sizes=sizes)
    ctx.sync()
    vr, Rr = oracle.test_schedulable(s, M, 1, KC, KM, cset, cmap, stride, k, csize, sizes=sizes)
    assert np.array_equal(_np(v), vr) and np.array_equal(_np(R), Rr)
    assert 0 < vr.sum() < nc
    bad = csize.copy()
    bad[0] = 8  # not in the list
    with pytest.raises(gpa.GpaError) as ei:
        ctx.test_schedulable(s, M, cset, cmap, bad, stride, k, sizes=sizes)
    assert ei.value.code == gpa.ERR_RANGE


@pytest.mark.parametrize("sched", ["DM", "EDF"])
def test_sizes_search_best(ctx, sched):
    s = gpa.gen_tasksets(seed=82, nsets=60, n_min=1, n_max=9, U_lo_ppm=500000, U_hi_ppm=3500000, deadline_pm=750,
                         T_lo=1000, T_hi=100000)
    M, g, kmin, kmax = 40, 2, 1, 4
    sizes = [4, 6, 10, 16, 24]
    out = ctx.search_best(gpa.to_device(s), M, g=g, k_c_pm=KC, k_m_pm=KM, kmin=kmin, kmax=kmax, sched=sched,
                          sizes=sizes)
    ctx.sync()
    ref = oracle.search_best(s, M, g, KC, KM, kmin, kmax, nthreads=8, sched=sched, sizes=sizes)
    _assert_equal(out, ref, BEST_KEYS, f"search sizes {sched}")
    assert 5 < ref["feasible"].sum() < 60
