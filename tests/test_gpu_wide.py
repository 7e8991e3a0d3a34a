"""GPU parity of the 256-task build (sets of 129..256 tasks, e.g. the 200-task
sets of the paper's Figs. 6 and 7) against the oracle, element by element:
the heuristic (fast path and merge loop, DM and EDF), the 1G baseline, the
candidate test, and the switch between the two builds at n_max = 128."""
import numpy as np
import pytest
import torch

import oracle
import paper_2105_10312_gb300 as gpa
from paper_2105_10312_gb300 import gen as G
from paper_2105_10312_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KC, KM = W.K_C, W.K_M
ALLOC_KEYS = ("verdict", "reason", "n_parts", "Pi", "W", "n_tests", "part_of_task", "size_of_part")


def _np(x):
    return x.cpu().numpy() if torch.is_tensor(x) else x


def _assert_equal(got, ref, keys, what):
    for k in keys:
        g, r = _np(got[k]), ref[k]
        if not np.array_equal(g, r):
            bad = np.nonzero(g != r)[0]
            raise AssertionError(f"{what}: {k} differs at {len(bad)} positions, first {bad[:8]}: "
                                 f"gpu {g[bad[:8]]} oracle {r[bad[:8]]}")


def _random_wide(seed, nsets=48):
    return gpa.gen_tasksets(seed=seed, nsets=nsets, n_min=120, n_max=256, U_lo_ppm=500000, U_hi_ppm=6000000,
                            deadline_pm=750, T_lo=1000, T_hi=100000, mu_dist="BETA25")


@pytest.mark.parametrize("policy,act,sched", [("SMS", False, "DM"), ("BF", True, "DM"), ("SMS", True, "EDF")])
def test_paper200_low_load_matches_oracle(ctx, policy, act, sched):
    """200-task sets of the paper's setting at U = 2..8 (the oracle's RTA on
    200 tasks takes seconds per set there): every merge of the heuristic."""
    s = gpa.gen_tasksets(**W.gen_params("paper200", nsets=34 * 2))
    sub = G.subset(s, np.array([0, 1, 2, 3, 34, 35, 36]))
    md = W.model("paper200")
    out = ctx.allocate(gpa.to_device(sub), **md, policy=policy, act=act, sched=sched)
    ctx.sync()
    ref = oracle.allocate(sub, md["M"], md["g"], KC, KM, policy=policy, act=act, nthreads=8, sched=sched)
    _assert_equal(out, ref, ALLOC_KEYS, f"paper200 {policy} act={act} {sched}")
    assert ref["n_tests"].min() > 1000


@pytest.mark.parametrize("sched", ["DM", "EDF"])
def test_wide_random_sets_match_oracle(ctx, sched):
    """120..256 tasks: on 512 SMs the fast path decides every set, on 256
    SMs in units of 2 almost every set merges; host and device inputs."""
    s = _random_wide(95)
    for M, g in ((512, 1), (256, 2)):
        ref = oracle.allocate(s, M, g, KC, KM, policy="BF", act=False, nthreads=8, sched=sched)
        out = ctx.allocate(gpa.to_device(s), M, g=g, k_c_pm=KC, k_m_pm=KM, policy="BF", sched=sched)
        ctx.sync()
        _assert_equal(out, ref, ALLOC_KEYS, f"wide device M={M} g={g} {sched}")
        out = ctx.allocate(s, M, g=g, k_c_pm=KC, k_m_pm=KM, policy="BF", sched=sched)
        _assert_equal(out, ref, ALLOC_KEYS, f"wide host M={M} g={g} {sched}")


@pytest.mark.parametrize("sched", ["DM", "EDF"])
def test_wide_one_gpu_matches_oracle(ctx, sched):
    s = _random_wide(96, nsets=200)
    out = ctx.allocate(gpa.to_device(s), 148, g=1, k_c_pm=KC, k_m_pm=KM, policy="ONE_GPU", sched=sched)
    ctx.sync()
    ref = oracle.allocate(s, 148, 1, KC, KM, policy="ONE_GPU", nthreads=8, sched=sched)
    _assert_equal(out, ref, ALLOC_KEYS, f"wide 1G {sched}")
    assert 0 < ref["verdict"].sum() < 200


@pytest.mark.parametrize("sched", ["DM", "EDF"])
def test_wide_candidates_match_oracle(ctx, sched):
    """Random splits and maps of 0..256-task sets into 6 parts: verdicts and
    per-task R."""
    rng = np.random.default_rng(97)
    s = gpa.gen_tasksets(seed=97, nsets=32, n_min=0, n_max=256, U_lo_ppm=100000, U_hi_ppm=12000000,
                         deadline_pm=750, mu_dist="BETA25", T_lo=1000, T_hi=100000)
    M, g, k, stride = 192, 2, 6, 256
    nc = 1500
    cset = rng.integers(0, 32, nc).astype(np.int64)
    cmap = rng.integers(0, k, nc * stride).astype(np.uint8)
    csize = (g * rng.integers(0, M // g // 4 + 1, nc * k)).astype(np.int32)
    v, R = ctx.test_schedulable(gpa.to_device(s), M, torch.from_numpy(cset).cuda(), torch.from_numpy(cmap).cuda(),
                                torch.from_numpy(csize).cuda(), stride, k, g=g, sched=sched)
    ctx.sync()
    vr, Rr = oracle.test_schedulable(s, M, g, KC, KM, cset, cmap, stride, k, csize, sched=sched)
    assert np.array_equal(_np(v), vr) and np.array_equal(_np(R), Rr)
    assert 0 < vr.sum() < nc


@pytest.mark.parametrize("n_top,n_maxes,policy", [(128, (128, 129, 256), "SMS"), (64, (64, 65, 128, 256), "SMS"),
                                                  (64, (64, 65, 256), "ONE_GPU")])
def test_builds_agree_at_the_switch(ctx, n_top, n_maxes, policy):
    """Sets of at most n_top tasks declared with every n_max that selects a
    different build (64-task, 128-task, 256-task): identical results, equal
    to the oracle's."""
    s = gpa.gen_tasksets(seed=98, nsets=600, n_min=0, n_max=n_top, U_lo_ppm=500000, U_hi_ppm=20000000,
                         deadline_pm=750, mu_dist="BETA25", T_lo=1000, T_hi=100000)
    M, g = 96, 2
    act = policy != "ONE_GPU"
    ref = oracle.allocate(s, M, g, KC, KM, policy=policy, act=act, nthreads=8)
    for n_max in n_maxes:
        d = gpa.to_device(s)
        d["n_max"] = n_max
        out = ctx.allocate(d, M, g=g, k_c_pm=KC, k_m_pm=KM, policy=policy, act=act)
        ctx.sync()
        _assert_equal(out, ref, ALLOC_KEYS, f"n_max={n_max} {policy}")


def test_wide_limits(ctx):
    """n_max 257 is rejected on the host; a device set longer than its
    batch's n_max (here above 128) is flagged invalid by the 256-task build."""
    s = _random_wide(99, nsets=4)
    off = s["set_off"]
    n = off[1:] - off[:-1]
    big = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}
    big["n_max"] = 257
    with pytest.raises(gpa.GpaError) as ei:
        ctx.allocate(big, 512, g=1, k_c_pm=KC, k_m_pm=KM)
    assert ei.value.code == gpa.ERR_RANGE
    short = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}
    short["n_max"] = int(n.max()) - 1
    out = ctx.allocate(gpa.to_device(short), 512, g=1, k_c_pm=KC, k_m_pm=KM)
    with pytest.raises(gpa.GpaError) as ei:
        ctx.sync()
    assert ei.value.code == gpa.ERR_RANGE
    assert _np(out["reason"])[int(np.argmax(n))] == gpa.REASON["INVALID"]


@pytest.mark.parametrize("slices,copy", [(3, 0), (2, 1)])
def test_wide_sets_through_sliced_host_buffers(ctx, slices, copy):
    """120..256-task sets (the 256-task build) from page-locked host buffers
    split into slices, by the staging kernel and by copies."""
    s = _random_wide(95)
    hs = {k: (torch.from_numpy(v).pin_memory().numpy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}
    M, g = 256, 2
    ref = oracle.allocate(s, M, g, KC, KM, policy="SMS", act=True, nthreads=8)
    ctx.set_option("HOST_SLICES", slices)
    ctx.set_option("HOST_COPY", copy)
    try:
        out = ctx.allocate(hs, M, g=g, k_c_pm=KC, k_m_pm=KM, policy="SMS", act=True)
    finally:
        ctx.set_option("HOST_SLICES", 0)
        ctx.set_option("HOST_COPY", 0)
    _assert_equal(out, ref, ALLOC_KEYS, f"wide sliced={slices} copy={copy}")
