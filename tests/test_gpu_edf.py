"""GPU parity of the EDF per-partition policy (processor-demand test) against
the CPU oracle: the candidate test, the heuristic, the 1G baseline and the
exhaustive search, element by element on seeded inputs."""
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


def _np(x):
    return x.cpu().numpy() if torch.is_tensor(x) else x


def _assert_equal(got, ref, keys, what):
    for k in keys:
        g, r = _np(got[k]), ref[k]
        if not np.array_equal(g, r):
            bad = np.nonzero(g != r)[0]
            raise AssertionError(f"{what}: {k} differs at {len(bad)} positions, first {bad[:8]}: "
                                 f"gpu {g[bad[:8]]} oracle {r[bad[:8]]}")


@pytest.mark.parametrize("seed", [0, 1])
def test_edf_random_candidates(ctx, seed):
    """Random splits and maps of 0..128-task sets: verdicts and the per-task
    R convention (0 in a passing part, -1 otherwise) equal the oracle's; EDF
    accepts every candidate DM accepts, and some that DM rejects."""
    rng = np.random.default_rng(seed)
    s = gpa.gen_tasksets(seed=60 + seed, nsets=64, n_min=0, n_max=128, U_lo_ppm=100000, U_hi_ppm=8000000,
                         deadline_pm=750, mu_dist="BETA25", T_lo=1000, T_hi=100000)
    M, g, k, stride = 96, 2, 5, 128
    nc = 3000
    cset = rng.integers(0, 64, nc).astype(np.int64)
    cmap = rng.integers(0, k, nc * stride).astype(np.uint8)
    csize = (g * rng.integers(0, M // g // 3 + 1, nc * k)).astype(np.int32)
    d = gpa.to_device(s)
    args = (torch.from_numpy(cset).cuda(), torch.from_numpy(cmap).cuda(), torch.from_numpy(csize).cuda(), stride, k)
    for with_R in (True, False):
        v, R = ctx.test_schedulable(d, M, *args, g=g, with_R=with_R, sched="EDF")
        ctx.sync()
        vr, Rr = oracle.test_schedulable(s, M, g, KC, KM, cset, cmap, stride, k, csize, with_R=with_R, sched="EDF")
        assert np.array_equal(_np(v), vr)
        if with_R:
            assert np.array_equal(_np(R), Rr)
    vd, _ = ctx.test_schedulable(d, M, *args, g=g, with_R=False)
    ctx.sync()
    vd = _np(vd)
    assert (vr >= vd).all()
    assert (vr > vd).sum() > 0 and 0 < vr.sum() < nc


@pytest.mark.parametrize("policy,act", [("SMS", False), ("SMS", True), ("BF", False), ("BF", True)])
def test_edf_allocate_paper_setting(ctx, policy, act):
    """The §7 setting under EDF: the merge loop runs (one-lane candidate
    sizing and the warp test both), results equal the oracle's."""
    s = gpa.gen_tasksets(**W.gen_params("paper50", nsets=34 * 3))
    md = W.model("paper50")
    out = ctx.allocate(gpa.to_device(s), **md, policy=policy, act=act, sched="EDF")
    ctx.sync()
    ref = oracle.allocate(s, md["M"], md["g"], KC, KM, policy=policy, act=act, nthreads=8, sched="EDF")
    _assert_equal(out, ref, ALLOC_KEYS, f"paper50 EDF {policy} act={act}")
    assert ref["n_tests"].sum() > 1000


def test_edf_allocate_binary_merge_tpc_and_batch(ctx):
    s = gpa.gen_tasksets(seed=61, nsets=400, n_min=1, n_max=40, U_lo_ppm=500000, U_hi_ppm=20000000,
                         deadline_pm=750, T_lo=1000, T_hi=100000)
    for md in (dict(M=40, g=2, k_c_pm=KC, k_m_pm=KM), dict(M=16, g=4, k_c_pm=1500, k_m_pm=4000)):
        for linear in (True, False):
            out = ctx.allocate(gpa.to_device(s), **md, linear=linear, sched="EDF")
            ctx.sync()
            ref = oracle.allocate(s, md["M"], md["g"], md["k_c_pm"], md["k_m_pm"], linear=linear, nthreads=8,
                                  sched="EDF")
            _assert_equal(out, ref, ALLOC_KEYS, f"EDF M={md['M']} g={md['g']} linear={linear}")
    b = gpa.gen_tasksets(**W.gen_params("batch", nsets=5000))
    md = W.model("batch")
    out = ctx.allocate(gpa.to_device(b), **md, sched="EDF")
    ctx.sync()
    ref = oracle.allocate(b, md["M"], md["g"], KC, KM, nthreads=8, sched="EDF")
    _assert_equal(out, ref, ALLOC_KEYS, "EDF batch")


def test_edf_one_gpu(ctx):
    s = gpa.gen_tasksets(**W.gen_params("sweep", nsets=3000))
    md = W.model("sweep")
    out = ctx.allocate(gpa.to_device(s), **md, policy="ONE_GPU", sched="EDF")
    ctx.sync()
    ref = oracle.allocate(s, md["M"], md["g"], KC, KM, policy="ONE_GPU", nthreads=8, sched="EDF")
    _assert_equal(out, ref, ALLOC_KEYS, "EDF 1G")
    dm = oracle.allocate(s, md["M"], md["g"], KC, KM, policy="ONE_GPU", nthreads=8)
    assert (ref["verdict"] >= dm["verdict"]).all() and 0 < ref["verdict"].sum() < 3000


def test_edf_search_best(ctx):
    s = gpa.gen_tasksets(seed=62, nsets=40, n_min=1, n_max=8, U_lo_ppm=500000, U_hi_ppm=3500000, deadline_pm=750,
                         T_lo=1000, T_hi=100000)
    M, g, kmin, kmax = 40, 2, 1, 4
    out = ctx.search_best(gpa.to_device(s), M, g=g, k_c_pm=KC, k_m_pm=KM, kmin=kmin, kmax=kmax, sched="EDF")
    ctx.sync()
    ref = oracle.search_best(s, M, g, KC, KM, kmin, kmax, nthreads=8, sched="EDF")
    _assert_equal(out, ref, BEST_KEYS, "EDF search")
    assert ref["feasible"].sum() > 10


def _crafted_batch(sets_tasks):
    """Sets of (T, D, C) tasks alternating types (no conflict at k = 1000),
    A = 1000 C and B = 0 so that C(1) = C."""
    off, cols = [0], {k: [] for k in ("T", "D", "A", "B", "u_ppm", "type")}
    for tasks in sets_tasks:
        for j, (T, D, C) in enumerate(tasks):
            cols["T"].append(T)
            cols["D"].append(D)
            cols["A"].append(1000 * C)
            cols["B"].append(0)
            cols["u_ppm"].append(10**6 * C // T)
            cols["type"].append(j % 2)
        off.append(off[-1] + len(tasks))
    out = {k: np.array(v, np.uint8 if k == "type" else np.int64) for k, v in cols.items()}
    out["set_off"] = np.array(off, np.int64)
    out["n_max"] = max(len(t) for t in sets_tasks)
    return out


def _one_part_candidates(s, m):
    nsets = len(s["set_off"]) - 1
    stride = int(s["n_max"])
    cset = np.arange(nsets, dtype=np.int64)
    cmap = np.zeros(nsets * stride, np.uint8)
    csize = np.full(nsets, m, np.int32)
    return cset, cmap, csize, stride


def _edf_candidate_parity(ctx, s, M=1, kc=1000, km=1000):
    cset, cmap, csize, stride = _one_part_candidates(s, 1)
    d = gpa.to_device(s)
    v, R = ctx.test_schedulable(d, M, torch.from_numpy(cset).cuda(), torch.from_numpy(cmap).cuda(),
                                torch.from_numpy(csize).cuda(), stride, 1, k_c_pm=kc, k_m_pm=km, sched="EDF")
    ctx.sync()
    vr, Rr = oracle.test_schedulable(s, M, 1, kc, km, cset, cmap, stride, 1, csize, sched="EDF")
    assert np.array_equal(_np(v), vr) and np.array_equal(_np(R), Rr)
    return vr


def test_edf_utilisation_one_edges(ctx):
    """Sets whose U equals 1 exactly or misses it by one unit of C: harmonic
    periods, 1/3 + 2/3 (the 2^64-scaled terms straddle 1, decided by the
    periods' least common multiple), pairs of large coprime periods (U - 1 a
    multiple of 1 / (T1 T2)); implicit deadlines, and a first deadline
    shortened by one and by a quarter.  Every verdict equals the oracle's
    exact test, and none is undecided."""
    base = [([3, 3], [1, 2]), ([1000003, 2000006], [600001, 800004]), ([7, 14, 28], [3, 4, 8]),
            ([1000, 4000, 500], [250, 1000, 250])]
    T1, T2 = 1329, 1048573
    for C1 in (1, 664, 1328):
        base.append(([T1, T2], [C1, (T2 * (T1 - C1)) // T1]))
    sets = []
    for T, C in base:
        for dc in (-1, 0, 1):
            CC = list(C[:-1]) + [C[-1] + dc]
            if not 1 <= CC[-1] <= T[-1]:
                continue
            for cut in (0, 1, T[0] // 4):
                D = [T[0] - cut] + list(T[1:])
                if CC[0] <= D[0]:
                    sets.append(list(zip(T, D, CC)))
    s = _crafted_batch(sets)
    v = _edf_candidate_parity(ctx, s)
    assert 0 < v.sum() < len(v) and (v <= 1).all()


def test_edf_near_one(ctx):
    """Eight tasks on periods in [10^5, 10^6] with U = 1 - 2^-k, k = 11..17
    (rounded to whole WCET units), constrained and implicit deadlines: the
    L_a bound and the QPA walk grow like 2^k; verdicts equal the oracle's."""
    rng = np.random.default_rng(11)
    sets = []
    for k in (11, 13, 15, 17):
        for trial in range(4):
            n = 8
            T = rng.integers(100_000, 1_000_000, n)
            w = rng.random(n)
            C = np.floor((1 - 2.0 ** -k) * w / w.sum() * T).astype(np.int64)
            C = np.maximum(C, 1)
            D = T if trial % 2 == 0 else np.maximum(C, (T * 0.9).astype(np.int64))
            sets.append(list(zip(T.tolist(), D.tolist(), C.tolist())))
    v = _edf_candidate_parity(ctx, _crafted_batch(sets))
    assert (v <= 1).all() and v.sum() > 0


def test_edf_busy_period_beyond_31_bits(ctx):
    """Many large tasks at U close to 1: the busy period and the QPA
    points pass 2^31, so the 64-bit division paths run; verdicts equal the
    oracle's."""
    rng = np.random.default_rng(7)
    sets = []
    for trial in range(24):
        n = int(rng.integers(60, 128))
        T = rng.integers(100_000_000, 400_000_000, n)
        target = 0.95 + 0.049 * rng.random()   # total U in [0.95, 0.999)
        w = rng.random(n)
        C = np.maximum(1, (target * w / w.sum() * T).astype(np.int64))
        C = np.minimum(C, 60_000_000)  # A = 1000 C stays within 2^36
        D = np.maximum(C, (T * rng.uniform(0.15, 1.0, n)).astype(np.int64))
        sets.append(list(zip(T.tolist(), D.tolist(), C.tolist())))
    s = _crafted_batch(sets)
    v = _edf_candidate_parity(ctx, s)
    assert v.sum() > 0
