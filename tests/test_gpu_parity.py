"""GPU-vs-oracle parity through the C ABI (bit-exact: the path is integer).

Every comparison is element by element against the CPU oracle on the same
seeded inputs: sizes that span several tiles and ragged tails, the full-size
batching workload, and edge cases (empty sets, 128-task sets, sets rejected by
Lemma 1 / Lemma 2, 1-task sets, extreme WCET parameters).
"""
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


def _edge_batch():
    """Hand-built edge cases: empty set, single tasks, Lemma 1 / Lemma 2
    rejects, a 128-task set, equal (D, T) ties, A = 0 and B = 0 tasks."""
    sets = []
    sets.append(dict(T=[], D=[], A=[], B=[], u=[], ty=[]))
    sets.append(dict(T=[1000], D=[1000], A=[500000], B=[0], u=[500000], ty=[0]))
    sets.append(dict(T=[10], D=[10], A=[2**36 - 1], B=[1], u=[2**32 - 1], ty=[1]))           # Lemma 2 fails
    sets.append(dict(T=[100] * 6, D=[100] * 6, A=[100000 * 20] * 6, B=[0] * 6, u=[20 * 10**6] * 6,
                     ty=[0, 1, 0, 1, 0, 1]))                                                  # Lemma 1 at small M
    sets.append(dict(T=[50, 50, 50, 50], D=[40, 40, 40, 40], A=[0, 0, 1000, 1000], B=[10000, 1, 0, 5000],
                     u=[200000, 1, 20000, 1], ty=[0, 0, 1, 1]))                               # ties, A = 0, B = 0
    rng = np.random.default_rng(5)
    T = rng.integers(1000, 100000, 128)
    sets.append(dict(T=list(T), D=list(T * 3 // 4), A=list(rng.integers(1, 50000, 128) * 1000),
                     B=list(rng.integers(0, 5000, 128)), u=list(rng.integers(0, 10**5, 128)),
                     ty=list(rng.integers(0, 2, 128))))
    off = [0]
    cols = {k: [] for k in ("T", "D", "A", "B", "u_ppm", "type")}
    for s in sets:
        off.append(off[-1] + len(s["T"]))
        cols["T"] += s["T"]
        cols["D"] += s["D"]
        cols["A"] += s["A"]
        cols["B"] += s["B"]
        cols["u_ppm"] += s["u"]
        cols["type"] += s["ty"]
    out = {k: np.array(v, np.uint8 if k == "type" else np.int64) for k, v in cols.items()}
    out["set_off"] = np.array(off, np.int64)
    out["n_max"] = 128
    return out


# ---------------------------------------------------------------- WCET tables

@pytest.mark.parametrize("M,g", [(8, 1), (80, 1), (40, 2), (148, 1), (1024, 4)])
def test_wcet_tables(ctx, M, g):
    s = gpa.gen_tasksets(seed=M + g, nsets=300, n_min=0, n_max=70, U_lo_ppm=100000, U_hi_ppm=9000000)
    Cn, Cc = ctx.build_wcet_tables(gpa.to_device(s), M, g, KC, KM)
    ctx.sync()
    rn, rc = oracle.wcet_tables(s, M, g, KC, KM)
    assert np.array_equal(_np(Cn), rn) and np.array_equal(_np(Cc), rc)


def test_wcet_tables_extreme_parameters(ctx):
    """A + B up to 2^36 and k up to 16000 at every m up to 1024: the
    reciprocal division by 10^6 m is exact over the whole validated range."""
    rng = np.random.default_rng(1)
    n = 128 * 16
    A = rng.integers(0, 2**36, n)
    B = rng.integers(0, 2**36, n)
    A = np.minimum(A, 2**36 - B)
    A[A + B == 0] = 1
    A[:4] = [2**36 - 1, 0, 1, 2**35]
    B[:4] = [1, 2**36, 0, 2**35]
    s = {"set_off": np.arange(0, n + 1, 128, dtype=np.int64), "T": np.full(n, 2**31 - 1, np.int64),
         "D": np.full(n, 2**31 - 1, np.int64), "A": A.astype(np.int64), "B": B.astype(np.int64),
         "u_ppm": np.zeros(n, np.int64), "type": rng.integers(0, 2, n).astype(np.uint8), "n_max": 128}
    for kc, km in ((1000, 1000), (16000, 16000), (1200, 2300)):
        Cn, Cc = ctx.build_wcet_tables(gpa.to_device(s), 1024, 1, kc, km)
        ctx.sync()
        rn, rc = oracle.wcet_tables(s, 1024, 1, kc, km)
        assert np.array_equal(_np(Cn), rn) and np.array_equal(_np(Cc), rc)


# ------------------------------------------------------- explicit candidates

def _single_candidates():
    maps = np.array([[(c >> t) & 1 for t in range(8)] for c in range(256)], np.uint8)
    sizes = np.array([[a, 8 - a] for a in range(1, 8)], np.int32)
    cset = np.zeros(7 * 256, np.int64)
    cmap = np.repeat(maps[None], 7, axis=0).reshape(-1)
    csize = np.repeat(sizes, 256, axis=0).reshape(-1)
    return cset, cmap, csize


def test_single_instance_all_1792_candidates(ctx):
    s = gpa.gen_tasksets(**W.gen_params("single"))
    cset, cmap, csize = _single_candidates()
    v, R = ctx.test_schedulable(gpa.to_device(s), 8, torch.from_numpy(cset).cuda(), torch.from_numpy(cmap).cuda(),
                                torch.from_numpy(csize).cuda(), 8, 2)
    ctx.sync()
    vr, Rr = oracle.test_schedulable(s, 8, 1, KC, KM, cset, cmap, 8, 2, csize)
    assert np.array_equal(_np(v), vr) and np.array_equal(_np(R), Rr)
    assert vr.sum() > 0


@pytest.mark.parametrize("seed", [0, 1])
def test_random_candidates(ctx, seed):
    rng = np.random.default_rng(seed)
    s = gpa.gen_tasksets(seed=20 + seed, nsets=64, n_min=0, n_max=128, U_lo_ppm=100000, U_hi_ppm=8000000,
                         deadline_pm=750, mu_dist="BETA25")
    M, g, k, stride = 96, 2, 5, 128
    nc = 3000
    cset = rng.integers(0, 64, nc).astype(np.int64)
    cmap = rng.integers(0, k, nc * stride).astype(np.uint8)
    csize = (g * rng.integers(0, M // g // 3 + 1, nc * k)).astype(np.int32)
    for with_R in (True, False):
        v, R = ctx.test_schedulable(gpa.to_device(s), M, torch.from_numpy(cset).cuda(), torch.from_numpy(cmap).cuda(),
                                    torch.from_numpy(csize).cuda(), stride, k, g=g, with_R=with_R)
        ctx.sync()
        vr, Rr = oracle.test_schedulable(s, M, g, KC, KM, cset, cmap, stride, k, csize, with_R=with_R)
        assert np.array_equal(_np(v), vr)
        if with_R:
            assert np.array_equal(_np(R), Rr)
    assert 0 < vr.sum() < nc


# ------------------------------------------------------------------ allocate

def _alloc_parity(ctx, s, md, policy, act, linear=True, what=""):
    out = ctx.allocate(gpa.to_device(s), **md, policy=policy, act=act, linear=linear)
    ctx.sync()
    ref = oracle.allocate(s, md["M"], md["g"], md["k_c_pm"], md["k_m_pm"], policy=policy, act=act, linear=linear,
                          nthreads=8)
    _assert_equal(out, ref, ALLOC_KEYS, f"{what} {policy} act={act}")
    return ref


def test_allocate_batch_workload_full_size(ctx):
    """The 100 000-set batching workload, every set, default launch shape."""
    s = gpa.gen_tasksets(**W.gen_params("batch"))
    ref = _alloc_parity(ctx, s, W.model("batch"), "SMS", False, what="batch")
    assert ref["verdict"].sum() > 0


@pytest.mark.parametrize("policy,act", [("SMS", False), ("SMS", True), ("BF", False), ("BF", True)])
def test_allocate_paper_setting_merges(ctx, policy, act):
    """The §7 setting (50 tasks, 68 SMs, U up to 68): the merge loop runs."""
    s = gpa.gen_tasksets(**W.gen_params("paper50", nsets=34 * 4))
    ref = _alloc_parity(ctx, s, W.model("paper50"), policy, act, what="paper50")
    assert ref["n_tests"].sum() > 1000
    assert len(set(ref["reason"].tolist())) >= 3


def test_allocate_binary_merge_search(ctx):
    s = gpa.gen_tasksets(**W.gen_params("paper50", nsets=68))
    _alloc_parity(ctx, s, W.model("paper50"), "SMS", False, linear=False, what="paper50-binary")


def test_allocate_tpc_units_and_small_gpu(ctx):
    s = gpa.gen_tasksets(seed=31, nsets=500, n_min=1, n_max=40, U_lo_ppm=500000, U_hi_ppm=20000000,
                         deadline_pm=750, T_lo=1000, T_hi=100000)
    for md in (dict(M=40, g=2, k_c_pm=KC, k_m_pm=KM), dict(M=16, g=4, k_c_pm=1500, k_m_pm=4000)):
        for policy in ("SMS", "BF"):
            _alloc_parity(ctx, s, md, policy, False, what=f"M={md['M']} g={md['g']}")


def test_allocate_one_gpu_sweep_sample(ctx):
    s = gpa.gen_tasksets(**W.gen_params("sweep", nsets=6000))
    ref = _alloc_parity(ctx, s, W.model("sweep"), "ONE_GPU", False, what="sweep")
    assert 0 < ref["verdict"].sum() < 6000


def test_allocate_edge_cases(ctx):
    s = _edge_batch()
    for M in (1, 3, 68, 1024):
        for policy in ("SMS", "BF", "ONE_GPU"):
            for act in (False, True):
                _alloc_parity(ctx, s, dict(M=M, g=1, k_c_pm=KC, k_m_pm=KM), policy, act, what=f"edge M={M}")


def test_allocate_host_path_equals_device_path(ctx):
    s = gpa.gen_tasksets(**W.gen_params("paper50", nsets=40))
    md = W.model("paper50")
    host = ctx.allocate({k: v for k, v in s.items()}, **md)
    dev = ctx.allocate(gpa.to_device(s), **md)
    ctx.sync()
    for k in ALLOC_KEYS:
        assert np.array_equal(host[k], _np(dev[k])), k


def test_allocate_launch_shapes_graph_and_per_set(ctx):
    """Every launch shape, the CUDA-graph replay and the one-launch-per-set
    form give the same results."""
    s = gpa.gen_tasksets(**W.gen_params("batch", nsets=3000))
    # mix in merge-heavy sets
    p = gpa.gen_tasksets(**W.gen_params("paper50", nsets=34))
    md = W.model("batch")
    ref = oracle.allocate(s, md["M"], md["g"], KC, KM, nthreads=8)
    refp = oracle.allocate(p, 68, 1, KC, KM, nthreads=8)
    d, dp = gpa.to_device(s), gpa.to_device(p)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()  # graph capture needs a non-default stream
    c2 = gpa.Context(0, stream=stream)
    try:
        for stages in (1, 2, 3, 5):
            for warps in (1, 2, 4, 8):
                for chunk in (1, 2, 3, 4, 8):
                    c2.set_option("FAST_STAGES", stages)
                    c2.set_option("FAST_WARPS", warps)
                    c2.set_option("FAST_CHUNK", chunk)
                    c2.set_option("FAST_BLOCKS", 7)
                    out = c2.allocate(d, **md)
                    c2.sync()
                    _assert_equal(out, ref, ALLOC_KEYS, f"shape {stages}x{warps}x{chunk}")
        for k in ("FAST_WARPS", "FAST_CHUNK", "FAST_BLOCKS", "FAST_STAGES"):
            c2.set_option(k, 0)
        c2.set_option("GRAPH", 1)
        for _ in range(3):
            out = c2.allocate(dp, M=68, g=1, k_c_pm=KC, k_m_pm=KM)
            c2.sync()
            _assert_equal(out, refp, ALLOC_KEYS, "graph")
        c2.set_option("GRAPH", 0)
        c2.set_option("AUTOTUNE", 1)
        out = c2.allocate(d, **md)
        c2.sync()
        _assert_equal(out, ref, ALLOC_KEYS, "autotuned")
        c2.set_option("AUTOTUNE", 0)
        c2.set_option("PER_SET_LAUNCH", 1)
        out = c2.allocate(dp, M=68, g=1, k_c_pm=KC, k_m_pm=KM)
        c2.sync()
        _assert_equal(out, refp, ALLOC_KEYS, "per-set")
    finally:
        c2.close()


def _shifted(dev, k, shift):
    """A copy of column k that starts `shift` elements into a fresh buffer
    (so that its base address loses the 16-byte alignment)."""
    v = dev[k]
    buf = torch.empty(v.numel() + shift, dtype=v.dtype, device=v.device)
    buf[shift:].copy_(v)
    return buf[shift:]


@pytest.mark.parametrize("stages", [1, 3])
def test_allocate_odd_task_count_and_unaligned_columns(ctx, stages):
    """Bulk-copied stages: sets that start on odd task indices, an odd task
    count (the last task and the type bytes past the last 16-byte boundary
    are not bulk-copied) and columns whose base addresses are not 16-byte
    aligned (the launcher then reads directly) all match the oracle."""
    s = gpa.gen_tasksets(seed=41, nsets=1501, n_min=1, n_max=33, U_lo_ppm=200000, U_hi_ppm=4000000,
                         deadline_pm=750, T_lo=1000, T_hi=100000)
    if int(s["set_off"][-1]) % 2 == 0:  # make the task count odd: drop the last task
        s = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}
        n_last = int(s["set_off"][-1] - s["set_off"][-2])
        assert n_last > 1
        s["set_off"][-1] -= 1
        for k in ("T", "D", "A", "B", "u_ppm", "type"):
            s[k] = s[k][:-1].copy()
    assert int(s["set_off"][-1]) % 2 == 1
    md = dict(M=80, g=1, k_c_pm=KC, k_m_pm=KM)
    ref = oracle.allocate(s, md["M"], md["g"], KC, KM, nthreads=8)
    d = gpa.to_device(s)
    stream = torch.cuda.Stream()
    c2 = gpa.Context(0, stream=stream)
    try:
        c2.set_option("FAST_STAGES", stages)
        for chunk in (1, 2, 4, 8):
            c2.set_option("FAST_CHUNK", chunk)
            out = c2.allocate(d, **md)
            c2.sync()
            _assert_equal(out, ref, ALLOC_KEYS, f"odd count chunk {chunk}")
        for k, shift in (("T", 1), ("u_ppm", 1), ("type", 1), ("type", 2)):
            d2 = dict(d)
            d2[k] = _shifted(d, k, shift)
            torch.cuda.synchronize()
            out = c2.allocate(d2, **md)
            c2.sync()
            _assert_equal(out, ref, ALLOC_KEYS, f"column {k} shifted by {shift}")
    finally:
        c2.close()


def test_host_input_out_of_bounds_computes_nothing(ctx):
    """A host batch with one task out of bounds: GPA_ERR_RANGE naming that
    set, from the kernels by default and from the check before computation
    with HOST_SLICES = 1, which writes no output; the next valid call works."""
    s = gpa.gen_tasksets(**W.gen_params("batch", nsets=2000))
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}
    bad["D"][int(bad["set_off"][1234]) + 1] = 0
    md = W.model("batch")
    with pytest.raises(gpa.GpaError) as ei:
        ctx.allocate(bad, **md)
    assert ei.value.code == gpa.ERR_RANGE and "1234" in str(ei.value)
    out = ctx.alloc_result(bad)
    for v in out.values():
        if v is not None:
            v.fill(77)
    ctx.set_option("HOST_SLICES", 1)
    try:
        with pytest.raises(gpa.GpaError) as ei:
            ctx.allocate(bad, **md, out=out)
    finally:
        ctx.set_option("HOST_SLICES", 0)
    assert ei.value.code == gpa.ERR_RANGE and "1234" in str(ei.value)
    for k, v in out.items():
        if v is not None:
            assert (v == 77).all(), k
    good = ctx.allocate(s, **md)
    ref = oracle.allocate(s, md["M"], md["g"], KC, KM, nthreads=8)
    _assert_equal(good, ref, ALLOC_KEYS, "after a rejected call")


def test_device_validation_flags_invalid_sets(ctx):
    s = _edge_batch()
    s["D"] = s["D"].copy()
    s["D"][s["set_off"][1]] = s["T"][s["set_off"][1]] + 1  # D > T in set 1
    out = ctx.allocate(gpa.to_device(s), M=68, g=1, k_c_pm=KC, k_m_pm=KM)
    with pytest.raises(gpa.GpaError) as ei:
        ctx.sync()
    assert ei.value.code == gpa.ERR_RANGE
    assert _np(out["reason"])[1] == gpa.REASON["INVALID"]
    assert _np(out["reason"])[0] == gpa.REASON["OK"]
    ctx.sync()  # the flag is cleared
    with pytest.raises(gpa.GpaError) as ei:
        ctx.allocate(s, M=68, g=1, k_c_pm=KC, k_m_pm=KM)  # host path: rejected by the kernels
    assert ei.value.code == gpa.ERR_RANGE


# ------------------------------------------------------- exhaustive optimum

def test_search_best_exhaustive_workload_sample(ctx):
    p = W.WORKLOADS["exhaustive"]
    s = gpa.gen_tasksets(**W.gen_params("exhaustive", nsets=300))
    md = W.model("exhaustive")
    out = ctx.search_best(gpa.to_device(s), **md, kmin=p["kmin"], kmax=p["kmax"])
    ctx.sync()
    ref = oracle.search_best(s, md["M"], md["g"], KC, KM, p["kmin"], p["kmax"], nthreads=8)
    _assert_equal(out, ref, BEST_KEYS, "exhaustive")
    assert ref["feasible"].sum() > 0


def test_search_best_tiny_and_edge(ctx):
    rng = np.random.default_rng(3)
    for trial in range(6):
        kmin = int(rng.integers(1, 3))
        kmax = int(rng.integers(kmin, 9))
        g = int(rng.choice([1, 2]))
        M = g * int(rng.integers(1, 20))
        s = gpa.gen_tasksets(seed=40 + trial, nsets=120, n_min=0, n_max=9, U_lo_ppm=100000, U_hi_ppm=5000000,
                             deadline_pm=750, T_lo=1000, T_hi=100000)
        out = ctx.search_best(gpa.to_device(s), M=M, g=g, k_c_pm=KC, k_m_pm=KM, kmin=kmin, kmax=kmax)
        ctx.sync()
        ref = oracle.search_best(s, M, g, KC, KM, kmin, kmax, nthreads=8)
        _assert_equal(out, ref, BEST_KEYS, f"tiny trial {trial}")


def test_search_best_single_instance_matches_explicit(ctx):
    """The single-instance workload: subset+RGS on the GPU equals the
    oracle's brute force over all 1 792 explicit candidates."""
    s = gpa.gen_tasksets(**W.gen_params("single"))
    out = ctx.search_best(gpa.to_device(s), M=8, g=1, k_c_pm=KC, k_m_pm=KM, kmin=2, kmax=2)
    ctx.sync()
    ref = oracle.search_best(s, 8, 1, KC, KM, 2, 2, explicit=True)
    _assert_equal(out, ref, BEST_KEYS, "single")
