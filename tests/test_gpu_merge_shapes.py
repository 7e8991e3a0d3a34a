"""Launch shapes of the merge and 1G kernels (GPU), the autotuner, and the
interference-term counter.

Every shape computes the same results: the merge kernel with one to eight
warps per task set (a set's candidate merges spread over its warps) and
several sets per CTA, with and without the SMS top-size round, for the 64-,
128- and 256-task builds, both orders (SMS, BF), with and without ACT, the
level-by-level and the binary search of Alg. 2; the 1G kernel with one to
eight warps per CTA.  Each is compared
element by element with the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2105_10312_gb300 as gpa
import paper_2105_10312_gb300.gen as G
from paper_2105_10312_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KC, KM = W.K_C, W.K_M
ALLOC_KEYS = ("verdict", "reason", "n_parts", "Pi", "W", "n_tests", "part_of_task", "size_of_part")
SHAPES = [(1, 1), (1, 2), (1, 4), (2, 2), (2, 4), (4, 4), (4, 8), (8, 8)]  # (warps per set, warps per CTA)


def _assert_equal(got, ref, what):
    for k in ALLOC_KEYS:
        g = got[k].cpu().numpy() if isinstance(got[k], torch.Tensor) else got[k]
        bad = np.flatnonzero(g != ref[k])
        assert bad.size == 0, f"{what}: {k} differs at {bad[:8]}"


def _batch(name, idx):
    s = gpa.gen_tasksets(**W.gen_params(name))
    return G.subset(s, np.asarray(idx))


@pytest.fixture(scope="module")
def batches():
    """Merge-heavy sets of each capacity build: paper50 (64-task build), the
    same setting with 100 tasks (128-task build), paper200 at low U (the
    256-task build; its high-U sets take the oracle minutes)."""
    p50 = _batch("paper50", np.arange(0, 3400, 23))
    p100 = gpa.gen_tasksets(**W.gen_params("paper50", nsets=60, n_min=100, n_max=100, U_steps=12,
                                           U_hi_ppm=24000000))
    p200 = _batch("paper200", [0, 34, 68, 1, 35, 2, 36])
    out = {}
    for name, s in (("p50", p50), ("p100", p100), ("p200", p200)):
        out[name] = s
    return out


@pytest.mark.parametrize("policy,act,linear", [("SMS", False, True), ("SMS", True, True), ("BF", False, True),
                                               ("BF", True, True), ("SMS", False, False), ("BF", False, False)])
def test_merge_shapes_match_the_oracle(ctx, batches, policy, act, linear):
    for name, s in batches.items():
        if name == "p200" and (act or not linear):
            continue  # one set with ACT pairs takes the oracle long; the variants run on the smaller builds
        ref = oracle.allocate(s, 68, 1, KC, KM, policy=policy, act=act, linear=linear, nthreads=8)
        d = gpa.to_device(s)
        for idx, (gw, wpb) in enumerate(SHAPES):
            top = 1 + (idx + len(name)) % 2  # the SMS top-size round off (1) or on (2), alternating
            ctx.set_option("MERGE_GROUP", gw)
            ctx.set_option("MERGE_WARPS", wpb)
            ctx.set_option("MERGE_TOPFIRST", top)
            try:
                out = ctx.allocate(d, 68, 1, KC, KM, policy=policy, act=act, linear=linear)
                ctx.sync()
            finally:
                for k in ("MERGE_GROUP", "MERGE_WARPS", "MERGE_TOPFIRST"):
                    ctx.set_option(k, 0)
            _assert_equal(out, ref, f"{name} {policy} act={act} linear={linear} shape={gw}x{wpb} top={top}")


@pytest.mark.parametrize("sched", ["DM", "EDF"])
def test_merge_shapes_edf_and_small_grids(ctx, batches, sched):
    s = batches["p50"]
    ref = oracle.allocate(s, 68, 1, KC, KM, sched=sched, nthreads=8)
    d = gpa.to_device(s)
    for gw, wpb, blocks in ((2, 4, 1), (8, 8, 3), (1, 1, 5)):
        ctx.set_option("MERGE_GROUP", gw)
        ctx.set_option("MERGE_WARPS", wpb)
        ctx.set_option("MERGE_BLOCKS", blocks)
        try:
            out = ctx.allocate(d, 68, 1, KC, KM, sched=sched)
            ctx.sync()
        finally:
            for k in ("MERGE_GROUP", "MERGE_WARPS", "MERGE_BLOCKS"):
                ctx.set_option(k, 0)
        _assert_equal(out, ref, f"{sched} {gw}x{wpb}x{blocks}")


def test_one_gpu_warps_and_autotuner(ctx):
    s = gpa.gen_tasksets(**W.gen_params("sweep", nsets=6000))
    md = W.model("sweep")
    d = gpa.to_device(s)
    ref1 = oracle.allocate(s, md["M"], 1, KC, KM, policy="ONE_GPU", nthreads=8)
    refh = oracle.allocate(s, md["M"], 1, KC, KM, policy="SMS", nthreads=8)
    for w in (1, 2, 4, 8):
        ctx.set_option("TEST_WARPS", w)
        out = ctx.allocate(d, **md, policy="ONE_GPU")
        ctx.sync()
        _assert_equal(out, ref1, f"1G warps={w}")
    ctx.set_option("TEST_WARPS", 0)
    stream = torch.cuda.Stream()
    c2 = gpa.Context(0, stream=stream)
    try:
        c2.set_option("AUTOTUNE", 1)
        c2.set_option("GRAPH", 1)
        for _ in range(2):
            with torch.cuda.stream(stream):
                o1 = c2.allocate(d, **md, policy="ONE_GPU")
                oh = c2.allocate(d, **md, policy="SMS")
            c2.sync()
            _assert_equal(o1, ref1, "autotuned 1G")
            _assert_equal(oh, refh, "autotuned heuristic")
        p = _batch("paper50", np.arange(0, 3400, 50))
        refp = oracle.allocate(p, 68, 1, KC, KM, nthreads=8)
        with torch.cuda.stream(stream):
            op = c2.allocate(gpa.to_device(p), 68, 1, KC, KM)
        c2.sync()
        _assert_equal(op, refp, "autotuned merges")
    finally:
        c2.close()


def _hand_terms(s, M, g, eps=0.0):
    """Interference terms of the 1G verdict test, by the iteration the warp
    runs: no iteration when a task has C > D or U > 1, when the hyperbolic
    bound prod (1 + C_i / D_i) <= 2 holds, or when the kernel's pre-pass
    settles every task by its response-time upper bound (below);
    otherwise tasks in deadline-monotonic order, and of those only the ones
    whose response-time upper bound (C_i + sum_{j<i} C_j) / (1 - U_hp)
    exceeds D_i, as the kernel rounds it (float32, the same operations in
    the same order).  Up to 16 such tasks are iterated one after another,
    each from the previous one's fixed point plus the WCETs between them
    (task i's step evaluates i terms); each first evaluates f(D_i) and is
    settled if that is at most D_i.  For longer lists (each task's first
    step the same evaluation at D_i), lane l
    starts with the l-th such task i at C_0 + ... + C_i, every lane stepping
    once per round (task i's step evaluates i terms); a lane whose task
    reached its fixed point takes the next unassigned one in lane order,
    starting at the latest iterate of the last task assigned before that
    round plus the WCETs between the two; every start is raised to the
    utilisation bound C_i / (1 - U_hp) (float32 as well); the test stops
    after the round in which some task passed its deadline."""
    import itertools
    import math
    from fractions import Fraction
    T, D, A, B, ty = (np.asarray(s[k], np.int64) for k in ("T", "D", "A", "B", "type"))
    n = len(T)
    order = sorted(range(n), key=lambda i: (D[i], T[i], i))
    nmem = int(ty.sum())
    k = [(KM if nmem >= 2 else 1000) if ty[i] else (KC if n - nmem >= 2 else 1000) for i in range(n)]
    Cr = [-(-(k[i] * (int(A[i]) + int(B[i]) * M)) // (1000000 * M)) for i in range(n)]
    C = [Cr[order[p]] for p in range(n)]
    Dp = [int(D[order[p]]) for p in range(n)]
    Tp = [int(T[order[p]]) for p in range(n)]
    U = sum(Fraction(C[p], Tp[p]) for p in range(n))
    assert abs(U - 1) > Fraction(1, 4096), "too close to 1 for a float-order-free count"
    if any(C[p] > Dp[p] for p in range(n)) or U > 1:
        return 0
    f32 = np.float32

    def quo(x, y):
        # a float quotient as the kernel forms it (within 2 ulp); eps scales
        # it to check that no decision sits at a rounding boundary
        return f32(f32(f32(x) / f32(y)) * f32(1 + eps))

    def util_pass(Ci, chp, uhp, Di):
        u = f32(uhp + f32(2.0 ** -14))
        if not u < 1:
            return False
        return bool(f32(f32(chp + Ci) * f32(1 + 2.0 ** -17)) <= f32(f32(Di) * f32(f32(1) - u)))

    # the kernel's hyperbolic test: prod (1 + C_i / D_i) <= 2 (with a 2^-13
    # margin) settles the set
    hyp = float(np.prod([1 + Fraction(Cr[i], int(D[i])) for i in range(n)]))
    assert abs(hyp - 2 * (1 - 2.0 ** -13)) > 2.0 ** -10, "too close to the hyperbolic threshold"
    if hyp <= 2 * (1 - 2.0 ** -13):
        return 0
    # the kernel's pre-pass: in the original task order, each task's bound
    # with every task whose deadline is at most its own (itself included) as
    # higher priority, float32 sums in index order (its own C / T taken out
    # of the utilisation), else one evaluation at its deadline over the same
    # tasks; all within their deadlines: no iteration
    Tr, Dr = [int(x) for x in T], [int(x) for x in D]
    fr = [quo(Cr[i], Tr[i]) for i in range(n)]
    settled = True
    for i in range(n):
        a, b = f32(0), f32(0)
        for j in range(n):
            if Dr[j] <= Dr[i]:
                a = f32(a + f32(Cr[j]))
                b = f32(b + fr[j])
        u = f32(f32(b - fr[i]) + f32(2.0 ** -14))
        ok = bool(u < 1) and bool(f32(a * f32(1 + 2.0 ** -13)) <= f32(f32(Dr[i]) * f32(f32(1) - u)))
        if not ok:
            # one evaluation at D_i over the same tasks, ceilings from 1 / T_j
            # raised by 2^-19, a fused multiply-add per term
            Dt, cs = f32(Dr[i]), f32(0)
            for j in range(n):
                if Dr[j] <= Dr[i]:
                    rT = f32(quo(1, Tr[j]) * f32(1 + 2.0 ** -19))
                    cs = f32(float(np.ceil(f32(Dt * rT))) * float(f32(Cr[j])) + float(cs))
            ok = bool(f32(cs * f32(1 + 2.0 ** -13)) <= Dt)
        settled = settled and ok
    if settled:
        return 0
    # float sums of C_j / T_j before each task, as the warp forms them:
    # chunks of 32, an inclusive Hillis-Steele scan per chunk plus a carry
    Uex, carry = [f32(0)] * n, f32(0)
    for c0 in range(0, n, 32):
        u = np.array([quo(C[p], Tp[p]) if p < n else f32(0) for p in range(c0, c0 + 32)], np.float32)
        incl = u.copy()
        for o in (1, 2, 4, 8, 16):
            nxt_incl = incl.copy()
            nxt_incl[o:] = incl[o:] + incl[:-o]
            incl = nxt_incl
        for l in range(32):
            if c0 + l < n:
                Uex[c0 + l] = f32(carry + f32(incl[l] - u[l]))
        carry = f32(carry + incl[31])

    def util_start(Ci, uhp):
        u = f32(uhp - f32(2.0 ** -14))
        if u <= 0:
            return Ci
        if u >= 1:
            return 2 ** 32
        b = f32(quo(Ci, f32(f32(1) - u)) * f32(1 - 2.0 ** -20))
        if not b < 2.0 ** 32:
            return 2 ** 32
        return max(int(b), Ci)

    # tasks the utilisation bound settles are never iterated; the others are
    # taken by the lanes in priority order
    Cin = list(itertools.accumulate(C))
    need = [p for p in range(n) if not util_pass(C[p], Cin[p] - C[p], Uex[p], Dp[p])]
    q = len(need)
    if q == 0:
        return 0
    if q <= 16:
        # short lists: one task at a time by the whole warp, each starting at
        # the previous listed task's fixed point plus the WCETs between them
        Rp, Cp, terms = 0, 0, 0
        for i in need:
            R = max(Rp + Cin[i] - Cp, util_start(C[i], Uex[i]))
            if R > Dp[i]:
                return terms
            # one evaluation at D_i first: f(D_i) <= D_i settles the task
            terms += i
            if C[i] + sum(math.ceil(Dp[i] / Tp[j]) * C[j] for j in range(i)) <= Dp[i]:
                Rp, Cp = R, Cin[i]
                continue
            while True:
                if R > Dp[i]:
                    return terms
                terms += i
                step = C[i] + sum(math.ceil(R / Tp[j]) * C[j] for j in range(i))
                if step == R:
                    break
                R = step
            Rp, Cp = R, Cin[i]
        return terms
    lane_task = [need[l] if l < q else -1 for l in range(32)]
    probe = [True] * 32  # a task's first step evaluates f(D_i)
    R = [max(Cin[i], util_start(C[i], Uex[i])) if i >= 0 else 0 for i in lane_task]
    Rcur = [0] * n
    nxt, terms = min(q, 32), 0
    while True:
        miss, conv = False, [False] * 32
        for l in range(32):
            i = lane_task[l]
            if i < 0:
                conv[l] = True
                continue
            if R[l] > Dp[i]:
                miss = True
            elif probe[l]:
                probe[l] = False
                terms += i
                conv[l] = C[i] + sum(math.ceil(Dp[i] / Tp[j]) * C[j] for j in range(i)) <= Dp[i]
            else:
                terms += i
                step = C[i] + sum(math.ceil(R[l] / Tp[j]) * C[j] for j in range(i))
                if step == R[l]:
                    conv[l] = True
                else:
                    R[l] = step
            Rcur[i] = min(R[l], 2**32 - 1)
        if miss:
            return terms
        if nxt >= q and all(conv):
            return terms
        prev = need[nxt - 1]
        rank, nfree = 0, sum(conv)
        for l in range(32):
            if not conv[l]:
                continue
            idx = nxt + rank
            rank += 1
            if idx < q:
                i = need[idx]
                lane_task[l], R[l] = i, max(Rcur[prev] + Cin[i] - Cin[prev], util_start(C[i], Uex[i]))
                probe[l] = True
            else:
                lane_task[l] = -1
        nxt = min(q, nxt + nfree)


def test_term_counter(ctx):
    """The counter of the 1G kernel equals a hand count of the iteration on
    single sets; it is zero when every set is decided by the fast kernel,
    and the same on a repeated call."""
    s = gpa.gen_tasksets(**W.gen_params("sweep", nsets=120))
    counts = []
    for i in (0, 19, 33, 37, 93, 99):
        sub = G.subset(s, np.array([i]))
        ctx.allocate(gpa.to_device(sub), 148, 1, KC, KM, policy="ONE_GPU")
        got = ctx.last_terms()
        cols = {k: sub[k] for k in ("T", "D", "A", "B", "type")}
        counts.append(_hand_terms(cols, 148, 1))
        # the same count with every float quotient 2^-21 off either way: no
        # decision of the set sits at a rounding boundary
        assert _hand_terms(cols, 148, 1, 2.0 ** -21) == counts[-1] == _hand_terms(cols, 148, 1, -(2.0 ** -21)), i
        assert got == counts[-1], i
    assert min(counts) == 0 and sum(c > 0 for c in counts) >= 4, counts  # settled and iterated sets both covered
    b = gpa.gen_tasksets(**W.gen_params("batch", nsets=2000))
    ref = oracle.allocate(b, 80, 1, KC, KM, nthreads=8)
    assert (ref["n_tests"] == 0).all()
    ctx.allocate(gpa.to_device(b), 80, 1, KC, KM)
    assert ctx.last_terms() == 0
    p = gpa.to_device(_batch("paper50", np.arange(0, 3400, 40)))
    ctx.allocate(p, 68, 1, KC, KM)
    t1 = ctx.last_terms()
    ctx.allocate(p, 68, 1, KC, KM)
    assert t1 > 0 and ctx.last_terms() == t1
    ctx.sync()


def test_alu_peak(ctx):
    pk = ctx.measure_alu_peak()
    assert pk["terms"] > 0 and 0.5 < pk["term_ms"] < 100
    props = torch.cuda.get_device_properties(0)
    # at most one term per SM lane and clock (each takes several instructions)
    assert 1e9 < pk["terms_per_s"] < props.multi_processor_count * 128 * 3.0e9
    assert 1e10 < pk["imad_per_s"] < props.multi_processor_count * 256 * 3.0e9
