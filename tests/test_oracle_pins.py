"""Pins of the CPU oracle against facts fixed outside it (no GPU).

Each test checks the oracle against the paper (worked example, constants),
closed forms, textbook scheduling results, brute force on tiny inputs, or an
independent restatement in ``refs.py`` -- never against the oracle itself.
"""
import itertools
import json
import math
import os
import random

import numpy as np
import pytest

import oracle
import refs
from paper_2105_10312_gb300 import gen_tasksets, workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KC, KM = 1200, 2300


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ------------------------------------------------------------ conflict rule

def test_conflict_worked_example():
    """§4.2: 9 compute + 1 memory kernel in one partition -> the memory kernel
    is not in conflict, the 9 compute kernels are (observed through W and R)."""
    g = golden("conflict_example.json")
    types = np.array(g["types"], np.uint8)
    n = len(types)
    for i in range(n):
        u = np.zeros(n, np.int64)
        u[i] = 1
        w = oracle.workload(u, types, np.ones(n, np.uint8), KC, KM)
        k_expected = (KM if types[i] == 1 else KC) if g["in_conflict"][i] else 1000
        assert w == k_expected, (i, w)
    # through the test: the memory kernel at top priority responds in C^n
    T = np.full(n, 10**6, np.int64)
    D = T.copy()
    D[9] = 1000  # highest priority under DM
    A = np.full(n, 7 * 1000, np.int64)
    B = np.zeros(n, np.int64)
    _, R = oracle.rta(T, D, A, B, types, np.ones(n, np.uint8), 1, KC, KM)
    assert R[9] == 7  # k = 1: not inflated
    # a compute kernel sees its own inflated WCET: 7 * 1.2 -> ceil 9 (8.4)
    _, R1 = oracle.rta(T, D, A, B, types, np.array([1, 0, 0, 0, 0, 0, 0, 0, 1, 0], np.uint8), 1, KC, KM)
    assert R1[0] == 9 and R1[8] == 18


def test_conflict_needs_same_type_partner():
    """A lone task of each type is never in conflict (k = 1 for both)."""
    types = np.array([0, 1], np.uint8)
    for i in range(2):
        u = np.zeros(2, np.int64)
        u[i] = 5
        assert oracle.workload(u, types, np.ones(2, np.uint8), KC, KM) == 5000


# ---------------------------------------------------------------- WCET model

def test_oracle_refuses_exactly_the_tasks_outside_the_input_bounds():
    """The library's documented input bounds (1 <= D <= T <= 2^31 - 1,
    A, B >= 0, 1 <= A + B <= 2^36, 0 <= u_ppm < 2^32, type in {0, 1}): a
    one-task set at each bound is decided, and one a unit beyond it is
    marked invalid (reason 5), as the kernels mark it."""
    base = dict(T=1000, D=1000, A=1000, B=0, u_ppm=1000, type=0)
    inside = [dict(D=1), dict(T=2**31 - 1, D=2**31 - 1), dict(A=2**36), dict(A=0, B=2**36), dict(A=1),
              dict(A=0, B=1), dict(A=2**35, B=2**35), dict(u_ppm=2**32 - 1), dict(u_ppm=0), dict(type=1)]
    outside = [dict(D=0), dict(D=1001), dict(T=2**31, D=2**31), dict(A=0, B=0), dict(A=2**36, B=1),
               dict(A=-1, B=5), dict(B=-1), dict(u_ppm=2**32), dict(u_ppm=-1), dict(type=2)]
    cases = [dict(base, **c) for c in inside + outside]
    s = {k: np.array([c[k] for c in cases], np.uint8 if k == "type" else np.int64)
         for k in ("T", "D", "A", "B", "u_ppm", "type")}
    s["set_off"] = np.arange(len(cases) + 1, dtype=np.int64)
    s["n_max"] = 1
    r = oracle.allocate(s, 8, 1, KC, KM, policy="ONE_GPU")
    assert [int(x) != 5 for x in r["reason"]] == [True] * len(inside) + [False] * len(outside), r["reason"]


def test_oracle_refuses_exactly_the_models_outside_the_bounds():
    """The documented model bounds (1 <= g, g | M, 1 <= M <= 1024, 1000 <=
    k_c, k_m <= 16000): accepted at each bound, refused one step beyond."""
    s = gen_tasksets(seed=3, nsets=4, n_min=1, n_max=4, U_lo_ppm=100000, U_hi_ppm=900000, deadline_pm=750)
    for M, g, kc, km in ((1, 1, 1000, 1000), (1024, 1, 16000, 16000), (1024, 1024, 1000, 16000), (12, 4, 1200, 2300)):
        oracle.allocate(s, M, g, kc, km)
    for M, g, kc, km in ((0, 1, 1200, 2300), (1025, 1, 1200, 2300), (12, 5, 1200, 2300), (12, 0, 1200, 2300),
                         (12, 1, 999, 2300), (12, 1, 1200, 999), (12, 1, 16001, 2300), (12, 1, 1200, 16001)):
        with pytest.raises(RuntimeError):
            oracle.allocate(s, M, g, kc, km)


def test_model_constants_golden():
    g = golden("model_constants.json")
    p = workloads.gen_params("paper50")
    assert p["beta_c_pm"] == g["beta_compute_pm"] and p["beta_m_pm"] == g["beta_memory_pm"]
    assert workloads.K_C == g["k_compute_pm"] and workloads.K_M == g["k_memory_pm"]
    assert p["deadline_pm"] == g["deadline_pm"] and p["prm_pm"] == g["prm_pm"]
    assert (p["T_lo"], p["T_hi"]) == (g["period_lo"], g["period_hi"])
    assert workloads.model("paper50")["M"] == g["M"]


def test_wcet_alpha_form_matches_rational_closed_form():
    rng = random.Random(1)
    for _ in range(3000):
        C1 = rng.choice([1, 2, 3, 999, 1000, 12345, rng.randrange(1, 1 << 26)])
        alpha = rng.randrange(0, 1001)
        k = rng.choice([1000, 1200, 2300, rng.randrange(1000, 16001)])
        m = rng.randrange(1, 1025)
        A, B = C1 * (1000 - alpha), C1 * alpha
        assert oracle.wcet(A, B, k, m) == refs.wcet_alpha(C1, alpha, k, m)


def test_wcet_paper_form_matches_rational_closed_form():
    rng = random.Random(2)
    for _ in range(3000):
        a = rng.randrange(1, 1 << 25)
        beta = rng.choice([20, 100])
        k = rng.choice([1000, 1200, 2300])
        m = rng.randrange(1, 69)
        assert oracle.wcet(1000 * a, beta * a, k, m) == refs.wcet_paper(a, beta, k, m)


def test_wcet_properties():
    """No timing anomaly (§4.1): non-increasing in m; m C^n(m) >= C^n(1)
    (Lemma 1's basis); inflation never shrinks the WCET; C(1) = C1 in the
    serial-fraction form."""
    rng = random.Random(3)
    for _ in range(300):
        C1 = rng.randrange(1, 1 << 22)
        alpha = rng.randrange(0, 1001)
        A, B = C1 * (1000 - alpha), C1 * alpha
        prev = None
        c1 = oracle.wcet(A, B, 1000, 1)
        assert c1 == C1
        for m in range(1, 150, 7):
            c = oracle.wcet(A, B, 1000, m)
            assert m * c >= c1
            assert oracle.wcet(A, B, 2300, m) >= oracle.wcet(A, B, 1200, m) >= c
            if prev is not None:
                assert c <= prev
            prev = c


def test_wcet_tables_layout():
    s = gen_tasksets(seed=11, nsets=5, n_min=0, n_max=7)
    Cn, Cc = oracle.wcet_tables(s, 12, 3, KC, KM)
    off = s["set_off"]
    Mu = 4
    for si in range(5):
        o, n = off[si], off[si + 1] - off[si]
        for mi in range(Mu):
            for t in range(n):
                m = 3 * (mi + 1)
                k = KM if s["type"][o + t] else KC
                assert Cn[o * Mu + mi * n + t] == refs.wcet_alpha(s["C1"][o + t], s["alpha_pm"][o + t], 1000, m)
                assert Cc[o * Mu + mi * n + t] == refs.wcet_alpha(s["C1"][o + t], s["alpha_pm"][o + t], k, m)


# ------------------------------------------------- per-partition test (§5.5)

def _no_inflation_set(rng, n, periods):
    T = np.array([rng.choice(periods) for _ in range(n)], np.int64)
    D = np.array([rng.randrange(max(1, t // 2), t + 1) for t in T], np.int64)
    C = np.array([rng.randrange(1, max(2, t // 3)) for t in T], np.int64)
    return T, D, C


def test_rta_matches_fixed_priority_simulation():
    """Response times equal the first job's completion in a unit-step FP
    schedule with synchronous release; misses match; for tasks that meet
    their deadline every job in the hyperperiod responds within R."""
    rng = random.Random(4)
    periods = [4, 5, 6, 8, 10, 12, 15, 20, 24, 30]
    checked_miss = checked_ok = 0
    for trial in range(400):
        n = rng.randrange(1, 6)
        T, D, C = _no_inflation_set(rng, n, periods)
        # A = 1000 C, B = 0 -> C^n(1) = C; k = 1000 everywhere: no inflation
        A, B = 1000 * C, np.zeros(n, np.int64)
        typ = np.array([i % 2 for i in range(n)], np.uint8)
        v, R = oracle.rta(T, D, A, B, typ, np.ones(n, np.uint8), 1, 1000, 1000)
        order = refs.dm_order(T, D, range(n))
        H = 1
        for t in T:
            H = H * int(t) // math.gcd(H, int(t))
        first, worst = refs.simulate_fp([(int(T[i]), int(D[i]), int(C[i])) for i in order], H + int(D.max()) + 1)
        for rank, i in enumerate(order):
            if R[i] >= 0:
                checked_ok += 1
                assert first[rank] == R[i], (trial, i)
                assert worst[rank] <= R[i]
                assert R[i] <= D[i]
            else:
                checked_miss += 1
                assert first[rank] is None or first[rank] > D[i], (trial, i)
        assert v == int((R >= 0).all())
    assert checked_ok > 200 and checked_miss > 50


def test_rta_harmonic_rm_utilisation_bound():
    """Harmonic periods, implicit deadlines (RM = DM): schedulable iff U <= 1."""
    rng = random.Random(5)
    for trial in range(300):
        n = rng.randrange(1, 7)
        base = rng.choice([1, 2, 3, 5])
        T = np.array([base * 2 ** rng.randrange(0, 6) for _ in range(n)], np.int64)
        C = np.array([rng.randrange(1, int(t) + 1) for t in T], np.int64)
        U = sum(__import__("fractions").Fraction(int(c), int(t)) for c, t in zip(C, T))
        v, _ = oracle.rta(T, T.copy(), 1000 * C, np.zeros(n, np.int64), np.zeros(n, np.uint8),
                          np.ones(n, np.uint8), 1, 1000, 1000)
        assert v == int(U <= 1), (trial, U)


def test_rta_single_task_is_its_wcet():
    rng = random.Random(6)
    for _ in range(200):
        C1 = rng.randrange(1, 10**6)
        alpha = rng.randrange(0, 1001)
        T = rng.randrange(1, 2**31 - 1)
        m = rng.randrange(1, 200)
        c = refs.wcet_alpha(C1, alpha, 1000, m)
        v, R = oracle.rta(np.array([T]), np.array([T]), np.array([C1 * (1000 - alpha)]), np.array([C1 * alpha]),
                          np.zeros(1, np.uint8), np.ones(1, np.uint8), m, KC, KM)
        assert (R[0] == c) if c <= T else (R[0] == -1)
        assert v == int(c <= T)


def test_rta_monotone_in_m_and_in_tasks():
    """No timing anomalies: passing at m implies passing at every m' > m;
    removing a task never breaks a passing partition."""
    s = gen_tasksets(seed=7, nsets=60, n_min=2, n_max=7, U_lo_ppm=300000, U_hi_ppm=3000000, deadline_pm=750)
    off = s["set_off"]
    for si in range(60):
        o, e = off[si], off[si + 1]
        args = [s[k][o:e] for k in ("T", "D", "A", "B", "type")]
        n = e - o
        allin = np.ones(n, np.uint8)
        res = [oracle.rta(*args, allin, m, KC, KM)[0] for m in range(1, 40)]
        assert all(res[j] <= res[j + 1] for j in range(len(res) - 1))
        for m in (1, 4, 16, 39):
            if oracle.rta(*args, allin, m, KC, KM)[0]:
                for drop in range(n):
                    sub = allin.copy()
                    sub[drop] = 0
                    assert oracle.rta(*args, sub, m, KC, KM)[0] == 1


# ------------------------------------------ EDF, the second per-partition policy

def _edf(T, D, C):
    """The oracle's EDF verdict for tasks with WCET C (k = 1, m = 1)."""
    n = len(T)
    return oracle.edf(np.asarray(T, np.int64), np.asarray(D, np.int64), 1000 * np.asarray(C, np.int64),
                      np.zeros(n, np.int64), np.zeros(n, np.uint8), np.ones(n, np.uint8), 1, 1000, 1000)


def _hyperperiod(T):
    H = 1
    for t in T:
        H = H * int(t) // math.gcd(H, int(t))
    return H


def test_edf_matches_edf_simulation():
    """Processor-demand verdicts equal a unit-step EDF schedule simulated
    over two hyperperiods (synchronous release, constrained deadlines), over
    the whole range of U, U = 1 included: random sets, and sets whose WCETs
    are completed so that U is exactly 1."""
    from fractions import Fraction
    rng = random.Random(41)
    periods = [3, 4, 5, 6, 8, 10, 12, 15, 20]
    ok = miss = at_one = 0
    for trial in range(900):
        n = rng.randrange(1, 6)
        T = [rng.choice(periods) for _ in range(n)]
        D = [rng.randrange(max(1, t // 3), t + 1) for t in T]
        C = [rng.randrange(1, max(2, (2 * t) // n)) for t in T]
        if trial % 3 == 0 and n >= 2:
            # complete the last WCET so that U = 1 exactly, when that is possible
            rest = 1 - sum(Fraction(c, t) for c, t in zip(C[:-1], T[:-1]))
            last = rest * T[-1]
            if rest > 0 and last.denominator == 1 and 1 <= last <= T[-1]:
                C[-1] = int(last)
        U = sum(Fraction(c, t) for c, t in zip(C, T))
        v = _edf(T, D, C)
        sim = refs.simulate_edf(list(zip(T, D, C)), 2 * _hyperperiod(T) + max(D) + 1)
        assert v == int(sim), (trial, T, D, C)
        ok += v
        miss += 1 - v
        at_one += U == 1
    assert ok > 150 and miss > 150 and at_one > 40


def test_both_tests_inflate_by_the_conflict_factors():
    """§4.2 inside the per-partition tests: with both task types present and
    factors above 1000, at several partition sizes m, the DM response times
    equal the first jobs' completions in a fixed-priority schedule, and the
    EDF verdict an EDF schedule, of the WCETs C_i(m) inflated by the
    conflict rule (restated in refs.conflict_k)."""
    rng = random.Random(57)
    periods = [4, 5, 6, 8, 10, 12, 15, 20]
    kc, km = 1500, 2500
    cnt = dict(dm_ok=0, dm_miss=0, edf_ok=0, edf_miss=0, inflated=0)
    for trial in range(500):
        n = rng.randrange(2, 6)
        m = rng.randrange(1, 5)
        T = [rng.choice(periods) for _ in range(n)]
        D = [rng.randrange(max(1, t // 2), t + 1) for t in T]
        typ = [rng.randrange(2) for _ in range(n)]
        A = [rng.randrange(1000, 3000 * m) for _ in range(n)]
        B = [rng.randrange(0, 1000) for _ in range(n)]
        C = [oracle.wcet(A[i], B[i], refs.conflict_k(typ, range(n), i, kc, km), m) for i in range(n)]
        cnt["inflated"] += C != [oracle.wcet(A[i], B[i], 1000, m) for i in range(n)]
        args = (np.array(T, np.int64), np.array(D, np.int64), np.array(A, np.int64), np.array(B, np.int64),
                np.array(typ, np.uint8), np.ones(n, np.uint8), m, kc, km)
        horizon = _hyperperiod(T) + max(D) + 1
        v, R = oracle.rta(*args)
        order = refs.dm_order(T, D, range(n))
        first, _ = refs.simulate_fp([(T[i], D[i], C[i]) for i in order], horizon)
        for rank, i in enumerate(order):
            if R[i] >= 0:
                assert first[rank] == R[i], (trial, T, D, C, i)
            else:
                assert first[rank] is None or first[rank] > D[i], (trial, T, D, C, i)
        cnt["dm_ok" if v else "dm_miss"] += 1
        ve = oracle.edf(*args)
        assert ve == int(refs.simulate_edf(list(zip(T, D, C)), 2 * _hyperperiod(T) + max(D) + 1)), (trial, T, D, C)
        cnt["edf_ok" if ve else "edf_miss"] += 1
    assert min(cnt.values()) > 50, cnt


def test_edf_exact_at_utilisation_one():
    """U is compared with 1 exactly: with D = T a set passes iff U <= 1, at
    U = 1 exactly and one unit of C either side of it, for harmonic pairs,
    for 1/3 + 2/3 (whose 2^64-scaled terms straddle 1), and for pairs of
    large coprime periods, where U - 1 is a multiple of 1 / (T1 T2)."""
    from fractions import Fraction
    cases = [([3, 3], [1, 2]), ([1000003, 2000006], [600001, 800004]), ([7, 14, 28], [3, 4, 8])]
    # large coprime periods: C2 chosen so that U straddles 1 by one unit
    T1, T2 = 1329, 1048573
    for C1 in (1, 664, 1328):
        C2 = (T2 * (T1 - C1)) // T1  # U <= 1 with the largest such C2
        cases.append(([T1, T2], [C1, C2]))
        cases.append(([T1, T2], [C1, C2 + 1]))
    seen = [0, 0, 0]  # below 1, at 1, above 1
    for T, C in cases:
        for dc in (-1, 0, 1):
            CC = list(C[:-1]) + [C[-1] + dc]
            if not 1 <= CC[-1] <= T[-1]:
                continue
            U = sum(Fraction(c, t) for c, t in zip(CC, T))
            assert _edf(T, T, CC) == int(U <= 1), (T, CC, U)
            seen[(U > 1) - (U < 1) + 1] += 1
    assert min(seen) >= 3


def test_edf_implicit_deadlines_utilisation_bound():
    """Liu & Layland: with D = T, EDF meets every deadline iff U <= 1."""
    from fractions import Fraction
    rng = random.Random(42)
    seen = [0, 0]
    for trial in range(400):
        n = rng.randrange(2, 9)
        T = np.array([rng.randrange(10, 100000) for _ in range(n)], np.int64)
        C = np.array([rng.randrange(1, int(t) * 8 // (5 * n) + 1) for t in T], np.int64)
        U = sum(Fraction(int(c), int(t)) for c, t in zip(C, T))
        v = _edf(T, T, C)
        assert v == int(U <= 1), (trial, U)
        seen[int(U <= 1)] += 1
    assert min(seen) > 50


def test_edf_dominates_dm_and_is_monotone():
    """EDF is optimal on one processor: a DM-schedulable partition passes the
    EDF test; the EDF test is monotone in m and in the
    task set, like the DM test (no timing anomalies)."""
    s = gen_tasksets(seed=43, nsets=80, n_min=2, n_max=8, U_lo_ppm=300000, U_hi_ppm=4000000, deadline_pm=750,
                     T_lo=1000, T_hi=100000)
    off = s["set_off"]
    dm_ok = strict = 0
    for si in range(80):
        o, e = off[si], off[si + 1]
        args = [s[k][o:e] for k in ("T", "D", "A", "B", "type")]
        n = e - o
        allin = np.ones(n, np.uint8)
        ed = [oracle.edf(*args, allin, m, KC, KM) for m in range(1, 30)]
        dm = [oracle.rta(*args, allin, m, KC, KM)[0] for m in range(1, 30)]
        assert all(ed[j] <= ed[j + 1] for j in range(len(ed) - 1))
        for a, b in zip(dm, ed):
            if a:
                dm_ok += 1
                assert b == 1
            strict += b and not a
        for m in (2, 8, 29):
            if oracle.edf(*args, allin, m, KC, KM):
                for drop in range(n):
                    sub = allin.copy()
                    sub[drop] = 0
                    assert oracle.edf(*args, sub, m, KC, KM) == 1
    assert dm_ok > 200 and strict > 0


def test_edf_single_task_and_minm():
    """One task passes iff C <= D (the same as Lemma 2); the EDF minimum size
    of a singleton is the Lemma 2 size, and of a set never above the DM one."""
    rng = random.Random(44)
    for _ in range(300):
        C1 = rng.randrange(1, 10**6)
        alpha = rng.randrange(0, 1001)
        T = rng.randrange(1, 2**31 - 1)
        D = rng.randrange(1, T + 1)
        m = rng.randrange(1, 200)
        c = refs.wcet_alpha(C1, alpha, 1000, m)
        v = oracle.edf(np.array([T]), np.array([D]), np.array([C1 * (1000 - alpha)]), np.array([C1 * alpha]),
                       np.zeros(1, np.uint8), np.ones(1, np.uint8), m, KC, KM)
        assert v == int(c <= D)
    s = gen_tasksets(seed=45, nsets=40, n_min=1, n_max=6, U_lo_ppm=300000, U_hi_ppm=5000000, deadline_pm=750,
                     T_lo=1000, T_hi=100000)
    for si in range(40):
        v, o, n = _set_view(s, si)
        mask = np.ones(n, np.uint8)
        me = oracle.minm(v["T"], v["D"], v["A"], v["B"], v["type"], mask, 1, 64, 1, KC, KM, sched="EDF")
        md = oracle.minm(v["T"], v["D"], v["A"], v["B"], v["type"], mask, 1, 64, 1, KC, KM)
        assert me == oracle.minm(v["T"], v["D"], v["A"], v["B"], v["type"], mask, 1, 64, 1, KC, KM, linear=False,
                                 sched="EDF")
        if md:
            assert 1 <= me <= md
        if n == 1:
            assert me == md


# ------------------------------------------------------------------- Lemmas

def test_lemma2_singleton_size_closed_form():
    """Lemma 2: smallest m with C^n(m) <= D; checked against the algebraic
    form A <= m (1000 D - B) rounded up to the unit g."""
    rng = random.Random(8)
    for _ in range(1500):
        C1 = rng.randrange(1, 10**6)
        alpha = rng.randrange(0, 1001)
        T = rng.randrange(1, 10**6)
        D = rng.randrange(1, T + 1)
        g = rng.choice([1, 2, 4])
        M = g * rng.randrange(1, 100)
        A, B = C1 * (1000 - alpha), C1 * alpha
        den = 1000 * D - B
        if den < 0 or (den == 0 and A > 0):
            expect = 0
        else:
            m1 = 1 if A == 0 else max(1, -(-A // den))
            mg = -(-m1 // g) * g
            expect = mg if mg <= M else 0
        got = oracle.minm([T], [D], [A], [B], [0], [1], g, M, g, KC, KM, linear=True)
        assert got == expect


def test_merge_search_linear_equals_binary():
    """Alg. 2's linear scan and the §5.2 binary search give the same size."""
    s = gen_tasksets(seed=9, nsets=80, n_min=2, n_max=8, U_lo_ppm=500000, U_hi_ppm=6000000, deadline_pm=750)
    off = s["set_off"]
    rng = random.Random(9)
    for si in range(80):
        o, e = off[si], off[si + 1]
        n = e - o
        args = [s[k][o:e] for k in ("T", "D", "A", "B", "type")]
        for _ in range(5):
            mask = np.array([rng.random() < 0.6 for _ in range(n)], np.uint8)
            if not mask.any():
                continue
            g = rng.choice([1, 2])
            lo = g * rng.randrange(1, 10)
            hi = lo + g * rng.randrange(0, 30)
            a = oracle.minm(*args, mask, lo, hi, g, KC, KM, linear=True)
            b = oracle.minm(*args, mask, lo, hi, g, KC, KM, linear=False)
            assert a == b
            if a:
                assert oracle.rta(*args, mask, a, KC, KM)[0] == 1
                if a > lo:
                    assert oracle.rta(*args, mask, a - g, KC, KM)[0] == 0


def test_lemma1_utilisation_bound():
    """Lemma 1 (necessary condition): a set whose total single-SM
    utilisation exceeds M has no schedulable partition of M SMs.  Pinned at
    the exact boundary (U = M passes, a hair above fails) and against the
    exhaustive search: whenever Lemma 1 rejects, no allocation is feasible."""
    for M in range(1, 7):
        for n, want in ((M, False), (M + 1, True)):
            T = [1000] * n
            A = [1000 * 1000] * n  # C^n(1) = 1000 = T: utilisation exactly 1 per task
            assert oracle.lemma1_rejects(T, A, [0] * n, M) == want, (M, n)
        T = [997, 1000]
        A = [1000 * 997 * M, 1000]  # U = M + 1/1000 in total
        assert oracle.lemma1_rejects(T, A, [0, 0], M)
    s = gen_tasksets(seed=10, nsets=120, n_min=2, n_max=6, U_lo_ppm=1000000, U_hi_ppm=9000000, deadline_pm=1000,
                     T_lo=1000, T_hi=100000)
    M, rejected = 6, 0
    r = oracle.search_best(s, M, 1, KC, KM, 1, 6)
    for si in range(120):
        v, o, n = _set_view(s, si)
        if oracle.lemma1_rejects(v["T"], v["A"], v["B"], M):
            rejected += 1
            assert r["feasible"][si] == 0, si
    assert rejected > 20


# ------------------------------------------------------ heuristic (Alg. 1-3)

def _set_view(s, si):
    o, e = s["set_off"][si], s["set_off"][si + 1]
    return {k: s[k][o:e] for k in ("T", "D", "A", "B", "u_ppm", "type")}, o, e - o


def _partitions_from(r, si, o, n):
    parts = {}
    for t in range(n):
        parts.setdefault(int(r["part_of_task"][o + t]), set()).add(t)
    sizes = [int(r["size_of_part"][o + p]) for p in range(r["n_parts"][si])]
    return parts, sizes


@pytest.mark.parametrize("policy,act,sched", [("SMS", False, "DM"), ("SMS", True, "DM"), ("BF", False, "DM"),
                                              ("BF", True, "DM"), ("SMS", False, "EDF"), ("BF", True, "EDF")])
def test_heuristic_matches_independent_restatement(policy, act, sched):
    """Alg. 1-3 restated over Python sets reaches the same final partitions,
    the same verdict and the same number of merge evaluations (under either
    per-partition policy)."""
    M, g = 12, 1
    s = gen_tasksets(seed=12, nsets=50, n_min=3, n_max=9, U_lo_ppm=1000000, U_hi_ppm=12000000, deadline_pm=750,
                     T_lo=50, T_hi=4000, T_dist="LIST", mode="PAPER")
    r = oracle.allocate(s, M, g, KC, KM, policy=policy, act=act, sched=sched)
    seen_merges = 0
    for si in range(50):
        v, o, n = _set_view(s, si)
        if oracle.lemma1_rejects(v["T"], v["A"], v["B"], M):
            assert r["reason"][si] == oracle.REASON["LEMMA1"]
            continue

        def single(i):
            return oracle.minm(v["T"], v["D"], v["A"], v["B"], v["type"], np.eye(n, dtype=np.uint8)[i], g, M, g,
                               KC, KM, sched=sched)

        def test_min(S, lo, hi):
            mask = np.array([i in S for i in range(n)], np.uint8)
            return oracle.minm(v["T"], v["D"], v["A"], v["B"], v["type"], mask, lo, hi, g, KC, KM, sched=sched)

        def W(S):
            return sum(refs.conflict_k(v["type"], S, i, KC, KM) * int(v["u_ppm"][i]) for i in S)

        status, parts, tests = refs.heuristic(n, [int(x) for x in v["u_ppm"]], M, g, single, test_min,
                                              policy=policy, act=act, W=W)
        assert oracle.REASON[status] == r["reason"][si], si
        assert tests == r["n_tests"][si], si
        if status == "LEMMA2":
            continue
        seen_merges += tests
        got, sizes = _partitions_from(r, si, o, n)
        want = sorted((sorted(P), z) for P, z in parts.items())
        have = sorted((sorted(got[p]), sizes[p]) for p in got)
        assert want == have, si
        assert r["Pi"][si] == sum(parts.values())
        assert r["W"][si] == sum(W(P) for P in parts)
    assert seen_merges > 50


def test_heuristic_invariants_paper_workload():
    """On the paper's setting: success => Lemma 3 (Pi <= M), every partition
    passes at its size, that size is its minimum (a merge never lands above
    the smallest passing size), partitions cover every task exactly once,
    and Lemma 1 passes."""
    p = workloads.gen_params("paper50", nsets=68)
    s = gen_tasksets(**p)
    md = workloads.model("paper50")
    r = oracle.allocate(s, md["M"], md["g"], KC, KM, policy="SMS", act=False, nthreads=4)
    n_ok = 0
    for si in range(68):
        v, o, n = _set_view(s, si)
        if r["reason"][si] in (oracle.REASON["LEMMA1"], oracle.REASON["LEMMA2"]):
            continue
        parts, sizes = _partitions_from(r, si, o, n)
        assert sorted(t for P in parts.values() for t in P) == list(range(n))
        assert sum(sizes) == r["Pi"][si]
        for p_, P in parts.items():
            mask = np.array([i in P for i in range(n)], np.uint8)
            z = sizes[p_]
            assert z >= 1 and oracle.rta(v["T"], v["D"], v["A"], v["B"], v["type"], mask, z, KC, KM)[0] == 1
            assert oracle.minm(v["T"], v["D"], v["A"], v["B"], v["type"], mask, 1, md["M"], 1, KC, KM) == z
        if r["verdict"][si]:
            n_ok += 1
            assert r["Pi"][si] <= md["M"]
            assert not oracle.lemma1_rejects(v["T"], v["A"], v["B"], md["M"])
        else:
            assert r["Pi"][si] > md["M"]
    assert n_ok > 10


def test_one_gpu_is_the_whole_set_at_M():
    """§7.2's baseline: the whole set as one partition of all M SMs.  The
    verdict is the (separately pinned) test at M; the workload is Def. 4's
    sum of k_i u_i written out from the §4.2 conflict rule (k_i is the
    type's factor when the set holds at least two tasks of that type, else
    1000); every task sits in part 0 of size M; one test per set; an empty
    set is decided schedulable with no partition."""
    s = gen_tasksets(seed=13, nsets=60, n_min=0, n_max=20, U_lo_ppm=100000, U_hi_ppm=6000000, deadline_pm=750,
                     mu_dist="BETA25")
    M = 148
    r = oracle.allocate(s, M, 1, KC, KM, policy="ONE_GPU")
    empty = nonempty = 0
    for si in range(60):
        v, o, n = _set_view(s, si)
        assert r["n_tests"][si] == 1
        if n == 0:
            empty += 1
            assert r["verdict"][si] == 1 and r["reason"][si] == 0
            assert r["n_parts"][si] == 0 and r["Pi"][si] == 0 and r["W"][si] == 0
            continue
        nonempty += 1
        ok, _ = oracle.rta(v["T"], v["D"], v["A"], v["B"], v["type"], np.ones(n, np.uint8), M, KC, KM)
        assert r["verdict"][si] == ok
        assert r["reason"][si] == (0 if ok else 4)  # GPA_REASON_OK / GPA_REASON_TEST
        assert r["n_parts"][si] == 1 and r["Pi"][si] == M
        typ = [int(t) for t in v["type"]]
        factor = {0: KC if typ.count(0) >= 2 else 1000, 1: KM if typ.count(1) >= 2 else 1000}
        assert r["W"][si] == sum(factor[t] * int(u) for t, u in zip(typ, v["u_ppm"]))
        assert (r["part_of_task"][o:o + n] == 0).all()
        assert r["size_of_part"][o] == M and (r["size_of_part"][o + 1:o + n] == 0).all()
    assert empty > 0 and nonempty > 40


# ------------------------------------------------------- exhaustive optimum

@pytest.mark.parametrize("sched", ["DM", "EDF"])
def test_exhaustive_explicit_equals_subset_form_and_bruteforce(sched):
    rng = random.Random(14)
    for trial in range(25):
        n = rng.randrange(1, 6)
        g = rng.choice([1, 2])
        M = g * rng.randrange(2, 5)
        kmin = rng.randrange(1, 3)
        kmax = rng.randrange(kmin, 4)
        s = gen_tasksets(seed=100 + trial, nsets=1, n_min=n, n_max=n, U_lo_ppm=300000, U_hi_ppm=2500000,
                         deadline_pm=750, T_lo=1000, T_hi=100000)
        a = oracle.search_best(s, M, g, KC, KM, kmin, kmax, explicit=False, sched=sched)
        b = oracle.search_best(s, M, g, KC, KM, kmin, kmax, explicit=True, sched=sched)
        for k in ("feasible", "W", "sum_minm", "n_blocks", "spare", "rgs", "minm_block"):
            assert np.array_equal(a[k], b[k]), (trial, k)
        v, o, _ = _set_view(s, 0)

        def passes(S, m):
            mask = np.array([i in S for i in range(n)], np.uint8)
            if sched == "EDF":
                return oracle.edf(v["T"], v["D"], v["A"], v["B"], v["type"], mask, m, KC, KM) == 1
            return oracle.rta(v["T"], v["D"], v["A"], v["B"], v["type"], mask, m, KC, KM)[0] == 1

        def minsize(S):
            for m in range(g, M + 1, g):
                if passes(S, m):
                    return m
            return 0

        def W(S):
            return sum(refs.conflict_k(v["type"], S, i, KC, KM) * int(v["u_ppm"][i]) for i in S)

        best = refs.exhaustive_bruteforce(n, M, g, kmin, kmax, passes, minsize, W)
        assert bool(a["feasible"][0]) == (best is not None)
        if best is not None:
            assert (a["W"][0], a["sum_minm"][0], tuple(a["rgs"][:n])) == best
            # the outputs derived from the optimum, as the header defines them
            nb = int(max(a["rgs"][:n])) + 1
            assert a["n_blocks"][0] == nb
            sizes = [minsize([i for i in range(n) if a["rgs"][i] == b]) for b in range(nb)]
            assert list(a["minm_block"][:kmax]) == sizes + [0] * (kmax - nb)
            assert a["spare"][0] == M - sum(sizes) - max(0, kmin - nb) * g


def test_explicit_candidate_count_single_workload():
    """7 SM splits x 2^8 maps = 1 792 explicit candidates for one 8-task set on
    8 SMs in exactly 2 partitions."""
    s = gen_tasksets(**workloads.gen_params("single"))
    r = oracle.search_best(s, 8, 1, KC, KM, 2, 2, explicit=True)
    assert r["candidates"] == math.comb(7, 1) * 2**8 == 1792


def test_exhaustive_removal_never_breaks_feasibility():
    s = gen_tasksets(seed=15, nsets=30, n_min=2, n_max=7, U_lo_ppm=500000, U_hi_ppm=4000000, deadline_pm=750,
                     T_lo=1000, T_hi=100000)
    M, g, kmin, kmax = 12, 2, 1, 3
    full = oracle.search_best(s, M, g, KC, KM, kmin, kmax)
    off = s["set_off"]
    for si in range(30):
        if not full["feasible"][si]:
            continue
        o, e = off[si], off[si + 1]
        for drop in range(e - o):
            keep = [t for t in range(o, e) if t != o + drop]
            sub = {k: s[k][keep] for k in ("T", "D", "A", "B", "u_ppm", "type")}
            sub["set_off"] = np.array([0, len(keep)], np.int64)
            r = oracle.search_best(sub, M, g, KC, KM, kmin, kmax)
            assert r["feasible"][0] == 1


def test_heuristic_success_implies_exhaustive_feasible_and_not_better():
    s = gen_tasksets(seed=16, nsets=60, n_min=2, n_max=8, U_lo_ppm=500000, U_hi_ppm=5000000, deadline_pm=750,
                     T_lo=1000, T_hi=100000)
    M, g = 16, 2
    h = oracle.allocate(s, M, g, KC, KM, policy="SMS")
    e = oracle.search_best(s, M, g, KC, KM, 1, 8)
    checked = 0
    for si in range(60):
        if h["verdict"][si]:
            assert e["feasible"][si] == 1
            assert e["W"][si] <= h["W"][si]
            checked += 1
    assert checked > 20


# ------------------------------------------- admissible partition sizes (§2)

def test_sizes_listing_every_multiple_of_g_changes_nothing():
    s = gen_tasksets(seed=70, nsets=60, n_min=2, n_max=10, U_lo_ppm=500000, U_hi_ppm=6000000, deadline_pm=750,
                     T_lo=1000, T_hi=100000)
    M, g = 24, 2
    every = list(range(g, M + 1, g))
    for policy, act in (("SMS", False), ("BF", True)):
        a = oracle.allocate(s, M, g, KC, KM, policy=policy, act=act)
        b = oracle.allocate(s, M, g, KC, KM, policy=policy, act=act, sizes=every)
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    small = gen_tasksets(seed=71, nsets=20, n_min=1, n_max=6, U_lo_ppm=500000, U_hi_ppm=3000000, deadline_pm=750,
                         T_lo=1000, T_hi=100000)
    a = oracle.search_best(small, M, g, KC, KM, 1, 3)
    b = oracle.search_best(small, M, g, KC, KM, 1, 3, sizes=every)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_sizes_singleton_is_next_admissible_lemma2_size():
    rng = random.Random(72)
    sizes = [3, 4, 7, 12, 20, 33]
    for _ in range(400):
        C1 = rng.randrange(1, 10**6)
        alpha = rng.randrange(0, 1001)
        T = rng.randrange(1000, 10**6)
        D = rng.randrange(max(1, T // 2), T + 1)
        A, B = C1 * (1000 - alpha), C1 * alpha
        m = oracle.minm(np.array([T]), np.array([D]), np.array([A]), np.array([B]), np.zeros(1, np.uint8),
                        np.ones(1, np.uint8), 1, 40, 1, KC, KM, sizes=sizes)
        plain = next((z for z in range(1, 41) if refs.wcet_alpha(C1, alpha, 1000, z) <= D), 0)
        want = next((z for z in sizes if z >= plain), 0) if plain else 0
        assert m == want, (C1, alpha, T, D)


@pytest.mark.parametrize("policy,act", [("SMS", False), ("BF", True)])
def test_sizes_heuristic_matches_restatement(policy, act):
    """Alg. 1-3 with partition sizes from a GPC-like list: the restatement
    (merges sized in [max(a, b), a + b - 1] over the list) agrees."""
    M, g, sizes = 16, 1, [2, 3, 5, 8, 11, 16]
    s = gen_tasksets(seed=73, nsets=40, n_min=3, n_max=8, U_lo_ppm=1000000, U_hi_ppm=12000000, deadline_pm=750,
                     T_lo=50, T_hi=4000, T_dist="LIST", mode="PAPER")
    r = oracle.allocate(s, M, g, KC, KM, policy=policy, act=act, sizes=sizes)
    merges = 0
    for si in range(40):
        v, o, n = _set_view(s, si)
        if oracle.lemma1_rejects(v["T"], v["A"], v["B"], M):
            assert r["reason"][si] == oracle.REASON["LEMMA1"]
            continue

        def test_min(S, lo, hi):
            mask = np.array([i in S for i in range(n)], np.uint8)
            return oracle.minm(v["T"], v["D"], v["A"], v["B"], v["type"], mask, lo, hi, g, KC, KM, sizes=sizes)

        def single(i):
            return test_min({i}, g, M)

        def W(S):
            return sum(refs.conflict_k(v["type"], S, i, KC, KM) * int(v["u_ppm"][i]) for i in S)

        status, parts, tests = refs.heuristic(n, [int(x) for x in v["u_ppm"]], M, g, single, test_min,
                                              policy=policy, act=act, W=W, gap=1)
        assert oracle.REASON[status] == r["reason"][si], si
        assert tests == r["n_tests"][si], si
        if status == "LEMMA2":
            continue
        merges += tests
        got, zs = _partitions_from(r, si, o, n)
        assert sorted((sorted(P), z) for P, z in parts.items()) == sorted((sorted(got[p]), zs[p]) for p in got)
        assert all(z in sizes for z in zs)
    assert merges > 20


def test_sizes_exhaustive_matches_bruteforce():
    rng = random.Random(74)
    for trial in range(20):
        n = rng.randrange(1, 5)
        M = rng.choice([6, 8, 10])
        sizes = sorted(rng.sample(range(1, M + 1), rng.randrange(1, min(M, 4) + 1)))
        kmin = rng.randrange(1, 3)
        kmax = rng.randrange(kmin, 4)
        s = gen_tasksets(seed=200 + trial, nsets=1, n_min=n, n_max=n, U_lo_ppm=300000, U_hi_ppm=2500000,
                         deadline_pm=750, T_lo=1000, T_hi=100000)
        a = oracle.search_best(s, M, 1, KC, KM, kmin, kmax, sizes=sizes)
        b = oracle.search_best(s, M, 1, KC, KM, kmin, kmax, explicit=True, sizes=sizes)
        for k in ("feasible", "W", "sum_minm", "n_blocks", "spare", "rgs", "minm_block"):
            assert np.array_equal(a[k], b[k]), (trial, k)
        v, o, _ = _set_view(s, 0)

        def passes(S, m):
            mask = np.array([i in S for i in range(n)], np.uint8)
            return oracle.rta(v["T"], v["D"], v["A"], v["B"], v["type"], mask, m, KC, KM)[0] == 1

        def minsize(S):
            return next((z for z in sizes if passes(S, z)), 0)

        def W(S):
            return sum(refs.conflict_k(v["type"], S, i, KC, KM) * int(v["u_ppm"][i]) for i in S)

        best = refs.exhaustive_bruteforce(n, M, 1, kmin, kmax, passes, minsize, W, sizes=sizes)
        assert bool(a["feasible"][0]) == (best is not None), trial
        if best is not None:
            assert (a["W"][0], a["sum_minm"][0], tuple(a["rgs"][:n])) == best


def test_sizes_candidate_part_must_be_admissible():
    s = gen_tasksets(seed=75, nsets=2, n_min=3, n_max=3)
    cset = np.array([0, 1], np.int64)
    cmap = np.zeros(6, np.uint8)
    v, _ = oracle.test_schedulable(s, 16, 1, KC, KM, cset, cmap, 3, 1, np.array([8, 8], np.int32), sizes=[4, 8, 16])
    assert len(v) == 2
    with pytest.raises(RuntimeError):
        oracle.test_schedulable(s, 16, 1, KC, KM, cset, cmap, 3, 1, np.array([8, 6], np.int32), sizes=[4, 8, 16])


def test_rgs_and_composition_counts():
    """Stirling numbers of the second kind (recurrence) and binomials."""
    def stirling(n, k):
        S = [[0] * (k + 1) for _ in range(n + 1)]
        S[0][0] = 1
        for i in range(1, n + 1):
            for j in range(1, k + 1):
                S[i][j] = j * S[i - 1][j] + S[i - 1][j - 1]
        return S[n][k]
    assert sum(stirling(12, k) for k in range(1, 5)) == 700075
    total = sum(math.comb(19, k - 1) * k**12 for k in range(1, 5))
    assert total == 16348076540  # explicit (split x map) candidates per 12-task set on 20 units
    assert [len(list(refs.compositions(8, 2)))] == [7]


# ------------------------------------------------------------- serving ops

def _check_state(t, M, g):
    """The tenant's allocation passes (Lemma 3), every partition passes at its
    size and that size is its minimum, Pi and W are consistent."""
    n = t.n
    if n == 0:
        assert t.n_parts == 0 and t.Pi == 0
        return
    parts = {}
    for i in range(n):
        parts.setdefault(int(t.part[i]), []).append(i)
    assert sorted(parts) == list(range(t.n_parts))
    # numbered by lowest task index
    assert [min(parts[p]) for p in range(t.n_parts)] == sorted(min(v) for v in parts.values())
    total = 0
    Wsum = 0
    for p, rows in parts.items():
        mask = np.zeros(n, np.uint8)
        mask[rows] = 1
        z = int(t.size[p])
        total += z
        args = [t.tasks[k] for k in ("T", "D", "A", "B", "type")]
        assert oracle.rta(*args, mask, z, KC, KM)[0] == 1
        assert oracle.minm(*args, mask, g, M, g, KC, KM) == z
        Wsum += sum(refs.conflict_k(t.tasks["type"], set(rows), i, KC, KM) * int(t.tasks["u_ppm"][i]) for i in rows)
    assert total == t.Pi <= M
    assert Wsum == t.W


def test_serving_operations_keep_minimal_passing_allocations():
    import serve_seq
    M, g = 148, 1
    ops = serve_seq.make_ops(12, 25, seed=3)
    paths = set()
    for seq in ops:
        t = oracle.Tenant(M, g, KC, KM)
        r = t.admit(seq[0][1])
        if not r["verdict"]:
            continue
        _check_state(t, M, g)
        for op, arg in seq[1:]:
            if op == "ADD" and t.n < 128:
                n0 = t.n
                r = t.add(arg)
                paths.add(r["path"])
                assert t.n == n0 + (1 if r["verdict"] else 0)
            elif op == "REMOVE" and t.n > 0:
                t.remove(int(arg * t.n))
            _check_state(t, M, g)
    assert {1, 3} <= paths  # fits and new partitions both occur


def test_serving_add_into_empty_tenant_takes_lemma2_size():
    t = oracle.Tenant(8, 1, KC, KM)
    empty = {k: np.zeros(0, np.uint8 if k == "type" else np.int64) for k in oracle.Tenant.COLS}
    assert t.admit(empty)["verdict"] == 1
    # C1 = 250 on a 100-tick deadline: alpha = 0 -> C(m) = ceil(250/m) -> m = 3
    r = t.add({"T": 100, "D": 100, "A": 250000, "B": 0, "u_ppm": 2500000, "type": 0})
    assert r["verdict"] == 1 and r["path"] == 3 and list(r["size_of_part"]) == [3] and r["Pi"] == 3
    # a second compute task: the fit at 3 SMs would put both in conflict (k = 1.2)
    r = t.add({"T": 100, "D": 100, "A": 100000, "B": 0, "u_ppm": 1000000, "type": 0})
    assert r["verdict"] == 1
    _check_state(t, 8, 1)
    r = t.remove(0)
    assert r["n_tasks"] == 1 and r["n_parts"] == 1
    _check_state(t, 8, 1)


def test_serving_paths_match_a_restatement():
    """ADD and REMOVE of the oracle's tenant against refs.serve_add /
    serve_remove (the FIT, GROW, NEW, REALLOC order and ranges restated over
    the pinned per-partition test): same path, partitions and sizes after
    every request of seeded sequences."""
    import serve_seq
    M, g = 148, 1
    paths = set()
    for seq in serve_seq.make_ops(12, 25, seed=3):
        t = oracle.Tenant(M, g, KC, KM)
        if not t.admit(seq[0][1])["verdict"]:
            continue
        for op, arg in seq[1:]:
            if op == "ADD" and t.n < 128:
                path, cols, part, size = refs.serve_add(t.tasks, t.part, t.size[:t.n_parts], arg, M, g, KC, KM)
                r = t.add(arg)
                paths.add(path)
                assert r["path"] == path and bool(r["verdict"]) == (path != 0)
            elif op == "REMOVE" and t.n > 0:
                idx = int(arg * t.n)
                cols, part, size = refs.serve_remove(t.tasks, t.part, t.size[:t.n_parts], idx, g, KC, KM)
                t.remove(idx)
            else:
                continue
            assert list(t.part) == list(part) and list(t.size[:t.n_parts]) == list(size)
            for k in ("T", "D", "A", "B", "u_ppm", "type"):
                assert np.array_equal(t.tasks[k], cols[k]), k
    assert {1, 3} <= paths


def test_serving_new_partition_may_take_every_spare_sm():
    """8 SMs, one compute task X held at its Lemma 2 size (A = 1000 * 100,
    B = 1000 * 60, T = D = 100: C = ceil(100 / m + 60) is 94 at 3 SMs, 110
    at 2): five SMs spare.  A compute task Y with A = 1000 * 500 needs
    exactly 5 SMs alone (C = 100).  Beside Y, X takes the compute conflict
    factor 1.2, at least ceil(1.2 * 72.5) = 87 even at 8 SMs, and Y at least
    75, so Y neither fits nor grows X's partition; a new partition of 5 SMs
    fits the 5 spare ones exactly, and the GPU is then full."""
    def task(a, b):
        return {"T": 100, "D": 100, "A": 1000 * a, "B": 1000 * b, "u_ppm": a * 10000, "type": 0}
    t = oracle.Tenant(8, 1, KC, KM)
    cols = {k: np.array([task(100, 60)[k]], np.uint8 if k == "type" else np.int64) for k in oracle.Tenant.COLS}
    assert t.admit(cols)["verdict"] == 1
    assert list(t.size[:t.n_parts]) == [3]
    r = t.add(task(500, 0))
    assert r["verdict"] == 1 and r["path"] == 3  # a new partition
    assert list(t.size[:t.n_parts]) == [3, 5] and r["Pi"] == 8


def test_serving_new_partition_must_fit_the_spare_sms():
    """8 SMs held as 3 + 4 (a compute task of C1 = 250 and a memory task of
    C1 = 350, both T = D = 100): one SM spare.  A compute task of C1 = 190
    needs 2 SMs alone, fails in both partitions at their sizes (with the
    other compute task: 100 + 76 > 100; beside the memory task: 88 + 48 > 100)
    and after growing into the spare SM (75 + 57, 70 + 38 > 100), so it may
    not open a new partition: the request reallocates within 8 SMs or is
    rejected with the state unchanged, as the restatement says."""
    def task(C1, typ):
        return {"T": 100, "D": 100, "A": 1000 * C1, "B": 0, "u_ppm": C1 * 10000, "type": typ}
    t = oracle.Tenant(8, 1, KC, KM)
    cols = {k: np.array([task(250, 0)[k], task(350, 1)[k]], np.uint8 if k == "type" else np.int64)
            for k in oracle.Tenant.COLS}
    assert t.admit(cols)["verdict"] == 1
    assert sorted(int(z) for z in t.size[:t.n_parts]) == [3, 4]
    path, _, part, size = refs.serve_add(t.tasks, t.part, t.size[:t.n_parts], task(190, 0), 8, 1, KC, KM)
    r = t.add(task(190, 0))
    assert path in (0, 4) and r["path"] == path
    assert r["Pi"] <= 8 and list(t.size[:t.n_parts]) == list(size)
