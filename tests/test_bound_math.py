"""The closed-form shortcuts of the GPU tests, checked against the oracle's
exact response-time analysis on the CPU (no GPU).

The kernels settle tasks and sets without iterating the fixed point of the
§5.5 test, and start the iteration at lower bounds of it.  Each shortcut is
a mathematical claim about the exact analysis; here every claim is checked
in exact rational arithmetic on seeded random sets (many equal periods and
deadlines, utilisations up to and above 1) against the oracle, which
iterates from the plain start value and knows none of them:

* upper bound: with U_hp < 1, X_i = (C_i + sum_{j in hp(i)} C_j) / (1 - U_hp)
  is at least the response time, so X_i <= D_i means task i meets D_i; the
  same holds when hp(i) is widened to every other task with D_j <= D_i;
* hyperbolic bound with deadlines as periods: prod (1 + C_i / D_i) <= 2
  means every task meets its deadline under DM;
* one evaluation at the deadline: f(D_i) <= D_i (f the iteration's
  function) means task i meets D_i, also with the higher-priority set
  widened to every task with D_j <= D_i;
* lower bounds: R_i >= C_i / (1 - U_hp), R_i >= R_{i-1} + C_i and
  R_i >= C_0 + ... + C_i for tasks whose fixed point is within D_i;
* the exhaustive search's cut: adding a task to a block adds at least the
  task's own workload alone.
"""
import math
from fractions import Fraction

import numpy as np

import oracle

PERIODS = [10, 12, 15, 20, 24, 30, 40, 60, 100, 120, 250, 1000]


def _random_set(rng):
    n = int(rng.integers(2, 13))
    T = rng.choice(PERIODS, n).astype(np.int64)
    D = np.array([int(rng.integers(max(1, t // 2), t + 1)) for t in T], np.int64)
    U = rng.uniform(0.3, 1.1)
    C = np.maximum(1, np.round(rng.dirichlet(np.ones(n)) * U * T)).astype(np.int64)
    C = np.minimum(C, D)  # C <= D, as the shortcuts assume (C > D decides a miss first)
    return T, D, C


def _oracle_R(T, D, C):
    n = len(T)
    v, R = oracle.rta(T, D, 1000 * C, np.zeros(n, np.int64), np.zeros(n, np.uint8), np.ones(n, np.uint8), 1,
                      1000, 1000)
    return v, R


def _dm_order(T, D):
    return sorted(range(len(T)), key=lambda i: (int(D[i]), int(T[i]), i))


def test_closed_form_shortcuts_agree_with_the_exact_analysis():
    rng = np.random.default_rng(2024)
    checked = dict(upper=0, upper_wide=0, hyperbolic=0, at_deadline=0, at_deadline_wide=0, lower=0)
    for _ in range(3000):
        T, D, C = _random_set(rng)
        n = len(T)
        v, R = _oracle_R(T, D, C)
        meets = [0 <= R[i] <= D[i] for i in range(n)]
        assert bool(v) == all(meets)
        order = _dm_order(T, D)
        # hyperbolic bound with the deadlines as periods
        if math.prod(1 + Fraction(int(C[i]), int(D[i])) for i in range(n)) <= 2:
            assert v == 1
            checked["hyperbolic"] += 1
        Rprev = 0
        for pos, i in enumerate(order):
            hp = order[:pos]
            Uhp = sum(Fraction(int(C[j]), int(T[j])) for j in hp)
            Chp = sum(int(C[j]) for j in hp)
            if Uhp < 1:
                X = Fraction(int(C[i]) + Chp, 1) / (1 - Uhp)
                if X <= D[i]:
                    assert meets[i], (T, D, C, i)
                    checked["upper"] += 1
                if meets[i]:
                    assert R[i] <= X
            wide = [j for j in range(n) if j != i and D[j] <= D[i]]
            Uw = sum(Fraction(int(C[j]), int(T[j])) for j in wide)
            if Uw < 1 and Fraction(int(C[i]) + sum(int(C[j]) for j in wide), 1) / (1 - Uw) <= D[i]:
                assert meets[i]
                checked["upper_wide"] += 1
            # f(D_i) = C_i + sum_{hp} ceil(D_i / T_j) C_j
            fD = int(C[i]) + sum(-(-int(D[i]) // int(T[j])) * int(C[j]) for j in hp)
            if fD <= D[i]:
                assert meets[i]
                checked["at_deadline"] += 1
            # the same over every task with D_j <= D_i, task i included
            fw = sum(-(-int(D[i]) // int(T[j])) * int(C[j]) for j in range(n) if D[j] <= D[i])
            if fw <= D[i]:
                assert meets[i]
                checked["at_deadline_wide"] += 1
            if meets[i]:
                if Uhp < 1:
                    assert R[i] >= Fraction(int(C[i]), 1) / (1 - Uhp)
                assert R[i] >= Chp + int(C[i])
                if pos > 0 and meets[order[pos - 1]]:
                    assert R[i] >= Rprev + int(C[i])
                checked["lower"] += 1
            Rprev = int(R[i])
    # every shortcut was exercised (and none claimed a pass the analysis refutes)
    assert all(c > 100 for c in checked.values()), checked


def test_a_task_adds_at_least_its_own_workload():
    """W(S + {k}) >= W(S) + W({k}) for the inflated workload of Def. 4, with
    the conflict factors of §4.2 (the exhaustive search's cut)."""
    rng = np.random.default_rng(7)
    for _ in range(2000):
        n = int(rng.integers(2, 12))
        u = rng.integers(0, 10**6, n).astype(np.int64)
        typ = rng.integers(0, 2, n).astype(np.uint8)
        kc, km = int(rng.integers(1000, 3000)), int(rng.integers(1000, 5000))
        S = rng.integers(0, 2, n).astype(np.uint8)
        k = int(rng.integers(0, n))
        S[k] = 0
        Sk = S.copy()
        Sk[k] = 1
        single = np.zeros(n, np.uint8)
        single[k] = 1
        assert oracle.workload(u, typ, Sk, kc, km) >= oracle.workload(u, typ, S, kc, km) + oracle.workload(
            u, typ, single, kc, km)
