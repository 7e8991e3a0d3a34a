"""Tests whose analysis cannot finish within the kernels' step limits are
reported as undecided, never as misses: a deadline-monotonic iteration
that needs more than 2^20 steps, and an EDF set whose U lies within n 2^-64
of 1 over periods whose least common multiple exceeds 2^62.  The first is
decided (a miss) by the oracle's unbounded iteration; the second is beyond
the oracle too (its busy period passes 2^100), so the test checks the
condition the header states instead."""
import math
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import paper_2105_10312_gb300 as gpa

pytestmark = pytest.mark.gpu


def _crafted(sets_tasks):
    """(T, D, C) tasks alternating types, A = 1000 C and B = 0 so C(1) = C."""
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


def _is_prime(p):
    if p < 2 or p % 2 == 0:
        return p == 2
    f = 3
    while f * f <= p:
        if p % f == 0:
            return False
        f += 2
    return True


def _near_one_set():
    """Three prime periods just below 2^26 and WCETs with sum C_i / T_i =
    1 - 1 / (T1 T2 T3) exactly: C_i = -(P / T_i)^-1 mod T_i makes the
    numerator -1 modulo P = T1 T2 T3; triples whose numerator is 2P - 1 are
    skipped."""
    primes = []
    p = (1 << 26) - 1
    while len(primes) < 12:
        if _is_prime(p):
            primes.append(p)
        p -= 2
    for a in range(len(primes)):
        for b in range(a + 1, len(primes)):
            for c in range(b + 1, len(primes)):
                T = [primes[a], primes[b], primes[c]]
                P = T[0] * T[1] * T[2]
                C = [(-pow(P // t, -1, t)) % t for t in T]
                U = sum(Fraction(ci, ti) for ci, ti in zip(C, T))
                if U == 1 - Fraction(1, P) and all(1 <= ci <= ti for ci, ti in zip(C, T)):
                    return T, C
    raise AssertionError("no triple found")


def test_dm_fixed_point_beyond_the_step_limit(ctx):
    """A higher-priority task with T = D = C = 1 in front of a task with
    C = 1 and D = T = 2^21: the second task's iteration R = 1 + ceil(R / 1)
    climbs by one per step, so it passes D only after about 2^21 steps.  The
    GPU gives up after 2^20 (candidate verdict 2, set reason UNDECIDED, sync
    GPA_ERR_TIMEOUT); the oracle's unbounded iteration finds the miss."""
    D2 = 1 << 21
    tasks = [(1, 1, 1), (D2, D2, 1)]
    s = _crafted([tasks])
    vr, Rr = oracle.test_schedulable(s, 1, 1, 1000, 1000, np.zeros(1, np.int64), np.zeros(2, np.uint8), 2, 1,
                                     np.ones(1, np.int32))
    assert vr[0] == 0 and list(Rr) == [1, -1]
    d = gpa.to_device(s)
    v, R = ctx.test_schedulable(d, 1, torch.zeros(1, dtype=torch.int64).cuda(),
                                torch.zeros(2, dtype=torch.uint8).cuda(), torch.ones(1, dtype=torch.int32).cuda(),
                                2, 1, k_c_pm=1000, k_m_pm=1000)
    with pytest.raises(gpa.GpaError) as ei:
        ctx.sync()
    assert ei.value.code == gpa.ERR_TIMEOUT
    assert v.cpu().numpy()[0] == 2
    out = ctx.allocate(d, 1, g=1, k_c_pm=1000, k_m_pm=1000, policy="ONE_GPU")
    with pytest.raises(gpa.GpaError):
        ctx.sync()
    assert out["reason"].cpu().numpy()[0] == gpa.REASON["UNDECIDED"] and out["verdict"].cpu().numpy()[0] == 0
    ctx.sync()  # the flag was cleared by the previous sync


def test_edf_utilisation_within_2_to_the_minus_64(ctx):
    """U = 1 - 1 / (T1 T2 T3) with T1 T2 T3 > 2^62 and D = T: the 2^64-scaled
    terms straddle 1 and the least common multiple is too large, so the GPU
    reports the test undecided, and decides the same periods with one unit
    of C more (U > 1 by far more than 2^-64: a miss) exactly."""
    T, C = _near_one_set()
    P = T[0] * T[1] * T[2]
    assert P > 1 << 62 and 1 - Fraction(1, P) > 1 - Fraction(3, 1 << 64)
    sets = [list(zip(T, T, C)), list(zip(T, T, C[:-1] + [C[-1] + 1]))]
    s = _crafted(sets)
    d = gpa.to_device(s)
    v, _ = ctx.test_schedulable(d, 1, torch.arange(2, dtype=torch.int64).cuda(),
                                torch.zeros(6, dtype=torch.uint8).cuda(), torch.ones(2, dtype=torch.int32).cuda(),
                                3, 1, k_c_pm=1000, k_m_pm=1000, sched="EDF")
    with pytest.raises(gpa.GpaError) as ei:
        ctx.sync()
    assert ei.value.code == gpa.ERR_TIMEOUT
    assert list(v.cpu().numpy()) == [2, 0]
    vr, _ = oracle.test_schedulable(s, 1, 1, 1000, 1000, np.array([1], np.int64), np.zeros(3, np.uint8), 3, 1,
                                    np.ones(1, np.int32), sched="EDF")
    assert vr[0] == 0
    ctx.sync()
