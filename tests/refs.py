"""Independent CPU references used to pin the oracle (test-only).

Each function restates a fact the paper or textbook scheduling theory fixes,
by a different route from the oracle's code:

* ``wcet_alpha`` / ``wcet_paper``: the execution-time model of §3.3 in the
  scaling-function form of §7.1, C = k (a/m + b), evaluated with exact
  rationals from the serial-fraction parameters (alpha) or the paper's b = beta a.
* ``simulate_fp``: a unit-step discrete-time simulation of a fixed-priority
  uniprocessor schedule with synchronous release (the partition of §5.5 run
  as one processor) -- response times by brute force, not by analysis.
* ``simulate_edf``: the same simulation under earliest-deadline-first
  dispatching -- deadline misses by brute force, not by a demand bound.
* ``heuristic``: Alg. 1-3 restated over Python frozensets (different data
  structures and loop order from the oracle), using a supplied per-partition
  test.
* ``exhaustive_bruteforce``: every composition of M/g into k parts times every
  task-to-part map, evaluated directly.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np


def wcet_alpha(C1, alpha_pm, k_pm, m):
    """ceil(k C1 (alpha + (1 - alpha) / m)) with alpha = alpha_pm / 1000 (exact)."""
    C1, alpha_pm, k_pm, m = int(C1), int(alpha_pm), int(k_pm), int(m)
    a = Fraction(alpha_pm, 1000)
    v = Fraction(k_pm, 1000) * C1 * (a + (1 - a) / m)
    return math.ceil(v)


def wcet_paper(a, beta_pm, k_pm, m):
    """ceil(k (a / m + b)) with b = beta a (exact), the §7.1 scaling function."""
    a, beta_pm, k_pm, m = int(a), int(beta_pm), int(k_pm), int(m)
    v = Fraction(k_pm, 1000) * (Fraction(a, m) + Fraction(beta_pm, 1000) * a)
    return math.ceil(v)


def simulate_fp(tasks, horizon):
    """tasks: list of (T, D, C) in priority order (index 0 highest).  Synchronous
    release at t = 0, unit time steps, work-conserving.  Returns (first, worst):
    the first job's response time of each task (None if not finished by
    ``horizon``) and the largest response time over jobs released before
    ``horizon`` that finished by ``horizon``."""
    n = len(tasks)
    pending = [[] for _ in range(n)]  # [release, remaining]
    first = [None] * n
    worst = [0] * n
    jobno = [0] * n
    for t in range(horizon):
        for i, (T, D, C) in enumerate(tasks):
            if t % T == 0:
                pending[i].append([t, C, jobno[i]])
                jobno[i] += 1
        for i in range(n):
            if pending[i]:
                job = pending[i][0]
                job[1] -= 1
                if job[1] == 0:
                    resp = t + 1 - job[0]
                    if job[2] == 0:
                        first[i] = resp
                    worst[i] = max(worst[i], resp)
                    pending[i].pop(0)
                break
    return first, worst


def simulate_edf(tasks, horizon):
    """tasks: list of (T, D, C).  Synchronous periodic release at t = 0, unit
    time steps, preemptive EDF (ties: lower task index).  Returns True iff no
    job misses its absolute deadline before ``horizon``."""
    jobs = []  # [absolute deadline, task index, remaining]
    for t in range(horizon):
        for i, (T, D, C) in enumerate(tasks):
            if t % T == 0:
                jobs.append([t + D, i, C])
        if jobs:
            jobs.sort(key=lambda j: (j[0], j[1]))
            jobs[0][2] -= 1
            if jobs[0][2] == 0:
                jobs.pop(0)
        for j in jobs:
            if j[0] <= t + 1 and j[2] > 0:
                return False
    return True


def dm_order(T, D, idx):
    return sorted(idx, key=lambda i: (D[i], T[i], i))


def conflict_k(types, S, i, kc, km):
    same = sum(1 for j in S if types[j] == types[i])
    if same >= 2:
        return km if types[i] == 1 else kc
    return 1000


def heuristic(n, u, M, g, single_size, test_min, policy="SMS", act=False, W=None, gap=None):
    """Alg. 1-3 over frozensets.  single_size(i) -> Lemma 2 size or 0;
    test_min(S, lo, hi) -> smallest passing size in [lo, hi] or 0;
    W(S) -> inflated workload (Def. 4 reading).  A merge of sizes a and b is
    sized in [max(a, b), a + b - gap] (gap = g by default).  Returns
    (ok, parts, tests) with parts a dict frozenset -> size; Lemma 1 is left
    to the caller."""
    gap = g if gap is None else gap
    parts = {}
    for i in range(n):
        z = single_size(i)
        if z == 0:
            return "LEMMA2", {}, 0
        parts[frozenset([i])] = z
    tests = 0
    act_pairs = set()
    if act and sum(parts.values()) > M:
        for i, j in itertools.combinations(range(n), 2):
            a, b = parts[frozenset([i])], parts[frozenset([j])]
            tests += 1
            if test_min(frozenset([i, j]), max(a, b), a + b - gap) == 0:
                act_pairs.add(frozenset([i, j]))
    failed = set()  # frozenset({P, Q})

    def forbidden(P, Q):
        if frozenset([P, Q]) in failed:
            return True
        return any(frozenset([i, j]) in act_pairs for i in P for j in Q)

    while sum(parts.values()) > M:
        order = sorted(parts, key=lambda P: (-sum(u[i] for i in P), min(P)))
        chosen = None
        for P in order:
            elig = [Q for Q in order if Q != P and not forbidden(P, Q)]
            if elig:
                chosen = (P, elig)
                break
        if chosen is None:
            return "NO_MERGE", parts, tests
        P, elig = chosen
        if policy == "SMS":
            results = []
            for pos, Q in enumerate(elig):
                tests += 1
                m3 = test_min(P | Q, max(parts[P], parts[Q]), parts[P] + parts[Q] - gap)
                if m3:
                    results.append((m3, pos, Q))
            if results:
                m3, _, Q = min(results, key=lambda r: (r[0], r[1]))
                del parts[P], parts[Q]
                parts[P | Q] = m3
            else:
                for Q in elig:
                    failed.add(frozenset([P, Q]))
        else:
            ranked = sorted(enumerate(elig), key=lambda pq: (W(P | pq[1]), pq[0]))
            for _, Q in ranked:
                tests += 1
                m3 = test_min(P | Q, max(parts[P], parts[Q]), parts[P] + parts[Q] - gap)
                if m3:
                    del parts[P], parts[Q]
                    parts[P | Q] = m3
                    break
                failed.add(frozenset([P, Q]))
    return "OK", parts, tests


def compositions(total, k):
    """All compositions of total into k positive parts, lexicographic."""
    if k == 1:
        yield (total,)
        return
    for first in range(1, total - k + 2):
        for rest in compositions(total - first, k - 1):
            yield (first,) + rest


def rgs_of(labels):
    seen = {}
    out = []
    for lab in labels:
        if lab not in seen:
            seen[lab] = len(seen)
        out.append(seen[lab])
    return tuple(out)


def exhaustive_bruteforce(n, M, g, kmin, kmax, passes, minsize, W, sizes=None):
    """passes(S, m) -> bool; minsize(S) -> minimal size in [g, M] or 0;
    W(S) -> workload.  Splits: compositions of M/g into k parts, or with an
    admissible size list every k sizes from it of sum <= M.  Returns None
    or (W, sum_minm, rgs)."""
    best = None
    Mu = M // g
    for k in range(kmin, kmax + 1):
        if k > Mu:
            break
        if sizes:
            splits = [c for c in itertools.product(sizes, repeat=k) if sum(c) <= M]
        else:
            splits = [tuple(x * g for x in c) for c in compositions(Mu, k)]
        for comp in splits:
            for labels in itertools.product(range(k), repeat=n):
                ok = True
                for p in range(k):
                    S = frozenset(i for i in range(n) if labels[i] == p)
                    if S and not passes(S, comp[p]):
                        ok = False
                        break
                if not ok:
                    continue
                rgs = rgs_of(labels)
                blocks = {}
                for i, b in enumerate(rgs):
                    blocks.setdefault(b, set()).add(i)
                key = (sum(W(frozenset(B)) for B in blocks.values()),
                       sum(minsize(frozenset(B)) for B in blocks.values()), rgs)
                if best is None or key < best:
                    best = key
    return best


# ------------------------------------------------------- serving, restated

_SCOLS = ("T", "D", "A", "B", "u_ppm", "type")


def _passes(cols, rows, m, kc, km):
    import oracle
    n = len(cols["T"])
    mask = np.zeros(n, np.uint8)
    mask[list(rows)] = 1
    return oracle.rta(*[cols[k] for k in ("T", "D", "A", "B", "type")], mask, m, kc, km)[0] == 1


def _smallest(cols, rows, lo, hi, g, kc, km):
    """Smallest multiple of g in [lo, hi] at which the rows pass, else 0."""
    m = -(-lo // g) * g
    while m <= hi:
        if _passes(cols, rows, m, kc, km):
            return m
        m += g
    return 0


def _canonical(part, size):
    """Partitions renumbered in the order of their lowest task index."""
    order = []
    for p in part:
        if p not in order:
            order.append(int(p))
    new = {p: k for k, p in enumerate(order)}
    return [new[int(p)] for p in part], [size[p] for p in order]


def serve_add(tasks, part, size, task, M, g, kc, km, policy="SMS", act=False):
    """ADD of one task to a tenant's allocation, restated: the first
    partition (in order) that still passes at its size takes it (FIT); else
    the first that passes after growing into the spare SMs, at its smallest
    such size (GROW); else a new partition of the task's Lemma 2 size if the
    spare SMs hold it (NEW); else Alg. 1 on every task (REALLOC); else the
    request is rejected and the state is unchanged.  Returns (path, tasks,
    part, size) with path 1..4, or (0, ...) with the old state."""
    import oracle
    cols = {k: np.concatenate([tasks[k], np.asarray([task[k]], tasks[k].dtype)]) for k in _SCOLS}
    n = len(tasks["T"])
    part, size = [int(p) for p in part], [int(z) for z in size]
    spare = M - sum(size)
    members = [[i for i in range(n) if part[i] == p] + [n] for p in range(len(size))]
    for p, rows in enumerate(members):
        if _passes(cols, rows, size[p], kc, km):
            return 1, cols, part + [p], size
    if spare >= g:
        for p, rows in enumerate(members):
            m = _smallest(cols, rows, size[p] + 1, size[p] + spare, g, kc, km)
            if m:
                size2 = list(size)
                size2[p] = m
                return 2, cols, part + [p], size2
    z = _smallest(cols, [n], g, M, g, kc, km)
    if z and z <= spare:
        return 3, cols, part + [len(size)], size + [z]
    one = {k: cols[k] for k in _SCOLS}
    one["set_off"] = np.array([0, n + 1], np.int64)
    r = oracle.allocate(one, M, g, kc, km, policy=policy, act=act)
    if r["verdict"][0]:
        k = int(r["n_parts"][0])
        return 4, cols, [int(p) for p in r["part_of_task"]], [int(z) for z in r["size_of_part"][:k]]
    return 0, tasks, part, size


def serve_remove(tasks, part, size, index, g, kc, km):
    """REMOVE of task `index`, restated: its partition disappears if it was
    the last task there, else shrinks to the smallest passing size at or
    below its size; partitions are then renumbered by lowest task index."""
    keep = [i for i in range(len(tasks["T"])) if i != index]
    cols = {k: tasks[k][keep] for k in _SCOLS}
    part2 = [int(part[i]) for i in keep]
    size2 = [int(z) for z in size]
    pr = int(part[index])
    if pr in part2:
        rows = [i for i, p in enumerate(part2) if p == pr]
        size2[pr] = _smallest(cols, rows, g, size2[pr], g, kc, km)
    else:
        part2 = [p - 1 if p > pr else p for p in part2]
        del size2[pr]
    part2, size2 = _canonical(part2, size2)
    return cols, part2, size2
