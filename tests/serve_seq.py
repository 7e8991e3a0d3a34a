"""Seeded request sequences for the serving tests (test-only helper).

A sequence per tenant: one ADMIT of a generated task set, then ADD (one task
from a generated pool) and REMOVE (an index drawn on the fly against the
tenant's current size) operations, and optionally an EVICT at the end.
"""
import numpy as np

from paper_2105_10312_gb300 import gen_tasksets
from paper_2105_10312_gb300 import workloads as W

COLS = ("T", "D", "A", "B", "u_ppm", "type")


def tenant_sets(ntenants, seed, n_min=4, n_max=40, M=148):
    p = W.gen_params("serve", nsets=ntenants, seed=seed, n_min=n_min, n_max=n_max)
    return gen_tasksets(**p)


def task_pool(npool, seed):
    p = W.gen_params("serve", nsets=npool, seed=seed + 1000, n_min=1, n_max=1, U_lo_ppm=20000, U_hi_ppm=1500000)
    return gen_tasksets(**p)


def set_of(s, k):
    o, e = s["set_off"][k], s["set_off"][k + 1]
    return {c: s[c][o:e].copy() for c in COLS}


def task_of(pool, j):
    return {c: pool[c][j] for c in COLS}


def make_ops(ntenants, nops, seed, evict=False):
    """Per tenant: [("ADMIT", tasks), ("ADD", task) | ("REMOVE", u) ...] where u in [0, 1)
    picks the index to remove as floor(u * n) at the time of the request."""
    rng = np.random.default_rng(seed)
    sets = tenant_sets(ntenants, seed)
    pool = task_pool(ntenants * nops + 1, seed)
    ops = []
    j = 0
    for k in range(ntenants):
        seq = [("ADMIT", set_of(sets, k))]
        for _ in range(nops):
            if rng.random() < 0.55:
                seq.append(("ADD", task_of(pool, j)))
                j += 1
            else:
                seq.append(("REMOVE", float(rng.random())))
        if evict:
            seq.append(("EVICT", None))
        ops.append(seq)
    return ops
