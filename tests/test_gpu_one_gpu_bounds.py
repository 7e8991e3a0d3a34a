"""1G parity on sets built around the shortcuts of the 1G kernel (GPU).

The 1G kernel decides most sets before the deadline-monotonic staging: a
miss when some task has C > D or the utilisation exceeds 1, a pass when every
task's response-time upper bound (C_i + sum C_hp) / (1 - U_hp) is within its
deadline, with every task of no later deadline counted as higher priority.
The sets here sit where such shortcuts could go wrong: many tasks sharing a
deadline (the tie rule), total utilisation just below and just above 1, and
constrained deadlines close to the response times.  Every verdict and output
must equal the oracle's exact test, under DM and under EDF, in the 64-, 128-
and 256-task builds.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2105_10312_gb300 as gpa

pytestmark = pytest.mark.gpu
ALLOC_KEYS = ("verdict", "reason", "n_parts", "Pi", "W", "n_tests", "part_of_task", "size_of_part")
PERIODS = np.array([100, 125, 200, 250, 400, 500, 800, 1000, 2000, 4000])  # divisors of 4000


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = gpa.Context(0)
    yield c
    c.close()


def _family(fam, seed, nsets, n_lo, n_hi):
    """Seeded sets of one family; C is exact at M = 1 with factors 1000 per
    mille (A = 1000 C, B = 0), so the family controls the WCETs directly."""
    rng = np.random.default_rng(seed)
    off, cols = [0], {k: [] for k in ("T", "D", "A", "B", "u_ppm", "type")}
    for _ in range(nsets):
        n = int(rng.integers(n_lo, n_hi + 1))
        if fam == "ties":  # three deadlines shared by all tasks, periods 0-2 ticks longer
            dv = rng.integers(100, 5000, 3)
            D = rng.choice(dv, n)
            T = D + rng.integers(0, 3, n)
            U = rng.uniform(0.5, 1.0)
        elif fam == "near1":  # implicit deadlines, U in [0.97, 1.03]
            T = rng.choice(PERIODS, n)
            D = T.copy()
            U = rng.uniform(0.97, 1.03)
        else:  # constrained deadlines, periods log-uniform
            T = np.exp(rng.uniform(np.log(1000), np.log(100000), n)).astype(np.int64)
            D = T * rng.integers(500, 1001, n) // 1000
            U = rng.uniform(0.3, 0.95)
        C = np.maximum(1, np.round(rng.dirichlet(np.ones(n)) * U * T)).astype(np.int64)
        for k, v in (("T", T), ("D", D), ("A", 1000 * C), ("B", np.zeros(n, np.int64)),
                     ("u_ppm", 10**6 * C // T), ("type", rng.integers(0, 2, n))):
            cols[k] += [int(x) for x in v]
        off.append(off[-1] + n)
    s = {k: np.array(v, np.uint8 if k == "type" else np.int64) for k, v in cols.items()}
    s["set_off"] = np.array(off, np.int64)
    s["n_max"] = int(np.diff(s["set_off"]).max())
    return s


def _check(ctx, s, sched, M=1, kc=1000, km=1000, what=""):
    out = ctx.allocate(gpa.to_device(s), M, 1, kc, km, policy="ONE_GPU", sched=sched)
    ctx.sync()
    ref = oracle.allocate(s, M, 1, kc, km, policy="ONE_GPU", nthreads=8, sched=sched)
    for k in ALLOC_KEYS:
        g, r = out[k].cpu().numpy(), ref[k]
        bad = np.nonzero(g != r)[0]
        assert len(bad) == 0, f"{what} {sched}: {k} differs at {bad[:8]}: gpu {g[bad[:8]]} oracle {r[bad[:8]]}"
    return ref


@pytest.mark.parametrize("sched", ["DM", "EDF"])
@pytest.mark.parametrize("fam", ["ties", "near1", "constrained"])
def test_one_gpu_shortcut_boundaries(ctx, fam, sched):
    for k, (n_lo, n_hi, nsets) in enumerate(((2, 64, 1500), (65, 128, 150), (129, 200, 60))):
        s = _family(fam, 100 * k + len(fam), nsets, n_lo, n_hi)
        ref = _check(ctx, s, sched, what=f"{fam} n={n_lo}..{n_hi}")
        if n_hi == 64:
            assert 0 < ref["verdict"].sum() < nsets, (fam, sched, ref["verdict"].sum())


def test_one_gpu_shortcuts_with_conflict_factors(ctx):
    """The same families on 8 SMs with the §7.1 factors: the WCETs the
    kernel derives at M (conflict factors by task type) feed the shortcuts."""
    for fam in ("ties", "near1", "constrained"):
        s = _family(fam, 7 + len(fam), 1000, 2, 64)
        s["A"] = s["A"] * 8 // 3  # C(8) = ceil(k A / (8 10^6)): about a third of C at factor 1000
        for sched in ("DM", "EDF"):
            _check(ctx, s, sched, M=8, kc=1200, km=2300, what=f"{fam} M=8")
