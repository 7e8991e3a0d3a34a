"""gpa_search_explicit (GPU) against the oracle: every explicit candidate
(an SM split times a task-to-partition map, the problem statement of §5)
enumerated and tested on the device.

The candidate order is restated here from its definition (compositions in
lexicographic order of their parts, then map codes with task i in part
(c / k^i) mod k), so each candidate's verdict is checked against the
oracle's test of that exact candidate; the optimum is checked against the
oracle's explicit brute force and its set-partition search."""
import itertools

import numpy as np
import pytest
import torch

import oracle
import paper_2105_10312_gb300 as gpa
from paper_2105_10312_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KC, KM = W.K_C, W.K_M
BEST_KEYS = ("feasible", "W", "sum_minm", "n_blocks", "spare", "rgs", "minm_block")


def _np(x):
    return x.cpu().numpy() if isinstance(x, torch.Tensor) else x


def _compositions(Mu, k):
    """Compositions of Mu into k positive parts, lexicographic in the parts."""
    for cuts in itertools.combinations(range(1, Mu), k - 1):
        edges = (0,) + cuts + (Mu,)
        yield [edges[i + 1] - edges[i] for i in range(k)]


def _candidates(n, Mu, kmin, kmax):
    """(k, parts, map) of every explicit candidate, in rank order."""
    for k in range(kmin, min(kmax, Mu) + 1):
        for parts in _compositions(Mu, k):
            for code in range(k ** n):
                yield k, parts, [(code // k ** i) % k for i in range(n)]


def _oracle_verdicts(s, M, g, kmin, kmax, sched="DM"):
    n = int(s["set_off"][1] - s["set_off"][0])
    out = []
    by_k = {}
    for k, parts, mp in _candidates(n, M // g, kmin, kmax):
        by_k.setdefault(k, []).append((parts, mp))
    for k in sorted(by_k):
        cands = by_k[k]
        cset = np.zeros(len(cands), np.int64)
        cmap = np.array([mp for _, mp in cands], np.uint8).reshape(-1)
        csize = np.array([[p * g for p in parts] for parts, _ in cands], np.int32).reshape(-1)
        v, _ = oracle.test_schedulable(s, M, g, KC, KM, cset, cmap, n, k, csize, with_R=False, sched=sched)
        out.append(v)
    return np.concatenate(out)


def test_single_instance_every_candidate_and_the_optimum(ctx):
    """The single-instance workload: 8 tasks on 8 SMs in exactly 2 parts,
    7 splits x 2^8 maps = 1 792 candidates, each verdict equal to the
    oracle's test of that candidate; the optimum equal to the oracle's
    explicit brute force and to its set-partition search."""
    wp = W.WORKLOADS["single"]
    s = gpa.gen_tasksets(**W.gen_params("single"))
    md = W.model("single")
    d = gpa.to_device(s)
    assert ctx.explicit_count(d, md["M"], md["g"], wp["kmin"], wp["kmax"]) == 1792
    out = ctx.search_explicit(d, **md, kmin=wp["kmin"], kmax=wp["kmax"], cand_verdict=True)
    ctx.sync()
    cv = _np(out["cand_verdict"]).reshape(-1)
    want = _oracle_verdicts(s, md["M"], md["g"], wp["kmin"], wp["kmax"])
    assert cv.shape == (1792,) and np.array_equal(cv, want)
    ref = oracle.search_best(s, md["M"], md["g"], KC, KM, wp["kmin"], wp["kmax"], explicit=True)
    ref2 = oracle.search_best(s, md["M"], md["g"], KC, KM, wp["kmin"], wp["kmax"])
    assert ref["candidates"] == 1792
    for k in BEST_KEYS:
        assert np.array_equal(_np(out[k]), ref[k]), k
        assert np.array_equal(ref2[k], ref[k]), k
    assert ctx.last_terms() > 0


@pytest.mark.parametrize("sched", ["DM", "EDF"])
@pytest.mark.parametrize("M,g,kmin,kmax", [(8, 1, 1, 3), (12, 2, 2, 3), (6, 1, 3, 4), (4, 1, 1, 8)])
def test_random_small_sets_match_the_oracle(ctx, sched, M, g, kmin, kmax):
    """60 seeded sets of 1..6 tasks (several utilisations), the optimum
    equal to the oracle's explicit brute force; every candidate verdict of
    the first sets equal to the oracle's test of the candidate."""
    s = gpa.gen_tasksets(seed=11, nsets=60, n_min=1, n_max=6, U_lo_ppm=200000, U_hi_ppm=2500000,
                         T_lo=1000, T_hi=100000, T_dist="LOGUNIFORM", deadline_pm=750, alpha_lo_pm=50,
                         alpha_hi_pm=300, mu_dist="UNIFORM", prm_pm=500, mode="ALPHA")
    d = gpa.to_device(s)
    out = ctx.search_explicit(d, M, g, KC, KM, kmin=kmin, kmax=kmax, sched=sched, cand_verdict=True)
    ctx.sync()
    ref = oracle.search_best(s, M, g, KC, KM, kmin, kmax, explicit=True, sched=sched)
    for k in BEST_KEYS:
        assert np.array_equal(_np(out[k]), ref[k]), k
    cv = _np(out["cand_verdict"])
    off = s["set_off"]
    for i in range(4):
        sub = {k: s[k][off[i]:off[i + 1]] for k in ("T", "D", "A", "B", "u_ppm", "type")}
        sub["set_off"] = np.array([0, off[i + 1] - off[i]], np.int64)
        sub["n_max"] = s["n_max"]
        want = _oracle_verdicts(sub, M, g, kmin, kmax, sched)
        assert np.array_equal(cv[i, :len(want)], want), i
        assert (cv[i, len(want):] == 255).all()


def test_host_buffers_equal_device_buffers(ctx):
    s = gpa.gen_tasksets(seed=12, nsets=40, n_min=2, n_max=7, U_lo_ppm=300000, U_hi_ppm=2000000,
                         T_lo=1000, T_hi=100000, T_dist="LOGUNIFORM", deadline_pm=750, alpha_lo_pm=50,
                         alpha_hi_pm=300, mu_dist="UNIFORM", prm_pm=500, mode="ALPHA")
    dev = ctx.search_explicit(gpa.to_device(s), 10, 1, KC, KM, kmin=1, kmax=3, cand_verdict=True)
    host = ctx.search_explicit(dict(s), 10, 1, KC, KM, kmin=1, kmax=3, cand_verdict=True)
    ctx.sync()
    for k in BEST_KEYS + ("cand_verdict",):
        assert np.array_equal(host[k], _np(dev[k])), k


def test_limits(ctx):
    s = gpa.gen_tasksets(**W.gen_params("exhaustive", nsets=2))
    with pytest.raises(gpa.GpaError) as ei:
        ctx.search_explicit(gpa.to_device(s), 40, 2, KC, KM, kmin=1, kmax=4)  # 12 tasks on 20 units: > 2^26
    assert ei.value.code == gpa.ERR_RANGE
    with pytest.raises(gpa.GpaError) as ei:
        ctx.search_explicit(gpa.to_device(s), 40, 2, KC, KM, kmin=1, kmax=9)
    assert ei.value.code == gpa.ERR_RANGE
