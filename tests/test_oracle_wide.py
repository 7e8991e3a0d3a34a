"""The oracle on sets of 200 and 256 tasks (the paper's Figs. 6-7 size and
the library's cap), CPU only: the heuristic's allocation is consistent with
the oracle's own per-partition test, and the cap is enforced.  Kept apart
from the pins that the mutation checks rerun, because one 200-task set costs
the oracle about a second."""
import numpy as np
import pytest

import oracle
import paper_2105_10312_gb300 as gpa
from paper_2105_10312_gb300 import gen as G
from paper_2105_10312_gb300 import workloads as W

KC, KM = W.K_C, W.K_M


def _parts_pass_at_their_sizes(s, r, M, g, sched):
    """Every partition of every allocated set passes the oracle's test at its
    size, the sizes sum to at most M, and each partition fails one unit g
    smaller (each size is the smallest that passes)."""
    off = s["set_off"]
    nsets = len(off) - 1
    for i in range(nsets):
        if not r["verdict"][i]:
            continue
        o, e = int(off[i]), int(off[i + 1])
        k = int(r["n_parts"][i])
        part = r["part_of_task"][o:e]
        size = r["size_of_part"][o:o + k].astype(np.int32)
        assert size.sum() <= M and (size >= g).all()
        one = G.subset(s, np.array([i]))
        stride = e - o
        # candidate 0: the allocation; candidate 1 + p: partition p alone one unit smaller
        cands, maps, sizes = [0], [part], [size]
        for p in range(k):
            if size[p] > g:
                smaller = np.zeros(k, np.int32)
                smaller[p] = size[p] - g
                cands.append(0)
                maps.append(np.where(part == p, p, 255).astype(np.uint8))
                sizes.append(smaller)
        cmap = np.concatenate(maps).astype(np.uint8)
        cmap[cmap == 255] = 0
        # tasks outside the tested partition go to a part of size 0 (empty parts are not tested)
        for c in range(1, len(maps)):
            p = int(np.nonzero(sizes[c])[0][0])
            block = cmap[c * stride:(c + 1) * stride]
            block[maps[c] == 255] = (p + 1) % k if k > 1 else 0
        v, _ = oracle.test_schedulable(one, M, g, KC, KM, np.array(cands, np.int64), cmap, stride, k,
                                       np.concatenate(sizes), with_R=False, sched=sched)
        assert v[0] == 1, f"set {i}: the allocation fails the per-partition test"
        assert not v[1:].any(), f"set {i}: a partition passes one unit smaller"


@pytest.mark.parametrize("sched", ["DM", "EDF"])
def test_200_task_allocations_are_consistent(sched):
    s = G.subset(gpa.gen_tasksets(**W.gen_params("paper200", nsets=34)), np.array([0, 1]))
    md = W.model("paper200")
    r = oracle.allocate(s, md["M"], md["g"], KC, KM, policy="BF", act=True, nthreads=2, sched=sched)
    assert r["verdict"].all() and (r["n_parts"] == md["M"]).all()
    _parts_pass_at_their_sizes(s, r, md["M"], md["g"], sched)


def test_256_tasks_accepted_257_flagged():
    s = gpa.gen_tasksets(seed=3, nsets=2, n_min=256, n_max=256, U_lo_ppm=500000, U_hi_ppm=2000000,
                         deadline_pm=750, T_lo=1000, T_hi=100000)
    # 240 SMs: the 256 singletons must merge (a candidate has at most 255 parts)
    r = oracle.allocate(s, 240, 1, KC, KM, nthreads=2)
    assert r["verdict"].all() and (r["n_parts"] <= 240).all() and (r["n_tests"] > 0).all()
    _parts_pass_at_their_sizes(s, r, 240, 1, "DM")
    t = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}
    for k in ("T", "D", "A", "B", "u_ppm", "type"):
        t[k] = np.concatenate([t[k], t[k][:1]])
    t["set_off"] = np.array([0, 257, 513], np.int64)
    # like the kernels, the oracle rejects the 257-task set alone (reason INVALID) and allocates the other
    r2 = oracle.allocate(t, 240, 1, KC, KM, nthreads=2)
    assert r2["reason"][0] == gpa.REASON["INVALID"] and r2["verdict"][0] == 0
    assert r2["verdict"][1] == 1
