"""The §7 figure data: host aggregation (CPU) and the GPU run against the
same aggregation over the oracle's results (GPU)."""
import numpy as np
import pytest

import oracle
from paper_2105_10312_gb300 import figures, gen_tasksets
from paper_2105_10312_gb300 import workloads as W


def test_workload_bounds_by_hand():
    sets = {"set_off": np.array([0, 2, 2, 5]), "u_ppm": np.array([100000, 300000, 50000, 50000, 400000]),
            "type": np.array([0, 1, 1, 0, 1], np.uint8)}
    best, worst = figures.workload_bounds(sets, 1200, 2300)
    assert np.allclose(best, [0.4, 0.0, 0.5])
    assert np.allclose(worst, [0.1 * 1.2 + 0.3 * 2.3, 0.0, 0.05 * 2.3 + 0.05 * 1.2 + 0.4 * 2.3])


def test_aggregate_by_hand():
    best = np.array([1.0, 2.0, 1.0, 2.0])
    worst = np.array([2.0, 4.0, 2.0, 4.0])
    res = {"X": {"verdict": np.array([1, 1, 0, 1]), "n_parts": np.array([3, 4, 9, 6]),
                 "W": np.array([1.5e9, 3.0e9, 0, 4.0e9])}}
    agg = figures.aggregate(res, best, worst, 2)
    x = agg["variants"]["X"]
    assert agg["best"] == [1.0, 2.0] and agg["worst"] == [2.0, 4.0]
    assert x["rate"] == [0.5, 1.0]
    assert x["parts"] == [3.0, 5.0]
    assert x["load"] == [1.5, 3.5]
    assert x["load_in_bounds"] == [0.5, 0.75]


@pytest.mark.gpu
def test_figure_data_matches_oracle_aggregation():
    """figures.run on 2 sets per U step equals the same aggregation of the
    oracle's allocations; the bounds hold for every allocated set and the
    heuristics schedule at least what 1G does."""
    agg = figures.run(sets_per_step=2)
    p = W.gen_params("paper50", nsets=68)
    s = gen_tasksets(**p)
    md = W.model("paper50")
    res = {}
    for name, policy, act in figures.VARIANTS:
        r = oracle.allocate(s, md["M"], md["g"], md["k_c_pm"], md["k_m_pm"], policy=policy, act=act, nthreads=8)
        res[name] = {k: r[k] for k in ("verdict", "n_parts", "W")}
    best, worst = figures.workload_bounds(s, md["k_c_pm"], md["k_m_pm"])
    ref = figures.aggregate(res, best, worst, p["U_steps"])
    assert agg["variants"] == ref["variants"] and agg["best"] == ref["best"] and agg["worst"] == ref["worst"]
    for name in ("SMS_ACT", "SMS_INA", "BF_ACT", "BF_INA"):
        v = agg["variants"][name]
        assert all(a >= b for a, b in zip(v["rate"], agg["variants"]["1G"]["rate"]))
        assert all(r is None or -1e-9 <= r <= 1 + 1e-9 for r in v["load_in_bounds"])


@pytest.mark.gpu
def test_figure_data_200_tasks():
    """Figs. 6 and 7's setting (200 tasks per set, 256-task build), one set per
    U step: the rates are fractions, the heuristics schedule at least what 1G
    does, and the scheduled load of each allocated set lies in its bounds."""
    agg = figures.run(sets_per_step=1, tasks=200)
    assert agg["tasks"] == 200 and len(agg["U"]) == 34
    for name in ("SMS_ACT", "SMS_INA", "BF_ACT", "BF_INA"):
        v = agg["variants"][name]
        assert all(r is None or 0.0 <= r <= 1.0 for r in v["rate"])
        assert all(a >= b for a, b in zip(v["rate"], agg["variants"]["1G"]["rate"]))
        assert all(r is None or -1e-9 <= r <= 1 + 1e-9 for r in v["load_in_bounds"])
    assert agg["variants"]["SMS_INA"]["rate"][0] == 1.0
