"""The synthetic workloads the library is measured and tested on.

Each entry gives the generator parameters and the GPU model.  Times are
integer microsecond ticks; utilisations are ppm; factors are per mille (§7.1:
k_c = 1.2, k_m = 2.3).  Inputs are synthetic and seeded: the paper's own
evaluation (§7) is synthetic too.

* ``single``   one set of 8 implicit-deadline tasks, U = 0.8, on 8 SMs split
               into exactly 2 partitions (7 splits x 2^8 maps = 1 792 explicit
               candidates).
* ``batch``    100 000 sets of U{16..32} tasks on an 80-SM GPU, U ~ U[0.5, 3.0],
               D = 0.75 T; the heuristic (SMS, INA) per set.
* ``exhaustive`` 20 000 sets of 12 tasks on 40 SMs in units of 2 (TPCs), split
               into 1..4 partitions; periods in [1 000, 100 000]; U ~ U[1.0, 3.5].
* ``sweep``    1 000 000 sets of U{4..64} tasks on 148 SMs; U = 0.1 .. 6.0 in
               steps of 0.1 (equal sets per step); memory intensity Beta(2, 5);
               heuristic vs 1G.
* ``serve``    admission queries of 4..128 tasks (log-uniform) on 148 SMs.
* ``paper50``  the paper's §7 setting: 68 SMs, 50 tasks, U = 2..68 in steps of 2,
               100 sets per step, D = 0.75 T, periods from the divisors of 4000 in
               [50, 4000], a 50 % memory-kernel ratio, b = 0.02 a / 0.1 a.
* ``paper200`` the same with 200 tasks per set (the paper's Figs. 6 and 7).
"""
from __future__ import annotations

K_C, K_M = 1200, 2300

COMMON = dict(T_lo=10000, T_hi=1000000, T_dist="LOGUNIFORM", alpha_lo_pm=50, alpha_hi_pm=300,
              mu_dist="UNIFORM", prm_pm=500, mode="ALPHA")

WORKLOADS = {
    "single": dict(
        gen=dict(COMMON, seed=0, nsets=1, n_min=8, n_max=8, U_lo_ppm=800000, U_hi_ppm=800000, deadline_pm=1000),
        model=dict(M=8, g=1, k_c_pm=K_C, k_m_pm=K_M), kmin=2, kmax=2),
    "batch": dict(
        gen=dict(COMMON, seed=2, nsets=100000, n_min=16, n_max=32, U_lo_ppm=500000, U_hi_ppm=3000000,
                 deadline_pm=750),
        model=dict(M=80, g=1, k_c_pm=K_C, k_m_pm=K_M), policy="SMS", act=False),
    "exhaustive": dict(
        gen=dict(COMMON, seed=3, nsets=20000, n_min=12, n_max=12, U_lo_ppm=1000000, U_hi_ppm=3500000,
                 T_lo=1000, T_hi=100000, deadline_pm=750),
        model=dict(M=40, g=2, k_c_pm=K_C, k_m_pm=K_M), kmin=1, kmax=4),
    "sweep": dict(
        gen=dict(COMMON, seed=4, nsets=1000000, n_min=4, n_max=64, U_steps=60, U_lo_ppm=100000,
                 U_hi_ppm=6000000, deadline_pm=750, mu_dist="BETA25"),
        model=dict(M=148, g=1, k_c_pm=K_C, k_m_pm=K_M), policy="SMS", act=False),
    "serve": dict(
        gen=dict(COMMON, seed=5, nsets=1, n_min=4, n_max=128, n_dist="LOGUNIFORM", U_lo_ppm=500000,
                 U_hi_ppm=6000000, deadline_pm=750),
        model=dict(M=148, g=1, k_c_pm=K_C, k_m_pm=K_M)),
    "paper50": dict(
        gen=dict(seed=6, nsets=3400, n_min=50, n_max=50, U_steps=34, U_lo_ppm=2000000, U_hi_ppm=68000000,
                 T_lo=50, T_hi=4000, T_dist="LIST", deadline_pm=750, mu_dist="UNIFORM", prm_pm=500,
                 mode="PAPER", beta_c_pm=20, beta_m_pm=100, alpha_lo_pm=0, alpha_hi_pm=0),
        model=dict(M=68, g=1, k_c_pm=K_C, k_m_pm=K_M)),
    "paper200": dict(
        gen=dict(seed=7, nsets=3400, n_min=200, n_max=200, U_steps=34, U_lo_ppm=2000000, U_hi_ppm=68000000,
                 T_lo=50, T_hi=4000, T_dist="LIST", deadline_pm=750, mu_dist="UNIFORM", prm_pm=500,
                 mode="PAPER", beta_c_pm=20, beta_m_pm=100, alpha_lo_pm=0, alpha_hi_pm=0),
        model=dict(M=68, g=1, k_c_pm=K_C, k_m_pm=K_M)),
}


def gen_params(name, **override):
    p = dict(WORKLOADS[name]["gen"])
    p.update(override)
    return p


def model(name):
    return dict(WORKLOADS[name]["model"])
