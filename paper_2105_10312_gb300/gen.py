"""Seeded synthetic task-set generator (ctypes over ``libgpa_gen.so``, built from ``csrc/gen.c``).

The generator is the only code both the CUDA path's callers and the CPU oracle's
tests share: it draws inputs and holds none of the method's arithmetic.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
GEN_PATH = os.path.join(_HERE, "libgpa_gen.so")

DIST = {"UNIFORM": 0, "LOGUNIFORM": 1, "LIST": 2, "BETA25": 3}
MODE = {"ALPHA": 0, "PAPER": 1}


class GenParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("nsets", ctypes.c_int64), ("n_min", ctypes.c_int32),
                ("n_max", ctypes.c_int32), ("n_dist", ctypes.c_int32), ("U_steps", ctypes.c_int32),
                ("U_lo_ppm", ctypes.c_int64), ("U_hi_ppm", ctypes.c_int64), ("T_lo", ctypes.c_int64),
                ("T_hi", ctypes.c_int64), ("T_dist", ctypes.c_int32), ("deadline_pm", ctypes.c_int32),
                ("alpha_lo_pm", ctypes.c_int32), ("alpha_hi_pm", ctypes.c_int32), ("mu_dist", ctypes.c_int32),
                ("prm_pm", ctypes.c_int32), ("mode", ctypes.c_int32), ("beta_c_pm", ctypes.c_int32),
                ("beta_m_pm", ctypes.c_int32), ("pad_", ctypes.c_int32), ("u_max_ppm", ctypes.c_int64),
                ("max_tries", ctypes.c_int32), ("nthreads", ctypes.c_int32)]


class GenOut(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in
                ("set_off", "T", "D", "A", "B", "u_ppm", "type", "C1", "alpha_pm", "mu_pm", "flags")]


_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(GEN_PATH):
            from ._build import build_gen_only
            build_gen_only()
        _lib = ctypes.CDLL(GEN_PATH)
        _lib.gpa_gen_tasksets.argtypes = [ctypes.POINTER(GenParams), ctypes.POINTER(GenOut),
                                          ctypes.POINTER(ctypes.c_int64)]
    return _lib


DEFAULTS = dict(seed=0, nsets=1, n_min=8, n_max=8, n_dist="UNIFORM", U_steps=0, U_lo_ppm=800000,
                U_hi_ppm=800000, T_lo=10000, T_hi=1000000, T_dist="LOGUNIFORM", deadline_pm=1000,
                alpha_lo_pm=50, alpha_hi_pm=300, mu_dist="UNIFORM", prm_pm=500, mode="ALPHA", beta_c_pm=20,
                beta_m_pm=100, u_max_ppm=0, max_tries=1, nthreads=os.cpu_count() or 1)


def gen_tasksets(**kw):
    """Generate a batch; returns a dict of numpy arrays (set_off, T, D, A, B, u_ppm, type, C1, alpha_pm, mu_pm,
    flags) plus ``n_max``."""
    p = dict(DEFAULTS)
    unknown = set(kw) - set(p)
    if unknown:
        raise TypeError(f"unknown generator parameters: {sorted(unknown)}")
    p.update(kw)
    gp = GenParams(int(p["seed"]) & (2**64 - 1), int(p["nsets"]), int(p["n_min"]), int(p["n_max"]),
                   DIST[p["n_dist"]], int(p["U_steps"]), int(p["U_lo_ppm"]), int(p["U_hi_ppm"]), int(p["T_lo"]),
                   int(p["T_hi"]), DIST[p["T_dist"]], int(p["deadline_pm"]), int(p["alpha_lo_pm"]),
                   int(p["alpha_hi_pm"]), DIST[p["mu_dist"]], int(p["prm_pm"]), MODE[p["mode"]],
                   int(p["beta_c_pm"]), int(p["beta_m_pm"]), 0, int(p["u_max_ppm"]), int(p["max_tries"]),
                   int(p["nthreads"]))
    lib = _load()
    nt = ctypes.c_int64()
    st = lib.gpa_gen_tasksets(ctypes.byref(gp), None, ctypes.byref(nt))
    if st != 0:
        raise ValueError(f"gpa_gen_tasksets rejected the parameters (status {st})")
    n = nt.value
    ns = int(p["nsets"])
    out = {
        "set_off": np.zeros(ns + 1, np.int64), "T": np.zeros(n, np.int64), "D": np.zeros(n, np.int64),
        "A": np.zeros(n, np.int64), "B": np.zeros(n, np.int64), "u_ppm": np.zeros(n, np.int64),
        "type": np.zeros(n, np.uint8), "C1": np.zeros(n, np.int64), "alpha_pm": np.zeros(n, np.int16),
        "mu_pm": np.zeros(n, np.int16), "flags": np.zeros(ns, np.uint8),
    }
    go = GenOut(*[out[k].ctypes.data for k in
                  ("set_off", "T", "D", "A", "B", "u_ppm", "type", "C1", "alpha_pm", "mu_pm", "flags")])
    st = lib.gpa_gen_tasksets(ctypes.byref(gp), ctypes.byref(go), ctypes.byref(nt))
    if st != 0:
        raise ValueError(f"gpa_gen_tasksets failed (status {st})")
    out["n_max"] = int(p["n_max"])
    return out


def subset(sets, idx):
    """The task sets with the given indices, as a new contiguous batch."""
    off = sets["set_off"]
    idx = np.asarray(idx, dtype=np.int64)
    sizes = off[idx + 1] - off[idx]
    new_off = np.zeros(len(idx) + 1, np.int64)
    np.cumsum(sizes, out=new_off[1:])
    take = np.concatenate([np.arange(off[i], off[i + 1]) for i in idx]) if len(idx) else np.zeros(0, np.int64)
    out = {"set_off": new_off}
    for k in ("T", "D", "A", "B", "u_ppm", "type", "C1", "alpha_pm", "mu_pm"):
        if k in sets:
            out[k] = np.ascontiguousarray(sets[k][take])
    out["n_max"] = sets.get("n_max", 128)
    return out
