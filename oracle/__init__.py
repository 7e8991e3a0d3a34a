"""CPU oracle for the contention-aware partition/allocation path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  It wraps ``oracle.c`` (plain C, built with
gcc into ``liboracle.so`` next to this file) through ctypes and takes numpy
arrays.  Nothing here imports the CUDA package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

POLICY = {"SMS": 0, "BF": 1, "ONE_GPU": 2}
SCHED = {"DM": 0, "EDF": 1}
REASON = {"OK": 0, "LEMMA1": 1, "LEMMA2": 2, "NO_MERGE": 3, "TEST": 4, "INVALID": 5}

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OracleRefused(RuntimeError):
    """The oracle declined an analysis that would not end in reasonable time
    (an EDF busy period beyond 2^100, or more than 2^34 demand terms)."""


class _Checked:
    """The loaded library, each of whose functions raises OracleRefused after
    a call during which the oracle refused an analysis."""

    def __init__(self, cdll):
        self._cdll = cdll

    def __getattr__(self, name):
        f = getattr(self._cdll, name)
        if name == "orc_take_refused":
            return f
        take = self._cdll.orc_take_refused

        def call(*args):
            r = f(*args)
            if take():
                raise OracleRefused(f"oracle {name}: an analysis was refused (too long to run)")
            return r
        return call


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
    return _Checked(_lib)


# Arrays converted for a call are kept alive in _KEEP until the next call
# starts: a pointer into a temporary copy must outlive the foreign call.
_KEEP = []


def _p(a):
    if a is None:
        return ctypes.c_void_p(0)
    _KEEP.append(a)
    return ctypes.c_void_p(a.ctypes.data)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _fresh():
    _KEEP.clear()


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def wcet(A, B, k, m):
    _fresh()
    out = ctypes.c_int64()
    _check(lib().orc_wcet(ctypes.c_int64(A), ctypes.c_int64(B), ctypes.c_int64(k), ctypes.c_int64(m),
                          ctypes.byref(out)), "wcet")
    return out.value


def wcet_tables(sets, M, g, kc, km):
    _fresh()
    off = _i64(sets["set_off"])
    ntasks = int(off[-1])
    Mu = M // g
    Cn = np.zeros(ntasks * Mu, dtype=np.int64)
    Cc = np.zeros(ntasks * Mu, dtype=np.int64)
    _check(lib().orc_wcet_tables(ctypes.c_int64(len(off) - 1), _p(off), _p(_i64(sets["A"])), _p(_i64(sets["B"])),
                                 _p(_u8(sets["type"])), ctypes.c_int64(M), ctypes.c_int64(g), ctypes.c_int64(kc),
                                 ctypes.c_int64(km), _p(Cn), _p(Cc)), "wcet_tables")
    return Cn, Cc


def rta(T, D, A, B, typ, in_mask, m, kc, km):
    """Per-partition test of the tasks selected by in_mask at m SMs -> (verdict, R)."""
    _fresh()
    n = len(T)
    R = np.full(n, -1, dtype=np.int64)
    v = lib().orc_rta(ctypes.c_int(n), _p(_i64(T)), _p(_i64(D)), _p(_i64(A)), _p(_i64(B)), _p(_u8(typ)),
                      _p(_u8(in_mask)), ctypes.c_int64(m), ctypes.c_int64(kc), ctypes.c_int64(km), _p(R))
    return int(v), R


def edf(T, D, A, B, typ, in_mask, m, kc, km):
    """EDF processor-demand test of the tasks selected by in_mask at m SMs -> verdict."""
    _fresh()
    return int(lib().orc_edf(ctypes.c_int(len(T)), _p(_i64(T)), _p(_i64(D)), _p(_i64(A)), _p(_i64(B)),
                             _p(_u8(typ)), _p(_u8(in_mask)), ctypes.c_int64(m), ctypes.c_int64(kc),
                             ctypes.c_int64(km)))


def _sizes(sizes):
    """(pointer, count) of an admissible size list; (None, 0) for every multiple of g."""
    if sizes is None or len(sizes) == 0:
        return None, 0
    arr = np.ascontiguousarray(sizes, dtype=np.int32)
    return _p(arr), len(arr)


def minm(T, D, A, B, typ, in_mask, lo, hi, g, kc, km, linear=True, sched="DM", sizes=None):
    _fresh()
    out = ctypes.c_int64()
    zp, zn = _sizes(sizes)
    _check(lib().orc_minm(ctypes.c_int(len(T)), _p(_i64(T)), _p(_i64(D)), _p(_i64(A)), _p(_i64(B)), _p(_u8(typ)),
                          _p(_u8(in_mask)), ctypes.c_int64(lo), ctypes.c_int64(hi), ctypes.c_int64(g),
                          ctypes.c_int64(kc), ctypes.c_int64(km), ctypes.c_int64(SCHED[sched]), zp,
                          ctypes.c_int64(zn), ctypes.c_int(1 if linear else 0), ctypes.byref(out)), "minm")
    return out.value


def workload(u, typ, in_mask, kc, km):
    _fresh()
    out = ctypes.c_int64()
    _check(lib().orc_workload(ctypes.c_int(len(u)), _p(_i64(u)), _p(_u8(typ)), _p(_u8(in_mask)), ctypes.c_int64(kc),
                              ctypes.c_int64(km), ctypes.byref(out)), "workload")
    return out.value


def lemma1_rejects(T, A, B, M):
    _fresh()
    return bool(lib().orc_lemma1_rejects(ctypes.c_int(len(T)), _p(_i64(T)), _p(_i64(A)), _p(_i64(B)),
                                         ctypes.c_int64(M)))


def test_schedulable(sets, M, g, kc, km, cand_set, part_of_task, map_stride, kparts, size_of_part, with_R=True,
                     sched="DM", sizes=None):
    _fresh()
    zp, zn = _sizes(sizes)
    off = _i64(sets["set_off"])
    cand_set = _i64(cand_set)
    nc = len(cand_set)
    pot = _u8(part_of_task)
    sop = np.ascontiguousarray(size_of_part, dtype=np.int32)
    verdict = np.zeros(nc, dtype=np.uint8)
    R = np.full(nc * map_stride, -1, dtype=np.int64) if with_R else None
    _check(lib().orc_test_schedulable(
        ctypes.c_int64(len(off) - 1), _p(off), _p(_i64(sets["T"])), _p(_i64(sets["D"])), _p(_i64(sets["A"])),
        _p(_i64(sets["B"])), _p(_u8(sets["type"])), ctypes.c_int64(M), ctypes.c_int64(g), ctypes.c_int64(kc),
        ctypes.c_int64(km), ctypes.c_int64(SCHED[sched]), zp, ctypes.c_int64(zn), ctypes.c_int64(nc), _p(cand_set),
        _p(pot),
        ctypes.c_int64(map_stride),
        ctypes.c_int64(kparts), _p(sop), _p(verdict), _p(R)), "test_schedulable")
    return verdict, R


def allocate(sets, M, g, kc, km, policy="SMS", act=False, linear=True, nthreads=1, sched="DM", sizes=None):
    _fresh()
    zp, zn = _sizes(sizes)
    off = _i64(sets["set_off"])
    nsets = len(off) - 1
    ntasks = int(off[-1])
    out = {
        "verdict": np.zeros(nsets, np.uint8), "reason": np.zeros(nsets, np.uint8),
        "n_parts": np.zeros(nsets, np.int32), "Pi": np.zeros(nsets, np.int32), "W": np.zeros(nsets, np.int64),
        "n_tests": np.zeros(nsets, np.int32), "part_of_task": np.zeros(ntasks, np.uint8),
        "size_of_part": np.zeros(ntasks, np.int16),
    }
    _check(lib().orc_allocate(
        ctypes.c_int64(nsets), _p(off), _p(_i64(sets["T"])), _p(_i64(sets["D"])), _p(_i64(sets["A"])),
        _p(_i64(sets["B"])), _p(_i64(sets["u_ppm"])), _p(_u8(sets["type"])), ctypes.c_int64(M), ctypes.c_int64(g),
        ctypes.c_int64(kc), ctypes.c_int64(km), ctypes.c_int64(SCHED[sched]), zp, ctypes.c_int64(zn),
        ctypes.c_int(POLICY[policy]),
        ctypes.c_int(1 if act else 0),
        ctypes.c_int(1 if linear else 0), _p(out["verdict"]), _p(out["reason"]), _p(out["n_parts"]), _p(out["Pi"]),
        _p(out["W"]), _p(out["n_tests"]), _p(out["part_of_task"]), _p(out["size_of_part"]),
        ctypes.c_int(nthreads)), "allocate")
    return out


def search_best(sets, M, g, kc, km, kmin, kmax, explicit=False, nthreads=1, sched="DM", sizes=None):
    _fresh()
    zp, zn = _sizes(sizes)
    off = _i64(sets["set_off"])
    nsets = len(off) - 1
    ntasks = int(off[-1])
    out = {
        "feasible": np.zeros(nsets, np.uint8), "W": np.zeros(nsets, np.int64),
        "sum_minm": np.zeros(nsets, np.int32), "n_blocks": np.zeros(nsets, np.int32),
        "spare": np.zeros(nsets, np.int32), "rgs": np.zeros(ntasks, np.uint8),
        "minm_block": np.zeros(nsets * kmax, np.int16),
    }
    args = [ctypes.c_int64(nsets), _p(off), _p(_i64(sets["T"])), _p(_i64(sets["D"])), _p(_i64(sets["A"])),
            _p(_i64(sets["B"])), _p(_i64(sets["u_ppm"])), _p(_u8(sets["type"])), ctypes.c_int64(M),
            ctypes.c_int64(g), ctypes.c_int64(kc), ctypes.c_int64(km), ctypes.c_int64(SCHED[sched]), zp,
            ctypes.c_int64(zn), ctypes.c_int(kmin), ctypes.c_int(kmax),
            _p(out["feasible"]), _p(out["W"]), _p(out["sum_minm"]), _p(out["n_blocks"]), _p(out["spare"]),
            _p(out["rgs"]), _p(out["minm_block"]), ctypes.c_int(nthreads)]
    if explicit:
        cand = ctypes.c_int64()
        _check(lib().orc_search_explicit(*args, ctypes.byref(cand)), "search_explicit")
        out["candidates"] = cand.value
    else:
        _check(lib().orc_search_best(*args), "search_best")
    return out


class Tenant:
    """One tenant of the serving loop, replayed on the CPU (ADMIT / ADD / REMOVE)."""

    COLS = ("T", "D", "A", "B", "u_ppm", "type")

    def __init__(self, M, g, kc, km, policy="SMS", act=False, sched="DM", sizes=None):
        self.M, self.g, self.kc, self.km = M, g, kc, km
        self.policy, self.act = POLICY[policy], 1 if act else 0
        self.sched = SCHED[sched]
        self.sizes = None if sizes is None or len(sizes) == 0 else np.ascontiguousarray(sizes, dtype=np.int32)

    def _model_args(self):
        zp = ctypes.c_void_p(self.sizes.ctypes.data) if self.sizes is not None else ctypes.c_void_p(0)
        return (ctypes.c_int64(self.sched), zp, ctypes.c_int64(0 if self.sizes is None else len(self.sizes)))
        self.tasks = {k: np.zeros(0, np.uint8 if k == "type" else np.int64) for k in self.COLS}
        self.part = np.zeros(0, np.uint8)
        self.size = np.zeros(0, np.int16)
        self.n_parts = 0
        self.Pi = 0
        self.W = 0
        self.alive = False

    @property
    def n(self):
        return len(self.tasks["T"])

    def _res(self, verdict, reason, path):
        return {"verdict": int(verdict), "reason": int(reason), "path": int(path), "n_tasks": self.n,
                "n_parts": self.n_parts, "Pi": self.Pi, "W": self.W, "part_of_task": self.part.copy(),
                "size_of_part": self.size[:self.n_parts].copy()}

    def admit(self, tasks):
        _fresh()
        n = len(tasks["T"])
        cols = {k: (_u8(tasks[k]) if k == "type" else _i64(tasks[k])) for k in self.COLS}
        v, r = ctypes.c_uint8(), ctypes.c_uint8()
        npart, Pi, W = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        part = np.zeros(max(n, 1), np.uint8)
        size = np.zeros(max(n, 1), np.int16)
        _check(lib().orc_serve_admit(ctypes.c_int(n), *[_p(cols[k]) for k in self.COLS], ctypes.c_int64(self.M),
                                     ctypes.c_int64(self.g), ctypes.c_int64(self.kc), ctypes.c_int64(self.km),
                                     *self._model_args(), ctypes.c_int(self.policy), ctypes.c_int(self.act),
                                     ctypes.byref(v),
                                     ctypes.byref(r), _p(part), _p(size), ctypes.byref(npart), ctypes.byref(Pi),
                                     ctypes.byref(W)), "serve_admit")
        if v.value:
            self.tasks = {k: cols[k].copy() for k in self.COLS}
            self.part, self.size = part[:n].copy(), size.copy()
            self.n_parts, self.Pi, self.W = npart.value, Pi.value, W.value
            self.alive = True
        return {"verdict": v.value, "reason": r.value, "path": 0, "n_tasks": n if v.value else 0,
                "n_parts": npart.value if v.value else 0, "Pi": Pi.value if v.value else 0,
                "W": W.value if v.value else 0, "part_of_task": part[:n].copy() if v.value else np.zeros(0, np.uint8),
                "size_of_part": size[:npart.value].copy() if v.value else np.zeros(0, np.int16)}

    def add(self, task):
        _fresh()
        n = self.n
        cols = {k: np.concatenate([self.tasks[k], np.asarray([task[k]], self.tasks[k].dtype)]) for k in self.COLS}
        v, r, path = ctypes.c_uint8(), ctypes.c_uint8(), ctypes.c_uint8()
        npart, Pi, W = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        part_in = np.ascontiguousarray(self.part, np.uint8) if n else np.zeros(1, np.uint8)
        size_in = np.ascontiguousarray(self.size, np.int16) if len(self.size) else np.zeros(1, np.int16)
        part = np.zeros(n + 1, np.uint8)
        size = np.zeros(n + 1, np.int16)
        _check(lib().orc_serve_add(ctypes.c_int(n), *[_p(cols[k]) for k in self.COLS], _p(part_in), _p(size_in),
                                   ctypes.c_int(self.n_parts), ctypes.c_int64(self.M), ctypes.c_int64(self.g),
                                   ctypes.c_int64(self.kc), ctypes.c_int64(self.km), *self._model_args(),
                                   ctypes.c_int(self.policy),
                                   ctypes.c_int(self.act), ctypes.byref(v), ctypes.byref(r), ctypes.byref(path),
                                   _p(part), _p(size), ctypes.byref(npart), ctypes.byref(Pi), ctypes.byref(W)),
               "serve_add")
        if v.value:
            self.tasks = cols
            self.part, self.size = part.copy(), size.copy()
            self.n_parts, self.Pi, self.W = npart.value, Pi.value, W.value
        return self._res(v.value, r.value, path.value)

    def remove(self, index):
        _fresh()
        n = self.n
        outs = {k: np.zeros(max(n - 1, 1), np.uint8 if k == "type" else np.int64) for k in self.COLS}
        part = np.zeros(max(n - 1, 1), np.uint8)
        size = np.zeros(max(n, 1), np.int16)
        npart, Pi, W = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(lib().orc_serve_remove(ctypes.c_int(n), *[_p(self.tasks[k]) for k in self.COLS], _p(self.part),
                                      _p(self.size), ctypes.c_int(self.n_parts), ctypes.c_int(index),
                                      ctypes.c_int64(self.M), ctypes.c_int64(self.g), ctypes.c_int64(self.kc),
                                      ctypes.c_int64(self.km), *self._model_args(), *[_p(outs[k]) for k in self.COLS],
                                      _p(part),
                                      _p(size), ctypes.byref(npart), ctypes.byref(Pi), ctypes.byref(W)),
               "serve_remove")
        self.tasks = {k: outs[k][:n - 1].copy() for k in self.COLS}
        self.part, self.size = part[:n - 1].copy(), size.copy()
        self.n_parts, self.Pi, self.W = npart.value, Pi.value, W.value
        return self._res(1, 0, 0)
