"""GB300-native contention-aware GPU-partition schedulability (arXiv 2105.10312).

A thin ctypes binding over ``libgpa.so`` (the C ABI declared in ``include/gpa.h``).
Every step of the computation runs in the library's CUDA kernels; this module
only marshals arguments: torch CUDA tensors go in as device pointers (GPA_DEVICE),
numpy arrays as host pointers (GPA_HOST: copied in and checked on the device,
synchronous).

The first call into the library raises ImportError if ``libgpa.so`` has not
been built (``python -c "import __graft_entry__ as g; g.build()"``): there is
no CPU fallback.  The generator (``gen``) and the workload presets need no GPU.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import gen as _gen
from .gen import gen_tasksets  # noqa: F401  (re-export)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpa.so")

# --- constants mirrored from gpa.h -------------------------------------------
OK, ERR_ARG, ERR_RANGE, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_BUSY, ERR_NOTFOUND = 0, -1, -2, -3, -4, -5, -6, -7
HOST, DEVICE = 0, 1
POLICY = {"SMS": 0, "BF": 1, "ONE_GPU": 2}
SCHED = {"DM": 0, "EDF": 1}
REASON = {"OK": 0, "LEMMA1": 1, "LEMMA2": 2, "NO_MERGE": 3, "TEST": 4, "INVALID": 5, "UNDECIDED": 6}
OPT = {"AUTOTUNE": 1, "GRAPH": 2, "FAST_WARPS": 3, "FAST_CHUNK": 4, "FAST_BLOCKS": 5, "PER_SET_LAUNCH": 6,
       "PROFILE": 7, "FAST_STAGES": 8, "HOST_SLICES": 9,
       "HOST_COPY": 10, "MERGE_WARPS": 11, "MERGE_GROUP": 12, "MERGE_BLOCKS": 13, "TEST_WARPS": 14,
       "MERGE_TOPFIRST": 15}
EXPLICIT_MAX = 1 << 26
NMAX, SERVE_NMAX, MMAX, SEARCH_NMAX, SEARCH_KMAX = 256, 128, 1024, 14, 8

_vp = ctypes.c_void_p


class GpaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gpa error {code}: {msg}")
        self.code = code


def _check(code):
    if code != OK:
        buf = ctypes.create_string_buffer(512)
        lib().gpa_last_error(buf, 512)
        raise GpaError(code, buf.value.decode(errors="replace"))


class Tasksets(ctypes.Structure):
    _fields_ = [("nsets", ctypes.c_int64), ("mem", ctypes.c_int32), ("n_max", ctypes.c_int32),
                ("set_off", _vp), ("T", _vp), ("D", _vp), ("A", _vp), ("B", _vp), ("u_ppm", _vp), ("type", _vp)]


class Model(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("g", ctypes.c_int32), ("k_c_pm", ctypes.c_int32), ("k_m_pm", ctypes.c_int32),
                ("sched", ctypes.c_int32), ("nsizes", ctypes.c_int32), ("sizes", _vp)]


def make_model(M, g, k_c_pm, k_m_pm, sched="DM", sizes=None):
    """The gpa_model of the arguments; the size list (if any) is kept alive
    on the returned structure."""
    if sizes is None or len(sizes) == 0:
        return Model(M, g, k_c_pm, k_m_pm, SCHED[sched], 0, None)
    arr = np.ascontiguousarray(sizes, dtype=np.int32)
    md = Model(M, g, k_c_pm, k_m_pm, SCHED[sched], len(arr), arr.ctypes.data)
    md._keep = arr
    return md


class Candidates(ctypes.Structure):
    _fields_ = [("ncands", ctypes.c_int64), ("mem", ctypes.c_int32), ("map_stride", ctypes.c_int32),
                ("kparts", ctypes.c_int32), ("pad_", ctypes.c_int32), ("set", _vp), ("part_of_task", _vp),
                ("size_of_part", _vp)]


class Params(ctypes.Structure):
    _fields_ = [("policy", ctypes.c_int32), ("act", ctypes.c_int32), ("linear_merge", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


class AllocResult(ctypes.Structure):
    _fields_ = [("mem", ctypes.c_int32), ("pad_", ctypes.c_int32), ("verdict", _vp), ("reason", _vp),
                ("n_parts", _vp), ("Pi", _vp), ("W", _vp), ("n_tests", _vp), ("part_of_task", _vp),
                ("size_of_part", _vp)]


class BestResult(ctypes.Structure):
    _fields_ = [("mem", ctypes.c_int32), ("pad_", ctypes.c_int32), ("feasible", _vp), ("W", _vp),
                ("sum_minm", _vp), ("n_blocks", _vp), ("spare", _vp), ("rgs", _vp), ("minm_block", _vp)]


_lib = None


class AluPeak(ctypes.Structure):
    _fields_ = [("terms_per_s", ctypes.c_double), ("imad_per_s", ctypes.c_double), ("term_ms", ctypes.c_double),
                ("terms", ctypes.c_int64)]


def _set_signatures(L):
    L.gpa_ctx_create.argtypes = [ctypes.c_int32, _vp, ctypes.POINTER(_vp)]
    L.gpa_ctx_destroy.argtypes = [_vp]
    L.gpa_ctx_set_stream.argtypes = [_vp, _vp]
    L.gpa_ctx_sync.argtypes = [_vp]
    L.gpa_ctx_launch_count.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
    L.gpa_ctx_set_option.argtypes = [_vp, ctypes.c_int32, ctypes.c_int64]
    L.gpa_ctx_last_timing.argtypes = [_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_int32)]
    L.gpa_last_error.argtypes = [ctypes.c_char_p, ctypes.c_int32]
    L.gpa_validate.argtypes = [ctypes.POINTER(Tasksets), ctypes.POINTER(Model), ctypes.POINTER(ctypes.c_int64)]
    L.gpa_build_wcet_tables.argtypes = [_vp, ctypes.POINTER(Tasksets), ctypes.POINTER(Model), _vp, _vp]
    L.gpa_test_schedulable.argtypes = [_vp, ctypes.POINTER(Tasksets), ctypes.POINTER(Model),
                                          ctypes.POINTER(Candidates), _vp, _vp]
    L.gpa_allocate.argtypes = [_vp, ctypes.POINTER(Tasksets), ctypes.POINTER(Model), ctypes.POINTER(Params),
                                  ctypes.POINTER(AllocResult)]
    L.gpa_allocate_multi.argtypes = [_vp, ctypes.POINTER(Tasksets), ctypes.POINTER(Model), ctypes.POINTER(Params),
                                     ctypes.c_int32, ctypes.POINTER(AllocResult)]
    L.gpa_search_best.argtypes = [_vp, ctypes.POINTER(Tasksets), ctypes.POINTER(Model), ctypes.c_int32,
                                     ctypes.c_int32, ctypes.POINTER(BestResult)]
    L.gpa_enumerate_partitions.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_uint64)]
    L.gpa_unrank_composition.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _vp]
    L.gpa_count_rgs.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64)]
    L.gpa_unrank_rgs.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _vp]
    L.gpa_allocate_noalloc.argtypes = [_vp, ctypes.POINTER(Tasksets), ctypes.POINTER(Model), ctypes.POINTER(Params),
                                       ctypes.POINTER(AllocResult)]
    L.gpa_allocate_noalloc_status.argtypes = [_vp]
    L.gpa_ctx_last_terms.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
    L.gpa_search_explicit.argtypes = [_vp, ctypes.POINTER(Tasksets), ctypes.POINTER(Model), ctypes.c_int32,
                                      ctypes.c_int32, ctypes.POINTER(BestResult), _vp, ctypes.POINTER(ctypes.c_int64)]
    L.gpa_measure_alu_peak.argtypes = [_vp, ctypes.POINTER(AluPeak)]


def lib():
    """The loaded libgpa.so; raises ImportError if the CUDA extension was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build the CUDA extension first "
                "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        _set_signatures(L)
        _lib = L
    return _lib


# --- array helpers --------------------------------------------------------------

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _mem_of(x):
    if _is_torch(x):
        return DEVICE if x.is_cuda else HOST
    return HOST


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        assert x.is_contiguous(), "tensors must be contiguous"
        return x.data_ptr()
    assert isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"], "numpy arrays must be C-contiguous"
    return x.ctypes.data


def _empty_like_mem(mem, n, np_dtype, device=None):
    if mem == DEVICE:
        import torch
        tdt = {np.uint8: torch.uint8, np.int16: torch.int16, np.int32: torch.int32, np.int64: torch.int64}[np_dtype]
        return torch.empty(max(n, 0), dtype=tdt, device=device)
    return np.zeros(max(n, 0), dtype=np_dtype)


def _len(x):
    return int(x.numel()) if _is_torch(x) else int(x.size)


def make_tasksets(sets, n_max=None):
    """Build the gpa_tasksets view over a dict of arrays (all numpy or all CUDA tensors)."""
    mem = _mem_of(sets["set_off"])
    nsets = _len(sets["set_off"]) - 1
    if n_max is None:
        n_max = sets.get("n_max")
    if n_max is None:
        # the largest set of the batch (the kernels are chosen by it: up to 128
        # tasks, or up to 256)
        off = sets["set_off"]
        n_max = int((off[1:] - off[:-1]).max()) if nsets > 0 else 0
    n_max = int(n_max)
    ts = Tasksets(nsets, mem, int(n_max), _ptr(sets["set_off"]), _ptr(sets["T"]), _ptr(sets["D"]),
                  _ptr(sets["A"]), _ptr(sets["B"]), _ptr(sets.get("u_ppm")), _ptr(sets["type"]))
    return ts, mem


def validate(sets, M=None, g=1, k_c_pm=1200, k_m_pm=2300):
    ts, mem = make_tasksets(sets)
    md = Model(M, g, k_c_pm, k_m_pm) if M is not None else None
    bad = ctypes.c_int64(-1)
    code = lib().gpa_validate(ctypes.byref(ts), ctypes.byref(md) if md is not None else None, ctypes.byref(bad))
    return code, bad.value


def enumerate_partitions(Mu, kmin, kmax):
    out = ctypes.c_uint64()
    _check(lib().gpa_enumerate_partitions(Mu, kmin, kmax, ctypes.byref(out)))
    return out.value


def unrank_composition(Mu, k, rank):
    parts = np.zeros(k, dtype=np.int32)
    _check(lib().gpa_unrank_composition(Mu, k, ctypes.c_uint64(rank), parts.ctypes.data))
    return parts


def count_rgs(n, kmax):
    out = ctypes.c_uint64()
    _check(lib().gpa_count_rgs(n, kmax, ctypes.byref(out)))
    return out.value


def unrank_rgs(n, kmax, rank):
    rgs = np.zeros(max(n, 1), dtype=np.uint8)
    _check(lib().gpa_unrank_rgs(n, kmax, ctypes.c_uint64(rank), rgs.ctypes.data))
    return rgs[:n]


class Context:
    """A gpa_ctx bound to one CUDA device and stream (default: torch's current stream)."""

    def __init__(self, device=0, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self._stream = stream
        h = _vp()
        _check(lib().gpa_ctx_create(device, _vp(stream.cuda_stream), ctypes.byref(h)))
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            lib().gpa_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._stream = stream
        _check(lib().gpa_ctx_set_stream(self._h, _vp(stream.cuda_stream)))

    def set_option(self, name, value):
        _check(lib().gpa_ctx_set_option(self._h, OPT[name], int(value)))

    def sync(self):
        _check(lib().gpa_ctx_sync(self._h))

    def launch_count(self):
        out = ctypes.c_int64()
        _check(lib().gpa_ctx_launch_count(self._h, ctypes.byref(out)))
        return out.value

    def last_timing(self):
        """Kernel times (ms) of the last call made with the PROFILE option on."""
        ms = (ctypes.c_float * 4)()
        cnt = ctypes.c_int32()
        _check(lib().gpa_ctx_last_timing(self._h, ms, 4, ctypes.byref(cnt)))
        return [ms[i] for i in range(cnt.value)]

    def last_terms(self):
        """Interference terms the kernels of the last device-buffer call evaluated."""
        out = ctypes.c_int64()
        _check(lib().gpa_ctx_last_terms(self._h, ctypes.byref(out)))
        return out.value

    def measure_alu_peak(self):
        """The device's rate of interference terms and of integer multiply-adds."""
        pk = AluPeak()
        _check(lib().gpa_measure_alu_peak(self._h, ctypes.byref(pk)))
        return {"terms_per_s": pk.terms_per_s, "imad_per_s": pk.imad_per_s, "term_ms": pk.term_ms,
                "terms": pk.terms}

    @property
    def handle(self):
        return self._h

    # --- entry points ----------------------------------------------------------

    def build_wcet_tables(self, sets, M, g=1, k_c_pm=1200, k_m_pm=2300, out=None):
        ts, mem = make_tasksets(sets)
        md = Model(M, g, k_c_pm, k_m_pm)
        ntasks = int(sets["set_off"][-1])
        size = ntasks * (M // g)
        dev = sets["T"].device if mem == DEVICE else None
        Cn = out[0] if out else _empty_like_mem(mem, size, np.int64, dev)
        Cc = out[1] if out else _empty_like_mem(mem, size, np.int64, dev)
        _check(lib().gpa_build_wcet_tables(self._h, ctypes.byref(ts), ctypes.byref(md), _ptr(Cn), _ptr(Cc)))
        return Cn, Cc

    def test_schedulable(self, sets, M, cand_set, part_of_task, size_of_part, map_stride, kparts, g=1,
                         k_c_pm=1200, k_m_pm=2300, with_R=True, sched="DM", sizes=None):
        ts, mem = make_tasksets(sets)
        md = make_model(M, g, k_c_pm, k_m_pm, sched, sizes)
        nc = _len(cand_set)
        cands = Candidates(nc, mem, int(map_stride), int(kparts), 0, _ptr(cand_set), _ptr(part_of_task),
                           _ptr(size_of_part))
        dev = sets["T"].device if mem == DEVICE else None
        verdict = _empty_like_mem(mem, nc, np.uint8, dev)
        R = _empty_like_mem(mem, nc * map_stride, np.int64, dev) if with_R else None
        _check(lib().gpa_test_schedulable(self._h, ctypes.byref(ts), ctypes.byref(md), ctypes.byref(cands),
                                         _ptr(verdict), _ptr(R)))
        return verdict, R

    def alloc_result(self, sets, with_tests=True):
        mem = _mem_of(sets["set_off"])
        nsets = _len(sets["set_off"]) - 1
        ntasks = int(sets["set_off"][-1])
        dev = sets["T"].device if mem == DEVICE else None
        return {
            "verdict": _empty_like_mem(mem, nsets, np.uint8, dev),
            "reason": _empty_like_mem(mem, nsets, np.uint8, dev),
            "n_parts": _empty_like_mem(mem, nsets, np.int32, dev),
            "Pi": _empty_like_mem(mem, nsets, np.int32, dev),
            "W": _empty_like_mem(mem, nsets, np.int64, dev),
            "n_tests": _empty_like_mem(mem, nsets, np.int32, dev) if with_tests else None,
            "part_of_task": _empty_like_mem(mem, ntasks, np.uint8, dev),
            "size_of_part": _empty_like_mem(mem, ntasks, np.int16, dev),
        }

    def allocate(self, sets, M, g=1, k_c_pm=1200, k_m_pm=2300, policy="SMS", act=False, linear=True, out=None,
                 sched="DM", sizes=None):
        ts, mem = make_tasksets(sets)
        md = make_model(M, g, k_c_pm, k_m_pm, sched, sizes)
        pr = Params(POLICY[policy], 1 if act else 0, 1 if linear else 0, 0)
        if out is None:
            out = self.alloc_result(sets)
        res = AllocResult(mem, 0, _ptr(out["verdict"]), _ptr(out["reason"]), _ptr(out["n_parts"]),
                          _ptr(out["Pi"]), _ptr(out["W"]), _ptr(out.get("n_tests")), _ptr(out["part_of_task"]),
                          _ptr(out["size_of_part"]))
        _check(lib().gpa_allocate(self._h, ctypes.byref(ts), ctypes.byref(md), ctypes.byref(pr), ctypes.byref(res)))
        return out

    def allocate_multi(self, sets, M, g=1, k_c_pm=1200, k_m_pm=2300, policies=("SMS", "ONE_GPU"), act=False,
                       linear=True, outs=None, sched="DM", sizes=None):
        """gpa_allocate_multi: the batch decided under every policy of
        ``policies`` (names, or (name, act) pairs) in one call; host inputs
        are copied to the device once for all of them.  Returns one result
        dict per policy, as ``allocate`` returns."""
        ts, mem = make_tasksets(sets)
        md = make_model(M, g, k_c_pm, k_m_pm, sched, sizes)
        pol = [(q, act) if isinstance(q, str) else (q[0], bool(q[1])) for q in policies]
        if outs is None:
            outs = [self.alloc_result(sets) for _ in pol]
        if len(outs) != len(pol):
            raise ValueError("allocate_multi: one result per policy")
        prs = (Params * len(pol))(*[Params(POLICY[q], 1 if a else 0, 1 if linear else 0, 0) for q, a in pol])
        res = (AllocResult * len(pol))(*[
            AllocResult(mem, 0, _ptr(o["verdict"]), _ptr(o["reason"]), _ptr(o["n_parts"]), _ptr(o["Pi"]),
                        _ptr(o["W"]), _ptr(o.get("n_tests")), _ptr(o["part_of_task"]), _ptr(o["size_of_part"]))
            for o in outs])
        _check(lib().gpa_allocate_multi(self._h, ctypes.byref(ts), ctypes.byref(md), prs, len(pol), res))
        return outs

    def best_result(self, sets, kmax):
        mem = _mem_of(sets["set_off"])
        nsets = _len(sets["set_off"]) - 1
        ntasks = int(sets["set_off"][-1])
        dev = sets["T"].device if mem == DEVICE else None
        return {
            "feasible": _empty_like_mem(mem, nsets, np.uint8, dev),
            "W": _empty_like_mem(mem, nsets, np.int64, dev),
            "sum_minm": _empty_like_mem(mem, nsets, np.int32, dev),
            "n_blocks": _empty_like_mem(mem, nsets, np.int32, dev),
            "spare": _empty_like_mem(mem, nsets, np.int32, dev),
            "rgs": _empty_like_mem(mem, ntasks, np.uint8, dev),
            "minm_block": _empty_like_mem(mem, nsets * kmax, np.int16, dev),
        }

    def search_best(self, sets, M, g=1, k_c_pm=1200, k_m_pm=2300, kmin=1, kmax=4, out=None, sched="DM", sizes=None):
        ts, mem = make_tasksets(sets)
        md = make_model(M, g, k_c_pm, k_m_pm, sched, sizes)
        if out is None:
            out = self.best_result(sets, kmax)
        res = BestResult(mem, 0, _ptr(out["feasible"]), _ptr(out["W"]), _ptr(out["sum_minm"]),
                         _ptr(out["n_blocks"]), _ptr(out["spare"]), _ptr(out["rgs"]), _ptr(out["minm_block"]))
        _check(lib().gpa_search_best(self._h, ctypes.byref(ts), ctypes.byref(md), kmin, kmax, ctypes.byref(res)))
        return out

    def explicit_count(self, sets, M, g=1, kmin=1, kmax=4, k_c_pm=1200, k_m_pm=2300, sched="DM"):
        """Explicit candidates per set for the batch's n_max (the cand_verdict stride)."""
        ts, _ = make_tasksets(sets)
        md = make_model(M, g, k_c_pm, k_m_pm, sched)
        n = ctypes.c_int64()
        empty = Tasksets(0, ts.mem, ts.n_max, ts.set_off, None, None, None, None, None, None)
        res = BestResult(ts.mem, 0, None, None, None, None, None, None, None)
        _check(lib().gpa_search_explicit(self._h, ctypes.byref(empty), ctypes.byref(md), kmin, kmax,
                                         ctypes.byref(res), None, ctypes.byref(n)))
        return n.value

    def search_explicit(self, sets, M, g=1, k_c_pm=1200, k_m_pm=2300, kmin=1, kmax=4, out=None, sched="DM",
                        cand_verdict=False):
        """The optimum over every explicit candidate (composition x map); with
        cand_verdict=True also every candidate's verdict, [nsets, count]."""
        ts, mem = make_tasksets(sets)
        md = make_model(M, g, k_c_pm, k_m_pm, sched)
        if out is None:
            out = self.best_result(sets, kmax)
        res = BestResult(mem, 0, _ptr(out["feasible"]), _ptr(out["W"]), _ptr(out["sum_minm"]),
                         _ptr(out["n_blocks"]), _ptr(out["spare"]), _ptr(out["rgs"]), _ptr(out["minm_block"]))
        cv = None
        if cand_verdict:
            stride = self.explicit_count(sets, M, g, kmin, kmax, k_c_pm, k_m_pm, sched)
            dev = sets["T"].device if mem == DEVICE else None
            cv = _empty_like_mem(mem, (_len(sets["set_off"]) - 1) * stride, np.uint8, dev)
        n = ctypes.c_int64()
        _check(lib().gpa_search_explicit(self._h, ctypes.byref(ts), ctypes.byref(md), kmin, kmax, ctypes.byref(res),
                                         _ptr(cv), ctypes.byref(n)))
        if cand_verdict:
            out["cand_verdict"] = cv.reshape(-1, n.value) if n.value else cv
        return out


NOALLOC_MAX_SETS = 262144
MULTI_MAX_POLICIES = 8


def allocate_noalloc(sets, out, M, g=1, k_c_pm=1200, k_m_pm=2300, policy="SMS", act=False, linear=True,
                     stream=None, sched="DM"):
    """gpa_allocate_noalloc: the heuristic for callers that may not allocate device
    memory.  No context; the library's static device scratch is used, so calls
    must not overlap on the GPU.  ``sets`` and ``out`` are CUDA tensors the caller
    allocated; work is enqueued on ``stream`` (default: torch's current stream).
    Problems found on the device are reported by allocate_noalloc_status."""
    import torch
    ts, mem = make_tasksets(sets)
    md = make_model(M, g, k_c_pm, k_m_pm, sched)
    pr = Params(POLICY[policy], 1 if act else 0, 1 if linear else 0, 0)
    res = AllocResult(mem, 0, _ptr(out["verdict"]), _ptr(out["reason"]), _ptr(out["n_parts"]), _ptr(out["Pi"]),
                      _ptr(out["W"]), _ptr(out.get("n_tests")), _ptr(out["part_of_task"]), _ptr(out["size_of_part"]))
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().gpa_allocate_noalloc(_vp(stream.cuda_stream), ctypes.byref(ts), ctypes.byref(md), ctypes.byref(pr),
                                      ctypes.byref(res)))
    return out


def allocate_noalloc_status(stream=None):
    """gpa_allocate_noalloc_status: waits for ``stream`` and raises GpaError
    (ERR_TIMEOUT: a set was left undecided; ERR_RANGE: a set failed
    validation) if the allocation-free calls since the last status recorded a
    problem on the current device; clears the record."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().gpa_allocate_noalloc_status(_vp(stream.cuda_stream)))


def to_device(sets, device="cuda"):
    """Copy a numpy task batch to CUDA tensors (plumbing for callers and tests)."""
    import torch
    out = {}
    for k, v in sets.items():
        if isinstance(v, np.ndarray):
            out[k] = torch.from_numpy(np.ascontiguousarray(v)).to(device)
        else:
            out[k] = v
    return out


# --- serving ------------------------------------------------------------------

SERVE_OP = {"ADMIT": 0, "ADD": 1, "REMOVE": 2, "EVICT": 3}
PATH = {"NONE": 0, "FIT": 1, "GROW": 2, "NEW": 3, "REALLOC": 4}


class ServeCfg(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("g", ctypes.c_int32), ("k_c_pm", ctypes.c_int32), ("k_m_pm", ctypes.c_int32),
                ("policy", ctypes.c_int32), ("act", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("nstreams", ctypes.c_int32), ("queue_cap", ctypes.c_int32), ("slots_per_chunk", ctypes.c_int32),
                ("max_tenants", ctypes.c_int64), ("reserve_bytes", ctypes.c_int64), ("sched", ctypes.c_int32),
                ("nsizes", ctypes.c_int32), ("sizes", _vp)]


class Request(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("n", ctypes.c_int32), ("tenant", ctypes.c_int64), ("index", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("T", _vp), ("D", _vp), ("A", _vp), ("B", _vp), ("u_ppm", _vp),
                ("type", _vp)]


class Response(ctypes.Structure):
    _fields_ = [("req_id", ctypes.c_uint64), ("status", ctypes.c_int32), ("verdict", ctypes.c_uint8),
                ("reason", ctypes.c_uint8), ("path", ctypes.c_uint8), ("pad_", ctypes.c_uint8),
                ("n_tasks", ctypes.c_int32), ("n_parts", ctypes.c_int32), ("Pi", ctypes.c_int32),
                ("W", ctypes.c_int64), ("part_of_task", ctypes.c_uint8 * SERVE_NMAX),
                ("size_of_part", ctypes.c_int16 * SERVE_NMAX),
                ("latency_us", ctypes.c_double)]

    def as_dict(self):
        n, k = self.n_tasks, self.n_parts
        return {"req_id": self.req_id, "status": self.status, "verdict": self.verdict, "reason": self.reason,
                "path": self.path, "n_tasks": n, "n_parts": k, "Pi": self.Pi, "W": self.W,
                "part_of_task": np.array(self.part_of_task[:n], np.uint8),
                "size_of_part": np.array(self.size_of_part[:k], np.int16), "latency_us": self.latency_us}


def _serve_sigs(L):
    L.gpa_serve_start.argtypes = [_vp, ctypes.POINTER(ServeCfg)]
    L.gpa_serve_submit.argtypes = [_vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    L.gpa_serve_poll.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(Response), ctypes.c_int64]
    L.gpa_serve_stop.argtypes = [_vp]
    L.gpa_serve_stats.argtypes = [_vp] + [ctypes.POINTER(ctypes.c_int64)] * 5


class Server:
    """The admission-control server of a Context (gpa_serve_*)."""

    def __init__(self, ctx, M, g=1, k_c_pm=1200, k_m_pm=2300, policy="SMS", act=False, max_batch=1024, nstreams=3,
                 queue_cap=1 << 20, slots_per_chunk=256, max_tenants=1 << 16, reserve_bytes=1 << 30, sched="DM",
                 sizes=None):
        _serve_sigs(lib())
        self.ctx = ctx
        zs = None if sizes is None or len(sizes) == 0 else np.ascontiguousarray(sizes, dtype=np.int32)
        cfg = ServeCfg(M, g, k_c_pm, k_m_pm, POLICY[policy], 1 if act else 0, max_batch, nstreams, queue_cap,
                       slots_per_chunk, max_tenants, reserve_bytes, SCHED[sched], 0 if zs is None else len(zs),
                       None if zs is None else zs.ctypes.data)
        _check(lib().gpa_serve_start(ctx.handle, ctypes.byref(cfg)))
        self.running = True

    def submit(self, op, tenant, tasks=None, index=0):
        """tasks: dict of numpy columns (T, D, A, B, u_ppm, type) for ADMIT (n tasks) or ADD (1 task)."""
        keep = []
        cols = [None] * 6
        n = 0
        if tasks is not None:
            for i, k in enumerate(("T", "D", "A", "B", "u_ppm", "type")):
                a = np.ascontiguousarray(tasks[k], np.uint8 if k == "type" else np.int64)
                keep.append(a)
                cols[i] = a.ctypes.data
            n = len(keep[0])
        rq = Request(SERVE_OP[op], n, int(tenant), int(index), 0, *cols)
        rid = ctypes.c_uint64()
        _check(lib().gpa_serve_submit(self.ctx.handle, ctypes.byref(rq), ctypes.byref(rid)))
        return rid.value

    def poll(self, req_id, timeout_us=10_000_000):
        r = Response()
        _check(lib().gpa_serve_poll(self.ctx.handle, ctypes.c_uint64(req_id), ctypes.byref(r), int(timeout_us)))
        return r.as_dict()

    def stats(self):
        v = [ctypes.c_int64() for _ in range(5)]
        _check(lib().gpa_serve_stats(self.ctx.handle, *[ctypes.byref(x) for x in v]))
        return dict(zip(("completed", "batches", "max_batch", "overlapped", "slots"), [x.value for x in v]))

    def stop(self):
        if self.running:
            _check(lib().gpa_serve_stop(self.ctx.handle))
            self.running = False


# ------------------------------------------------- measured WCET curves (§3)

PROBE = {"VADD": 0, "TRANSPOSE": 1, "STENCIL": 2, "COMPUTE": 3}


class ProbeCfg(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("interfere", ctypes.c_int32), ("n", ctypes.c_int64),
                ("reps", ctypes.c_int32), ("ctas", ctypes.c_int32)]


def _probe_sigs(L):
    L.gpa_measure_wcet.argtypes = [_vp, ctypes.POINTER(ProbeCfg), _vp, ctypes.c_int32, _vp, _vp]
    L.gpa_probe_run.argtypes = [_vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _vp, _vp, _vp]
    L.gpa_fit_wcet.argtypes = [_vp, _vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double)]


def probe_run(ctx, kernel, n, a, b=None, ctas=0):
    """gpa_probe_run: probe `kernel` once on the whole GPU on host float32
    data a (and b); returns its output."""
    _probe_sigs(lib())
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = None if b is None else np.ascontiguousarray(b, dtype=np.float32)
    out = np.empty_like(a)
    _check(lib().gpa_probe_run(ctx.handle, PROBE[kernel], int(n), int(ctas), a.ctypes.data,
                               None if b is None else b.ctypes.data, out.ctypes.data))
    return out


def measure_wcet(ctx, kernel, m, n, reps=5, interfere=False, ctas=0):
    """gpa_measure_wcet: median device time (ms) of probe `kernel` on each m
    SMs (the rest held by the blocker, idle or streaming HBM), and the SMs it
    ran on (-1 where no repetition passed the placement check)."""
    _probe_sigs(lib())
    mm = np.ascontiguousarray(m, dtype=np.int32)
    ms = np.zeros(len(mm), np.float64)
    used = np.zeros(len(mm), np.int32)
    cfg = ProbeCfg(PROBE[kernel], 1 if interfere else 0, int(n), int(reps), int(ctas))
    _check(lib().gpa_measure_wcet(ctx.handle, ctypes.byref(cfg), mm.ctypes.data, len(mm), ms.ctypes.data,
                                  used.ctypes.data))
    return ms, used


def fit_wcet(m, ms):
    """gpa_fit_wcet: least squares of ms = a / m + b; returns (a, b)."""
    _probe_sigs(lib())
    mm = np.ascontiguousarray(m, dtype=np.int32)
    t = np.ascontiguousarray(ms, dtype=np.float64)
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().gpa_fit_wcet(mm.ctypes.data, t.ctypes.data, len(mm), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value
