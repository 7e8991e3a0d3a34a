"""The C ABI on the host (no GPU): exported symbols, validation, enumeration."""
import ctypes
import itertools
import math
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2105_10312_gb300 as gpa
import refs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*int32_t\s+(gpa_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_entry_point():
    names = _declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(gpa.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_header_documents_every_entry_point():
    text = open(os.path.join(ROOT, "include", "gpa.h")).read()
    for n in _declared_functions():
        i = re.search(r"^\s*int32_t\s+" + n + r"\s*\(", text, flags=re.M).start()
        before = text[max(0, i - 400):i]
        assert "/*" in before or "*/" in before, n


def _entry_points(with_ctx):
    """(name, ctypes argument types) of every declared entry point whose first
    parameter is (with_ctx) or is not the context, from the header."""
    text = open(os.path.join(ROOT, "include", "gpa.h")).read()
    out = []
    for name, params in re.findall(r"^\s*int32_t\s+(gpa_\w+)\s*\(([^)]*)\)\s*;", text, flags=re.M):
        ps = [q.strip() for q in params.split(",") if q.strip()]
        if bool(ps) and ps[0].startswith("gpa_ctx*") != with_ctx:
            continue
        types = []
        for q in ps:
            if "*" in q:
                types.append(ctypes.c_void_p)
            elif q.startswith("uint64_t"):
                types.append(ctypes.c_uint64)
            elif q.startswith("int64_t"):
                types.append(ctypes.c_int64)
            else:
                assert q.startswith("int32_t"), (name, q)
                types.append(ctypes.c_int32)
        out.append((name, types))
    return out


def test_every_context_entry_point_rejects_a_null_context():
    """No entry point dereferences a NULL context: each returns GPA_ERR_ARG
    (gpa_ctx_destroy: GPA_OK, nothing to free) before any CUDA call, so this
    runs without a GPU."""
    fns = _entry_points(True)
    assert len(fns) >= 15 and "gpa_allocate_multi" in [n for n, _ in fns]
    lib = ctypes.CDLL(gpa.LIB_PATH)
    for name, types in fns:
        f = getattr(lib, name)
        f.argtypes, f.restype = types, ctypes.c_int32
        code = f(*[None if t is ctypes.c_void_p else 0 for t in types])
        assert code == (gpa.OK if name == "gpa_ctx_destroy" else gpa.ERR_ARG), (name, code)


def test_every_other_entry_point_rejects_null_arguments():
    """The entry points without a context, given NULL pointers and zero
    sizes, return an error status instead of dereferencing them (the
    allocation-free call's status read is left out: a NULL stream is the
    default stream, valid wherever a GPU is)."""
    fns = [(n, t) for n, t in _entry_points(False) if n != "gpa_allocate_noalloc_status"]
    assert {"gpa_validate", "gpa_gen_tasksets", "gpa_allocate_noalloc", "gpa_fit_wcet"} <= {n for n, _ in fns}
    lib = ctypes.CDLL(gpa.LIB_PATH)
    for name, types in fns:
        f = getattr(lib, name)
        f.argtypes, f.restype = types, ctypes.c_int32
        code = f(*[None if t is ctypes.c_void_p else 0 for t in types])
        assert code < 0, (name, code)


def test_ctx_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    code = gpa.lib().gpa_ctx_create(0, None, ctypes.byref(h))
    assert code in (gpa.ERR_CUDA, gpa.ERR_ARG)
    buf = ctypes.create_string_buffer(256)
    assert gpa.lib().gpa_last_error(buf, 256) == 0 and buf.value


def test_host_validation_bounds():
    s = gpa.gen_tasksets(seed=1, nsets=20, n_min=0, n_max=12)
    assert gpa.validate(s, M=80)[0] == gpa.OK
    for col, idx, val in (("D", 3, 0), ("T", 5, 2**31), ("A", 2, -1), ("B", 4, 2**36 + 1), ("type", 1, 2)):
        bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}
        if col == "D":
            bad["D"][idx] = val
        elif col == "T":
            bad["T"][idx] = val
            bad["D"][idx] = 1
        else:
            bad[col][idx] = val
        code, bad_set = gpa.validate(bad, M=80)
        assert code == gpa.ERR_RANGE
        assert bad["set_off"][bad_set] <= idx < bad["set_off"][bad_set + 1]
    # D > T
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}
    bad["D"][0] = bad["T"][0] + 1
    assert gpa.validate(bad, M=80)[0] == gpa.ERR_RANGE
    # model bounds: k < 1000 (an inflation factor below 1), g not dividing M, M too large
    assert gpa.validate(s, M=80, k_c_pm=999)[0] == gpa.ERR_RANGE
    assert gpa.validate(s, M=81, g=2)[0] == gpa.ERR_RANGE
    assert gpa.validate(s, M=1025)[0] == gpa.ERR_RANGE


def test_composition_count_and_unrank_lexicographic():
    assert gpa.enumerate_partitions(8, 2, 2) == 7
    assert gpa.enumerate_partitions(20, 1, 4) == sum(math.comb(19, k - 1) for k in range(1, 5))
    for Mu, k in ((8, 2), (7, 3), (10, 4), (6, 6), (5, 1)):
        want = list(refs.compositions(Mu, k))
        got = [tuple(gpa.unrank_composition(Mu, k, r)) for r in range(len(want))]
        assert got == want
        with pytest.raises(gpa.GpaError):
            gpa.unrank_composition(Mu, k, len(want))


def test_rgs_count_and_unrank_lexicographic():
    def all_rgs(n, kmax):
        out = []
        for labels in itertools.product(range(kmax), repeat=n):
            r = refs.rgs_of(labels)
            if tuple(labels) == r:
                out.append(r)
        return sorted(out)
    assert gpa.count_rgs(12, 4) == 700075
    for n, kmax in ((1, 1), (4, 2), (5, 3), (6, 4), (7, 7)):
        want = all_rgs(n, kmax)
        assert gpa.count_rgs(n, kmax) == len(want)
        got = [tuple(int(x) for x in gpa.unrank_rgs(n, kmax, r)) for r in range(len(want))]
        assert got == want


def test_generator_is_deterministic_and_shaped():
    a = gpa.gen_tasksets(seed=7, nsets=300, n_min=4, n_max=64, U_steps=60, U_lo_ppm=100000, U_hi_ppm=6000000,
                         mu_dist="BETA25", deadline_pm=750, nthreads=1)
    b = gpa.gen_tasksets(seed=7, nsets=300, n_min=4, n_max=64, U_steps=60, U_lo_ppm=100000, U_hi_ppm=6000000,
                         mu_dist="BETA25", deadline_pm=750, nthreads=5)
    for k in ("set_off", "T", "D", "A", "B", "u_ppm", "type", "C1"):
        assert np.array_equal(a[k], b[k]), k
    n = np.diff(a["set_off"])
    assert n.min() >= 4 and n.max() <= 64
    assert (a["D"] == a["T"] * 750 // 1000).all()
    assert (a["T"] >= 10000).all() and (a["T"] <= 1000000).all()
    # Beta(2,5) intensity with prm = 0.5: P(memory) = 7/64
    frac = a["type"].mean()
    assert 0.07 < frac < 0.15
    # stepped total utilisation: U = 0.1 (s mod 60 + 1)
    C1, T = a["C1"], a["T"]
    for s in range(0, 300, 37):
        o, e = a["set_off"][s], a["set_off"][s + 1]
        U = (C1[o:e] / T[o:e]).sum()
        assert abs(U - 0.1 * (s % 60 + 1)) < 0.02 * (e - o) / 10 + 0.01


def test_generator_follows_the_stated_input_recipe():
    """The recipe the workloads are described by: the paper's setting takes
    its periods from the divisors of 4000 in [50, 4000], D = 0.75 T, 50
    tasks, U = 2, 4, .. 68 by set index and memory intensity uniform (half
    the tasks memory-bound); the sweep's periods are log-uniform on
    [10^4, 10^6] and its intensity Beta(2, 5); utilisations are uniform on the simplex sum u = U, whose
    marginal u_i / U is Beta(1, n - 1): variance (n - 1) / (n^2 (n + 1)) and
    P(u_i / U > 2 / n) = (1 - 2 / n)^(n - 1)."""
    from paper_2105_10312_gb300 import workloads as W
    p = gpa.gen_tasksets(**W.gen_params("paper50", nsets=680))
    div = [d for d in range(50, 4001) if 4000 % d == 0]
    assert set(p["T"].tolist()) <= set(div) and len(set(p["T"].tolist())) > 10
    assert (p["D"] == p["T"] * 750 // 1000).all() and (np.diff(p["set_off"]) == 50).all()
    assert 0.45 < p["type"].mean() < 0.55
    for k in range(0, 680, 23):
        o, e = p["set_off"][k], p["set_off"][k + 1]
        assert abs((p["C1"][o:e] / p["T"][o:e]).sum() - 2 * (k % 34 + 1)) < 0.1
    w = gpa.gen_tasksets(**W.gen_params("sweep", nsets=3000))
    lt = np.log10(w["T"])
    assert lt.min() >= 4 and lt.max() <= 6 and abs(lt.mean() - 5) < 0.02 and abs((lt < 5).mean() - 0.5) < 0.02
    # Beta(2, 5) intensity (second order statistic of six uniforms) >= 0.5
    # when at most one of the six is below 0.5: probability 7 / 64
    assert abs(w["type"].mean() - 7 / 64) < 0.005
    n = 8
    u = gpa.gen_tasksets(seed=11, nsets=3000, n_min=n, n_max=n, U_lo_ppm=2000000, U_hi_ppm=2000000,
                         deadline_pm=750, T_lo=1000000, T_hi=10000000)
    share = (u["C1"] / u["T"]).reshape(-1, n)
    share = share / share.sum(axis=1, keepdims=True)
    assert abs(share.var() / ((n - 1) / (n * n * (n + 1))) - 1) < 0.05
    assert abs((share > 2 / n).mean() - (1 - 2 / n) ** (n - 1)) < 0.015


def test_task_limits():
    """Sets of up to 256 tasks pass the host check and the generator; 257
    do not (the serving tenants' 128-task limit is checked on the GPU)."""
    t = gpa.gen_tasksets(seed=1, nsets=3, n_min=256, n_max=256)
    assert np.array_equal(np.diff(t["set_off"]), [256, 256, 256])
    assert gpa.validate(t, M=512) == (0, -1)
    t["n_max"] = 257
    assert gpa.validate(t, M=512)[0] == gpa.ERR_RANGE
    with pytest.raises(ValueError):
        gpa.gen_tasksets(seed=1, nsets=2, n_min=1, n_max=257)
    assert gpa.NMAX == 256 and gpa.SERVE_NMAX == 128


def test_binding_constants_match_the_header():
    """Every enum value the binding mirrors equals the header's."""
    text = open(os.path.join(ROOT, "include", "gpa.h")).read()
    hdr = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(GPA_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}
    defines = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(GPA_[A-Z0-9_]+)\s+(-?\d+)", text)}
    from paper_2105_10312_gb300 import gen as G
    serve = {k: v for k, v in hdr.items() if k.startswith("GPA_SERVE_") and k != "GPA_SERVE_NMAX"}
    assert {k[len("GPA_SERVE_"):]: v for k, v in serve.items()} == gpa.SERVE_OP
    for prefix, table in (("GPA_OPT_", gpa.OPT), ("GPA_POLICY_", gpa.POLICY), ("GPA_SCHED_", gpa.SCHED),
                          ("GPA_REASON_", gpa.REASON), ("GPA_PROBE_", gpa.PROBE), ("GPA_PATH_", gpa.PATH),
                          ("GPA_DIST_", G.DIST), ("GPA_GEN_", G.MODE)):
        declared = {k[len(prefix):]: v for k, v in hdr.items() if k.startswith(prefix)}
        assert declared == table, prefix
    errs = {k: v for k, v in hdr.items() if k.startswith("GPA_ERR_") or k == "GPA_OK"}
    assert errs == {"GPA_OK": gpa.OK, "GPA_ERR_ARG": gpa.ERR_ARG, "GPA_ERR_RANGE": gpa.ERR_RANGE,
                    "GPA_ERR_NOMEM": gpa.ERR_NOMEM, "GPA_ERR_CUDA": gpa.ERR_CUDA, "GPA_ERR_TIMEOUT": gpa.ERR_TIMEOUT,
                    "GPA_ERR_BUSY": gpa.ERR_BUSY, "GPA_ERR_NOTFOUND": gpa.ERR_NOTFOUND}
    assert (defines["GPA_NMAX"], defines["GPA_SERVE_NMAX"], defines["GPA_MMAX"], defines["GPA_SEARCH_NMAX"],
            defines["GPA_SEARCH_KMAX"]) == (gpa.NMAX, gpa.SERVE_NMAX, gpa.MMAX, gpa.SEARCH_NMAX, gpa.SEARCH_KMAX)
    m = re.search(r"#define\s+GPA_EXPLICIT_MAX\s+\(1ll << (\d+)\)", text)
    assert m and 1 << int(m.group(1)) == gpa.EXPLICIT_MAX


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the size and field offsets of
    the header's C structs (gcc compiles offsetof / sizeof of each)."""
    import shutil
    from paper_2105_10312_gb300 import gen as G
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    pairs = {"gpa_tasksets": gpa.Tasksets, "gpa_model": gpa.Model, "gpa_candidates": gpa.Candidates,
             "gpa_params": gpa.Params, "gpa_alloc_result": gpa.AllocResult, "gpa_best_result": gpa.BestResult,
             "gpa_serve_cfg": gpa.ServeCfg, "gpa_request": gpa.Request, "gpa_response": gpa.Response,
             "gpa_probe_cfg": gpa.ProbeCfg, "gpa_gen_params": G.GenParams, "gpa_gen_out": G.GenOut,
             "gpa_alu_peak": gpa.AluPeak}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gpa.h"', "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            if fname.startswith("pad"):
                continue
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, field, value = ln.split()
        got[(cname, field)] = int(value)
    for cname, cls in pairs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            if not fname.startswith("pad"):
                assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
