"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of oracle.c (a dropped term, a
flipped comparison, a swapped operand, an off-by-one), builds it into a
temporary library, points the oracle module at it and runs the pins of
tests/test_oracle_pins.py, quickest first, until one fails: at least one
must.  The real oracle is untouched; all of this runs on the CPU."""
import ctypes
import inspect
import itertools
import os
import subprocess
import time

import pytest

import oracle
import test_oracle_pins as pins

MUTANTS = [
    ("wcet drops m from the b term", "(i128)A + (i128)B * (i128)m", "(i128)A + (i128)B"),
    ("wcet rounds down", "return (int64_t)((num + den - 1) / den);", "return (int64_t)(num / den);"),
    ("a task conflicts with itself", "return same >= 2;", "return same >= 1;"),
    ("conflict factors swapped", "return s->type[i] == 1 ? md->km : md->kc;",
     "return s->type[i] == 1 ? md->kc : md->km;"),
    ("priority order reversed", "if (s->D[j] != s->D[i]) return s->D[j] < s->D[i];",
     "if (s->D[j] != s->D[i]) return s->D[j] > s->D[i];"),
    ("interference rounded down", "((r + s->T[j] - 1) / s->T[j])", "(r / s->T[j])"),
    ("Lemma 1 boundary", "return sum > (i128)1000000 * md->M;", "return sum >= (i128)1000000 * md->M;"),
    ("BF ties to the later candidate", "while (j >= 0 && w[j] > xw)", "while (j >= 0 && w[j] >= xw)"),
    ("par_list increasing", "if (ux != uy) return ux > uy;", "if (ux != uy) return ux < uy;"),
    ("demand bound drops the first job", "dbf += ((t - s->D[j]) / s->T[j] + 1) * (i128)C[j];",
     "dbf += ((t - s->D[j]) / s->T[j]) * (i128)C[j];"),
    ("size search skips lo", "for (int64_t m = lo; m <= hi; m++)", "for (int64_t m = lo + 1; m <= hi; m++)"),
    ("merge may keep the sum", "+ Q->m - 1;", "+ Q->m;"),
    ("workload ignores conflicts", "if (in[i]) w += kfactor(s, md, in, i) * s->u[i];",
     "if (in[i]) w += 1000 * s->u[i];"),
    ("SMS ties to the later candidate", "if (m3 > 0 && (best < 0 || m3 < best_m))",
     "if (m3 > 0 && (best < 0 || m3 <= best_m))"),
    ("search forgets empty parts", "if (sm + empty * smallest_size(w->md) > w->md->M) return;",
     "if (sm > w->md->M) return;"),
    ("EDF task needs slack", "if (C[idx[a]] > s->D[idx[a]]) return 0;", "if (C[idx[a]] >= s->D[idx[a]]) return 0;"),
    ("sizes ignore the unit g", "if (md->nsizes == 0) return m % md->g == 0;", "if (md->nsizes == 0) return 1;"),
    ("EDF demand equal to t fails", "      if (dbf > t) return 0;", "      if (dbf >= t) return 0;"),
    ("EDF demand counts tasks not yet due", "if (s->D[j] <= t) dbf +=", "if (1) dbf +="),
    ("EDF rejects U = 1", "if (utilisation_vs_one(s, C, idx, k) > 0) return 0;",
     "if (utilisation_vs_one(s, C, idx, k) >= 0) return 0;"),
    ("EDF utilisation test dropped", "if (utilisation_vs_one(s, C, idx, k) > 0) return 0;", ""),
    ("EDF utilisation adds C unscaled", "big_mul(&t, &q, (uint32_t)C[i]);", "big_set(&t, (uint32_t)C[i]);"),
    ("multi-limb product drops its top limb", "  out->n = a->n;\n  if (carry) out->d[out->n++] = (uint32_t)carry;",
     "  out->n = a->n;"),
    ("EDF busy period by floor", "next += ((L + s->T[i] - 1) / s->T[i]) * (i128)C[i];",
     "next += (L / s->T[i]) * (i128)C[i];"),
    ("serving GROW leaves one spare SM unused", "size_in[p] + 1, size_in[p] + spare);",
     "size_in[p] + 1, size_in[p] + spare - 1);"),
    ("serving NEW ignores the spare SMs", "if (z && z <= spare) { part_out[nw]", "if (z) { part_out[nw]"),
    ("serving REMOVE keeps the size", "size_out[pr] = (int16_t)minm_linear(&s, &md, in, g, size_in[pr]);",
     "size_out[pr] = size_in[pr];"),
    ("equal deadlines ordered by the longer period", "if (s->T[j] != s->T[i]) return s->T[j] < s->T[i];",
     "if (s->T[j] != s->T[i]) return s->T[j] > s->T[i];"),
    ("full ties ordered by the later index", "  return j < i;\n}", "  return j > i;\n}"),
    ("optimum ties to the larger size sum", "if (sm != b->sum_minm) return sm < b->sum_minm;",
     "if (sm != b->sum_minm) return sm > b->sum_minm;"),
    ("optimum ties to the later RGS", "if (rgs[i] != b->rgs[i]) return rgs[i] < b->rgs[i];",
     "if (rgs[i] != b->rgs[i]) return rgs[i] > b->rgs[i];"),
    ("response time equal to D misses", "      if (r > s->D[i]) { ok = 0; break; }",
     "      if (r >= s->D[i]) { ok = 0; break; }"),
    ("interference from lower-priority tasks", "if (in[j] && j != i && higher_prio(s, j, i)) next +=",
     "if (in[j] && j != i) next +="),
    ("start value counts lower-priority tasks", "if (in[j] && j != i && higher_prio(s, j, i)) r += C[j];",
     "if (in[j] && j != i) r += C[j];"),
    ("binary size search skips its top check", "if (nc == 0 || !test(s, md, in, cand[nc - 1])) return 0;",
     "if (nc == 0) return 0;"),
    ("Lemma 1 at M SMs", "wcet(s->A[i], s->B[i], 1000, 1) * 1000000", "wcet(s->A[i], s->B[i], 1000, md->M) * 1000000"),
    ("Alg. 1 merges until the sum is below M", "  while (Pi > md->M) {", "  while (Pi >= md->M) {"),
    ("success needs a sum below M", "  if (Pi <= md->M) { r->verdict = 1;", "  if (Pi < md->M) { r->verdict = 1;"),
    ("ACT runs when no merge is needed", "if (act && Pi > md->M) {", "if (act) {"),
    ("forbidden pair matched one way only",
     "    if (same_tasks(pl->v[k].a, Q->in, s->n) && same_tasks(pl->v[k].b, P->in, s->n)) return 1;\n", ""),
    ("1G tests at one SM", "  int ok = test(s, md, in, md->M);", "  int ok = test(s, md, in, 1);"),
    ("1G workload left out", "  r->W = workload(s, md, in);\n  size_of_part[0]", "  r->W = 0;\n  size_of_part[0]"),
    ("EDF skips each task's first deadline", "for (i128 t = s->D[i]; t <= L; t += s->T[i]) {",
     "for (i128 t = s->D[i] + s->T[i]; t <= L; t += s->T[i]) {"),
    ("EDF ignores conflicts", "      C[i] = wcet(s->A[i], s->B[i], kfactor(s, md, in, i), m);\n      idx[k++] = i;",
     "      C[i] = wcet(s->A[i], s->B[i], 1000, m);\n      idx[k++] = i;"),
    ("DM ignores conflicts", "    if (in[i]) C[i] = wcet(s->A[i], s->B[i], kfactor(s, md, in, i), m);",
     "    if (in[i]) C[i] = wcet(s->A[i], s->B[i], 1000, m);"),
    ("EDF busy period from zero", "  for (int a = 0; a < k; a++) L += C[idx[a]];\n", ""),
    ("EDF demand rounds its job count up", "dbf += ((t - s->D[j]) / s->T[j] + 1) * (i128)C[j];",
     "dbf += ((t - s->D[j] + s->T[j] - 1) / s->T[j] + 1) * (i128)C[j];"),
    ("RGS allows kmax + 1 blocks", "int top = used < w->kmax ? used : w->kmax - 1;",
     "int top = used <= w->kmax ? used : w->kmax;"),
    ("search counts an unschedulable block as size 0", "    if (w->minm_sub[mask[b]] == 0) return;\n", ""),
    ("search rejects a size sum equal to M", "if (sm + empty * smallest_size(w->md) > w->md->M) return;",
     "if (sm + empty * smallest_size(w->md) >= w->md->M) return;"),
    ("compositions skip the largest first part", "for (int64_t v = 1; v <= left - (w->k - 1 - part); v++) {",
     "for (int64_t v = 1; v < left - (w->k - 1 - part); v++) {"),
    ("optimum keyed by size sum before W",
     "  if (W != b->W) return W < b->W;\n  if (sm != b->sum_minm) return sm < b->sum_minm;",
     "  if (sm != b->sum_minm) return sm < b->sum_minm;\n  if (W != b->W) return W < b->W;"),
    ("optimum's block sizes left out",
     "for (int b = 0; b < 8; b++) w->best->minm_block[b] = b < nb ? w->minm_sub[mask[b]] : 0;",
     "for (int b = 0; b < 8; b++) w->best->minm_block[b] = 0;"),
    ("spare SMs ignore empty parts", "(j->md.M - best.sum_minm - empty * smallest_size(&j->md))",
     "(j->md.M - best.sum_minm)"),
    ("serving NEW rejects a partition equal to the spare SMs", "if (z && z <= spare) {", "if (z && z < spare) {"),
    ("serving REMOVE leaves a gap in the numbering", "      if (part_out[i] > pr) part_out[i]--;\n", ""),
    ("serving summary misses the last partition", "  for (int p = 0; p < np; p++) {\n    pi += size[p];",
     "  for (int p = 0; p + 1 < np; p++) {\n    pi += size[p];"),
    ("serving REMOVE skips the renumbering", "  canonical(n2, part_out, size_out, np);\n", ""),
    ("validation admits D > T", "if (s->D[i] < 1 || s->D[i] > s->T[i] || s->T[i] > 2147483647LL) return 0;",
     "if (s->D[i] < 1 || s->T[i] > 2147483647LL) return 0;"),
    ("validation refuses A + B = 2^36", "s->A[i] + s->B[i] > ((int64_t)1 << 36)) return 0;",
     "s->A[i] + s->B[i] >= ((int64_t)1 << 36)) return 0;"),
    ("validation admits u = 2^32", "s->u[i] >= ((int64_t)1 << 32))) return 0;", "s->u[i] > ((int64_t)1 << 32))) return 0;"),
    ("WCET tables at sizes in units of one SM", "        int64_t m = g * (mi + 1);\n", "        int64_t m = mi + 1;\n"),
    ("WCET tables swap the factors by type", "int64_t kx = type[o + t] == 1 ? km : kc;",
     "int64_t kx = type[o + t] == 1 ? kc : km;"),
    ("WCET tables transposed", "Cc[o * Mu + mi * n + t] = wcet(", "Cc[o * Mu + t * Mu + mi] = wcet("),
    ("model admits M = 1025", "md->M > 1024 ||", "md->M > 1025 ||"),
    ("model admits g not dividing M", " || md->M % md->g != 0) return 0;", ") return 0;"),
    ("model admits a compute factor below 1000", "if (md->kc < 1000 ||", "if (md->kc < 999 ||"),
    ("ACT counts each pair twice",
     "        tests++;\n        if (minm(s, md, in, lo, hi, linear) == 0) act_pair",
     "        tests += 2;\n        if (minm(s, md, in, lo, hi, linear) == 0) act_pair"),
    ("SMS counts only passing candidates",
     "        int64_t m3 = minm(s, md, in, lo, hi, linear);\n        tests++;\n        if (m3 > 0 && (best < 0",
     "        int64_t m3 = minm(s, md, in, lo, hi, linear);\n        if (m3 > 0) tests++;\n        if (m3 > 0 && (best < 0"),
    ("par_list never re-sorted", "  while (Pi > md->M) {\n    sort_par_list(s, list, np);", "  while (Pi > md->M) {"),
    ("BF tries its candidates unsorted",
     "        while (j >= 0 && w[j] > xw) { elig[j + 1] = elig[j]; w[j + 1] = w[j]; j--; }", "        while (0) { }"),
]


def _pin_calls():
    """(name, function, kwargs) for every pin, parametrised ones expanded."""
    calls = []
    for name, f in inspect.getmembers(pins, inspect.isfunction):
        if not name.startswith("test_") or f.__module__ != pins.__name__:
            continue
        marks = [m for m in getattr(f, "pytestmark", []) if m.name == "parametrize"]
        if not marks:
            calls.append((name, f, {}))
            continue
        grids = []
        for m in marks:
            argnames = [a.strip() for a in (m.args[0].split(",") if isinstance(m.args[0], str) else m.args[0])]
            grids.append([dict(zip(argnames, v if isinstance(v, (tuple, list)) and len(argnames) > 1 else (v,)))
                          for v in m.args[1]])
        for combo in itertools.product(*grids):
            kw = {}
            for d in combo:
                kw.update(d)
            calls.append((name, f, kw))
    return calls


# seconds each pin took in the last full run (the control below), so that
# a run that stops at its first failing pin tries the quick pins first
_PIN_SECONDS = {}


def _failing_pins(source, tmp_path, first_only=False):
    """Names of the pins that fail with the oracle built from `source` (only
    the first one with first_only)."""
    c_path = tmp_path / "mutant.c"
    so_path = tmp_path / "libmutant.so"
    c_path.write_text(source)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so_path), str(c_path), "-lpthread"],
                   check=True)
    oracle.lib()
    saved = oracle._lib
    oracle._lib = ctypes.CDLL(str(so_path))
    failed = []
    calls = sorted(_pin_calls(), key=lambda c: _PIN_SECONDS.get(c[0] + repr(c[2]), 0.0))
    try:
        for name, f, kw in calls:
            t0 = time.perf_counter()
            try:
                f(**kw)
            # an AssertionError, a status the mutant made the oracle return, or
            # pytest.raises finding no error (pytest's Failed is no Exception)
            except (Exception, pytest.fail.Exception):
                failed.append(name)
                if first_only:
                    break
            if not first_only:
                _PIN_SECONDS[name + repr(kw)] = time.perf_counter() - t0
    finally:
        oracle._lib = saved
    return failed


def test_unmutated_copy_passes_every_pin(tmp_path):
    """Control: the same harness on an unchanged copy fails no pin."""
    assert _failing_pins(open(oracle._SRC).read(), tmp_path) == []


@pytest.mark.parametrize("label,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(label, old, new, tmp_path):
    src = open(oracle._SRC).read()
    assert old in src, label
    assert _failing_pins(src.replace(old, new), tmp_path, first_only=True), \
        f"no pin caught the planted mistake: {label}"
