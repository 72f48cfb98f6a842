"""CPU-side checks of the C ABI: the library builds, loads, exports every
symbol include/ms.h declares, the ctypes mirrors match the C structs, and the
argument checks that run before any device work reject bad input."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2009_12638_gb300 import _build, _lib, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ms.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^MS_API\s+[\w\s\*]*?\b(ms_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_exports():
    assert declared_functions() == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True, check=True)
    exported = set(re.findall(r"\sT\s+(ms_\w+)", out.stdout))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)
    # nothing but the ABI is exported
    assert exported == set(declared_functions())


def test_ctypes_structs_match_c_layout(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "ms.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(ms_opts), offsetof(ms_opts, outer_tol),
         offsetof(ms_opts, res_hist), offsetof(ms_opts, slow_ns), offsetof(ms_opts, time_limit_ms),
         offsetof(ms_opts, variant), offsetof(ms_opts, inner_adapt), offsetof(ms_opts, overlap),
         offsetof(ms_opts, gmres_restart), offsetof(ms_opts, wait_polls), offsetof(ms_opts, trace_cap),
         offsetof(ms_opts, trace), offsetof(ms_opts, sum_polls));
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(ms_stats), offsetof(ms_stats, lups), offsetof(ms_stats, per_rhs_rel),
         offsetof(ms_stats, slots), offsetof(ms_stats, variant), offsetof(ms_stats, inner_rtol_final),
         offsetof(ms_stats, trace_count));
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(ms_trace_rec), offsetof(ms_trace_rec, sweep),
         offsetof(ms_trace_rec, block), offsetof(ms_trace_rec, rhs), offsetof(ms_trace_rec, inner_its),
         offsetof(ms_trace_rec, block_rr), offsetof(ms_trace_rec, t_ns));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    a, b, c = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:3]
    O, S, T = _lib.Opts, _lib.Stats, _lib.TraceRec
    assert [int(v) for v in a.split()] == [ctypes.sizeof(O), O.outer_tol.offset, O.res_hist.offset,
                                          O.slow_ns.offset, O.time_limit_ms.offset, O.variant.offset,
                                          O.inner_adapt.offset, O.overlap.offset, O.gmres_restart.offset,
                                          O.wait_polls.offset, O.trace_cap.offset, O.trace.offset,
                                          O.sum_polls.offset]
    assert [int(v) for v in b.split()] == [ctypes.sizeof(S), S.lups.offset, S.per_rhs_rel.offset, S.slots.offset,
                                          S.variant.offset, S.inner_rtol_final.offset, S.trace_count.offset]
    from paper_2009_12638_gb300 import TRACE_DTYPE
    want = [ctypes.sizeof(T)] + [getattr(T, n).offset for n in ("sweep", "block", "rhs", "inner_its", "block_rr", "t_ns")]
    assert [int(v) for v in c.split()] == want
    assert TRACE_DTYPE.itemsize == ctypes.sizeof(T)
    assert [TRACE_DTYPE.fields[n][1] for n in ("sweep", "block", "rhs", "inner_its", "block_rr", "t_ns")] == want[1:]


def test_default_opts(lib):
    o = _lib.Opts()
    lib.ms_default_opts(ctypes.byref(o))
    assert (o.mode, o.precision, o.inner_rtol, o.inner_maxit, o.outer_tol) == (0, 1, 1e-6, 50, 1e-8)
    assert o.slow_block == -1 and o.use_graph == 1
    assert o.variant == -1 and o.inner_adapt == 0 and o.overlap == 0
    assert o.inner_method == 0 and o.gmres_restart == 10
    assert o.wait_polls == 0 and o.trace_cap == 0 and not o.trace and o.sum_polls == 0


def test_resident_variant_table(lib):
    from paper_2009_12638_gb300 import resident_variants
    rows = resident_variants()
    assert len(rows) >= 2
    for r in rows:
        assert r["threads"] in (256, 512, 1024) and r["strips"] >= 1 and r["planes"] >= 1
        assert r["d_smem"] in (0, 1) and r["q_regs"] in (0, 1) and r["one_reduction"] in (0, 1)
        # the single-reduction CG keeps d in shared memory and has no separate q
        assert not r["one_reduction"] or (r["d_smem"] and not r["q_regs"])
    # every two-reduction layout that keeps q in registers has a twin that does
    # not (the GPU tests compare the two bit for bit)
    key = lambda r: (r["threads"], r["strips"], r["planes"], r["d_smem"])  # noqa: E731
    plain = {key(r) for r in rows if not r["q_regs"] and not r["one_reduction"]}
    assert all(key(r) in plain for r in rows if r["q_regs"])
    assert any(r["one_reduction"] for r in rows)
    n = ctypes.c_int(0)
    t = ctypes.c_int(0)
    assert lib.ms_resident_variant(len(rows), ctypes.byref(n), ctypes.byref(t), None, None, None, None, None) == \
        _lib.MS_ERR_ARG
    assert n.value == len(rows)
    assert lib.ms_resident_variant(-1, None, None, None, None, None, None, None) == _lib.MS_ERR_ARG


def test_boundary_size(lib):
    for n in [(1, 1, 1), (3, 4, 5), (384, 320, 256)]:
        assert lib.ms_boundary_size(*n) == inputs.boundary_size(*n)


def _grid(lib, *dims):
    h = ctypes.c_void_p()
    rc = lib.ms_create_grid(*dims, ctypes.byref(h))
    return rc, h


def test_create_rejects_bad_sizes(lib):
    for dims in [(0, 4, 4, 1), (4, -1, 4, 1), (4, 4, 4, 0)]:
        rc, h = _grid(lib, *dims)
        assert rc == _lib.MS_ERR_ARG and not h.value
        assert b"sizes" in lib.ms_last_error(None)


def test_partition_equal_split_and_errors(lib):
    rc, h = _grid(lib, 10, 7, 5, 2)
    assert rc == 0
    try:
        assert lib.ms_partition(h, 3, 2, 5, None, None, None) == 0
        cx, cy, cz = (ctypes.c_int * 4)(), (ctypes.c_int * 3)(), (ctypes.c_int * 6)()
        assert lib.ms_get_cuts(h, cx, cy, cz) == 0
        assert list(cx) == list(inputs.equal_cuts(10, 3))
        assert list(cy) == list(inputs.equal_cuts(7, 2))
        assert list(cz) == list(inputs.equal_cuts(5, 5))
        bad = (ctypes.c_int * 4)(0, 5, 5, 10)
        assert lib.ms_partition(h, 3, 1, 1, bad, None, None) == _lib.MS_ERR_ARG
        assert b"strictly" in lib.ms_last_error(h)
        wrong_end = (ctypes.c_int * 3)(0, 4, 9)
        assert lib.ms_partition(h, 2, 1, 1, wrong_end, None, None) == _lib.MS_ERR_ARG
        assert lib.ms_partition(h, 11, 1, 1, None, None, None) == _lib.MS_ERR_ARG
        assert lib.ms_partition(h, 0, 1, 1, None, None, None) == _lib.MS_ERR_ARG
        good = (ctypes.c_int * 3)(0, 3, 10)
        assert lib.ms_partition(h, 2, 1, 1, good, None, None) == 0
    finally:
        lib.ms_destroy(h)


def test_solve_rejects_bad_arguments_before_device_work(lib):
    rc, h = _grid(lib, 4, 4, 4, 1)
    try:
        o = _lib.Opts()
        lib.ms_default_opts(ctypes.byref(o))
        assert lib.ms_solve(h, None, None, None, ctypes.byref(o), None, None) == _lib.MS_ERR_ARG
        dummy = ctypes.c_void_p(16)  # never dereferenced: options are checked first
        for field, value in [("mode", 7), ("precision", 3), ("inner_maxit", -1), ("threads", 100),
                             ("cluster", 17), ("outer_tol", -1.0), ("time_limit_ms", -5.0), ("variant", -2),
                             ("variant", 10000), ("inner_adapt", 2), ("overlap", -1), ("inner_method", 2),
                             ("sum_polls", -1)]:
            o2 = _lib.Opts()
            lib.ms_default_opts(ctypes.byref(o2))
            setattr(o2, field, value)
            assert lib.ms_solve(h, None, None, dummy, ctypes.byref(o2), None, None) == _lib.MS_ERR_ARG, field
        # the inner-tolerance controller runs between sweeps: not in the asynchronous mode
        o2 = _lib.Opts()
        lib.ms_default_opts(ctypes.byref(o2))
        o2.inner_adapt, o2.mode = 1, 1
        assert lib.ms_solve(h, None, None, dummy, ctypes.byref(o2), None, None) == _lib.MS_ERR_ARG
        # GMRES: restart range, sync mode, streaming engine
        for fields in [dict(inner_method=1, gmres_restart=0), dict(inner_method=1, gmres_restart=51),
                       dict(inner_method=1, mode=1), dict(inner_method=1, engine=2)]:
            o2 = _lib.Opts()
            lib.ms_default_opts(ctypes.byref(o2))
            for k2, v2 in fields.items():
                setattr(o2, k2, v2)
            assert lib.ms_solve(h, None, None, dummy, ctypes.byref(o2), None, None) == _lib.MS_ERR_ARG, fields
        # overlapping blocks: sync mode and the streaming engine only
        for mode, eng in [(1, 0), (0, 2)]:
            o2 = _lib.Opts()
            lib.ms_default_opts(ctypes.byref(o2))
            o2.overlap, o2.mode, o2.engine = 1, mode, eng
            assert lib.ms_solve(h, None, None, dummy, ctypes.byref(o2), None, None) == _lib.MS_ERR_ARG
        # a resident layout with FP64 or the streaming engine is rejected before device work
        for prec, eng in [(0, 0), (1, 1)]:
            o2 = _lib.Opts()
            lib.ms_default_opts(ctypes.byref(o2))
            o2.variant, o2.precision, o2.engine = 0, prec, eng
            assert lib.ms_solve(h, None, None, dummy, ctypes.byref(o2), None, None) == _lib.MS_ERR_ARG
        assert lib.ms_residual(h, None, None, None, None, None) == _lib.MS_ERR_ARG
        # global CG: NULL x and negative tolerances or caps are rejected before device work
        assert lib.ms_gcg_solve(h, None, None, None, ctypes.byref(o), None, None) == _lib.MS_ERR_ARG
        for field, value in [("outer_tol", -1.0), ("outer_maxit", -1), ("time_limit_ms", -1.0)]:
            o2 = _lib.Opts()
            lib.ms_default_opts(ctypes.byref(o2))
            setattr(o2, field, value)
            assert lib.ms_gcg_solve(h, None, None, dummy, ctypes.byref(o2), None, None) == _lib.MS_ERR_ARG, field
        assert lib.ms_face_gather(h, None, None, None) == _lib.MS_ERR_ARG
    finally:
        lib.ms_destroy(h)
    assert lib.ms_destroy(None) == 0


def test_python_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.load(str(tmp_path / "missing.so"))


def test_inputs_uneven_cuts_rule():
    rng = np.random.default_rng(12638)
    cx = inputs.uneven_cuts(384, 5, 40, 96, rng)
    cy = inputs.uneven_cuts(320, 6, 40, 96, rng)
    cz = inputs.uneven_cuts(256, 4, 40, 96, rng)
    for c, n, p in [(cx, 384, 5), (cy, 320, 6), (cz, 256, 4)]:
        e = np.diff(c)
        assert c[0] == 0 and c[-1] == n and len(e) == p and e.min() >= 40 and e.max() <= 96
