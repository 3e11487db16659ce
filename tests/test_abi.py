"""The C-ABI library: it loads, exports every symbol include/qdtrace.h
declares, its struct layouts match the binding's, and the host-side
even-odd map is bit-exact against the oracle.  No GPU needed."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import lattice
from paper_1909_12234_gb300 import build as qbuild
from paper_1909_12234_gb300 import qdtrace as qd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qdtrace.h")


@pytest.fixture(scope="session", autouse=True)
def library():
    if not os.path.exists(qd.LIB_PATH):
        qbuild.build()
    return qd.load()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qd_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(library):
    names = _declared()
    assert len(names) >= 25
    for n in names:
        assert hasattr(library, n), f"{n} missing from libqdtrace.so"
    assert set(names) == set(qd.SIGNATURES), "binding and header disagree"


def test_every_declaration_is_documented():
    # each function the header declares has a comment block right before it
    # (or before the group of declarations it belongs to)
    lines = open(HEADER).read().split("\n")
    decl = re.compile(r"^(?:const\s+)?(?:int|void|long long|double|char|size_t)\b[\s*]*(qd_[a-z0-9_]+)\s*\(")
    missing = []
    for i, line in enumerate(lines):
        m = decl.match(line)
        if not m:
            continue
        j = i - 1
        while j >= 0 and (not lines[j].strip() or lines[j].startswith(" ") or decl.match(lines[j])
                          or lines[j].rstrip().endswith(");")):
            if lines[j].rstrip().endswith("*/"):
                break
            j -= 1
        if j < 0 or not lines[j].rstrip().endswith("*/"):
            missing.append(m.group(1))
    assert not missing, missing


def test_abi_version(library):
    assert library.qd_abi_version() == 6


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "qdtrace.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(qd_mg_params), offsetof(qd_mg_params, null_tol),
         offsetof(qd_mg_params, coarsest_direct), offsetof(qd_mg_params, use_graphs), offsetof(qd_mg_params, coarse_tc),
         offsetof(qd_mg_params, coarse_smoother_steps), offsetof(qd_mg_params, null_f32));
  printf("%zu %zu %zu\n", sizeof(qd_solve_stats), offsetof(qd_solve_stats, true_rel_residual),
         offsetof(qd_solve_stats, stagnated));
  printf("%zu %zu %zu %zu\n", sizeof(qd_defl_params), offsetof(qd_defl_params, seed),
         offsetof(qd_defl_params, tau_restart), offsetof(qd_defl_params, fail_first));
  printf("%zu %zu %zu\n", sizeof(qd_trace_params), offsetof(qd_trace_params, solver),
         offsetof(qd_trace_params, dilution));
  printf("%zu %zu %zu %zu %zu\n", sizeof(qd_solver_params), offsetof(qd_solver_params, inner_tol),
         offsetof(qd_solver_params, max_refine), offsetof(qd_solver_params, stag_window),
         offsetof(qd_solver_params, schur));
  printf("%zu %zu %zu\n", sizeof(qd_trace_result), offsetof(qd_trace_result, nsamples), offsetof(qd_trace_result, UhKZ));
  printf("%zu %zu %zu %zu\n", sizeof(qd_smoother_params), offsetof(qd_smoother_params, seed),
         offsetof(qd_smoother_params, mr_steps), offsetof(qd_smoother_params, layers));
  printf("%zu %zu\n", sizeof(qd_smoother_info), offsetof(qd_smoother_info, enabled));
  printf("%zu %zu %zu %zu %zu\n", sizeof(qd_batch_item), offsetof(qd_batch_item, m0), offsetof(qd_batch_item, params),
         offsetof(qd_batch_item, result), offsetof(qd_batch_item, status));
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [list(map(int, l.split())) for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines()]
    want = [
        [ctypes.sizeof(qd.MGParams), qd.MGParams.null_tol.offset, qd.MGParams.coarsest_direct.offset,
         qd.MGParams.use_graphs.offset, qd.MGParams.coarse_tc.offset, qd.MGParams.coarse_smoother_steps.offset,
         qd.MGParams.null_f32.offset],
        [ctypes.sizeof(qd.SolveStats), qd.SolveStats.true_rel_residual.offset, qd.SolveStats.stagnated.offset],
        [ctypes.sizeof(qd.DeflParams), qd.DeflParams.seed.offset, qd.DeflParams.tau_restart.offset,
         qd.DeflParams.fail_first.offset],
        [ctypes.sizeof(qd.TraceParams), qd.TraceParams.solver.offset, qd.TraceParams.dilution.offset],
        [ctypes.sizeof(qd.SolverParams), qd.SolverParams.inner_tol.offset, qd.SolverParams.max_refine.offset,
         qd.SolverParams.stag_window.offset, qd.SolverParams.schur.offset],
        [ctypes.sizeof(qd.TraceResult), qd.TraceResult.nsamples.offset, qd.TraceResult.UhKZ.offset],
        [ctypes.sizeof(qd.SmootherParams), qd.SmootherParams.seed.offset, qd.SmootherParams.mr_steps.offset,
         qd.SmootherParams.layers.offset],
        [ctypes.sizeof(qd.SmootherInfo), qd.SmootherInfo.enabled.offset],
        [ctypes.sizeof(qd.BatchItem), qd.BatchItem.m0.offset, qd.BatchItem.params.offset, qd.BatchItem.result.offset,
         qd.BatchItem.status.offset],
    ]
    assert got == want


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (8, 4, 6, 2), (6, 6, 6, 6), (4, 3, 5, 2)])
def test_eo_index_bit_exact(dims):
    assert np.array_equal(qd.eo_index(dims), lattice.eo_index(dims))


def test_eo_index_rejects_odd_lx():
    with pytest.raises(qd.QDError) as e:
        qd.eo_index((3, 4, 4, 4))
    assert e.value.code == qd.QD_ERR_INVALID


def test_defaults(library):
    p = qd.mg_params()
    assert p.null_tol == 1e-2 and p.null_maxit == 200 and p.nv[0] == 12
    assert tuple(p.block[0]) == (2, 2, 2, 2)
    d = qd.defl_params()
    assert d.kind == qd.QD_DEFL_MG_OBLIQUE and d.k == 24
    sp = qd.solver_params()
    assert sp.tol == 1e-8 and sp.precision == qd.QD_PREC_F64 and sp.inner_tol == 1e-5 and sp.schur == 0
    assert p.coarsest_direct == 16384 and p.coarsest_bf16 == 1 and p.use_graphs == 1
    sm = qd.smoother_params()
    assert sm.nsamples == 8 and sm.solve_tol == 1e-6 and sm.seed == 4242 and sm.mr_steps == 2 and sm.layers == 1


def test_autotune_table_host_side(library):
    # no GPU work: an empty table reports nothing; the mode switch is host state
    qd.autotune_clear()
    assert qd.autotune_report() == {}
    qd.autotune_set(0)
    qd.autotune_set(1)
    n = library.qd_autotune_report(None, 0)
    assert n == 1  # the terminating NUL only
