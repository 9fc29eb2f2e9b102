"""C-ABI checks that need no GPU: every function declared in include/gmrf.h is
exported by libgmrf.so, the ctypes structures match the C layout, and
argument validation happens before any device work."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gmrf.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gmrf_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def g():
    from paper_1312_1476_gb300 import _build
    _build.build()
    from paper_1312_1476_gb300 import gmrf
    return gmrf


def test_every_declared_symbol_is_exported(g):
    names = _declared_functions()
    assert "gmrf_create" in names and "gmrf_sample" in names and "gmrf_logdet" in names
    out = subprocess.run(["nm", "-D", "--defined-only", g.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(gmrf_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(g.LIB_PATH)
    for n in names:
        assert getattr(lib, n) is not None


def test_struct_layout_matches_c(g):
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "gmrf.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(gmrf_desc), sizeof(gmrf_sample_opts), sizeof(gmrf_result_info),
         sizeof(gmrf_logdet_opts));
  printf("%zu %zu %zu %zu\n", offsetof(gmrf_desc, kappa2), offsetof(gmrf_desc, tau),
         offsetof(gmrf_desc, precision), offsetof(gmrf_sample_opts, z_in));
  printf("%zu %zu\n", offsetof(gmrf_result_info, err_est), offsetof(gmrf_logdet_opts, probes_in));
  printf("%zu %zu %zu\n", sizeof(gmrf_solve_opts), offsetof(gmrf_solve_opts, nrhs),
         offsetof(gmrf_solve_opts, reserved));
  printf("%zu %zu %zu %zu\n", sizeof(gmrf_sparse_desc), offsetof(gmrf_sparse_desc, f_rowptr),
         offsetof(gmrf_sparse_desc, tau), offsetof(gmrf_sparse_desc, reserved));
  printf("%zu %zu %zu %zu %zu\n", sizeof(gmrf_tuning), offsetof(gmrf_tuning, vec_steps_per_s),
         offsetof(gmrf_tuning, host_loop), sizeof(gmrf_server_opts), offsetof(gmrf_server_opts, tol));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        exe = os.path.join(d, "p")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    cs = ctypes.sizeof
    assert vals[:4] == [cs(g.GmrfDesc), cs(g.GmrfSampleOpts), cs(g.GmrfResultInfo), cs(g.GmrfLogdetOpts)]
    assert vals[4:] == [g.GmrfDesc.kappa2.offset, g.GmrfDesc.tau.offset, g.GmrfDesc.precision.offset,
                        g.GmrfSampleOpts.z_in.offset, g.GmrfResultInfo.err_est.offset,
                        g.GmrfLogdetOpts.probes_in.offset, cs(g.GmrfSolveOpts), g.GmrfSolveOpts.nrhs.offset,
                        g.GmrfSolveOpts.reserved.offset, cs(g.GmrfSparseDesc), g.GmrfSparseDesc.f_rowptr.offset,
                        g.GmrfSparseDesc.tau.offset, g.GmrfSparseDesc.reserved.offset,
                        cs(g.GmrfTuning), g.GmrfTuning.vec_steps_per_s.offset, g.GmrfTuning.host_loop.offset,
                        cs(g.GmrfServerOpts), g.GmrfServerOpts.tol.offset]


def test_invalid_descriptors_rejected_on_host(g):
    lib = g.lib()
    h = ctypes.c_void_p()
    base = dict(dim=2, bc=0, op=0, precond=0, nx=8, ny=8, nz=1, kappa2=None, kappa2_const=0.5, tau=1.0,
                kappa2_precond=0.0, precision=0, reserved=0)
    bad = [dict(dim=4), dict(bc=7), dict(op=3), dict(nx=1), dict(tau=0.0), dict(tau=float("nan")),
           dict(kappa2_const=-1.0), dict(kappa2_const=float("inf")), dict(precision=5), dict(reserved=1),
           dict(bc=0, kappa2_const=0.0)]  # periodic with kappa2 = 0 is singular
    for b in bad:
        d = g.GmrfDesc(**{**base, **b})
        assert lib.gmrf_create(ctypes.byref(d), None, ctypes.byref(h)) == g.ERR_INVALID, b
    # preconditioning needs 2-D power-of-two grids
    for b in (dict(precond=1, nx=12), dict(precond=2, dim=3, nz=8)):
        d = g.GmrfDesc(**{**base, **b})
        assert lib.gmrf_create(ctypes.byref(d), None, ctypes.byref(h)) == g.ERR_UNSUPPORTED, b
    assert lib.gmrf_sample(None, None, None, None) == g.ERR_INVALID
    assert lib.gmrf_solve(None, None, None, None, None) == g.ERR_INVALID
    assert lib.gmrf_sample_logdet(None, None, None, None, None, None, None, None, None) == g.ERR_INVALID
    assert lib.gmrf_submit_sample(None, None, None, None, None) == g.ERR_INVALID
    assert lib.gmrf_poll(None, 1, None, None) == g.ERR_INVALID and lib.gmrf_wait(None, 1, None) == g.ERR_INVALID
    assert g.strerror(g.ERR_NOT_SPD).startswith("operator")
    assert g.strerror(g.ERR_TIMEOUT) == "device wait timed out"
