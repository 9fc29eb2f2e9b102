"""Host-side logic of the sparse path (no GPU): the library's threshold
incomplete Cholesky (gmrf_ichol, Section 5.2) against the oracle's, and its
input validation."""
import ctypes

import numpy as np
import pytest

from oracle import sparse as osp
from paper_1312_1476_gb300 import gmrf, inputs


def _lib_factor(Q, droptol, shift=0.0):
    rp, ci, va = gmrf.ichol(Q, droptol=-1.0 if droptol is None else droptol, shift=shift)
    return osp.csr(rp, ci, va)


def _compare(Fl, Fo):
    Fl = Fl.tocsr()
    Fo = Fo.tocsr()
    Fl.sort_indices()
    Fo.sort_indices()
    np.testing.assert_array_equal(Fl.indptr, Fo.indptr)
    np.testing.assert_array_equal(Fl.indices, Fo.indices)
    np.testing.assert_allclose(Fl.data, Fo.data, rtol=1e-11, atol=1e-12 * np.abs(Fo.data).max())


CASES = [
    (dict(nx=9, ny=7, squared=False), None, 0.0),
    (dict(nx=9, ny=7, squared=False), 1e-2, 0.0),
    (dict(nx=9, ny=7, squared=False), 0.0, 0.0),
    (dict(nx=9, ny=7, squared=True), None, 0.05),
    (dict(nx=9, ny=7, squared=True), 1e-3, 0.1),
    (dict(nx=9, ny=7, squared=True), np.inf, 0.0),
    (dict(nx=16, ny=11, squared=True), 1e-4, 0.05),
]


@pytest.mark.parametrize("shape,droptol,shift", CASES)
def test_library_ichol_matches_oracle(shape, droptol, shift):
    Q = osp.csr(*inputs.random_sparse_spd(shape["nx"], shape["ny"], seed=13, squared=shape["squared"]))
    _compare(_lib_factor(Q, droptol, shift), osp.ichol(Q, droptol=droptol, shift=shift))


@pytest.mark.parametrize("droptol,shift", [(0.0, 0.0), (1e-3, 1e-3), (1e-5, 1e-4), (None, 0.01)])
def test_library_ichol_matches_oracle_figure3(droptol, shift):
    Q = osp.csr(*inputs.figure3_matrix())
    _compare(_lib_factor(Q, droptol, shift), osp.ichol(Q, droptol=droptol, shift=shift))


def test_rows_end_with_the_diagonal():
    rp, ci, va = gmrf.ichol(inputs.random_sparse_spd(8, 8, seed=3), droptol=1e-2)
    for i in range(len(rp) - 1):
        cols = ci[rp[i]:rp[i + 1]]
        assert cols[-1] == i and np.all(np.diff(cols) > 0) and va[rp[i + 1] - 1] > 0


def test_breakdown_reports_the_oracle_pivot():
    Q = inputs.figure3_matrix()
    with pytest.raises(osp.NotFactorable) as ei:
        osp.ichol(osp.csr(*Q), droptol=None)
    col = int(str(ei.value).split()[1])
    n, rp, ci, va = gmrf._csr_parts(Q)
    nnz = ctypes.c_int64()
    rc = gmrf.lib().gmrf_ichol(n, gmrf._ptr(rp), gmrf._ptr(ci), gmrf._ptr(va), -1.0, 0.0, 0, None, None, None,
                               ctypes.byref(nnz))
    assert rc == gmrf.ERR_NOT_SPD and nnz.value == col


def _call(rp, ci, va, droptol=0.0, shift=0.0, cap=0, out=False):
    n = len(rp) - 1
    nnz = ctypes.c_int64()
    fr = np.zeros(n + 1, dtype=np.int64)
    fc = np.zeros(max(cap, 1), dtype=np.int32)
    fv = np.zeros(max(cap, 1), dtype=np.float64)
    rc = gmrf.lib().gmrf_ichol(n, gmrf._ptr(np.ascontiguousarray(rp, dtype=np.int64)),
                               gmrf._ptr(np.ascontiguousarray(ci, dtype=np.int32)),
                               gmrf._ptr(np.ascontiguousarray(va, dtype=np.float64)), droptol, shift, cap,
                               gmrf._ptr(fr), gmrf._ptr(fc) if out else None, gmrf._ptr(fv) if out else None,
                               ctypes.byref(nnz))
    return rc, nnz.value


def test_size_query_and_capacity():
    rp, ci, va = inputs.random_sparse_spd(5, 4, seed=2)
    rc, nnz = _call(rp, ci, va)
    assert rc == gmrf.OK and nnz > 20
    assert _call(rp, ci, va, cap=nnz - 1, out=True) == (gmrf.ERR_INVALID, nnz)
    assert _call(rp, ci, va, cap=nnz, out=True) == (gmrf.OK, nnz)


def test_invalid_inputs():
    rp, ci, va = inputs.random_sparse_spd(5, 4, seed=2)
    # asymmetric values
    va2 = va.copy()
    k = np.nonzero(ci[rp[0]:rp[1]] != 0)[0][0]
    va2[rp[0] + k] *= 1.5
    assert _call(rp, ci, va2)[0] == gmrf.ERR_INVALID
    # column out of range, duplicate column, non-finite value
    ci2 = ci.copy()
    ci2[0] = len(rp) - 1
    assert _call(rp, ci2, va)[0] == gmrf.ERR_INVALID
    ci3 = ci.copy()
    ci3[rp[0] + 1] = ci3[rp[0]]
    assert _call(rp, ci3, va)[0] == gmrf.ERR_INVALID
    va3 = va.copy()
    va3[3] = np.nan
    assert _call(rp, ci, va3)[0] == gmrf.ERR_INVALID
    # bad options
    assert _call(rp, ci, va, droptol=float("nan"))[0] == gmrf.ERR_INVALID
    assert _call(rp, ci, va, shift=-1.0)[0] == gmrf.ERR_INVALID
    # non-positive diagonal
    d = [e for e in range(rp[2], rp[3]) if ci[e] == 2][0]
    va4 = va.copy()
    va4[d] = 0.0
    assert _call(rp, ci, va4)[0] == gmrf.ERR_INVALID


def test_explicit_zeros_and_unsorted_rows():
    # explicit zeros are outside Q's pattern for IC(0) on both sides, and the
    # column order within a row does not matter
    rp, ci, va = inputs.random_sparse_spd(8, 7, seed=5, squared=True)
    Q = osp.csr(rp, ci, va).tolil()
    n = Q.shape[0]
    rng = np.random.default_rng(1)
    for _ in range(20):  # symmetric explicit zeros at positions outside the pattern
        i, j = rng.integers(0, n, 2)
        if i != j and Q[i, j] == 0:
            Q[i, j] = 1.0
            Q[j, i] = 1.0
    Qz = Q.tocsr()
    Qz.data[Qz.data == 1.0] = 0.0  # stored, but zero
    rows = []
    for i in range(n):  # reverse the column order of every row
        s, e = Qz.indptr[i], Qz.indptr[i + 1]
        rows.append((Qz.indices[s:e][::-1], Qz.data[s:e][::-1]))
    ci2 = np.concatenate([r[0] for r in rows]).astype(np.int32)
    va2 = np.concatenate([r[1] for r in rows])
    Fl = osp.csr(*gmrf.ichol((Qz.indptr.astype(np.int64), ci2, va2), droptol=-1.0, shift=0.1))
    Fo = osp.ichol(Qz, droptol=None, shift=0.1)
    _compare(Fl, Fo)
    for dt in (0.0, 1e-3):
        _compare(osp.csr(*gmrf.ichol((Qz.indptr.astype(np.int64), ci2, va2), droptol=dt, shift=0.1)),
                 osp.ichol(Qz, droptol=dt, shift=0.1))
