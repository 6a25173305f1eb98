"""The CSR DGEMV(sparse) task and the CG loop of the case study (Sec. 7),
through the C ABI, against the float64 oracle.

SpMV: every row within 1e-14 of the sum of |a_ik||x_k| behind it (a few
float64 roundings of ~27 products).  CG: the relative residual, recomputed
by the oracle from the returned x, meets the tolerance; the iteration count
matches the oracle's CG within one (the two sum in different orders); on a
small grid the solution matches a direct solve.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cg as CG

pytestmark = pytest.mark.gpu


def _dev(row_ptr, col, vals):
    return (torch.from_numpy(row_ptr).cuda(), torch.from_numpy(col).cuda(), torch.from_numpy(vals).cuda())


@pytest.mark.parametrize("side", [3, 17, 51])
def test_spmv_matches_oracle(arol, side):
    row_ptr, col, vals, b = W.stencil27_csr(side, seed=7)
    solver = arol.ConjugateGradient(*_dev(row_ptr, col, vals))
    x = W.rng(8).standard_normal(side ** 3)
    y = solver.spmv(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = CG.spmv(row_ptr, col, vals, x)
    scale = CG.spmv_abs(row_ptr, col, vals, x)
    assert np.all(np.abs(y - ref) <= 1e-14 * scale + 1e-300)


@pytest.mark.parametrize("lpr", [1, 2, 4, 8])
def test_spmv_ragged_rows_every_lane_count(arol, monkeypatch, lpr):
    """Empty rows, single entries and rows longer than four steps of every
    lane group; the lane count is forced through AROL_SPMV_LPR."""
    monkeypatch.setenv("AROL_SPMV_LPR", str(lpr))
    for n, max_row in ((1, 1), (37, 9), (3000, 70)):
        row_ptr, col, vals = W.ragged_csr(n, seed=lpr * 10 + n % 7, max_row=max_row)
        x = W.rng(n).standard_normal(n)
        y = arol.ConjugateGradient(*_dev(row_ptr, col, vals)).spmv(torch.from_numpy(x).cuda()).cpu().numpy()
        ref = CG.spmv(row_ptr, col, vals, x)
        scale = CG.spmv_abs(row_ptr, col, vals, x)
        assert np.all(np.abs(y - ref) <= 1e-14 * scale + 1e-300), (n, lpr)
        assert np.all(y[np.diff(row_ptr) == 0] == 0.0)


@pytest.mark.parametrize("lpr", [1, 4, 8])
def test_cg_every_lane_count(arol, monkeypatch, lpr):
    monkeypatch.setenv("AROL_SPMV_LPR", str(lpr))
    row_ptr, col, vals, b = W.stencil27_csr(17, seed=3)
    solver = arol.ConjugateGradient(*_dev(row_ptr, col, vals))
    x, iters, rel = solver.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_iter=500)
    res = np.linalg.norm(b - CG.spmv(row_ptr, col, vals, x.cpu().numpy())) / np.linalg.norm(b)
    _, k_ref, _ = CG.cg(row_ptr, col, vals, b, tol=1e-10)
    assert res <= 1.5e-10 and abs(iters - k_ref) <= 1, (res, iters, k_ref)


def test_cg_full_size_case_study(arol):
    """N = 132651, NNZ = 3442951, tol = 1e-10 (Table 1's system size)."""
    row_ptr, col, vals, b = W.stencil27_csr(51)
    solver = arol.ConjugateGradient(*_dev(row_ptr, col, vals))
    bd = torch.from_numpy(b).cuda()
    x, iters, rel = solver.solve(bd, tol=1e-10, max_iter=1000)
    x = x.cpu().numpy()
    res = np.linalg.norm(b - CG.spmv(row_ptr, col, vals, x)) / np.linalg.norm(b)
    _, k_ref, _ = CG.cg(row_ptr, col, vals, b, tol=1e-10)
    assert rel <= 1e-10 and res <= 1.5e-10, (rel, res)
    assert abs(iters - k_ref) <= 1, (iters, k_ref)
    # deterministic: the same call gives the same bits
    x2, iters2, rel2 = solver.solve(bd, tol=1e-10, max_iter=1000)
    assert iters2 == iters and np.array_equal(x2.cpu().numpy(), x)


def test_cg_small_grid_matches_direct_solve_and_respects_limits(arol):
    row_ptr, col, vals, b = W.stencil27_csr(6, seed=9)
    A = np.zeros((216, 216))
    for i in range(216):
        A[i, col[row_ptr[i]:row_ptr[i + 1]]] = vals[row_ptr[i]:row_ptr[i + 1]]
    solver = arol.ConjugateGradient(*_dev(row_ptr, col, vals))
    bd = torch.from_numpy(b).cuda()
    x, iters, rel = solver.solve(bd, tol=1e-13, max_iter=500)
    np.testing.assert_allclose(x.cpu().numpy(), np.linalg.solve(A, b), rtol=1e-10, atol=1e-11)
    x, iters, rel = solver.solve(bd, tol=1e-13, max_iter=3)          # stops at the limit
    assert iters == 3 and rel > 1e-13
    x0 = torch.from_numpy(np.linalg.solve(A, b)).cuda()               # already solved: no iteration
    x, iters, rel = solver.solve(bd, x0.clone(), tol=1e-8, max_iter=50)
    assert iters == 0


def test_malformed_csr_is_refused(arol):
    """A column index outside [0, n), a decreasing row_ptr or a wrong end
    value is refused before any product runs (AROL_ERR_INVALID)."""
    row_ptr, col, vals, b = W.stencil27_csr(5, seed=1)
    good = _dev(row_ptr, col, vals)
    arol.arol_csr_check(len(row_ptr) - 1, len(vals), good[0], good[1])
    bad_col = col.copy()
    bad_col[17] = len(row_ptr) - 1                      # == n: out of range
    bad_rp = row_ptr.copy()
    bad_rp[10], bad_rp[11] = bad_rp[11], bad_rp[10]      # decreasing
    bad_end = row_ptr.copy()
    bad_end[-1] -= 1                                     # row_ptr[n] != nnz
    for rp, c in ((row_ptr, bad_col), (bad_rp, col), (bad_end, col)):
        with pytest.raises(arol.ArolError) as e:
            arol.ConjugateGradient(*_dev(rp, c, vals))
        assert e.value.status == 1
