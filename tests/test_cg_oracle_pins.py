"""Pins of the sparse/CG oracle (CPU): the paper's printed sizes, dense
closed forms, a textbook solver and the finite-termination property."""
import numpy as np

import workloads as W
from oracle import cg as CG


def test_generator_has_the_papers_size_and_nnz():
    # Sec. 7 / Table 1: N = 132651, NNZ = 3442951 (a 27-point stencil on 51^3)
    row_ptr, col, vals, b = W.stencil27_csr(51)
    assert len(row_ptr) - 1 == 132651 == 51 ** 3
    assert row_ptr[-1] == 3442951 == (3 * 51 - 2) ** 3
    assert col.dtype == np.int32 and np.all(np.diff(row_ptr) <= 27)


def _dense(row_ptr, col, vals, n):
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            A[i, col[k]] += vals[k]
    return A


def test_small_matrix_is_symmetric_positive_definite_and_spmv_is_matvec():
    row_ptr, col, vals, b = W.stencil27_csr(5, seed=3)
    A = _dense(row_ptr, col, vals, 125)
    assert np.allclose(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0
    x = W.rng(4).standard_normal(125)
    np.testing.assert_allclose(CG.spmv(row_ptr, col, vals, x), A @ x, rtol=1e-13, atol=1e-12)


def test_cg_matches_a_direct_solve():
    row_ptr, col, vals, b = W.stencil27_csr(6, seed=5)
    A = _dense(row_ptr, col, vals, 216)
    x, k, hist = CG.cg(row_ptr, col, vals, b, tol=1e-12)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-10)
    assert hist[-1] <= 1e-12 * np.linalg.norm(b) and k < 216


def test_cg_terminates_in_n_steps_on_a_small_spd_system():
    # in exact arithmetic CG ends in at most n steps; on a well-conditioned
    # 12 x 12 system the residual after 12 steps is at rounding level
    g = W.rng(6)
    M = g.standard_normal((12, 12))
    A = M @ M.T + 12 * np.eye(12)
    rows, cols = np.nonzero(np.ones((12, 12)))
    row_ptr = np.arange(0, 145, 12, dtype=np.int64)
    b = g.standard_normal(12)
    x, k, hist = CG.cg(row_ptr, cols.astype(np.int32), A[rows, cols], b, tol=1e-14, max_iter=12)
    assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b)


def test_planted_cg_mistake_is_caught(monkeypatch):
    # a wrong beta (rr_new / rr replaced by rr / rr_new) must break convergence
    row_ptr, col, vals, b = W.stencil27_csr(6, seed=5)
    A = _dense(row_ptr, col, vals, 216)

    def bad_cg(row_ptr, col_idx, vals, b, x0=None, tol=1e-10, max_iter=1000):
        x = np.zeros_like(b)
        r = b.copy()
        p = r.copy()
        rr = r @ r
        for _ in range(60):
            ap = CG.spmv(row_ptr, col_idx, vals, p)
            alpha = rr / (p @ ap)
            x += alpha * p
            r -= alpha * ap
            rr_new = r @ r
            p = r + (rr / rr_new) * p
            rr = rr_new
        return x
    xb = bad_cg(row_ptr, col, vals, b)
    assert not np.allclose(xb, np.linalg.solve(A, b), rtol=1e-6)


def test_spmv_ragged_rows_match_dense_product():
    """Empty rows, single entries and long rows: the reduceat path of the
    oracle against a dense matrix-vector product built entry by entry."""
    for n, max_row in ((1, 1), (37, 9), (400, 70)):
        row_ptr, col, vals = W.ragged_csr(n, seed=n, max_row=max_row)
        A = np.zeros((n, n))
        for i in range(n):
            for k in range(row_ptr[i], row_ptr[i + 1]):
                A[i, col[k]] += vals[k]
        x = W.rng(n + 1).standard_normal(n)
        np.testing.assert_allclose(CG.spmv(row_ptr, col, vals, x), A @ x, rtol=1e-12, atol=1e-12)
        assert np.all(CG.spmv(row_ptr, col, vals, x)[np.diff(row_ptr) == 0] == 0.0)
