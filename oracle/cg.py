"""Sparse matrix-vector product and conjugate gradient — TEST INFRASTRUCTURE.

Sec. 7 of the paper: the conjugate gradient method (Golub and Van Loan, cited
there) solves a symmetric positive definite system stored in Compressed
Sparse Row format; its DGEMV(sparse) step is a repetitive task over the rows
(row i gathers the columns of its nonzeros), the scalar steps run between
them, and a continue-condition ends the loop.  Everything here is float64,
written from the definitions; nothing in the product path imports it.
"""
from __future__ import annotations

import numpy as np


def spmv(row_ptr, col_idx, vals, x):
    """y_i = sum over k in [row_ptr[i], row_ptr[i+1]) of vals[k] * x[col_idx[k]]."""
    prod = np.asarray(vals, np.float64) * np.asarray(x, np.float64)[np.asarray(col_idx)]
    n = len(row_ptr) - 1
    y = np.zeros(n)
    starts = np.asarray(row_ptr[:-1])
    nonempty = np.asarray(row_ptr[1:]) > starts
    y[nonempty] = np.add.reduceat(prod, starts[nonempty])
    return y


def spmv_abs(row_ptr, col_idx, vals, x):
    """sum of |vals[k]| |x[col_idx[k]]| per row: the scale of each product's rounding."""
    return spmv(row_ptr, col_idx, np.abs(vals), np.abs(x))


def cg(row_ptr, col_idx, vals, b, x0=None, tol=1e-10, max_iter=1000):
    """Conjugate gradient (Hestenes-Stiefel form): stop when
    ||r_k|| <= tol * ||b||.  Returns (x, iterations, residual norms)."""
    b = np.asarray(b, np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64)
    r = b - spmv(row_ptr, col_idx, vals, x)
    p = r.copy()
    rr = float(r @ r)
    bnorm = float(np.sqrt(b @ b))
    hist = [np.sqrt(rr)]
    k = 0
    while np.sqrt(rr) > tol * bnorm and k < max_iter:
        ap = spmv(row_ptr, col_idx, vals, p)
        alpha = rr / float(p @ ap)
        x += alpha * p
        r -= alpha * ap
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        k += 1
        hist.append(np.sqrt(rr))
    return x, k, np.array(hist)
