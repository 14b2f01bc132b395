"""The property the QR's row band rests on, checked on the column problems of
the benchmark's structure with a textbook Householder QR in numpy (no GPU):
with H_k the last row that holds an entry of columns 0..k of B, the
reflectors 0..k leave every row after H_k of [B c] exactly as it was, so
reflector k may be restricted to rows k..H_k (and, for the large class, to
the columns whose first row is at most H_k) without changing R or Q^T c.
Rows are the shadow rows in ascending order, as the kernels hold them."""
import numpy as np

import oracle
from paper_2406_17656_gb300 import workloads as W


def _column_problem(ak, a0, cp, ri, j):
    """B = A_k(I, J), c = A_0(I, j), I ascending (the kernels' row order)."""
    J = ri[cp[j]:cp[j + 1]]
    A = ak.to_scipy().tocsc()
    I = np.unique(np.concatenate([A.indices[A.indptr[c]:A.indptr[c + 1]] for c in J]))
    B = A[I][:, J].toarray()
    c = a0.to_scipy().tocsc()[I][:, [j]].toarray()[:, 0]
    return B, c


def _householder(T, band=None, cols=None):
    """In-place textbook Householder QR of T (Golub & Van Loan Alg. 5.2.1 with
    the right-hand side as the last column); band[k] (exclusive row bound)
    and cols[k] (exclusive column bound, the last column always included)
    restrict reflector k when given.  Returns the tile after each reflector."""
    m, ncol = T.shape
    snaps = []
    for k in range(ncol - 1):
        re = m if band is None else band[k]
        x = T[k:re, k].copy()
        alpha, sigma = x[0], float(np.dot(x[1:], x[1:]))
        if sigma != 0.0:
            beta = -np.copysign(np.sqrt(alpha * alpha + sigma), alpha)
            u = x.copy()
            u[0] = alpha - beta
            tau = -1.0 / (beta * u[0])
            ce = ncol - 1 if cols is None else cols[k]
            sel = list(range(k + 1, ce)) + [ncol - 1]
            w = u @ T[k:re, sel]
            T[k:re, sel] -= tau * np.outer(u, w)
            T[k, k] = beta
            T[k + 1:re, k] = 0.0
        snaps.append(T.copy())
    return snaps


def _bands(B):
    last = np.array([np.flatnonzero(B[:, c]).max() if np.any(B[:, c]) else -1 for c in range(B.shape[1])])
    first = np.array([np.flatnonzero(B[:, c]).min() if np.any(B[:, c]) else B.shape[0] for c in range(B.shape[1])])
    H = np.maximum(np.maximum.accumulate(last), np.arange(B.shape[1]))
    band = H + 1
    cols = np.array([max(k + 1, 1 + max([t for t in range(B.shape[1]) if first[t] <= H[k]], default=k)) for k in
                     range(B.shape[1])])
    return H, band, cols


def test_reflectors_leave_rows_after_the_band_untouched():
    seq = W.config2(nx=16, nmat=2, level=2)
    a0, a1 = seq.mats
    cp, ri = oracle.pattern(a1, 2)
    n = a1.n
    for j in (0, 5, n // 2 + 7, n - 1):  # a corner, a boundary and interior columns
        B, c = _column_problem(a1, a0, cp, ri, j)
        T0 = np.column_stack([B, c])
        H, band, cols = _bands(B)
        snaps = _householder(T0.copy())
        for k, Tk in enumerate(snaps):
            # rows after H_k of every column, c included, are as they were
            assert np.array_equal(Tk[H[k] + 1:], T0[H[k] + 1:]), (j, k)
        # the banded sweep (rows and columns) gives the same R and Q^T c
        full, banded = snaps[-1], _householder(T0.copy(), band, cols)[-1]
        nJ = B.shape[1]
        scale = np.abs(full).max()
        assert np.allclose(np.triu(full[:nJ, :nJ]), np.triu(banded[:nJ, :nJ]), rtol=0, atol=1e-13 * scale)
        assert np.allclose(full[:nJ, -1], banded[:nJ, -1], rtol=0, atol=1e-13 * scale)


def test_interior_band_is_narrow():
    """On an interior 49 x 25 column of the 9-point level-2 structure the
    band ends at most 21 rows after the pivot: every reflector fits a head
    of 7 row slots of 4 rows (the register tile of size class 3)."""
    seq = W.config2(nx=16, nmat=2, level=2)
    a0, a1 = seq.mats
    cp, ri = oracle.pattern(a1, 2)
    j = 8 * 16 + 8
    B, _ = _column_problem(a1, a0, cp, ri, j)
    assert B.shape == (49, 25)
    H, _, _ = _bands(B)
    slots = H // 4 - np.arange(25) // 4 + 1
    assert slots.max() <= 7 and slots.sum() < 0.6 * sum(13 - k // 4 for k in range(25))
