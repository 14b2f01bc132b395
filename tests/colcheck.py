"""Column-by-column comparison of a GPU map with the oracle's.

The method solves one least-squares problem per column (Sec. 2), so parity
is checked per column, not only through one norm of the whole map:

* values: ||m_j^gpu - m_j^orc|| <= eps ||m_j^orc|| for every column j, with
  eps = 1e-12 for the FP64 build and 1e-10 for FP32 QR + FP64 refinement
  (the accuracy target the refinement's guard enforces per column); a
  column whose oracle solution is exactly zero must be exactly zero;
* squared residuals res2[j] = ||B_j m_j - c_j||^2 + (target entries outside
  the shadow rows)^2: the GPU reports the residual of its own map.  With
  rho_j the oracle's residual norm and gamma_j = ||A_0(:, j)||, the GPU
  value differs by at most 2 eps rho_j gamma_j + (eps gamma_j)^2: the
  second-order term ||B_j (m^gpu - m^orc)||^2 <= (kappa eps ||c_j||)^2 of a
  least-squares residual, plus the rounding of r = c - B m in FP64 (and of
  the FP32 product B d of the last correction, about u_32 kappa^2 u_32
  kappa ||c_j|| for the refined build), each well below eps gamma_j in the
  first-order term 2 rho_j |delta r_j|.

Test infrastructure only."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

EPS = {"fp64": 1e-12, "fp32r": 1e-10}


def csr_to_csc_values(n, ip, ix, dv, cp, ri):
    """Values of a CSR map in the CSC order of the pattern (cp, ri); the
    structure must be the pattern's transpose (asserted)."""
    m = sp.csr_matrix((np.asarray(dv, np.float64), np.asarray(ix), np.asarray(ip)), shape=(n, n)).tocsc()
    m.sort_indices()
    assert np.array_equal(m.indptr, cp) and np.array_equal(m.indices, ri), "map structure differs from the pattern"
    return m.data


def column_errors(cp, got, want, cols=None):
    """Per-column ||got_j - want_j|| / ||want_j|| over CSC values (cols:
    only these columns); columns with want_j = 0 give 0 if got_j = 0 too,
    else inf."""
    cp = np.asarray(cp, np.int64)
    if cols is None:
        cols = np.arange(len(cp) - 1)
        idx = np.arange(cp[-1])
    else:
        cols = np.asarray(cols, np.int64)
        idx = np.concatenate([np.arange(cp[j], cp[j + 1]) for j in cols]) if len(cols) else np.zeros(0, np.int64)
    lens = cp[cols + 1] - cp[cols]
    if len(idx) == 0:
        return np.zeros(len(cols))
    starts = np.minimum(np.concatenate([[0], np.cumsum(lens)[:-1]]), max(len(idx) - 1, 0))
    d2 = np.add.reduceat((got[idx] - want[idx]) ** 2, starts)
    w2 = np.add.reduceat(want[idx] ** 2, starts)
    d2 = np.where(lens > 0, d2, 0.0)
    w2 = np.where(lens > 0, w2, 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        err = np.sqrt(d2 / w2)
    err = np.where(w2 > 0, err, np.where(d2 > 0, np.inf, 0.0))
    return err


def assert_columns(cp, got, want, precision, cols=None, what="map"):
    err = column_errors(cp, got, want, cols)
    eps = EPS[precision]
    bad = np.flatnonzero(err > eps)
    assert len(bad) == 0, "%s: %d columns above %.0e (worst %.3e at column %d)" % (
        what, len(bad), eps, float(err.max()), int((cols if cols is not None else np.arange(len(err)))[np.argmax(err)]))
    return float(err.max()) if len(err) else 0.0


def target_column_norms(A0):
    """||A_0(:, j)|| for every column j."""
    s = A0.to_scipy().tocsc()
    return np.sqrt(np.asarray(s.multiply(s).sum(axis=0)).ravel())


def assert_res2(got, want, gamma, precision, what="res2"):
    """Per-column squared residuals against the oracle's (see the module
    docstring for the bar)."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    eps = EPS[precision]
    rho = np.sqrt(np.maximum(want, 0.0))
    tol = 2.0 * eps * rho * gamma + (eps * gamma) ** 2
    diff = np.abs(got - want)
    bad = np.flatnonzero(diff > tol)
    assert len(bad) == 0, "%s: %d columns off (worst excess %.3e at column %d)" % (
        what, len(bad), float((diff - tol).max()), int(np.argmax(diff - tol)))
