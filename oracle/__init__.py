"""FP64 CPU oracle for Sparse Approximate Map construction (arXiv 2406.17656).

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this module; the product path never
does, and it shares no code with the CUDA library (neither imports the
other).  The arithmetic lives in `sam_oracle.c` (plain C, FP64, textbook
Householder QR); this file compiles it with gcc on first use and marshals
numpy arrays through ctypes.

Matrices are passed as any object with attributes `n`, `indptr`, `indices`,
`data` (CSR, 0-based, column indices ascending within a row).

Pins: every function here is checked against something other than itself in
`tests/test_oracle_pins.py` (paper-printed pattern counts, closed forms,
brute force on tiny graphs, LAPACK least squares, exact recovery, dense
residuals).  The adjoint functions are pinned by finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sam_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

_i32p = ctypes.POINTER(ctypes.c_int)
_f64p = ctypes.POINTER(ctypes.c_double)


def build_oracle(force: bool = False) -> str:
    """Compile sam_oracle.c into a shared library (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_oracle())
            lib.so_free.argtypes = [ctypes.c_void_p]
            lib.so_max_threads.restype = ctypes.c_int
            lib.so_check_csr.argtypes = [ctypes.c_int, _i32p, _i32p]
            lib.so_pattern.argtypes = [ctypes.c_int, _i32p, _i32p, ctypes.c_int,
                                       ctypes.POINTER(_i32p), ctypes.POINTER(_i32p)]
            lib.so_shadow.argtypes = [ctypes.c_int, _i32p, _i32p, _i32p, _i32p,
                                      ctypes.POINTER(_i32p), ctypes.POINTER(_i32p)]
            lib.so_build.argtypes = [ctypes.c_int, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p,
                                     _i32p, _i32p, ctypes.c_int, _f64p, _f64p, _f64p]
            lib.so_build_cols.argtypes = [ctypes.c_int, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p,
                                          _i32p, _i32p, ctypes.c_int, _i32p, ctypes.c_int, _f64p, _f64p, _f64p]
            lib.so_adjoint.argtypes = [ctypes.c_int, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p, _i32p, _i32p,
                                       _f64p, _f64p, ctypes.c_double, _f64p, _f64p, _f64p]
            lib.so_residual.argtypes = [ctypes.c_int, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p,
                                        _i32p, _i32p, _f64p, _f64p, _f64p]
            lib.so_sparsify.argtypes = [ctypes.c_int, _i32p, _i32p, _f64p, ctypes.c_int, ctypes.c_double, _i32p]
            _lib = lib
    return _lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_i32p)


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_f64p)


def _take(ptr, count, dtype):
    lib = _load()
    out = np.ctypeslib.as_array(ptr, shape=(max(int(count), 1),))[: int(count)].astype(dtype, copy=True)
    lib.so_free(ctypes.cast(ptr, ctypes.c_void_p))
    return out


def _check(st, what):
    if st != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, st))


def max_threads() -> int:
    return int(_load().so_max_threads())


def pattern(A, level: int):
    """Level-`level` neighbour pattern of every column of G(A) (Sec. 3),
    as a CSC structure (colptr[n+1], rowidx[nnz]) with ascending rows."""
    lib = _load()
    rp, rpp = _i32(A.indptr)
    ci, cip = _i32(A.indices)
    cp, ri = _i32p(), _i32p()
    _check(lib.so_pattern(int(A.n), rpp, cip, int(level), ctypes.byref(cp), ctypes.byref(ri)), "pattern")
    colptr = _take(cp, A.n + 1, np.int32)
    rowidx = _take(ri, colptr[-1], np.int32)
    return colptr, rowidx


def shadow(A, colptr, rowidx):
    """Shadow rows I_j (rows where A(:, J_j) has stored entries), CSC form."""
    lib = _load()
    rp, rpp = _i32(A.indptr)
    ci, cip = _i32(A.indices)
    jc, jcp = _i32(colptr)
    jr, jrp = _i32(rowidx)
    ic, ir = _i32p(), _i32p()
    _check(lib.so_shadow(int(A.n), rpp, cip, jcp, jrp, ctypes.byref(ic), ctypes.byref(ir)), "shadow")
    icp = _take(ic, A.n + 1, np.int32)
    iri = _take(ir, icp[-1], np.int32)
    return icp, iri


def build(Ak, A0, colptr, rowidx, nthreads: int = 0):
    """SAM build (Eq. (approx_map), column decomposition of Sec. 2) in FP64.

    Returns a dict with `mval` (map values in the pattern's CSC order),
    `res2[j]` = ||B_j m_j - c_j||^2 and `out2[j]` = squared A_0 entries of
    column j outside the shadow rows."""
    lib = _load()
    n = int(Ak.n)
    a = [_i32(Ak.indptr), _i32(Ak.indices), _f64(Ak.data), _i32(A0.indptr), _i32(A0.indices), _f64(A0.data)]
    jc, jcp = _i32(colptr)
    jr, jrp = _i32(rowidx)
    mval = np.zeros(int(colptr[-1]), dtype=np.float64)
    res2 = np.zeros(n, dtype=np.float64)
    out2 = np.zeros(n, dtype=np.float64)
    st = lib.so_build(n, a[0][1], a[1][1], a[2][1], a[3][1], a[4][1], a[5][1], jcp, jrp, int(nthreads),
                      mval.ctypes.data_as(_f64p), res2.ctypes.data_as(_f64p), out2.ctypes.data_as(_f64p))
    _check(st, "build")
    return {"mval": mval, "res2": res2, "out2": out2}


def build_cols(Ak, A0, colptr, rowidx, cols, nthreads: int = 0):
    """`build` for the listed columns only (a sample of a large problem).
    Returns mval (entries of other columns are NaN), res2, out2."""
    lib = _load()
    n = int(Ak.n)
    a = [_i32(Ak.indptr), _i32(Ak.indices), _f64(Ak.data), _i32(A0.indptr), _i32(A0.indices), _f64(A0.data)]
    jc, jcp = _i32(colptr)
    jr, jrp = _i32(rowidx)
    cl, clp = _i32(cols)
    mval = np.full(int(colptr[-1]), np.nan, dtype=np.float64)
    res2 = np.full(n, np.nan, dtype=np.float64)
    out2 = np.full(n, np.nan, dtype=np.float64)
    st = lib.so_build_cols(n, a[0][1], a[1][1], a[2][1], a[3][1], a[4][1], a[5][1], jcp, jrp, int(nthreads),
                           clp, int(len(cl)), mval.ctypes.data_as(_f64p), res2.ctypes.data_as(_f64p),
                           out2.ctypes.data_as(_f64p))
    _check(st, "build_cols")
    return {"mval": mval, "res2": res2, "out2": out2}


def to_csr(n, colptr, rowidx, mval):
    """Map values in CSC order -> CSR arrays (indptr, indices, data) of N_k."""
    import scipy.sparse as sp

    m = sp.csc_matrix((np.asarray(mval, np.float64), np.asarray(rowidx), np.asarray(colptr)), shape=(n, n)).tocsr()
    m.sort_indices()
    return m.indptr.astype(np.int32), m.indices.astype(np.int32), m.data.astype(np.float64)


def residual(Ak, colptr, rowidx, mval, A0):
    """||R_k||_F and ||R_k||_F / ||A_0||_F for R_k = A_k N_k - A_0 (Eq. (res)),
    evaluated from the definition column by column."""
    lib = _load()
    n = int(Ak.n)
    a = [_i32(Ak.indptr), _i32(Ak.indices), _f64(Ak.data), _i32(colptr), _i32(rowidx), _f64(mval),
         _i32(A0.indptr), _i32(A0.indices), _f64(A0.data)]
    fro2, a02 = ctypes.c_double(), ctypes.c_double()
    st = lib.so_residual(n, *(x[1] for x in a), ctypes.byref(fro2), ctypes.byref(a02))
    _check(st, "residual")
    fro = float(np.sqrt(fro2.value))
    return fro, fro / float(np.sqrt(a02.value))


def adjoint(Ak, A0, colptr, rowidx, mval, gbar=None, rho=0.0, want_dmres=False):
    """Gradients of sum(gbar * N) + rho ||A_k N - A_0||_F^2 with respect to
    the stored values of A_k and A_0 (CSR orders), N the SAM on the pattern
    with values mval (CSC order); gbar in CSC order or None.  Returns
    (dA_k, dA_0[, dmres])."""
    lib = _load()
    n = int(Ak.n)
    a = [_i32(Ak.indptr), _i32(Ak.indices), _f64(Ak.data), _i32(A0.indptr), _i32(A0.indices), _f64(A0.data),
         _i32(colptr), _i32(rowidx), _f64(mval)]
    g = _f64(gbar) if gbar is not None else (None, None)
    dak = np.zeros(len(Ak.data), dtype=np.float64)
    da0 = np.zeros(len(A0.data), dtype=np.float64)
    dm = np.zeros(int(colptr[-1]), dtype=np.float64) if want_dmres else None
    st = lib.so_adjoint(n, *(x[1] for x in a), g[1], float(rho), dak.ctypes.data_as(_f64p),
                        da0.ctypes.data_as(_f64p), dm.ctypes.data_as(_f64p) if dm is not None else None)
    _check(st, "adjoint")
    return (dak, da0, dm) if want_dmres else (dak, da0)


def apply(indptr, indices, data, x):
    """y = N_k x for N_k in CSR (the preconditioner application, Sec. 1)."""
    import scipy.sparse as sp

    n = len(indptr) - 1
    return sp.csr_matrix((data, indices, indptr), shape=(n, n)) @ np.asarray(x, np.float64)


SPARSIFY_MODES = {"global": 0, "tau": 1, "lfil": 2}


def sparsify(A, mode: str, param: float):
    """Sparsified A~ of Sec. 4 (mode "global" thresh, "tau" column threshold,
    "lfil" entries per column; readings in sam_oracle.c).  Returns a CSR
    triple (indptr, indices, data) of the kept entries, rows ascending."""
    lib = _load()
    n = int(A.n)
    rp, rpp = _i32(A.indptr)
    ci, cip = _i32(A.indices)
    v, vp = _f64(A.data)
    keep = np.zeros(max(len(ci), 1), dtype=np.int32)
    _check(lib.so_sparsify(n, rpp, cip, vp, int(SPARSIFY_MODES[mode]), ctypes.c_double(float(param)),
                           keep.ctypes.data_as(_i32p)), "sparsify")
    keep = keep[: len(ci)].astype(bool)
    rows = np.repeat(np.arange(n), np.diff(rp))
    kept_rows = rows[keep]
    indptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(indptr, kept_rows + 1, 1)
    return np.cumsum(indptr).astype(np.int32), ci[keep].copy(), v[keep].copy()


def gmres(A, b, x0=None, M=None, p0=None, restart: int = 30, maxiter: int = 1000, rtol: float = 1e-8, P0=None):
    """Restarted GMRES with right preconditioning for A x = b, as a Krylov
    solve with a SAM would run it: the preconditioner is z = M (P_0 v), M a
    map (CSR object, None = identity) and P_0 either the diagonal p0 or a
    sparse operator P0 (CSR object; None for both = identity).  Textbook steps (Saad, "Iterative Methods for Sparse Linear
    Systems", right-preconditioned GMRES with modified Gram-Schmidt Arnoldi
    and Givens rotations), FP64, scipy sparse products as the only library
    primitive.  Stops when the least-squares residual estimate |g_{j+1}|
    falls to rtol ||b|| or after maxiter Arnoldi steps.
    Returns x, the number of Arnoldi steps, and the estimate after each step
    divided by ||b||."""
    import scipy.sparse as sp

    n = int(A.n)
    As = sp.csr_matrix((A.data, A.indices, A.indptr), shape=(n, n))
    Ms = None if M is None else sp.csr_matrix((M.data, M.indices, M.indptr), shape=(n, n))
    d = None if p0 is None else np.asarray(p0, np.float64)
    Ps = None if P0 is None else sp.csr_matrix((P0.data, P0.indices, P0.indptr), shape=(n, n))

    def prec(v):
        u = v if d is None else d * v
        u = u if Ps is None else Ps @ u
        return u if Ms is None else Ms @ u

    b = np.asarray(b, np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, np.float64)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return np.zeros(n), 0, []
    its, hist = 0, []
    m = int(restart)
    while its < maxiter:
        r = b - As @ x
        beta = float(np.linalg.norm(r))
        if beta <= rtol * bnorm:
            break
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        done = False
        for j in range(m):
            w = As @ prec(V[j])
            for i in range(j + 1):
                H[i, j] = float(V[i] @ w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):  # previous rotations on the new column
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = float(np.hypot(H[j, j], H[j + 1, j]))
            cs[j], sn[j] = (1.0, 0.0) if den == 0.0 else (H[j, j] / den, H[j + 1, j] / den)
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if hist[-1] <= rtol or its >= maxiter:
                done = True
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):  # back substitution with the rotated H
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + prec(V[:k].T @ y)
        if done:
            break
    return x, its, hist
