"""Pins for the oracle's adjoint: central finite differences of the oracle
build itself (a different computation: only forward solves), on every
parameter of a small instance and on seeded random directions of the
32x32 instance of the adjoint workload.  CPU only."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2406_17656_gb300 import workloads as W


def _with_values(m, data):
    return W.CSR(m.n, m.indptr, m.indices, np.asarray(data, dtype=np.float64))


def _loss(ak, a0, cp, ri, gbar, rho, v=None):
    out = oracle.build(ak, a0, cp, ri)
    val = float(np.dot(gbar, out["mval"])) if gbar is not None else 0.0
    if rho:
        val += rho * float(np.sum(out["res2"] + out["out2"]))
    if v is not None:
        m = sp.csc_matrix((out["mval"], ri, cp), shape=(ak.n, ak.n))
        val += float(np.sum((m @ v) ** 2))
    return val


def _fd_grad(ak, a0, cp, ri, gbar, rho, h=1e-6, v=None):
    gk = np.zeros_like(ak.data)
    g0 = np.zeros_like(a0.data)
    for arr, which in ((gk, "k"), (g0, "0")):
        base = ak.data if which == "k" else a0.data
        for e in range(len(base)):
            d = base.copy()
            step = h * max(1.0, abs(d[e]))
            d[e] += step
            lp = _loss(_with_values(ak, d) if which == "k" else ak, _with_values(a0, d) if which == "0" else a0,
                       cp, ri, gbar, rho, v)
            d[e] -= 2 * step
            lm = _loss(_with_values(ak, d) if which == "k" else ak, _with_values(a0, d) if which == "0" else a0,
                       cp, ri, gbar, rho, v)
            arr[e] = (lp - lm) / (2 * step)
    return gk, g0


@pytest.mark.parametrize("rho", [0.0, 1.0])
@pytest.mark.parametrize("level", [1, 2])
def test_adjoint_matches_finite_differences_everywhere(level, rho):
    seq = W.config2(nx=5, nmat=2)
    a0, ak = seq.mats
    cp, ri = oracle.pattern(ak, level)
    out = oracle.build(ak, a0, cp, ri)
    gbar = np.random.default_rng(level).standard_normal(len(ri))
    dk, d0 = oracle.adjoint(ak, a0, cp, ri, out["mval"], gbar, rho)
    fk, f0 = _fd_grad(ak, a0, cp, ri, gbar, rho)
    scale = max(np.abs(fk).max(), np.abs(f0).max())
    assert np.abs(dk - fk).max() <= 1e-6 * scale
    assert np.abs(d0 - f0).max() <= 1e-6 * scale


def test_adjoint_nonsymmetric_and_non_nested():
    """Upwinded (nonsymmetric) source, target whose pattern is not inside the
    source's (entries outside the shadow rows)."""
    seq = W.config4(ncell=4, nmat=4, flip_frac=0.5)
    a0, ak = seq.mats[0], seq.mats[3]
    cp, ri = oracle.pattern(ak, 0)
    out = oracle.build(ak, a0, cp, ri)
    assert np.any(out["out2"] > 0)
    gbar = np.random.default_rng(9).standard_normal(len(ri))
    dk, d0 = oracle.adjoint(ak, a0, cp, ri, out["mval"], gbar, 0.5)
    fk, f0 = _fd_grad(ak, a0, cp, ri, gbar, 0.5)
    scale = max(np.abs(fk).max(), np.abs(f0).max())
    assert np.abs(dk - fk).max() <= 1e-6 * scale
    assert np.abs(d0 - f0).max() <= 1e-6 * scale


def test_adjoint_random_directions_32x32_workload_loss():
    """The adjoint workload's loss ||A_1 M_1 - A_0||_F^2 + ||M_1 v||^2 on a
    32x32 instance: directional derivatives along 12 seeded directions."""
    a0, a1 = W.config5_pair(0, nx=32)
    v = W.config5_vector(a0.n)
    cp, ri = oracle.pattern(a1, 1)
    out = oracle.build(a1, a0, cp, ri)
    m = sp.csc_matrix((out["mval"], ri, cp), shape=(a1.n, a1.n))
    mv = m @ v
    cols = np.repeat(np.arange(a1.n), np.diff(cp))
    gbar = 2.0 * mv[ri] * v[cols]  # d ||M v||^2 / dM on the pattern (CSC order)
    _, _, dmres = oracle.adjoint(a1, a0, cp, ri, out["mval"], gbar, 1.0, want_dmres=True)
    # the residual's own dependence on M vanishes at the least-squares solution
    assert np.abs(dmres).max() <= 1e-9 * np.abs(gbar).max()
    dk, d0 = oracle.adjoint(a1, a0, cp, ri, out["mval"], gbar + dmres, 1.0)
    rng = np.random.default_rng(5)
    for _ in range(12):
        uk = rng.standard_normal(len(a1.data))
        u0 = rng.standard_normal(len(a0.data))
        h = 1e-6
        lp = _loss(_with_values(a1, a1.data + h * uk), _with_values(a0, a0.data + h * u0), cp, ri, None, 1.0, v)
        lm = _loss(_with_values(a1, a1.data - h * uk), _with_values(a0, a0.data - h * u0), cp, ri, None, 1.0, v)
        fd = (lp - lm) / (2 * h)
        ad = float(np.dot(dk, uk) + np.dot(d0, u0))
        assert abs(fd - ad) <= 1e-6 * max(abs(fd), 1e-12)


def test_adjoint_linear_in_target():
    """N is linear in A_0 (Sec. 2: each column solves a least-squares problem
    with right-hand side A_0(:, j)), so <gbar, N> has an exact A_0 gradient
    that a single finite difference with a large step reproduces."""
    seq = W.config2(nx=8, nmat=3)
    a0, ak = seq.mats[0], seq.mats[2]
    cp, ri = oracle.pattern(ak, 2)
    out = oracle.build(ak, a0, cp, ri)
    gbar = np.random.default_rng(2).standard_normal(len(ri))
    _, d0 = oracle.adjoint(ak, a0, cp, ri, out["mval"], gbar, 0.0)
    u0 = np.random.default_rng(3).standard_normal(len(a0.data))
    l0 = _loss(ak, a0, cp, ri, gbar, 0.0)
    l1 = _loss(ak, _with_values(a0, a0.data + 0.7 * u0), cp, ri, gbar, 0.0)
    assert abs((l1 - l0) / 0.7 - np.dot(d0, u0)) <= 1e-10 * max(1.0, abs(l1 - l0))
