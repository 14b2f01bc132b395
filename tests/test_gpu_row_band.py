"""The QR's row band (each Householder reflector kept to the rows that hold
entries of its columns) depends on the order of a column problem's rows,
which follows the source's numbering; the map does not.  A symmetric
permutation P A P^T of a sequence permutes every column problem's rows and
columns, so its maps are P M P^T: with the grid numbering the band stays
inside the reflectors' head of row slots, with a random numbering it spans
the tail too.  Both builds meet the per-column bar against the oracle, and
agree with each other column by column."""
import numpy as np
import pytest
import scipy.sparse as sp

import colcheck
import oracle
from paper_2406_17656_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sam():
    import torch

    from paper_2406_17656_gb300 import build, sam as S

    build.build()
    assert torch.cuda.is_available()
    return S


@pytest.fixture(scope="module")
def handle(sam):
    h = sam.Handle()
    yield h
    h.close()


def _permuted(a: W.CSR, p: np.ndarray) -> W.CSR:
    """A'[i, j] = A[p[i], p[j]], column indices sorted."""
    m = a.to_scipy()[p][:, p].tocsr()
    m.sort_indices()
    return W.CSR.from_scipy(m)


def _build(sam, handle, ak, a0, precision, steps):
    Ak, A0 = sam.Csr.from_host(ak), sam.Csr.from_host(a0)
    S = handle.sam_pattern_build(Ak, 2)
    rp, ci, v = handle.sam_build(Ak, A0, S, precision, steps)
    return rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp32r", "fp64"])
def test_row_order_does_not_change_the_map(sam, handle, precision):
    seq = W.config2(nx=40, nmat=2, level=2)
    a0, a1 = seq.mats
    n = a0.n
    p = np.random.default_rng(11).permutation(n)
    a0p, a1p = _permuted(a0, p), _permuted(a1, p)
    steps = 1 if precision == "fp32r" else 0
    rp, ci, v = _build(sam, handle, a1, a0, precision, steps)
    rpp, cip, vp = _build(sam, handle, a1p, a0p, precision, steps)
    # each build against the oracle of its own numbering, column by column
    for (ak, tgt, ip, ix, dv, what) in ((a1, a0, rp, ci, v, "grid order"), (a1p, a0p, rpp, cip, vp, "permuted")):
        cp, ri = oracle.pattern(ak, 2)
        ref = oracle.build(ak, tgt, cp, ri)
        got = colcheck.csr_to_csc_values(n, ip, ix, dv, cp, ri)
        colcheck.assert_columns(cp, got, ref["mval"], precision, what=what)
    # P M P^T against the permuted build, column by column (dense: n = 1600)
    md = sp.csr_matrix((v, ci, rp), shape=(n, n)).toarray()[np.ix_(p, p)]
    mpd = sp.csr_matrix((vp, cip, rpp), shape=(n, n)).toarray()
    err = np.linalg.norm(md - mpd, axis=0) / np.maximum(np.linalg.norm(md, axis=0), 1e-300)
    assert float(np.max(err)) <= 2 * colcheck.EPS[precision]
