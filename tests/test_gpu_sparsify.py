"""Sec. 4 sparsifications on the GPU (sam_sparsify) against the oracle:
kept structure and values bit-exact, the paper's CD2D pattern counts, and a
map built on the pattern of the sparsified source."""
import os

import numpy as np
import pytest

import oracle
from paper_2406_17656_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cd2d_sparsified_nnz.txt")


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


def _random_with_ties(seed, n=300):
    rng = np.random.default_rng(seed)
    p = rng.random((n, n)) < 0.03
    d = np.where(p, rng.uniform(-1.0, 1.0, (n, n)), 0.0)
    d[p & (rng.random((n, n)) < 0.3)] = 0.5  # equal magnitudes inside columns
    np.fill_diagonal(d, np.where(rng.random(n) < 0.8, 2.0 + rng.random(n), 0.0))  # some diagonals missing
    return W.CSR.from_dense(d)


MATS = {
    "poisson32": lambda: W.poisson5(32),
    "q1_24": lambda: W.config2(nx=24, nmat=1).mats[0],
    "fem_24": lambda: W.config4(ncell=24, nmat=1).mats[0],
    "upwind_9": lambda: W.config3(nx=9, nmat=2).mats[1],
    "random_ties": lambda: _random_with_ties(5),
}
MODES = [("global", 0.1), ("global", 0.01), ("global", 1e-4), ("tau", 0.6), ("tau", 0.8), ("tau", 0.95),
         ("lfil", 1), ("lfil", 3), ("lfil", 5), ("lfil", 7)]


@pytest.mark.parametrize("mode,param", MODES)
@pytest.mark.parametrize("mat", sorted(MATS))
def test_sparsify_matches_oracle(sam, handle, mat, mode, param):
    A = MATS[mat]()
    ip, ix, dv = oracle.sparsify(A, mode, param)
    S = handle.sam_sparsify(sam.Csr.from_host(A), mode, param)
    assert np.array_equal(S.indptr.cpu().numpy(), ip)
    assert np.array_equal(S.indices.cpu().numpy(), ix)
    assert np.array_equal(S.data.cpu().numpy(), dv)


def test_paper_cd2d_counts(sam, handle):
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        side, mode, param, power, nnz = line.split()
        A = sam.Csr.from_host(W.poisson5(int(side)))
        At = handle.sam_sparsify(A, mode, float(param))
        P = handle.sam_pattern_build(At, int(power))
        assert P.nnz == int(nnz), line


@pytest.mark.parametrize("mode,param,level", [("tau", 0.5, 2), ("lfil", 4, 2), ("global", 0.05, 2)])
def test_map_on_sparsified_pattern(sam, handle, mode, param, level):
    """The paper's use: pattern = level-L neighbours of A~_k, map built
    from the full A_k (FP32 QR + FP64 refinement) against the oracle."""
    seq = W.config4(ncell=24, nmat=3, flip_frac=0.05)
    A0, Ak = seq.mats[0], seq.mats[2]
    ip, ix, dv = oracle.sparsify(Ak, mode, param)
    cp, ri = oracle.pattern(W.CSR(Ak.n, ip, ix, dv), level)
    ref = oracle.build(Ak, A0, cp, ri)
    _, rx, rv = oracle.to_csr(Ak.n, cp, ri, ref["mval"])
    At = handle.sam_sparsify(sam.Csr.from_host(Ak), mode, param)
    S = handle.sam_pattern_build(At, level)
    assert np.array_equal(S.colptr().cpu().numpy(), cp) and np.array_equal(S.rowidx().cpu().numpy(), ri)
    _, mx, mv = handle.sam_build(sam.Csr.from_host(Ak), sam.Csr.from_host(A0), S, "fp32r", 1)
    assert np.array_equal(mx.cpu().numpy(), rx)
    mv = mv.cpu().numpy()
    assert np.linalg.norm(mv - rv) <= 1e-10 * np.linalg.norm(rv)


def test_bad_parameters_are_rejected(sam, handle):
    A = sam.Csr.from_host(W.poisson5(8))
    for mode, param in (("tau", 1.5), ("tau", -0.1), ("lfil", -1), ("global", float("nan"))):
        with pytest.raises(sam.SamError):
            handle.sam_sparsify(A, mode, param)


@pytest.mark.parametrize("mode,param", [("global", 0.01), ("tau", 0.8), ("lfil", 3)])
def test_batched_sparsify_equals_per_matrix(sam, handle, mode, param):
    """K matrices sparsified in one call: map k's kept entries, row pointers
    and values equal, bit for bit, the single call's and the oracle's."""
    mats = W.config2(nx=24, nmat=3).mats  # three matrices of order 576
    out = handle.sam_sparsify_batched([sam.Csr.from_host(a) for a in mats], mode, param)
    for a, got in zip(mats, out):
        ip, ix, dv = oracle.sparsify(a, mode, param)
        assert np.array_equal(got.indptr.cpu().numpy(), ip)
        assert np.array_equal(got.indices.cpu().numpy(), ix)
        assert np.array_equal(got.data.cpu().numpy(), dv)
        one = handle.sam_sparsify(sam.Csr.from_host(a), mode, param)
        assert np.array_equal(one.data.cpu().numpy(), got.data.cpu().numpy())


@pytest.mark.parametrize("mode,param", [("global", 0.05), ("tau", 0.7), ("lfil", 2)])
def test_batched_sparsify_of_different_structures(sam, handle, mode, param):
    """One call over three matrices of one order with different structures
    and entry counts (each read through its own offsets): every map's kept
    entries equal the oracle's and the single call's, bit for bit."""
    import scipy.sparse as sp

    a = W.config4(ncell=24, nmat=1).mats[0].to_scipy().tocoo()
    n = a.shape[0]
    drop = (a.row != a.col) & ((a.row + 2 * a.col) % 5 == 0)
    b = sp.csr_matrix((a.data[~drop], (a.row[~drop], a.col[~drop])), shape=(n, n))
    rng = np.random.default_rng(11)
    extra = sp.random(n, n, density=3.0 / n, random_state=rng, format="csr")
    c = (a.tocsr() + extra).tocsr()
    mats = [W.CSR.from_scipy(m.tocsr()) for m in (a.tocsr(), b, c)]
    assert len({m.indptr[-1] for m in mats}) == 3
    out = handle.sam_sparsify_batched([sam.Csr.from_host(m) for m in mats], mode, param)
    for m, got in zip(mats, out):
        ip, ix, dv = oracle.sparsify(m, mode, param)
        assert np.array_equal(got.indptr.cpu().numpy(), ip)
        assert np.array_equal(got.indices.cpu().numpy(), ix)
        assert np.array_equal(got.data.cpu().numpy(), dv)
        one = handle.sam_sparsify(sam.Csr.from_host(m), mode, param)
        assert np.array_equal(one.indices.cpu().numpy(), ix) and np.array_equal(one.data.cpu().numpy(), dv)
