"""One pattern for a whole sequence.  When the sparsity of A_k does not
change along the sequence (the paper's setting of Sec. 2, where the subset
property S(A_0) = S(A_k) holds), the level-L pattern built once from A_0
serves every map: the batched build given that one pattern K times returns,
bit for bit, what it returns with K separately built (equal) patterns, and
matches the oracle."""
import numpy as np
import pytest

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


# level 3 of the 5-point stencil has 25 unknowns per column (and 41 shadow
# rows), within the register tiles; level 3 of the 9-point stencil has 49
# and of the 7-point stencil 63, which the large class (one thread block
# per column) serves
SEQS = {"q1_36_L1": (lambda: W.config2(nx=36, nmat=4), 1), "q1_36_L2": (lambda: W.config2(nx=36, nmat=4), 2),
        "poisson5_32_L3": (lambda: W.config1(nx=32), 3), "q1_24_L3": (lambda: W.config2(nx=24, nmat=3), 3),
        "upwind7_9_L3": (lambda: W.config3(nx=9, nmat=3), 3)}


@pytest.mark.parametrize("case", sorted(SEQS))
def test_one_pattern_serves_a_fixed_sparsity_sequence(sam, case):
    make, level = SEQS[case]
    seq = make()
    with sam.Handle() as h:
        aks = [sam.Csr.from_host(m) for m in seq.mats]
        a0 = aks[0]
        per_map = h.sam_pattern_build_batched(aks, level)
        once = h.sam_pattern_build(a0, level)
        assert all(p.nnz == once.nnz for p in per_map)
        o1, rp1, ci1, v1, f1 = h.sam_build_batched(aks, a0, per_map, "fp32r", 1, want_fro=True)
        o2, rp2, ci2, v2, f2 = h.sam_build_batched(aks, a0, [once] * len(aks), "fp32r", 1, want_fro=True)
        assert np.array_equal(o1, o2)
        for x, y in ((rp1, rp2), (ci1, ci2), (v1, v2)):
            assert bool((x == y).all())
        assert np.array_equal(f1, f2)
        # the last map against the oracle on the pattern of A_0
        k = len(aks) - 1
        cp, ri = oracle.pattern(seq.mats[0], level)
        ref = oracle.build(seq.mats[k], seq.mats[0], cp, ri)
        ip, ix, dv = oracle.to_csr(seq.mats[0].n, cp, ri, ref["mval"])
        n = seq.mats[0].n
        assert np.array_equal(rp2[k * (n + 1):(k + 1) * (n + 1)].cpu().numpy(), ip)
        assert np.array_equal(ci2[o2[k]:o2[k + 1]].cpu().numpy(), ix)
        got = v2[o2[k]:o2[k + 1]].cpu().numpy()
        assert np.linalg.norm(got - dv) <= 1e-10 * np.linalg.norm(dv)
        csc = colcheck.csr_to_csc_values(n, ip, ix, got, cp, ri)
        colcheck.assert_columns(cp, csc, ref["mval"], "fp32r")


def _drop_pair(a, i, j):
    """a with the entries (i, j) and (j, i) removed (structure changes, the
    matrix stays structurally symmetric)."""
    d = a.dense()
    d[i, j] = d[j, i] = 0.0
    return W.CSR.from_dense(d)


@pytest.mark.parametrize("level", [1, 2])
def test_one_differing_structure_disables_sharing(sam, level):
    """Structure work is shared only when every matrix of the batch has the
    same structure: one matrix with two entries fewer gets its own pattern,
    shadow rows and map, each equal to the oracle's."""
    seq = W.config2(nx=20, nmat=3)
    mats = list(seq.mats)
    mats[1] = _drop_pair(mats[1], 45, 46)
    n = mats[0].n
    with sam.Handle() as h:
        aks = [sam.Csr.from_host(m) for m in mats]
        pats = h.sam_pattern_build_batched(aks, level)
        offs, rp, ci, v, fro = h.sam_build_batched(aks, aks[0], pats, "fp32r", 1, want_fro=True)
        for k, m in enumerate(mats):
            cp, ri = oracle.pattern(m, level)
            assert pats[k].nnz == int(cp[-1])
            assert np.array_equal(pats[k].colptr().cpu().numpy(), cp)
            assert np.array_equal(pats[k].rowidx().cpu().numpy(), ri)
            ref = oracle.build(m, mats[0], cp, ri)
            ip, ix, dv = oracle.to_csr(n, cp, ri, ref["mval"])
            assert np.array_equal(rp[k * (n + 1):(k + 1) * (n + 1)].cpu().numpy(), ip)
            assert np.array_equal(ci[offs[k]:offs[k + 1]].cpu().numpy(), ix)
            got = v[offs[k]:offs[k + 1]].cpu().numpy()
            assert np.linalg.norm(got - dv) <= 1e-10 * np.linalg.norm(dv)


def test_shared_and_per_column_shadow_agree_in_the_adjoint(sam):
    """The adjoint of a batch of one structure (shadow data shared) equals,
    bit for bit, the adjoint computed one map at a time."""
    seq = W.config2(nx=24, nmat=3)
    with sam.Handle() as h:
        aks = [sam.Csr.from_host(m) for m in seq.mats]
        a0 = aks[0]
        pats = h.sam_pattern_build_batched(aks, 2)
        offs, rp, ci, mv, _ = h.sam_build_batched(aks, a0, pats, "fp32r", 1)
        import torch

        g = torch.randn(mv.numel(), dtype=torch.float64, device="cuda", generator=torch.Generator(device="cuda").manual_seed(1))
        dak, da0 = h.sam_build_backward_batched(aks, [a0] * len(aks), pats, mv, g, "fp32r", 1, 1.0, offsets=offs)
        koff = np.cumsum([0] + [a.nnz for a in aks])
        for k in range(len(aks)):
            one = h.sam_pattern_build(aks[k], 2)
            dk, d0 = h.sam_build_backward(aks[k], a0, one, mv[offs[k]:offs[k + 1]], g[offs[k]:offs[k + 1]], "fp32r", 1,
                                          1.0)
            assert bool((dk == dak[koff[k]:koff[k + 1]]).all())
            assert bool((d0 == da0[k * a0.nnz:(k + 1) * a0.nnz]).all())


HOST_SEQS = {"q1_40_one_structure": lambda: W.config2(nx=40, nmat=5),
             "fem_24_changing": lambda: W.config4(ncell=24, nmat=5, flip_frac=0.2)}


@pytest.mark.parametrize("case", sorted(HOST_SEQS))
@pytest.mark.parametrize("level", [1, 2])
def test_host_batch_patterns_equal_device_ones(sam, case, level):
    """Batched pattern builds from host arrays (map 0's structure first, the
    others copied while map 0's pattern is built; that pattern is dropped
    when the structures differ) give the device build's patterns, bit for
    bit, for a sequence of one structure and one whose structure changes."""
    seq = HOST_SEQS[case]()
    with sam.Handle() as h:
        dev = h.sam_pattern_build_batched([sam.Csr.from_host(m) for m in seq.mats], level)
        host = h.sam_pattern_build_batched([sam.Csr(m.indptr, m.indices, m.data, n=m.n) for m in seq.mats], level)
        for a, b in zip(dev, host):
            assert a.nnz == b.nnz
            assert bool((a.colptr() == b.colptr()).all()) and bool((a.rowidx() == b.rowidx()).all())


def test_host_batch_with_a_bad_later_map_is_rejected(sam):
    """A later map with unsorted column indices, given as host arrays, is
    rejected after map 0's pattern was built speculatively; the handle stays
    usable."""
    seq = W.config2(nx=24, nmat=4)
    bad = seq.mats[2]
    ci = bad.indices.copy()
    r = 5
    b, e = bad.indptr[r], bad.indptr[r + 1]
    ci[b:e] = ci[b:e][::-1]
    mats = [sam.Csr(m.indptr, m.indices, m.data, n=m.n) for m in seq.mats]
    mats[2] = sam.Csr(bad.indptr, ci, bad.data, n=bad.n)
    with sam.Handle() as h:
        with pytest.raises(sam.SamError) as err:
            h.sam_pattern_build_batched(mats, 2)
        assert err.value.status == sam.SAM_ERR_BAD_CSR
        ok = h.sam_pattern_build_batched([sam.Csr.from_host(m) for m in seq.mats], 2)
        assert len(ok) == 4 and all(p.nnz == ok[0].nnz for p in ok)
