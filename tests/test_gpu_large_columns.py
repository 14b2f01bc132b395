"""Column problems past the register tiles (more than 64 shadow rows, 27
unknowns or 512 stored entries): the large size class, one thread block per
column with the tile in shared memory (FP64, or FP32 with FP64 refinement
steps), against the oracle column by column.  Workloads: level-3 patterns of the 9-point and 7-point stencils
(the paper's "level 2" of Sec. 5.1: 49 and 63 unknowns per interior column)
and a banded source with about 85 entries per column at level 1 (the NWP
density of Sec. 5.2: up to 96 unknowns and 201 shadow rows)."""
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


@pytest.fixture(scope="module")
def handle(sam):
    h = sam.Handle()
    yield h
    h.close()


CASES = {
    "q1_24_L3": lambda: (W.config2(nx=24, nmat=3), 3),
    "upwind7_9_L3": lambda: (W.config3(nx=9, nmat=3), 3),
    "wide_band_85_L1": lambda: (W.wide_band(), 1),
    "fem_20_L3": lambda: (W.config4(ncell=20, nmat=3, flip_frac=0.1), 3),
}


def _sizes(A, level):
    import bench

    return bench.column_sizes([A], level)[0]


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_large_columns_match_the_oracle(sam, handle, case, precision):
    import torch

    seq, level = CASES[case]()
    A0 = seq.mats[0]
    gamma = colcheck.target_column_norms(A0)
    for Ak in seq.mats[1:]:
        I, J, nB = _sizes(Ak, level)
        assert (I > 64).any() or (J > 27).any() or (nB > 512).any()  # the large class is used
        cp, ri = oracle.pattern(Ak, level)
        ref = oracle.build(Ak, A0, cp, ri)
        S = handle.sam_pattern_build(sam.Csr.from_host(Ak), level)
        st = torch.full((Ak.n,), -1, dtype=torch.int32, device="cuda")
        r2 = torch.empty(Ak.n, dtype=torch.float64, device="cuda")
        ip, ix, dv = handle.sam_build(sam.Csr.from_host(Ak), sam.Csr.from_host(A0), S, precision, 1, col_status=st,
                                      res2=r2)
        handle.sam_sync()
        assert int(st.abs().max()) == 0
        eip, eix, _ = oracle.to_csr(Ak.n, cp, ri, ref["mval"])
        assert np.array_equal(ip.cpu().numpy(), eip) and np.array_equal(ix.cpu().numpy(), eix)
        got = colcheck.csr_to_csc_values(Ak.n, ip.cpu().numpy(), ix.cpu().numpy(), dv.cpu().numpy(), cp, ri)
        colcheck.assert_columns(cp, got, ref["mval"], precision)
        big = (I > 64) | (J > 27) | (nB > 512)
        colcheck.assert_columns(cp, got, ref["mval"], precision, cols=np.flatnonzero(big), what="large class")
        colcheck.assert_res2(r2.cpu().numpy(), ref["res2"] + ref["out2"], gamma, precision)
        if precision == "fp32r":
            # the large class's FP32 tile with one guarded step: every column kept its one-step
            # solution or was re-solved in FP64, and the FP32 tile served large columns
            one, two, fp64 = handle.sam_refine_stats()
            assert one + two + fp64 == Ak.n and two == 0
            assert fp64 < int(big.sum()), (one, fp64, int(big.sum()))


def test_large_columns_in_a_shared_batch_multi_target_and_plan(sam, handle):
    """A level-3 sequence of one structure (shadow data shared across maps),
    the same maps against one target per map, and the captured plan: the
    large class reads every map's values at its own offsets."""
    import torch

    seq = W.config2(nx=20, nmat=3)
    aks = [sam.Csr.from_host(m) for m in seq.mats]
    a0 = aks[0]
    n = seq.mats[0].n
    pats = handle.sam_pattern_build_batched(aks, 3)
    offs, rp, ci, v, fro = handle.sam_build_batched(aks, a0, pats, "fp32r", 1, want_fro=True)
    offs2, rp2, ci2, v2, fro2 = handle.sam_build_batched(aks, [a0] * 3, pats, "fp32r", 1, want_fro=True)
    assert torch.equal(v, v2) and np.array_equal(fro, fro2)
    plan = handle.sam_plan_create(aks, a0, pats, "fp32r", 1)
    plan.execute()
    handle.sam_sync()
    assert torch.equal(plan.M_val, v)
    plan.destroy()
    rp, ci, v = rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy()
    for k, Ak in enumerate(seq.mats):
        cp, ri = oracle.pattern(Ak, 3)
        ref = oracle.build(Ak, seq.mats[0], cp, ri)
        got = colcheck.csr_to_csc_values(n, rp[k * (n + 1):(k + 1) * (n + 1)], ci[offs[k]:offs[k + 1]],
                                         v[offs[k]:offs[k + 1]], cp, ri)
        colcheck.assert_columns(cp, got, ref["mval"], "fp32r", what="map %d" % k)


@pytest.mark.parametrize("precision,steps", [("fp64", 0), ("fp32r", 2)])
def test_adjoint_of_large_columns_matches_oracle(sam, handle, precision, steps):
    """Level-3 maps mix register-class columns (the boundary) and large
    columns (the interior); the adjoint of both against the oracle's FP64
    adjoint, batched and single calls bit for bit."""
    import scipy.sparse as sp
    import torch

    seq = W.config2(nx=14, nmat=2)
    a0, a1 = seq.mats[0], seq.mats[1]
    n = a1.n
    I, J, nB = _sizes(a1, 3)
    assert ((I > 64) | (J > 27) | (nB > 512)).sum() > 20
    cp, ri = oracle.pattern(a1, 3)
    fwd = oracle.build(a1, a0, cp, ri)
    gbar = np.random.default_rng(9).standard_normal(len(ri))
    want_k, want_0, want_m = oracle.adjoint(a1, a0, cp, ri, fwd["mval"], gbar, 0.7, want_dmres=True)

    def csr_vals(vals_csc):
        m = sp.csc_matrix((vals_csc, ri, cp), shape=(n, n)).tocsr()
        m.sort_indices()
        return m.data

    A1, A0 = sam.Csr.from_host(a1), sam.Csr.from_host(a0)
    S = handle.sam_pattern_build(A1, 3)
    m_csr = torch.from_numpy(csr_vals(fwd["mval"])).cuda()
    g_csr = torch.from_numpy(csr_vals(gbar)).cuda()
    dmres = torch.empty_like(m_csr)
    dk, d0 = handle.sam_build_backward(A1, A0, S, m_csr, g_csr, precision, steps, 0.7, dM_resid=dmres)
    handle.sam_sync()
    scale = max(np.abs(want_k).max(), np.abs(want_0).max())
    tol = 1e-10
    assert np.abs(dk.cpu().numpy() - want_k).max() <= tol * scale
    assert np.abs(d0.cpu().numpy() - want_0).max() <= tol * scale
    mm = sp.csc_matrix((want_m, ri, cp), shape=(n, n)).tocsr()
    mm.sort_indices()
    assert np.abs(dmres.cpu().numpy() - mm.data).max() <= 1e-9 * max(np.abs(gbar).max(), 1.0)
    # batched (two maps, one structure) = single calls, bit for bit
    A2 = sam.Csr.from_host(seq.mats[1])
    pats = handle.sam_pattern_build_batched([A1, A2], 3)
    mm2 = torch.cat([m_csr, m_csr])
    gg2 = torch.cat([g_csr, g_csr])
    dkb, d0b = handle.sam_build_backward_batched([A1, A2], [A0, A0], pats, mm2, gg2, precision, steps, 0.7)
    handle.sam_sync()
    assert torch.equal(dkb[:a1.nnz], dk) and torch.equal(dkb[a1.nnz:], dk)
    assert torch.equal(d0b[:a0.nnz], d0) and torch.equal(d0b[a0.nnz:], d0)
    for p in pats:
        p.destroy()
