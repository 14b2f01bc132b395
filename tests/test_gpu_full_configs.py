"""Full-size parity of the remaining workloads, each in its batched launch
configuration: every map of a sequence (or every pair of the adjoint batch)
in one call, then sampled maps compared with the oracle -- patterns and CSR
structure bit-exact on whole maps, values of every sampled column within
the per-column bar (and the sample within the relative Frobenius bar), the
squared residual of every sampled column against the oracle's (bar derived
in colcheck.py), the residual of each sampled map against the oracle's
residual of the GPU's own map."""
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _check_map(k, Ak, A0, level, Ss, offs, rp, ci, v, fro, ncols, seed, tol=1e-10, r2=None):
    n = A0.n
    cp, ri = oracle.pattern(Ak, level)
    assert np.array_equal(Ss[k].colptr().cpu().numpy(), cp)
    assert np.array_equal(Ss[k].rowidx().cpu().numpy(), ri)
    m = sp.csr_matrix((v[offs[k]:offs[k + 1]], ci[offs[k]:offs[k + 1]], rp[k * (n + 1):(k + 1) * (n + 1)]),
                      shape=(n, n)).tocsc()
    m.sort_indices()
    assert np.array_equal(m.indptr, cp) and np.array_equal(m.indices, ri)
    rng = np.random.default_rng(seed)
    cols = np.unique(np.concatenate([rng.choice(n, ncols, replace=False), [0, n - 1]])).astype(np.int32)
    ref = oracle.build_cols(Ak, A0, cp, ri, cols)
    idx = np.concatenate([np.arange(cp[j], cp[j + 1]) for j in cols])
    err = _rel(m.data[idx], ref["mval"][idx])
    assert err <= tol, (k, err)
    colcheck.assert_columns(cp, m.data, ref["mval"], "fp32r", cols=cols, what="map %d" % k)
    if r2 is not None:
        got = r2[k * n:(k + 1) * n][cols]
        want = (ref["res2"] + ref["out2"])[cols]
        colcheck.assert_res2(got, want, colcheck.target_column_norms(A0)[cols], "fp32r", what="res2 of map %d" % k)
    own, _ = oracle.residual(Ak, m.indptr, m.indices, m.data, A0)
    assert abs(fro[k] - own) <= 1e-10 * own + 1e-13 * np.linalg.norm(A0.data)
    return err


def test_config3_upwind7_64cube_20maps_level2(sam, handle):
    """7-point upwind convection-diffusion on 64^3, 20 matrices, level-2
    patterns, all maps in one batched launch with the autotuned schedule."""
    seq = W.config3()
    A0 = seq.mats[0]
    Aks = [sam.Csr.from_host(m) for m in seq.mats]
    a0 = sam.Csr.from_host(A0)
    Ss = handle.sam_pattern_build_batched(Aks, 2)
    handle.sam_tune(Aks, a0, Ss, "fp32r", 1)
    import torch

    r2 = torch.empty(len(Aks) * A0.n, dtype=torch.float64, device="cuda")
    offs, rp, ci, v, fro = handle.sam_build_batched(Aks, a0, Ss, "fp32r", 1, want_fro=True, res2=r2)
    rp, ci, v, r2 = rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy(), r2.cpu().numpy()
    for k in (0, 10, 19):
        _check_map(k, seq.mats[k], A0, 2, Ss, offs, rp, ci, v, fro, 1200, 300 + k, r2=r2)
    # M_0 = I: the first map of a sequence is the identity
    assert fro[0] <= 1e-12 * np.linalg.norm(A0.data)


def test_config4_p1_fem_512_16maps_level2(sam, handle):
    """Jittered P1 FEM with reaction on 512^2 cells, 16 matrices whose
    pattern changes by edge flips (non-nested), level-2 patterns; direct
    call and captured plan."""
    import torch

    seq = W.config4()
    A0 = seq.mats[0]
    Aks = [sam.Csr.from_host(m) for m in seq.mats]
    a0 = sam.Csr.from_host(A0)
    Ss = handle.sam_pattern_build_batched(Aks, 2)
    r2 = torch.empty(len(Aks) * A0.n, dtype=torch.float64, device="cuda")
    offs, rp, ci, v, fro = handle.sam_build_batched(Aks, a0, Ss, "fp32r", 1, want_fro=True, res2=r2)
    # the CUDA-graph-captured pipeline gives the same maps bit for bit
    plan = handle.sam_plan_create(Aks, a0, Ss, "fp32r", 1)
    plan.execute()
    handle.sam_sync()
    assert torch.equal(plan.M_val, v) and torch.equal(plan.M_col_idx, ci) and torch.equal(plan.M_row_ptr, rp)
    plan.destroy()
    rp, ci, v, r2 = rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy(), r2.cpu().numpy()
    for k in (1, 8, 15):
        _check_map(k, seq.mats[k], A0, 2, Ss, offs, rp, ci, v, fro, 1200, 400 + k, r2=r2)


def test_config5_pairs_512_forward_and_adjoint(sam, handle):
    """The adjoint workload: 32 independent (A_0, A_1) 9-point pairs on
    512^2, level 1, forward in one sam_build_multi call and backward of
    L = ||A_1 M_1 - A_0||_F^2 + ||M_1 v||^2 in one batched adjoint call;
    sampled pairs against the oracle (forward columns, and the whole
    gradient of one pair)."""
    import torch

    pairs = [W.config5_pair(b) for b in range(32)]
    n = pairs[0][0].n
    A0s = [sam.Csr.from_host(p[0]) for p in pairs]
    A1s = [sam.Csr.from_host(p[1]) for p in pairs]
    Ss = handle.sam_pattern_build_batched(A1s, 1)
    r2 = torch.empty(32 * n, dtype=torch.float64, device="cuda")
    offs, rp, ci, v, fro = handle.sam_build_batched(A1s, A0s, Ss, "fp32r", 2, want_fro=True, res2=r2)
    rph, cih, vh, r2h = rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy(), r2.cpu().numpy()
    for b in (0, 17, 31):
        _check_map(b, pairs[b][1], pairs[b][0], 1, Ss, offs, rph, cih, vh, fro, 1500, 500 + b, r2=r2h)
    # gradient of the loss: dL/dM from the ||M v||^2 term, residual term direct
    vec = torch.from_numpy(W.config5_vector(n)).cuda()
    rows = torch.repeat_interleave(torch.arange(32 * n, device="cuda"),
                                   (rp.view(32, n + 1)[:, 1:] - rp.view(32, n + 1)[:, :-1]).reshape(-1).long())
    colg = ci.long()
    mv = torch.zeros(32 * n, dtype=torch.float64, device="cuda").index_add_(0, rows, v * vec[colg])
    gbar = 2.0 * mv[rows] * vec[colg]
    dmres = torch.empty_like(v)
    dk, d0 = handle.sam_build_backward_batched(A1s, A0s, Ss, v, gbar, "fp32r", 2, 1.0, offsets=offs, dM_resid=dmres)
    dk, d0 = dk.cpu().numpy(), d0.cpu().numpy()
    koff = np.concatenate([[0], np.cumsum([p[1].nnz for p in pairs])])
    zoff = np.concatenate([[0], np.cumsum([p[0].nnz for p in pairs])])
    b = 17
    a0h, a1h = pairs[b]
    cp, ri = oracle.pattern(a1h, 1)
    fwd = oracle.build(a1h, a0h, cp, ri)
    mm = sp.csc_matrix((fwd["mval"], ri, cp), shape=(n, n))
    vv = W.config5_vector(n)
    g_or = 2.0 * (mm @ vv)[ri] * vv[np.repeat(np.arange(n), np.diff(cp))]
    wk, w0 = oracle.adjoint(a1h, a0h, cp, ri, fwd["mval"], g_or, 1.0)
    scale = max(np.abs(wk).max(), np.abs(w0).max())
    assert np.abs(dk[koff[b]:koff[b + 1]] - wk).max() <= 1e-9 * scale
    assert np.abs(d0[zoff[b]:zoff[b + 1]] - w0).max() <= 1e-9 * scale


def test_config4_every_column_against_the_fp64_build(sam, handle):
    """Every column of the full P1 FEM sequence (16 maps, level 2, the
    workload with the worst-conditioned column problems): FP32 QR + one
    guarded FP64 step against the plain FP64 GPU build, whose columns meet
    the oracle to 1e-12 (the parity tests): the per-column bar, with the
    FP64 build's own error as margin."""
    import torch

    seq = W.config4()
    A0 = seq.mats[0]
    Aks = [sam.Csr.from_host(m) for m in seq.mats]
    a0 = sam.Csr.from_host(A0)
    n = A0.n
    Ss = handle.sam_pattern_build_batched(Aks, 2)
    offs, rp, ci, v32, _ = handle.sam_build_batched(Aks, a0, Ss, "fp32r", 1)
    _, _, _, v64, _ = handle.sam_build_batched(Aks, a0, Ss, "fp64", 0, offsets=offs)
    worst = 0.0
    for k in range(len(Aks)):
        a, b = v32[offs[k]:offs[k + 1]], v64[offs[k]:offs[k + 1]]
        c = ci[offs[k]:offs[k + 1]].long()
        d2 = torch.zeros(n, dtype=torch.float64, device="cuda").index_add_(0, c, (a - b) ** 2)
        w2 = torch.zeros(n, dtype=torch.float64, device="cuda").index_add_(0, c, b * b)
        assert bool((w2 > 0).all())
        worst = max(worst, float(torch.sqrt(d2 / w2).max()))
    assert worst <= colcheck.EPS["fp32r"] + colcheck.EPS["fp64"], worst
