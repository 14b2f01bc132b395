"""GPU adjoint (sam_build_backward and the autograd wrappers) against the
oracle's adjoint and against finite differences of the GPU's FP64 forward
build."""
import numpy as np
import pytest
import scipy.sparse as sp

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


def _csc_to_csr_values(n, cp, ri, vals_csc):
    m = sp.csc_matrix((vals_csc, ri, cp), shape=(n, n)).tocsr()
    m.sort_indices()
    return m.data


def _csr_to_csc_values(n, ip, ix, vals_csr):
    m = sp.csr_matrix((vals_csr, ix, ip), shape=(n, n)).tocsc()
    m.sort_indices()
    return m.data


CASES = {
    "q1_20_L1": lambda: (W.config2(nx=20, nmat=2), 1),
    "q1_20_L2": lambda: (W.config2(nx=20, nmat=2), 2),
    "upwind_8_L2": lambda: (W.config3(nx=8, nmat=3), 2),
    "fem_16_L1": lambda: (W.config4(ncell=16, nmat=3, flip_frac=0.2), 1),
}


@pytest.mark.parametrize("rho", [0.0, 0.7])
@pytest.mark.parametrize("precision,steps", [("fp64", 0), ("fp32r", 1), ("fp32r", 2)])
@pytest.mark.parametrize("case", sorted(CASES))
def test_adjoint_matches_oracle(sam, handle, case, precision, steps, rho):
    import torch

    seq, level = CASES[case]()
    a0, ak = seq.mats[0], seq.mats[-1]
    n = ak.n
    cp, ri = oracle.pattern(ak, level)
    fwd = oracle.build(ak, a0, cp, ri)
    gbar = np.random.default_rng(7).standard_normal(len(ri))
    want_k, want_0, want_m = oracle.adjoint(ak, a0, cp, ri, fwd["mval"], gbar, rho, want_dmres=True)
    S = handle.sam_pattern_build(sam.Csr.from_host(ak), level)
    ip, ix, _ = oracle.to_csr(n, cp, ri, fwd["mval"])
    m_csr = torch.from_numpy(_csc_to_csr_values(n, cp, ri, fwd["mval"])).cuda()
    g_csr = torch.from_numpy(_csc_to_csr_values(n, cp, ri, gbar)).cuda()
    dmres = torch.empty_like(m_csr)
    dk, d0 = handle.sam_build_backward(sam.Csr.from_host(ak), sam.Csr.from_host(a0), S, m_csr, g_csr, precision,
                                       steps, rho, dM_resid=dmres)
    handle.sam_sync()
    dk, d0 = dk.cpu().numpy(), d0.cpu().numpy()
    scale = max(np.abs(want_k).max(), np.abs(want_0).max())
    # lambda from the FP32 R converges like the forward refinement: ~u32 kappa^2 per step
    tol = {("fp64", 0): 1e-10, ("fp32r", 1): 1e-7, ("fp32r", 2): 1e-10}[(precision, steps)]
    assert np.abs(dk - want_k).max() <= tol * scale
    assert np.abs(d0 - want_0).max() <= tol * scale
    got_m = _csr_to_csc_values(n, ip, ix, dmres.cpu().numpy())
    assert np.abs(got_m - want_m).max() <= 1e-9 * max(np.abs(gbar).max(), 1.0)


def test_adjoint_is_deterministic(sam, handle):
    import torch

    seq = W.config2(nx=24, nmat=2)
    a0, ak = seq.mats
    cp, ri = oracle.pattern(ak, 2)
    fwd = oracle.build(ak, a0, cp, ri)
    S = handle.sam_pattern_build(sam.Csr.from_host(ak), 2)
    m = torch.from_numpy(_csc_to_csr_values(ak.n, cp, ri, fwd["mval"])).cuda()
    g = torch.randn(len(ri), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    outs = [handle.sam_build_backward(sam.Csr.from_host(ak), sam.Csr.from_host(a0), S, m, g, "fp32r", 1, 0.3)
            for _ in range(3)]
    for dk, d0 in outs[1:]:
        assert torch.equal(dk, outs[0][0]) and torch.equal(d0, outs[0][1])


def test_autograd_loss_matches_finite_differences_32x32(sam, handle):
    """The adjoint workload's loss ||A_1 M_1 - A_0||_F^2 + ||M_1 v||^2 on a
    32x32 instance through the autograd wrappers (FP32 QR + refinement),
    against central differences of the GPU's FP64 build along seeded
    directions, and against the oracle's adjoint."""
    import torch

    from paper_2406_17656_gb300.autograd import SamMap

    a0, a1 = W.config5_pair(0, nx=32)
    v = torch.from_numpy(W.config5_vector(a0.n)).cuda()
    A1, A0 = sam.Csr.from_host(a1), sam.Csr.from_host(a0)
    S = handle.sam_pattern_build(A1, 1)

    def loss(fn, k_val, z_val):
        m = fn(k_val, z_val)
        return fn.residual_sq(k_val, z_val, m) + (fn.matvec(m, v) ** 2).sum()

    f32 = SamMap(handle, (A1.indptr, A1.indices), (A0.indptr, A0.indices), S, "fp32r", 2)
    kv = A1.data.clone().requires_grad_(True)
    zv = A0.data.clone().requires_grad_(True)
    L = loss(f32, kv, zv)
    L.backward()
    gk, g0 = kv.grad.cpu().numpy(), zv.grad.cpu().numpy()
    # oracle adjoint of the same loss
    cp, ri = oracle.pattern(a1, 1)
    fwd = oracle.build(a1, a0, cp, ri)
    mm = sp.csc_matrix((fwd["mval"], ri, cp), shape=(a1.n, a1.n))
    vh = v.cpu().numpy()
    gbar = 2.0 * (mm @ vh)[ri] * vh[np.repeat(np.arange(a1.n), np.diff(cp))]
    _, _, dmres = oracle.adjoint(a1, a0, cp, ri, fwd["mval"], gbar, 1.0, want_dmres=True)
    wk, w0 = oracle.adjoint(a1, a0, cp, ri, fwd["mval"], gbar + dmres, 1.0)
    scale = max(np.abs(wk).max(), np.abs(w0).max())
    assert np.abs(gk - wk).max() <= 1e-8 * scale
    assert np.abs(g0 - w0).max() <= 1e-8 * scale
    # finite differences of the FP64 GPU forward
    f64 = SamMap(handle, (A1.indptr, A1.indices), (A0.indptr, A0.indices), S, "fp64", 0)
    gen = torch.Generator("cuda").manual_seed(11)
    h = 1e-6
    for _ in range(8):
        uk = torch.randn(A1.nnz, dtype=torch.float64, device="cuda", generator=gen)
        u0 = torch.randn(A0.nnz, dtype=torch.float64, device="cuda", generator=gen)
        with torch.no_grad():
            lp = float(loss(f64, A1.data + h * uk, A0.data + h * u0))
            lm = float(loss(f64, A1.data - h * uk, A0.data - h * u0))
        fd = (lp - lm) / (2 * h)
        ad = float(np.dot(gk, uk.cpu().numpy()) + np.dot(g0, u0.cpu().numpy()))
        assert abs(fd - ad) <= 1e-6 * abs(fd)


def test_batched_adjoint_equals_single_calls(sam, handle):
    """sam_build_backward_batched over several pairs gives, bit for bit, the
    gradients of one sam_build_backward call per pair."""
    import torch

    pairs = [W.config5_pair(b, nx=16) for b in range(3)]
    A0s = [sam.Csr.from_host(p[0]) for p in pairs]
    A1s = [sam.Csr.from_host(p[1]) for p in pairs]
    Ss = handle.sam_pattern_build_batched(A1s, 2)
    offs, rp, ci, v, _ = handle.sam_build_batched(A1s, A0s, Ss, "fp32r", 1)
    g = torch.randn(v.numel(), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    dk, d0 = handle.sam_build_backward_batched(A1s, A0s, Ss, v, g, "fp32r", 1, 0.4, offsets=offs)
    ko = np.concatenate([[0], np.cumsum([a.nnz for a in A1s])])
    zo = np.concatenate([[0], np.cumsum([a.nnz for a in A0s])])
    for k in range(3):
        sk, s0 = handle.sam_build_backward(A1s[k], A0s[k], Ss[k], v[offs[k]:offs[k + 1]], g[offs[k]:offs[k + 1]],
                                           "fp32r", 1, 0.4)
        assert torch.equal(sk, dk[ko[k]:ko[k + 1]])
        assert torch.equal(s0, d0[zo[k]:zo[k + 1]])
