"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle
on the same seeded inputs.

Bars: patterns, shadow-derived CSR structure and row pointers bit-exact;
map values column by column within a relative error of 1e-12 (SAM_FP64)
and 1e-10 (SAM_FP32_REFINE), and the whole map within the same relative
Frobenius error; per-column squared residuals within the bar derived in
colcheck.py."""
import numpy as np
import pytest
import scipy.sparse as sp

import colcheck
import oracle
from paper_2406_17656_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32r": 1e-10}


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


def dev(sam, m):
    return sam.Csr.from_host(m)


def oracle_map(Ak, A0, level):
    cp, ri = oracle.pattern(Ak, level)
    out = oracle.build(Ak, A0, cp, ri)
    ip, ix, dv = oracle.to_csr(Ak.n, cp, ri, out["mval"])
    return {"cp": cp, "ri": ri, "ip": ip, "ix": ix, "dv": dv, "res2": out["res2"] + out["out2"],
            "mval": out["mval"]}


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CASES = {
    "poisson5_32_L1": lambda: (W.config1(), 1),
    "q1_40_L1": lambda: (W.config2(nx=40, nmat=3), 1),
    "q1_40_L2": lambda: (W.config2(nx=40, nmat=3), 2),
    "upwind7_11_L2": lambda: (W.config3(nx=11, nmat=4), 2),
    "fem_36_L1": lambda: (W.config4(ncell=36, nmat=3, flip_frac=0.05), 1),
    "fem_36_L2": lambda: (W.config4(ncell=36, nmat=3, flip_frac=0.05), 2),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_pattern_bit_exact(sam, handle, case):
    seq, level = CASES[case]()
    for Ak in seq.mats:
        cp, ri = oracle.pattern(Ak, level)
        S = handle.sam_pattern_build(dev(sam, Ak), level)
        assert S.nnz == len(ri)
        assert np.array_equal(S.colptr().cpu().numpy(), cp)
        assert np.array_equal(S.rowidx().cpu().numpy(), ri)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_pattern_random_nonsymmetric(sam, handle, seed, level):
    rng = np.random.default_rng(100 + seed)
    n = 300
    p = (rng.random((n, n)) < 0.01) | np.eye(n, dtype=bool)
    p[:, rng.integers(0, n, 3)] = False  # a few empty columns
    a = np.where(p, rng.uniform(1.0, 2.0, (n, n)), 0.0)
    A = W.CSR.from_dense(a)
    cp, ri = oracle.pattern(A, level)
    S = handle.sam_pattern_build(dev(sam, A), level)
    assert np.array_equal(S.colptr().cpu().numpy(), cp)
    assert np.array_equal(S.rowidx().cpu().numpy(), ri)


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_build_matches_oracle(sam, handle, case, precision):
    import torch

    seq, level = CASES[case]()
    A0 = seq.mats[0]
    for Ak in seq.mats[1:]:
        ref = oracle_map(Ak, A0, level)
        S = handle.sam_pattern_build(dev(sam, Ak), level)
        st = torch.empty(Ak.n, dtype=torch.int32, device="cuda")
        r2 = torch.empty(Ak.n, dtype=torch.float64, device="cuda")
        ip, ix, dv = handle.sam_build(dev(sam, Ak), dev(sam, A0), S, precision, refine_steps=1,
                                      col_status=st, res2=r2)
        handle.sam_sync()
        assert np.array_equal(ip.cpu().numpy(), ref["ip"])
        assert np.array_equal(ix.cpu().numpy(), ref["ix"])
        assert int(st.abs().max()) == 0
        err = rel_fro(dv.cpu().numpy(), ref["dv"])
        assert err <= TOL[precision], err
        got = colcheck.csr_to_csc_values(Ak.n, ip.cpu().numpy(), ix.cpu().numpy(), dv.cpu().numpy(), ref["cp"],
                                         ref["ri"])
        colcheck.assert_columns(ref["cp"], got, ref["mval"], precision)
        colcheck.assert_res2(r2.cpu().numpy(), ref["res2"], colcheck.target_column_norms(A0), precision)


@pytest.mark.parametrize("steps", [0, 1, 2])
def test_refinement_steps_converge(sam, handle, steps):
    seq = W.config2(nx=32, nmat=4)
    Ak, A0 = seq.mats[3], seq.mats[0]
    ref = oracle_map(Ak, A0, 2)
    S = handle.sam_pattern_build(dev(sam, Ak), 2)
    ip, ix, dv = handle.sam_build(dev(sam, Ak), dev(sam, A0), S, "fp32r", refine_steps=steps)
    err = rel_fro(dv.cpu().numpy(), ref["dv"])
    bound = {0: 1e-5, 1: 1e-10, 2: 1e-13}[steps]
    assert err <= bound, err
    if steps >= 1:  # guarded: every column within the bar
        got = colcheck.csr_to_csc_values(Ak.n, ip.cpu().numpy(), ix.cpu().numpy(), dv.cpu().numpy(), ref["cp"],
                                         ref["ri"])
        colcheck.assert_columns(ref["cp"], got, ref["mval"], "fp32r")


def test_batched_build_matches_oracle(sam, handle):
    seq = W.config2(nx=36, nmat=5, level=2)
    A0 = seq.mats[0]
    Aks = [dev(sam, m) for m in seq.mats]
    Ss = handle.sam_pattern_build_batched(Aks, 2)
    import torch

    n = A0.n
    r2 = torch.empty(len(Aks) * n, dtype=torch.float64, device="cuda")
    offs, rp, ci, v, fro = handle.sam_build_batched(Aks, dev(sam, A0), Ss, "fp32r", 1, want_fro=True, res2=r2)
    rp, ci, v, r2 = rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy(), r2.cpu().numpy()
    gamma = colcheck.target_column_norms(A0)
    for k, Ak in enumerate(seq.mats):
        ref = oracle_map(Ak, A0, 2)
        assert np.array_equal(rp[k * (n + 1):(k + 1) * (n + 1)], ref["ip"])
        assert np.array_equal(ci[offs[k]:offs[k + 1]], ref["ix"])
        assert rel_fro(v[offs[k]:offs[k + 1]], ref["dv"]) <= 1e-10
        got = colcheck.csr_to_csc_values(n, rp[k * (n + 1):(k + 1) * (n + 1)], ci[offs[k]:offs[k + 1]],
                                         v[offs[k]:offs[k + 1]], ref["cp"], ref["ri"])
        colcheck.assert_columns(ref["cp"], got, ref["mval"], "fp32r", what="map %d" % k)
        colcheck.assert_res2(r2[k * n:(k + 1) * n], ref["res2"], gamma, "fp32r", what="res2 of map %d" % k)
        # the reported residual is the residual of the map that was built ...
        m = sp.csr_matrix((v[offs[k]:offs[k + 1]], ci[offs[k]:offs[k + 1]], rp[k * (n + 1):(k + 1) * (n + 1)]),
                          shape=(n, n)).tocsc()
        m.sort_indices()
        own, _ = oracle.residual(Ak, m.indptr, m.indices, m.data, A0)
        assert abs(fro[k] - own) <= 1e-10 * own + 1e-13 * np.linalg.norm(A0.data)
        # ... and differs from the oracle map's residual by at most ||A_k (M - M_oracle)||_F
        ofro, _ = oracle.residual(Ak, ref["cp"], ref["ri"], ref["mval"], A0)
        a_abs = abs(Ak.to_scipy())
        a2 = np.sqrt(a_abs.sum(0).max() * a_abs.sum(1).max())  # >= ||A_k||_2
        assert abs(fro[k] - ofro) <= 1e-10 * ofro + a2 * np.linalg.norm(m.data - ref["mval"]) + 1e-14 * ofro


def test_identity_map_when_source_is_target(sam, handle):
    A = W.config2(nx=30, nmat=1).mats[0]
    S = handle.sam_pattern_build(dev(sam, A), 2)
    for prec in ("fp64", "fp32r"):
        ip, ix, dv = handle.sam_build(dev(sam, A), dev(sam, A), S, prec, 1)
        m = sp.csr_matrix((dv.cpu().numpy(), ix.cpu().numpy(), ip.cpu().numpy()), shape=(A.n, A.n))
        assert abs(m - sp.eye(A.n)).max() < 1e-12


def test_residual_matches_oracle(sam, handle):
    seq = W.config4(ncell=30, nmat=4, flip_frac=0.2)
    Ak, A0 = seq.mats[3], seq.mats[0]
    for level in (0, 1, 2):
        ref = oracle_map(Ak, A0, level)
        M = sam.Csr.from_host(W.CSR(Ak.n, ref["ip"], ref["ix"], ref["dv"]))
        fro, rel = handle.sam_residual(dev(sam, Ak), M, dev(sam, A0))
        ofro, orel = oracle.residual(Ak, ref["cp"], ref["ri"], ref["mval"], A0)
        assert abs(fro - ofro) <= 1e-12 * ofro
        assert abs(rel - orel) <= 1e-12 * orel


def test_apply_matches_sparse_product(sam, handle):
    import torch

    seq = W.config2(nx=24, nmat=2)
    ref = oracle_map(seq.mats[1], seq.mats[0], 2)
    M = sam.Csr.from_host(W.CSR(seq.mats[1].n, ref["ip"], ref["ix"], ref["dv"]))
    x = np.random.default_rng(3).standard_normal(seq.mats[1].n)
    y = handle.sam_apply(M, torch.from_numpy(x).cuda()).cpu().numpy()
    want = oracle.apply(ref["ip"], ref["ix"], ref["dv"], x)
    assert np.max(np.abs(y - want)) <= 1e-14 * np.max(np.abs(want))


def test_host_buffers_give_the_device_result(sam, handle):
    """The same C-ABI call with host (numpy) inputs and outputs."""
    seq = W.config2(nx=20, nmat=2)
    Ak, A0 = seq.mats[1], seq.mats[0]
    S = handle.sam_pattern_build(dev(sam, Ak), 2)
    ipd, ixd, dvd = handle.sam_build(dev(sam, Ak), dev(sam, A0), S, "fp32r", 1)
    hk = sam.Csr(Ak.indptr, Ak.indices, Ak.data)
    h0 = sam.Csr(A0.indptr, A0.indices, A0.data)
    out = (np.empty(Ak.n + 1, np.int32), np.empty(S.nnz, np.int32), np.empty(S.nnz, np.float64))
    handle.sam_build(hk, h0, S, "fp32r", 1, out=out)
    assert np.array_equal(out[0], ipd.cpu().numpy())
    assert np.array_equal(out[1], ixd.cpu().numpy())
    assert np.array_equal(out[2], dvd.cpu().numpy())


@pytest.mark.parametrize("nmat,host_inputs,steps", [(4, False, 1), (5, True, 1), (4, True, "auto")])
def test_chunked_host_outputs_give_the_device_result(sam, handle, nmat, host_inputs, steps):
    """A one-structure sequence large enough (4 or 5 maps of 65536 columns)
    that a build into host arrays solves its large size classes in chunks of
    maps (3 + 1, or 4 + 1: the last chunk is the smallest) and copies each
    chunk's values while the next is solved (with host inputs, their values
    are copied while the structure work runs; the automatic refinement mode
    re-solves columns after all the solves and is not chunked): the same bits
    as the build into device arrays, residuals and column status included."""
    import torch

    seq = W.config2(nx=256, nmat=nmat)
    aks = [sam.Csr.from_host(m) for m in seq.mats]
    ps = handle.sam_pattern_build_batched(aks, 2)
    K, n = nmat, aks[0].n
    st_d = torch.empty(K * n, dtype=torch.int32, device="cuda")
    r2_d = torch.empty(K * n, dtype=torch.float64, device="cuda")
    offs, rp_d, ci_d, mv_d, fro_d = handle.sam_build_batched(aks, aks[0], ps, "fp32r", steps, col_status=st_d,
                                                             res2=r2_d, want_fro=True)
    tot = int(offs[-1])
    out = [torch.full((K * (n + 1),), -1, dtype=torch.int32).pin_memory(),
           torch.full((tot,), -1, dtype=torch.int32).pin_memory(),
           torch.full((tot,), np.nan, dtype=torch.float64).pin_memory(),
           torch.full((K * n,), -1, dtype=torch.int32).pin_memory(),
           torch.full((K * n,), np.nan, dtype=torch.float64).pin_memory()]
    src = aks
    if host_inputs:
        pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        src = [sam.Csr(pin(m.indptr), pin(m.indices), pin(m.data), n=n) for m in seq.mats]
    _, _, _, _, fro_h = handle.sam_build_batched(src, src[0], ps, "fp32r", steps, M_row_ptr=out[0], M_col_idx=out[1],
                                                 M_val=out[2], col_status=out[3], res2=out[4], want_fro=True,
                                                 offsets=offs)
    for p in ps:
        p.destroy()
    for got, want in zip(out, (rp_d, ci_d, mv_d, st_d, r2_d)):
        assert torch.equal(got, want.cpu())
    assert np.array_equal(fro_h, fro_d)


def test_changing_structure_host_batch_gives_the_device_result(sam, handle):
    """A batch whose sources change structure from map to map (P1 FEM with
    flipped diagonals), with host inputs (values copied while the structure
    work runs) and host outputs: the same bits as with device arrays."""
    seq = W.config4(ncell=40, nmat=4, flip_frac=0.2)
    aks = [sam.Csr.from_host(m) for m in seq.mats]
    ps = handle.sam_pattern_build_batched(aks, 2)
    offs, rp_d, ci_d, mv_d, fro_d = handle.sam_build_batched(aks, aks[0], ps, "fp32r", 1, want_fro=True)
    n = aks[0].n
    hk = [sam.Csr(m.indptr, m.indices, m.data, n=n) for m in seq.mats]
    out = (np.full(4 * (n + 1), -1, np.int32), np.full(int(offs[-1]), -1, np.int32),
           np.full(int(offs[-1]), np.nan))
    _, _, _, _, fro_h = handle.sam_build_batched(hk, hk[0], ps, "fp32r", 1, M_row_ptr=out[0], M_col_idx=out[1],
                                                 M_val=out[2], want_fro=True, offsets=offs)
    for p in ps:
        p.destroy()
    assert np.array_equal(out[0], rp_d.cpu().numpy())
    assert np.array_equal(out[1], ci_d.cpu().numpy())
    assert np.array_equal(out[2], mv_d.cpu().numpy())
    assert np.array_equal(fro_h, fro_d)


# ------------------------------------------------------------- edge cases


def test_empty_matrix_is_rejected(sam, handle):
    """An empty matrix (n = 0) is an invalid argument wherever a matrix is
    taken, and the handle stays usable."""
    import torch

    E = sam.Csr(torch.zeros(1, dtype=torch.int32, device="cuda"), torch.zeros(0, dtype=torch.int32, device="cuda"),
                torch.zeros(0, dtype=torch.float64, device="cuda"), n=0)
    for call in (lambda: handle.sam_pattern_build(E, 1), lambda: handle.sam_sparsify(E, "tau", 0.5),
                 lambda: handle.sam_residual(E, E, E)):
        with pytest.raises(sam.SamError) as err:
            call()
        assert err.value.status == sam.SAM_ERR_INVALID_ARG
    A = W.config1().mats[1]
    S = handle.sam_pattern_build(dev(sam, A), 1)
    assert S.nnz > A.n


def test_one_by_one(sam, handle):
    A = W.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0]))
    B = W.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0]))
    S = handle.sam_pattern_build(dev(sam, A), 1)
    for prec in ("fp64", "fp32r"):
        ip, ix, dv = handle.sam_build(dev(sam, A), dev(sam, B), S, prec, 1)
        assert abs(float(dv.cpu()[0]) - 0.75) < 1e-15


def test_non_nested_target_entries_enter_the_residual(sam, handle):
    seq = W.config4(ncell=20, nmat=6, flip_frac=0.3)
    Ak, A0 = seq.mats[5], seq.mats[0]
    ref = oracle_map(Ak, A0, 0)
    assert ref["res2"].sum() > 0
    import torch

    S = handle.sam_pattern_build(dev(sam, Ak), 0)
    r2 = torch.empty(Ak.n, dtype=torch.float64, device="cuda")
    ip, ix, dv = handle.sam_build(dev(sam, Ak), dev(sam, A0), S, "fp64", 0, res2=r2)
    assert rel_fro(dv.cpu().numpy(), ref["dv"]) <= 1e-12
    got = colcheck.csr_to_csc_values(Ak.n, ip.cpu().numpy(), ix.cpu().numpy(), dv.cpu().numpy(), ref["cp"], ref["ri"])
    colcheck.assert_columns(ref["cp"], got, ref["mval"], "fp64")
    assert np.allclose(r2.cpu().numpy(), ref["res2"], rtol=1e-10, atol=1e-14)
    colcheck.assert_res2(r2.cpu().numpy(), ref["res2"], colcheck.target_column_norms(A0), "fp64")


def test_rank_deficient_column_is_reported(sam, handle):
    import torch

    A = W.config1().mats[1].to_scipy().tolil()
    A[:, 5] = 0.0  # column 5 has no stored entries -> its problem has no rows
    A = W.CSR.from_scipy(A.tocsr())
    S = handle.sam_pattern_build(dev(sam, A), 1)
    st = torch.zeros(A.n, dtype=torch.int32, device="cuda")
    handle.sam_build(dev(sam, A), dev(sam, W.config1().mats[0]), S, "fp32r", 1, col_status=st)
    with pytest.raises(sam.SamError) as e:
        handle.sam_sync()
    assert e.value.status == sam.SAM_ERR_RANK_DEFICIENT
    assert int(st.cpu().numpy()[5]) == sam.SAM_ERR_RANK_DEFICIENT


def test_oversized_column_is_unsupported(sam, handle):
    n = 200
    a = np.eye(n) * 200.0
    a[0, 1:150] = -1.0  # column 0 of the level-1 pattern has 150 unknowns, past every size class
    a[1:150, 0] = -1.0
    A = W.CSR.from_dense(a)
    S = handle.sam_pattern_build(dev(sam, A), 1)
    handle.sam_build(dev(sam, A), dev(sam, A), S, "fp32r", 1)
    with pytest.raises(sam.SamError) as e:
        handle.sam_sync()
    assert e.value.status == sam.SAM_ERR_UNSUPPORTED


def test_malformed_csr_is_rejected_without_running_kernels(sam, handle):
    A = W.config1().mats[0]
    bad = W.CSR(A.n, A.indptr.copy(), A.indices.copy(), A.data.copy())
    bad.indices[3], bad.indices[4] = bad.indices[4], bad.indices[3]  # unsorted row
    with pytest.raises(sam.SamError) as e:
        handle.sam_pattern_build(dev(sam, bad), 1)
    assert e.value.status == sam.SAM_ERR_BAD_CSR
    bad2 = W.CSR(A.n, A.indptr.copy(), A.indices.copy(), A.data.copy())
    bad2.indices[7] = A.n + 5  # out of range
    with pytest.raises(sam.SamError) as e:
        handle.sam_pattern_build(dev(sam, bad2), 1)
    assert e.value.status == sam.SAM_ERR_BAD_CSR


# ------------------------------------------- full size, sampled columns


def test_full_size_q1_256_level2_sampled(sam, handle):
    """The 256x256 Q1 diffusion sequence (10 matrices, level 2) in the
    benchmark's launch configuration; 1500 sampled columns per map against
    the oracle."""
    import torch

    seq = W.config2(nx=256, nmat=10, level=2)
    A0 = seq.mats[0]
    Aks = [dev(sam, m) for m in seq.mats]
    Ss = handle.sam_pattern_build_batched(Aks, 2)
    offs, rp, ci, v, fro = handle.sam_build_batched(Aks, dev(sam, A0), Ss, "fp32r", 1, want_fro=True)
    n = A0.n
    rp, ci, v = rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy()
    rng = np.random.default_rng(77)
    for k in (1, 5, 9):
        Ak = seq.mats[k]
        cp, ri = oracle.pattern(Ak, 2)
        assert np.array_equal(Ss[k].colptr().cpu().numpy(), cp)
        cols = np.sort(rng.choice(n, 1500, replace=False)).astype(np.int32)
        cols = np.unique(np.concatenate([cols, [0, n - 1, 255, n - 256]]).astype(np.int32))
        ref = oracle.build_cols(Ak, A0, cp, ri, cols)
        m = sp.csr_matrix((v[offs[k]:offs[k + 1]], ci[offs[k]:offs[k + 1]], rp[k * (n + 1):(k + 1) * (n + 1)]),
                          shape=(n, n)).tocsc()
        m.sort_indices()
        assert np.array_equal(m.indptr, cp) and np.array_equal(m.indices, ri)
        idx = np.concatenate([np.arange(cp[j], cp[j + 1]) for j in cols])
        assert rel_fro(m.data[idx], ref["mval"][idx]) <= 1e-10
        colcheck.assert_columns(cp, m.data, ref["mval"], "fp32r", cols=cols, what="map %d" % k)


def test_multi_target_batch_matches_per_pair_oracle(sam, handle):
    """sam_build_multi: each map against its own target, small pairs."""
    pairs = [W.config5_pair(b, nx=20) for b in range(3)]
    A0s = [dev(sam, p[0]) for p in pairs]
    A1s = [dev(sam, p[1]) for p in pairs]
    for level in (1, 2):
        Ss = handle.sam_pattern_build_batched(A1s, level)
        offs, rp, ci, v, fro = handle.sam_build_batched(A1s, A0s, Ss, "fp32r", 1, want_fro=True)
        n = pairs[0][0].n
        rp, ci, v = rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy()
        for k, (a0, a1) in enumerate(pairs):
            ref = oracle_map(a1, a0, level)
            assert np.array_equal(rp[k * (n + 1):(k + 1) * (n + 1)], ref["ip"])
            assert np.array_equal(ci[offs[k]:offs[k + 1]], ref["ix"])
            assert rel_fro(v[offs[k]:offs[k + 1]], ref["dv"]) <= 1e-10
            got = colcheck.csr_to_csc_values(n, rp[k * (n + 1):(k + 1) * (n + 1)], ci[offs[k]:offs[k + 1]],
                                             v[offs[k]:offs[k + 1]], ref["cp"], ref["ri"])
            colcheck.assert_columns(ref["cp"], got, ref["mval"], "fp32r", what="pair %d" % k)
            assert abs(fro[k] ** 2 - ref["res2"].sum()) <= 1e-9 * ref["res2"].sum()


def _banded_nonsymmetric(seed, offsets, n=400):
    """Diagonally dominant matrix with a few nonsymmetric off-diagonals,
    each entry kept with probability 0.8."""
    rng = np.random.default_rng(seed)
    a = np.zeros((n, n))
    for o in offsets:
        i = np.arange(max(0, -o), min(n, n - o))
        keep = rng.random(len(i)) < 0.8
        a[i[keep], i[keep] + o] = rng.uniform(-1.0, 1.0, keep.sum())
    a[np.arange(n), np.arange(n)] = 4.0 + rng.random(n)
    return W.CSR.from_dense(a)


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_nonsymmetric_structure_takes_the_general_transpose(sam, handle, precision):
    """Structurally nonsymmetric source and target go through the
    atomic-fill + sort transposes (symmetric ones through the mirror
    lookup); against the oracle."""
    import torch

    A1 = _banded_nonsymmetric(31, (1, -2, 4, -7))
    A0 = _banded_nonsymmetric(32, (1, -1, 3))
    s1 = abs(A1.to_scipy())
    assert (s1 != s1.T).nnz > 0
    for level in (1, 2):
        ref = oracle_map(A1, A0, level)
        S = handle.sam_pattern_build(dev(sam, A1), level)
        st = torch.empty(A1.n, dtype=torch.int32, device="cuda")
        ip, ix, dv = handle.sam_build(dev(sam, A1), dev(sam, A0), S, precision, refine_steps=1, col_status=st)
        handle.sam_sync()
        assert int(st.abs().max()) == 0
        assert np.array_equal(ip.cpu().numpy(), ref["ip"]) and np.array_equal(ix.cpu().numpy(), ref["ix"])
        assert rel_fro(dv.cpu().numpy(), ref["dv"]) <= TOL[precision]
        got = colcheck.csr_to_csc_values(A1.n, ip.cpu().numpy(), ix.cpu().numpy(), dv.cpu().numpy(), ref["cp"],
                                         ref["ri"])
        colcheck.assert_columns(ref["cp"], got, ref["mval"], precision)


@pytest.mark.parametrize("seqname", ["fem_changing_structure", "q1_one_structure"])
def test_trusted_inputs_give_the_same_maps(sam, seqname):
    """A trusted handle skips validation (and so the symmetry detection; the
    structure comparison that lets a sequence of one structure share its
    structure work runs on its own): its maps equal the validated handle's
    bit for bit."""
    import torch

    seq = (W.config4(ncell=24, nmat=3, flip_frac=0.1) if seqname == "fem_changing_structure"
           else W.config2(nx=30, nmat=4))
    outs = []
    for trusted in (False, True):
        h = sam.Handle(trusted=trusted)
        try:
            Aks = [dev(sam, m) for m in seq.mats]
            Ss = h.sam_pattern_build_batched(Aks, 2)
            offs, rp, ci, v, _ = h.sam_build_batched(Aks, dev(sam, seq.mats[0]), Ss, "fp32r", 1)
            outs.append((rp, ci, v))
        finally:
            h.close()
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def test_dense_target_columns_use_the_shadow_row_search(sam, handle):
    """Target columns with more stored entries than the precomputed local-row
    capacity (32), inside and outside the shadow rows, against the oracle."""
    seq = W.config2(nx=24, nmat=2)
    a0, a1 = seq.mats
    d = a0.dense()
    rng = np.random.default_rng(12)
    for j in rng.choice(a0.n, 12, replace=False):
        rows = rng.choice(a0.n, 45, replace=False)
        d[rows, j] += rng.uniform(-0.5, 0.5, 45)
    A0 = W.CSR.from_dense(d)
    assert np.diff(A0.to_scipy().tocsc().indptr).max() > 32
    for precision in ("fp64", "fp32r"):
        ref = oracle_map(a1, A0, 2)
        S = handle.sam_pattern_build(dev(sam, a1), 2)
        r2 = __import__("torch").empty(a1.n, dtype=__import__("torch").float64, device="cuda")
        ip, ix, dv = handle.sam_build(dev(sam, a1), dev(sam, A0), S, precision, refine_steps=1, res2=r2)
        assert rel_fro(dv.cpu().numpy(), ref["dv"]) <= TOL[precision]
        got = colcheck.csr_to_csc_values(a1.n, ip.cpu().numpy(), ix.cpu().numpy(), dv.cpu().numpy(), ref["cp"],
                                         ref["ri"])
        colcheck.assert_columns(ref["cp"], got, ref["mval"], precision)
        colcheck.assert_res2(r2.cpu().numpy(), ref["res2"], colcheck.target_column_norms(A0), precision)


def test_dense_target_columns_in_a_shared_batch(sam, handle):
    """A batch of one structure (shadow data shared across the maps) whose
    target has columns longer than the precomputed local rows (32 entries):
    every map searches the target's rows among map 0's shadow rows, and
    matches the oracle column by column."""
    import torch

    seq = W.config2(nx=24, nmat=3)
    d = seq.mats[0].dense()
    rng = np.random.default_rng(21)
    for j in rng.choice(d.shape[0], 10, replace=False):
        rows = rng.choice(d.shape[0], 45, replace=False)
        d[rows, j] += rng.uniform(-0.5, 0.5, 45)
    A0 = W.CSR.from_dense(d)
    n = A0.n
    aks = [dev(sam, m) for m in seq.mats]
    Ss = handle.sam_pattern_build_batched(aks, 2)
    r2 = torch.empty(len(aks) * n, dtype=torch.float64, device="cuda")
    offs, rp, ci, v, _ = handle.sam_build_batched(aks, dev(sam, A0), Ss, "fp32r", 1, res2=r2)
    rp, ci, v, r2 = rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy(), r2.cpu().numpy()
    gamma = colcheck.target_column_norms(A0)
    for k, Ak in enumerate(seq.mats):
        ref = oracle_map(Ak, A0, 2)
        got = colcheck.csr_to_csc_values(n, rp[k * (n + 1):(k + 1) * (n + 1)], ci[offs[k]:offs[k + 1]],
                                         v[offs[k]:offs[k + 1]], ref["cp"], ref["ri"])
        colcheck.assert_columns(ref["cp"], got, ref["mval"], "fp32r", what="map %d" % k)
        colcheck.assert_res2(r2[k * n:(k + 1) * n], ref["res2"], gamma, "fp32r", what="res2 of map %d" % k)
