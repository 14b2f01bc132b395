"""The factor tape (sam_factor_tape_bytes / sam_set_factor_tape): a build
records every register-class column's triangular factor R, and an adjoint
replays it instead of gathering B into a tile and factoring it again.
Checked here: the tape's size and layout against the oracle's column
problems (R^T R = B^T B, |R_kk| against LAPACK's QR), replayed adjoints
equal to recomputing ones bit for bit (single, batched over one structure,
batched over changing structures, FP64, FP32 with 1 / 2 / automatic steps,
through autograd), and the error paths."""
import numpy as np
import pytest

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


def _slot(nj):
    """Elements of one column's slot: the packed triangle, rounded up to a
    multiple of four (columns past the register tiles: none)."""
    return ((nj * (nj + 1) // 2 + 3) // 4) * 4 if 1 <= nj <= 27 else 0


def _tape(torch, nbytes):
    return torch.zeros((nbytes + 15) // 16 * 2, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precision", ["fp32r", "fp64"])
def test_tape_size_and_contents_against_the_oracle(sam, handle, precision):
    import torch

    seq = W.config2(nx=12, nmat=2)
    level = 2
    mats = seq.mats
    pats = handle.sam_pattern_build_batched([sam.Csr.from_host(m) for m in mats], level)
    esize = 4 if precision == "fp32r" else 8
    slots, cols = [], []
    for k, A in enumerate(mats):
        cp, ri = oracle.pattern(A, level)
        nj = np.diff(cp)
        slots.append(np.array([_slot(int(x)) for x in nj], dtype=np.int64))
        cols.append((A, cp, ri))
    sizes = np.concatenate(slots)
    nbytes = handle.sam_factor_tape_bytes(pats, precision)
    assert nbytes == int(sizes.sum()) * esize
    off = np.concatenate([[0], np.cumsum(sizes)])
    tape = _tape(torch, nbytes)
    aks = [sam.Csr.from_host(m) for m in mats]
    handle.sam_set_factor_tape(sam.SAM_TAPE_RECORD, tape)
    try:
        handle.sam_build_batched(aks, aks[0], pats, precision, 1)
        handle.sam_sync()
    finally:
        handle.sam_set_factor_tape(sam.SAM_TAPE_OFF)
    raw = tape.cpu().numpy().view(np.float32 if esize == 4 else np.float64)
    n = mats[0].n
    tol = 2e-6 if esize == 4 else 1e-13
    rng = np.random.default_rng(11)
    for k, (A, cp, ri) in enumerate(cols):
        dense = A.to_scipy().toarray()
        for j in rng.choice(n, 40, replace=False):
            J = ri[cp[j]:cp[j + 1]]
            I = np.flatnonzero(np.abs(dense[:, J]).sum(axis=1) > 0)
            B = dense[np.ix_(I, J)]
            nj = len(J)
            base = off[k * n + j]
            R = np.zeros((nj, nj))
            p = base
            for r in range(nj):  # packed: row r from its diagonal
                R[r, r:] = raw[p:p + nj - r]
                p += nj - r
            G = B.T @ B
            assert np.abs(R.T @ R - G).max() <= tol * np.abs(G).max() * nj, (k, j)
            Rl = np.linalg.qr(B, mode="r")
            assert np.allclose(np.abs(np.diag(R)), np.abs(np.diag(Rl)), rtol=50 * tol, atol=0)
    for p in pats:
        p.destroy()


CASES = {
    # one structure for the batch: shadow data shared across the maps
    "q1_shared_L2": lambda: (W.config2(nx=20, nmat=3), 2),
    # every map its own structure
    "fem_changing_L2": lambda: (W.config4(ncell=16, nmat=3, flip_frac=0.2), 2),
    "upwind_L2": lambda: (W.config3(nx=8, nmat=2), 2),
}


@pytest.mark.parametrize("precision,steps", [("fp64", 0), ("fp32r", 1), ("fp32r", 2), ("fp32r", "auto")])
@pytest.mark.parametrize("case", sorted(CASES))
def test_replayed_adjoint_equals_recomputing_adjoint(sam, handle, case, precision, steps):
    import torch

    seq, level = CASES[case]()
    aks = [sam.Csr.from_host(m) for m in seq.mats]
    K = len(aks)
    pats = handle.sam_pattern_build_batched(aks, level)
    tape = _tape(torch, handle.sam_factor_tape_bytes(pats, precision))
    handle.sam_set_factor_tape(sam.SAM_TAPE_RECORD, tape)
    try:
        offs, _, _, mv, _ = handle.sam_build_batched(aks, aks[0], pats, precision, steps)
    finally:
        handle.sam_set_factor_tape(sam.SAM_TAPE_OFF)
    offs2, _, _, mv2, _ = handle.sam_build_batched(aks, aks[0], pats, precision, steps)
    assert torch.equal(mv, mv2)  # recording changes nothing in the build
    gbar = torch.randn(mv.numel(), dtype=torch.float64, device="cuda",
                       generator=torch.Generator(device="cuda").manual_seed(2))
    targets = [aks[0]] * K
    dk0, d00 = handle.sam_build_backward_batched(aks, targets, pats, mv, gbar, precision, steps, 0.5, offsets=offs)
    handle.sam_set_factor_tape(sam.SAM_TAPE_REPLAY, tape)
    try:
        dk1, d01 = handle.sam_build_backward_batched(aks, targets, pats, mv, gbar, precision, steps, 0.5,
                                                     offsets=offs)
        # a single map replays its own slots: map 0's come first on the tape
        dk1s, d01s = handle.sam_build_backward(aks[0], aks[0], pats[0], mv[offs[0]:offs[1]], gbar[offs[0]:offs[1]],
                                               precision, steps, 0.5)
    finally:
        handle.sam_set_factor_tape(sam.SAM_TAPE_OFF)
    handle.sam_sync()
    assert torch.equal(dk0, dk1) and torch.equal(d00, d01)
    dk0s, d00s = handle.sam_build_backward(aks[0], aks[0], pats[0], mv[offs[0]:offs[1]], gbar[offs[0]:offs[1]],
                                           precision, steps, 0.5)
    assert torch.equal(dk0s, dk1s) and torch.equal(d00s, d01s)
    for p in pats:
        p.destroy()


def test_tape_errors_leave_the_handle_usable(sam, handle):
    import torch

    seq = W.config2(nx=16, nmat=2)
    aks = [sam.Csr.from_host(m) for m in seq.mats]
    pats = handle.sam_pattern_build_batched(aks, 2)
    nbytes = handle.sam_factor_tape_bytes(pats, "fp32r")
    tape = _tape(torch, nbytes)
    # misaligned, host memory, unknown mode
    with pytest.raises(sam.SamError) as e:
        handle.sam_set_factor_tape(sam.SAM_TAPE_RECORD, tape.view(torch.float32)[1:])
    assert e.value.status == sam.SAM_ERR_INVALID_ARG
    with pytest.raises(sam.SamError) as e:
        handle.sam_set_factor_tape(sam.SAM_TAPE_RECORD, torch.zeros(nbytes // 8 + 2, dtype=torch.float64))
    assert e.value.status == sam.SAM_ERR_INVALID_ARG
    with pytest.raises(sam.SamError) as e:
        handle.sam_set_factor_tape(7, tape)
    assert e.value.status == sam.SAM_ERR_INVALID_ARG
    # a tape one slot too small: the build refuses before its solves
    small = tape[: (nbytes - 16) // 8]
    handle.sam_set_factor_tape(sam.SAM_TAPE_RECORD, small)
    try:
        with pytest.raises(sam.SamError) as e:
            handle.sam_build_batched(aks, aks[0], pats, "fp32r", 1)
        assert e.value.status == sam.SAM_ERR_INVALID_ARG
    finally:
        handle.sam_set_factor_tape(sam.SAM_TAPE_OFF)
    # FP64 factors need twice the bytes
    assert handle.sam_factor_tape_bytes(pats, "fp64") == 2 * nbytes
    offs, _, _, mv, _ = handle.sam_build_batched(aks, aks[0], pats, "fp32r", 1)
    handle.sam_set_factor_tape(sam.SAM_TAPE_REPLAY, small)
    try:
        with pytest.raises(sam.SamError) as e:
            handle.sam_build_backward_batched(aks, [aks[0]] * 2, pats, mv, mv, "fp32r", 1, 0.0, offsets=offs)
        assert e.value.status == sam.SAM_ERR_INVALID_ARG
    finally:
        handle.sam_set_factor_tape(sam.SAM_TAPE_OFF)
    handle.sam_build_backward_batched(aks, [aks[0]] * 2, pats, mv, mv, "fp32r", 1, 0.0, offsets=offs)
    handle.sam_sync()
    for p in pats:
        p.destroy()


def test_autograd_keep_factors_gives_the_same_gradients(sam, handle):
    import torch

    from paper_2406_17656_gb300.autograd import SamMap

    seq = W.config2(nx=16, nmat=2)
    a0, a1 = seq.mats[0], seq.mats[1]
    A1, A0 = sam.Csr.from_host(a1), sam.Csr.from_host(a0)
    S = handle.sam_pattern_build(A1, 2)
    v = torch.randn(a1.n, dtype=torch.float64, device="cuda", generator=torch.Generator(device="cuda").manual_seed(4))
    grads = []
    for keep in (False, True):
        f = SamMap(handle, (A1.indptr, A1.indices), (A0.indptr, A0.indices), S, "fp32r", 1, keep_factors=keep)
        ak = A1.data.clone().requires_grad_(True)
        az = A0.data.clone().requires_grad_(True)
        m = f(ak, az)
        loss = (f.matvec(m, v) ** 2).sum() + f.residual_sq(ak, az, m)
        loss.backward()
        grads.append((ak.grad.clone(), az.grad.clone()))
    assert torch.equal(grads[0][0], grads[1][0]) and torch.equal(grads[0][1], grads[1][1])


def test_zero_pivot_is_reported_through_the_tape(sam, handle):
    """A column of A_k whose stored values are all zero makes the problems
    that gather it rank deficient; the replaying adjoint meets the same zero
    pivots as the recomputing one and reports the same status."""
    import torch

    seq = W.config2(nx=12, nmat=2)
    a = seq.mats[1].to_scipy().tocsc()
    a.data[a.indptr[40]:a.indptr[41]] = 0.0  # stored, numerically zero
    ak = W.CSR.from_scipy(a.tocsr())
    A1, A0 = sam.Csr.from_host(ak), sam.Csr.from_host(seq.mats[0])
    S = handle.sam_pattern_build(A1, 1)
    tape = _tape(torch, handle.sam_factor_tape_bytes([S], "fp32r"))
    st = torch.zeros(ak.n, dtype=torch.int32, device="cuda")
    handle.sam_set_factor_tape(sam.SAM_TAPE_RECORD, tape)
    try:
        _, _, mv = handle.sam_build(A1, A0, S, "fp32r", 1, col_status=st)
        with pytest.raises(sam.SamError) as e:
            handle.sam_sync()
    finally:
        handle.sam_set_factor_tape(sam.SAM_TAPE_OFF)
    assert e.value.status == sam.SAM_ERR_RANK_DEFICIENT
    bad = np.flatnonzero(st.cpu().numpy() != 0)
    assert len(bad) > 0
    statuses = []
    for mode in (None, sam.SAM_TAPE_REPLAY):
        if mode is not None:
            handle.sam_set_factor_tape(mode, tape)
        try:
            with pytest.raises(sam.SamError) as e:
                handle.sam_build_backward(A1, A0, S, mv, mv, "fp32r", 1, 0.0)
                handle.sam_sync()
            statuses.append(e.value.status)
        finally:
            handle.sam_set_factor_tape(sam.SAM_TAPE_OFF)
    assert statuses == [sam.SAM_ERR_RANK_DEFICIENT] * 2


def test_tape_with_large_columns(sam, handle):
    """A level-3 batch mixes register-class columns (the boundary: tape
    slots) and large columns (no slot for more than 27 unknowns; their
    adjoint factors B again in FP64): replaying equals recomputing."""
    import torch

    seq = W.config2(nx=14, nmat=2)
    aks = [sam.Csr.from_host(m) for m in seq.mats]
    pats = handle.sam_pattern_build_batched(aks, 3)
    n = seq.mats[0].n
    sizes = []
    for A in seq.mats:
        cp, _ = oracle.pattern(A, 3)
        sizes += [_slot(int(x)) for x in np.diff(cp)]
    nbytes = handle.sam_factor_tape_bytes(pats, "fp32r")
    assert nbytes == 4 * int(np.sum(sizes))
    assert any(s == 0 for s in sizes) and any(s > 0 for s in sizes)
    tape = _tape(torch, nbytes)
    handle.sam_set_factor_tape(sam.SAM_TAPE_RECORD, tape)
    try:
        offs, _, _, mv, _ = handle.sam_build_batched(aks, aks[0], pats, "fp32r", 1)
    finally:
        handle.sam_set_factor_tape(sam.SAM_TAPE_OFF)
    gbar = torch.randn(mv.numel(), dtype=torch.float64, device="cuda",
                       generator=torch.Generator(device="cuda").manual_seed(6))
    dk0, d00 = handle.sam_build_backward_batched(aks, [aks[0]] * 2, pats, mv, gbar, "fp32r", 1, 0.3, offsets=offs)
    handle.sam_set_factor_tape(sam.SAM_TAPE_REPLAY, tape)
    try:
        dk1, d01 = handle.sam_build_backward_batched(aks, [aks[0]] * 2, pats, mv, gbar, "fp32r", 1, 0.3,
                                                     offsets=offs)
    finally:
        handle.sam_set_factor_tape(sam.SAM_TAPE_OFF)
    handle.sam_sync()
    assert torch.equal(dk0, dk1) and torch.equal(d00, d01)
    assert n == aks[0].n
    for p in pats:
        p.destroy()
