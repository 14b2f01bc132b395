"""The captured build (sam_plan_*): a replay gives, bit for bit, what the
direct batched call gives, re-reads the source values on every replay, and
rejects what it cannot capture."""
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


@pytest.mark.parametrize("precision,steps", [("fp32r", 1), ("fp32r", 2), ("fp64", 0)])
@pytest.mark.parametrize("level", [1, 2])
def test_replay_equals_direct_build(sam, handle, precision, steps, level):
    import torch

    seq = W.config2(nx=40, nmat=4, level=level)
    a0 = sam.Csr.from_host(seq.mats[0])
    aks = [sam.Csr.from_host(m) for m in seq.mats]
    Ss = handle.sam_pattern_build_batched(aks, level)
    plan = handle.sam_plan_create(aks, a0, Ss, precision, steps, want_status=True, want_res2=True)
    assert plan.launches() > 0
    for _ in range(2):
        plan.execute()
    st = torch.empty_like(plan.col_status)
    r2 = torch.empty_like(plan.res2)
    offs, rp, ci, v, fro = handle.sam_build_batched(aks, a0, Ss, precision, steps, col_status=st, res2=r2,
                                                    want_fro=True)
    handle.sam_sync()
    assert torch.equal(plan.M_row_ptr, rp) and torch.equal(plan.M_col_idx, ci)
    assert torch.equal(plan.M_val, v)
    assert torch.equal(plan.col_status, st) and torch.equal(plan.res2, r2)
    f2 = plan.fro2.cpu().numpy()
    assert np.allclose(np.sqrt(f2), fro, rtol=1e-15, atol=0)


def test_replay_reads_new_values(sam, handle):
    """Values changed in place between replays (same structure) give the map
    of the new values; per-map targets; patterns destroyed after capture."""
    import torch

    pairs = [W.config5_pair(b, nx=24) for b in range(3)]
    A0s = [sam.Csr.from_host(p[0]) for p in pairs]
    A1s = [sam.Csr.from_host(p[1]) for p in pairs]
    Ss = handle.sam_pattern_build_batched(A1s, 2)
    plan = handle.sam_plan_create(A1s, A0s, Ss, "fp32r", 1)
    cps = [(S.colptr().cpu().numpy(), S.rowidx().cpu().numpy()) for S in Ss]
    for S in Ss:
        S.destroy()
    gen = torch.Generator("cuda").manual_seed(5)
    n = pairs[0][0].n
    for rnd in range(2):
        for a in A1s + A0s:  # new values, same structure (stays diagonally dominant: positive scaling)
            a.data.mul_(1.0 + 0.2 * torch.rand(a.data.shape, dtype=torch.float64, device="cuda", generator=gen))
        plan.execute()
        handle.sam_sync()
        v = plan.M_val.cpu().numpy()
        ci = plan.M_col_idx.cpu().numpy()
        rp = plan.M_row_ptr.cpu().numpy()
        for k in range(3):
            ak = W.CSR(n, A1s[k].indptr.cpu().numpy(), A1s[k].indices.cpu().numpy(), A1s[k].data.cpu().numpy())
            az = W.CSR(n, A0s[k].indptr.cpu().numpy(), A0s[k].indices.cpu().numpy(), A0s[k].data.cpu().numpy())
            cp, ri = cps[k]
            ref = oracle.build(ak, az, cp, ri)
            _, ix, dv = oracle.to_csr(n, cp, ri, ref["mval"])
            sl = slice(plan.offsets[k], plan.offsets[k + 1])
            assert np.array_equal(ci[sl], ix)
            assert np.linalg.norm(v[sl] - dv) <= 1e-10 * np.linalg.norm(dv)
            assert abs(plan.fro2[k].item() - (ref["res2"] + ref["out2"]).sum()) <= 1e-9 * (ref["res2"] + ref["out2"]).sum()
    plan.destroy()


def test_launch_counter_advances_per_replay(sam, handle):
    seq = W.config2(nx=20, nmat=2, level=1)
    a0 = sam.Csr.from_host(seq.mats[0])
    aks = [sam.Csr.from_host(m) for m in seq.mats]
    Ss = handle.sam_pattern_build_batched(aks, 1)
    plan = handle.sam_plan_create(aks, a0, Ss, "fp32r", 1)
    handle.sam_profile(True)
    plan.execute()
    plan.execute()
    launches, _, _ = handle.sam_profile_read()
    handle.sam_profile(False)
    assert launches == 2 * plan.launches()
    plan.destroy()


def test_host_arrays_are_rejected(sam, handle):
    seq = W.config1()
    a0, a1 = seq.mats
    h0, h1 = sam.Csr.from_host(a0, device="cpu"), sam.Csr.from_host(a1, device="cpu")
    S = handle.sam_pattern_build(sam.Csr.from_host(a1), 1)
    with pytest.raises(sam.SamError):
        handle.sam_plan_create([h1], h0, [S], "fp32r", 1)
