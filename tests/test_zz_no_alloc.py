"""sam_residual_static, the entry point for callers that cannot allocate
device memory (its workspace is a fixed file-scope device array), against
the oracle's residual and sam_residual, the handle-based entry point that
allocates from a memory pool.  Collected last on purpose: it must pass on
its own in a fresh process and after every other test."""
import numpy as np
import pytest

import oracle
from paper_2406_17656_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the tolerance of the residual parity tests


def _setup():
    import torch  # noqa: F401

    from paper_2406_17656_gb300 import build, sam

    build.build()
    return sam


def _map_case():
    """A P1 FEM pair with a changing pattern, the oracle's level-1 map of it,
    and the oracle's residual of that map."""
    seq = W.config4(ncell=40, nmat=4, flip_frac=0.1)
    a0, ak = seq.mats[0], seq.mats[3]
    cp, ri = oracle.pattern(ak, 1)
    fwd = oracle.build(ak, a0, cp, ri)
    fro_orc, rel_orc = oracle.residual(ak, cp, ri, fwd["mval"], a0)
    ip, ix, dv = oracle.to_csr(ak.n, cp, ri, fwd["mval"])
    return a0, ak, W.CSR(ak.n, ip, ix, dv), fro_orc, rel_orc


def _call(sam, A_k, M, A_0):
    import torch

    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    sam.sam_residual_static(A_k, M, A_0, out, status)
    torch.cuda.synchronize()
    return out.cpu().numpy(), int(status.item())


def test_static_residual_equals_oracle_and_pooled_residual_twice():
    sam = _setup()
    a0, ak, mh, fro_orc, rel_orc = _map_case()
    A_k, A_0, M = sam.Csr.from_host(ak), sam.Csr.from_host(a0), sam.Csr.from_host(mh)
    with sam.Handle() as h:
        fro_ref, rel_ref = h.sam_residual(A_k, M, A_0)
    for _ in range(2):  # the second call reuses the same workspace
        (fro, rel), st = _call(sam, A_k, M, A_0)
        assert st == 0
        assert abs(fro - fro_ref) <= TOL * fro_ref
        assert abs(rel - rel_ref) <= TOL * rel_ref
        assert abs(fro - fro_orc) <= TOL * fro_orc
        assert abs(rel - rel_orc) <= TOL * rel_orc


def test_static_residual_rejects_oversized_empty_and_host_inputs():
    import torch

    sam = _setup()
    big = sam.SAM_STATIC_MAX_ROWS + 1
    rp = torch.zeros(big + 1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    v = torch.zeros(1, dtype=torch.float64, device="cuda")
    A = sam.Csr(rp, ci[:0], v[:0], n=big)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(sam.SamError) as e:
        sam.sam_residual_static(A, A, A, out)
    assert e.value.status == sam.SAM_ERR_INVALID_ARG
    E = sam.Csr(rp[:1], ci[:0], v[:0], n=0)  # an empty matrix, as for every other call
    with pytest.raises(sam.SamError) as e:
        sam.sam_residual_static(E, E, E, out)
    assert e.value.status == sam.SAM_ERR_INVALID_ARG
    a = W.config1().mats[0]
    H = sam.Csr(a.indptr, a.indices, a.data)  # host arrays cannot be staged without allocating
    with pytest.raises(sam.SamError) as e:
        sam.sam_residual_static(H, H, H, out)
    assert e.value.status == sam.SAM_ERR_INVALID_ARG


def test_static_residual_device_errors_then_recovers():
    """Malformed structures the host cannot see are caught by the validation
    kernel (status word + NaN outputs, nothing read out of bounds); an
    oversized row of R is reported as unsupported; the next valid call
    clears the status word and matches sam_residual."""
    import torch

    sam = _setup()
    a0, ak, mh, fro_orc, _ = _map_case()
    A_k, A_0, M = sam.Csr.from_host(ak), sam.Csr.from_host(a0), sam.Csr.from_host(mh)
    # row_ptr[n] one short of nnz: every row stays inside the arrays
    rp_bad = A_k.indptr.clone()
    rp_bad[-1] -= 1
    (fro, rel), st = _call(sam, sam.Csr(rp_bad, A_k.indices, A_k.data, n=ak.n), M, A_0)
    assert st == sam.SAM_ERR_BAD_CSR
    assert np.isnan(fro) and np.isnan(rel)
    # two column indices of one row swapped (unsorted): caught the same way
    ci_bad = M.indices.clone()
    r = int(np.argmax(np.diff(mh.indptr) >= 2))
    p = int(mh.indptr[r])
    ci_bad[p], ci_bad[p + 1] = M.indices[p + 1], M.indices[p]
    (fro, rel), st = _call(sam, A_k, sam.Csr(M.indptr, ci_bad, M.data, n=ak.n), A_0)
    assert st == sam.SAM_ERR_BAD_CSR
    assert np.isnan(fro) and np.isnan(rel)
    (fro, rel), st = _call(sam, A_k, M, A_0)
    assert st == 0 and abs(fro - fro_orc) <= TOL * fro_orc
    # a valid input whose row 0 of R has 40 x 40 = 1600 candidate entries
    n = 48
    d = np.zeros((n, n))
    d[0, :40] = 1.0 + np.arange(40) / 64.0
    d[np.arange(n), np.arange(n)] += 4.0
    m = np.eye(n)
    m[:40, :40] += 0.01
    import scipy.sparse as sp

    def dev(x):
        c = sp.csr_matrix(x)
        return sam.Csr.from_host(W.CSR(n, c.indptr.astype(np.int32), c.indices.astype(np.int32), c.data))

    (fro, rel), st = _call(sam, dev(d), dev(m), dev(d))
    assert st == sam.SAM_ERR_UNSUPPORTED
    assert np.isnan(fro) and np.isnan(rel)
    (fro, rel), st = _call(sam, A_k, M, A_0)
    assert st == 0 and abs(fro - fro_orc) <= TOL * fro_orc


def test_static_residual_rejects_arrays_of_another_device():
    import torch

    if torch.cuda.device_count() < 2:
        pytest.skip("one visible GPU")
    sam = _setup()
    a0, ak, mh, _, _ = _map_case()
    torch.cuda.set_device(0)
    A_k, A_0 = sam.Csr.from_host(ak, "cuda:0"), sam.Csr.from_host(a0, "cuda:0")
    M1 = sam.Csr.from_host(mh, "cuda:1")  # checked on the host: nothing is launched with it
    out = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    with pytest.raises(sam.SamError) as e:
        sam.sam_residual_static(A_k, M1, A_0, out)
    assert e.value.status == sam.SAM_ERR_INVALID_ARG
