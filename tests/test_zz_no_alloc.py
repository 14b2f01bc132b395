"""sam_residual_static, the entry point for callers that cannot allocate
device memory (its workspace is a fixed file-scope device array), against
sam_residual, the handle-based entry point that allocates from a memory
pool.  Collected last on purpose: it must pass on its own in a fresh process
and after every other test."""
import numpy as np
import pytest

import oracle
from paper_2406_17656_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_static_residual_equals_pooled_residual_twice():
    import torch

    from paper_2406_17656_gb300 import build, sam

    build.build()
    seq = W.config4(ncell=40, nmat=4, flip_frac=0.1)
    a0, ak = seq.mats[0], seq.mats[3]
    cp, ri = oracle.pattern(ak, 1)
    fwd = oracle.build(ak, a0, cp, ri)
    ip, ix, dv = oracle.to_csr(ak.n, cp, ri, fwd["mval"])
    A_k, A_0 = sam.Csr.from_host(ak), sam.Csr.from_host(a0)
    M = sam.Csr.from_host(W.CSR(ak.n, ip, ix, dv))
    with sam.Handle() as h:
        fro_ref, rel_ref = h.sam_residual(A_k, M, A_0)
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for _ in range(2):  # the second call reuses the same workspace
        out.fill_(-1.0)
        status.fill_(-1)
        sam.sam_residual_static(A_k, M, A_0, out, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        fro, rel = out.cpu().numpy()
        assert abs(fro - fro_ref) <= 1e-12 * fro_ref  # the tolerance of the residual parity test
        assert abs(rel - rel_ref) <= 1e-12 * rel_ref


def test_static_residual_rejects_oversized_and_host_inputs():
    import torch

    from paper_2406_17656_gb300 import build, sam

    build.build()
    big = sam.SAM_STATIC_MAX_ROWS + 1
    rp = torch.zeros(big + 1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    v = torch.zeros(1, dtype=torch.float64, device="cuda")
    A = sam.Csr(rp, ci[:0], v[:0], n=big)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(sam.SamError) as e:
        sam.sam_residual_static(A, A, A, out)
    assert e.value.status == sam.SAM_ERR_INVALID_ARG
    a = W.config1().mats[0]
    H = sam.Csr(a.indptr, a.indices, a.data)  # host arrays cannot be staged without allocating
    with pytest.raises(sam.SamError) as e:
        sam.sam_residual_static(H, H, H, out)
    assert e.value.status == sam.SAM_ERR_INVALID_ARG
