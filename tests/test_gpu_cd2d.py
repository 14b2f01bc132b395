"""The CD2D stand-in (Sec. 5.1, 66 Jacobians, n = 4096) through the GPU path:
sparsification of every source, the square and cube of S(A~) as map
patterns, and all 66 maps onto A_0 in one batched build, against the oracle
(patterns and map structure bit-exact, values within 1e-10 relative
Frobenius), with the value-dependent pattern counts of Tables 1-2 on every
matrix."""
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
def seq():
    return W.cd2d()


def test_table_counts_on_every_matrix(sam, seq):
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            side, mode, param, power, nnz = line.split()
            rows.append((mode, float(param), int(power), int(nnz)))
    with sam.Handle() as h:
        for a in seq.mats:
            A = sam.Csr.from_host(a)
            for mode, param, power, nnz in rows:
                assert h.sam_pattern_build(h.sam_sparsify(A, mode, param), power).nnz == nnz


@pytest.mark.parametrize("mode,param,power", [("tau", 0.8, 2), ("lfil", 3, 2), ("lfil", 5, 3)])
def test_all_maps_on_sparsified_patterns(sam, seq, mode, param, power):
    mats = seq.mats
    n, K = mats[0].n, len(mats)
    with sam.Handle() as h:
        aks = [sam.Csr.from_host(a) for a in mats]
        pats = [h.sam_pattern_build(h.sam_sparsify(a, mode, param), power) for a in aks]
        offs, rp, ci, mv, fro = h.sam_build_batched(aks, aks[0], pats, "fp32r", 1, want_fro=True)
        rp, ci, mv = rp.cpu().numpy(), ci.cpu().numpy(), mv.cpu().numpy()
    nrm0 = np.linalg.norm(mats[0].data)
    for k in (1, 4, 9, 29, 44, 65):
        ip, ix, dv = oracle.sparsify(mats[k], mode, param)
        cp, ri = oracle.pattern(W.CSR(n, ip, ix, dv), power)
        ref = oracle.build(mats[k], mats[0], cp, ri)
        rip, rix, rdv = oracle.to_csr(n, cp, ri, ref["mval"])
        assert np.array_equal(rp[k * (n + 1):(k + 1) * (n + 1)], rip)
        assert np.array_equal(ci[offs[k]:offs[k + 1]], rix)
        got = mv[offs[k]:offs[k + 1]]
        assert np.linalg.norm(got - rdv) <= 1e-10 * np.linalg.norm(rdv)
        rel_ref = np.sqrt(np.sum(ref["res2"] + ref["out2"])) / nrm0
        assert fro[k] / nrm0 == pytest.approx(rel_ref, rel=1e-8, abs=1e-14)
