"""Tile variants and the autotuner: every FP32 tile shape meets the same
parity bar against the oracle, sam_tune keeps a valid choice per size class,
and its cache file round-trips."""
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CASES = {
    # level-2 patterns put columns in every size class
    "q1_40_L2": lambda: (W.config2(nx=40, nmat=3), 2),
    "upwind7_11_L2": lambda: (W.config3(nx=11, nmat=3), 2),
    "fem_36_L2": lambda: (W.config4(ncell=36, nmat=3, flip_frac=0.05), 2),
}


@pytest.mark.parametrize("variants", [[0, 1, 1, 1, 1, 0], [0, 1, 0, 1, 0, 0], [0, 0, 1, 0, 1, 0]])
@pytest.mark.parametrize("case", sorted(CASES))
def test_every_variant_matches_oracle(sam, case, variants):
    seq, level = CASES[case]()
    A0 = seq.mats[0]
    h = sam.Handle()
    try:
        h.sam_set_tile_variants(variants)
        assert h.sam_get_tile_variants() == variants
        Aks = [sam.Csr.from_host(m) for m in seq.mats[1:]]
        Ss = h.sam_pattern_build_batched(Aks, level)
        offs, rp, ci, v, _ = h.sam_build_batched(Aks, sam.Csr.from_host(A0), Ss, "fp32r", 1)
        n = A0.n
        rp, ci, v = rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy()
        for k, Ak in enumerate(seq.mats[1:]):
            cp, ri = oracle.pattern(Ak, level)
            ref = oracle.build(Ak, A0, cp, ri)
            ip, ix, dv = oracle.to_csr(n, cp, ri, ref["mval"])
            assert np.array_equal(rp[k * (n + 1):(k + 1) * (n + 1)], ip)
            assert np.array_equal(ci[offs[k]:offs[k + 1]], ix)
            assert _rel(v[offs[k]:offs[k + 1]], dv) <= 1e-10
    finally:
        h.close()


def test_out_of_range_variants_are_rejected(sam):
    h = sam.Handle()
    try:
        for bad in ([1, 0, 0, 0, 0, 0], [0, 2, 0, 0, 0, 0], [0, 0, 0, 0, -1, 0], [0, 0, 0, 0, 0, 1]):
            with pytest.raises(sam.SamError):
                h.sam_set_tile_variants(bad)
        assert h.sam_get_tile_variants() == [0] * 6
    finally:
        h.close()


def test_tune_chooses_valid_variants_and_caches_them(sam, tmp_path):
    seq = W.config2(nx=48, nmat=3, level=2)
    A0 = sam.Csr.from_host(seq.mats[0])
    Aks = [sam.Csr.from_host(m) for m in seq.mats]
    cache = str(tmp_path / "tune.txt")
    h = sam.Handle()
    try:
        Ss = h.sam_pattern_build_batched(Aks, 2)
        h.sam_profile(True)
        chosen = h.sam_tune(Aks, A0, Ss, "fp32r", 1, cache_path=cache)
        assert chosen[0] == 0 and all(c in (0, 1) for c in chosen)
        # the tuner leaves the caller's tracing counters alone
        launches, _, per_bin = h.sam_profile_read()
        assert launches == 0 and per_bin == [0] * 6
        lines = open(cache).read().splitlines()
        sched = h.sam_get_bin_schedule()
        assert len(lines) == 1 and lines[0].split()[-12:-6] == [str(c) for c in chosen]
        assert lines[0].split()[-6:] == [str(c) for c in sched]
        # the key holds the histogram of natural size classes
        assert sum(1 for t in lines[0].split() if t.startswith("h")) == 6
        assert all(b <= t <= 4 for b, t in enumerate(sched[:5])) and sched[5] == 5
        # the build after tuning still meets the parity bar
        offs, _, _, v, _ = h.sam_build_batched(Aks, A0, Ss, "fp32r", 1)
        v = v.cpu().numpy()
        cp, ri = oracle.pattern(seq.mats[1], 2)
        ref = oracle.build(seq.mats[1], seq.mats[0], cp, ri)
        _, _, dv = oracle.to_csr(seq.mats[0].n, cp, ri, ref["mval"])
        assert _rel(v[offs[1]:offs[2]], dv) <= 1e-10
    finally:
        h.close()
    # a new handle finds the family in the cache: same choice, no new line
    h2 = sam.Handle()
    try:
        Ss = h2.sam_pattern_build_batched(Aks, 2)
        assert h2.sam_tune(Aks, A0, Ss, "fp32r", 1, cache_path=cache) == chosen
        assert h2.sam_get_bin_schedule() == sched
        assert len(open(cache).read().splitlines()) == 1
        # a family of the same sizes but other column sizes (level 1 instead
        # of level 2: a different histogram) gets its own line
        Ss1 = h2.sam_pattern_build_batched(Aks, 1)
        h2.sam_tune(Aks, A0, Ss1, "fp32r", 1, cache_path=cache)
        keys = [" ".join(l.split()[:-12]) for l in open(cache).read().splitlines()]
        assert len(keys) == 2 and keys[0] != keys[1]
        # FP64 has a single shape: nothing changes
        h2.sam_set_tile_variants([0] * 6)
        assert h2.sam_tune(Aks, A0, Ss, "fp64", 0) == [0] * 6
    finally:
        h2.close()


SCHEDULES = [[0, 1, 2, 3, 4, 5], [1, 1, 3, 3, 4, 5], [3, 3, 3, 3, 4, 5], [4, 4, 4, 4, 4, 5]]


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("case", sorted(CASES))
def test_every_bin_schedule_matches_oracle(sam, case, schedule):
    """Columns handed to a larger register tile by the bin schedule give the
    same maps within the bar, column by column."""
    import colcheck

    seq, level = CASES[case]()
    A0 = seq.mats[0]
    h = sam.Handle()
    try:
        h.sam_set_bin_schedule(schedule)
        assert h.sam_get_bin_schedule() == schedule
        Aks = [sam.Csr.from_host(m) for m in seq.mats[1:]]
        Ss = h.sam_pattern_build_batched(Aks, level)
        offs, rp, ci, v, _ = h.sam_build_batched(Aks, sam.Csr.from_host(A0), Ss, "fp32r", 1)
        n = A0.n
        rp, ci, v = rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy()
        for k, Ak in enumerate(seq.mats[1:]):
            cp, ri = oracle.pattern(Ak, level)
            ref = oracle.build(Ak, A0, cp, ri)
            got = colcheck.csr_to_csc_values(n, rp[k * (n + 1):(k + 1) * (n + 1)], ci[offs[k]:offs[k + 1]],
                                             v[offs[k]:offs[k + 1]], cp, ri)
            colcheck.assert_columns(cp, got, ref["mval"], "fp32r", what="map %d" % k)
    finally:
        h.close()


def test_bad_bin_schedules_are_rejected(sam):
    h = sam.Handle()
    try:
        for bad in ([1, 0, 2, 3, 4, 5], [0, 1, 2, 3, 5, 5], [0, 1, 2, 3, 4, 4], [0, 1, 2, 2, 4, 5], [0, 1, 2, 3, 4]):
            with pytest.raises(sam.SamError):
                h.sam_set_bin_schedule(bad)
        assert h.sam_get_bin_schedule() == [0, 1, 2, 3, 4, 5]
    finally:
        h.close()
