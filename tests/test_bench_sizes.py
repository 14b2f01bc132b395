"""The column sizes behind the benchmark's roofline figures.

bench.py derives |J_j| (pattern), |I_j| (shadow rows) and nnz(B_j) (stored
entries of A_k(I_j, J_j)) from sparse matrix products; here they are checked
against the oracle's explicit pattern and shadow sets, and the algorithmic
FP32 flop count against the closed form of Householder QR + Q^T c + back
solve + correction solves for a dense column problem."""
import numpy as np
import pytest

import bench
import oracle
from paper_2406_17656_gb300 import workloads as W

CASES = {"q1_20_L2": (lambda: W.config2(nx=20, nmat=2).mats[1], 2),
         "poisson5_16_L3": (lambda: W.config1(nx=16).mats[1], 3),
         "fem_12_L2": (lambda: W.config4(ncell=12, nmat=2, flip_frac=0.3).mats[1], 2),
         "upwind_6_L1": (lambda: W.config3(nx=6, nmat=2).mats[1], 1)}


@pytest.mark.parametrize("case", sorted(CASES))
def test_column_sizes_match_the_oracle_sets(case):
    make, level = CASES[case]
    A = make()
    I, J, nB = bench.column_sizes([A], level)[0]
    cp, ri = oracle.pattern(A, level)
    icp, iri = oracle.shadow(A, cp, ri)
    assert np.array_equal(J, np.diff(cp))
    assert np.array_equal(I, np.diff(icp))
    # nnz(B_j): stored entries of A in the rows I_j and the columns J_j
    csc = A.to_scipy().tocsc()
    want = np.array([sum(csc.indptr[c + 1] - csc.indptr[c] for c in ri[cp[j]:cp[j + 1]]) for j in range(A.n)])
    assert np.array_equal(nB, want)


def test_algorithmic_flops_closed_form():
    I, J, nB = np.array([49, 10]), np.array([25, 4]), np.array([222, 30])
    f32, f64 = bench.algorithmic_flops(I, J, nB, "fp32r", 1)
    m, n = I.astype(float), J.astype(float)
    qr = 2 * n * n * (m - n / 3) + 4 * m * n - 2 * n * n + n * n
    assert np.allclose(f32, qr + (4 * m * n - n * n))
    assert np.allclose(f64, 2 * nB + m)
    f32_0, f64_0 = bench.algorithmic_flops(I, J, nB, "fp64", 0)
    assert np.allclose(f64_0, qr) and np.allclose(f32_0, 0)


def test_bench_size_classes_are_the_librarys():
    """bench.py's roofline selects the columns of a size class by the
    library's own limits (no copy of the kernel's constants)."""
    from paper_2406_17656_gb300 import build, sam

    build.build()
    c = sam.size_classes()
    assert bench.size_classes() == c
    assert len(c["max_rows"]) == sam.SAM_NUM_SIZE_CLASSES
    # every class boundary: a column just inside goes to that class (or an
    # earlier one), just outside to a later one
    for q in range(sam.SAM_NUM_SIZE_CLASSES):
        I = np.array([c["max_rows"][q]])
        J = np.array([min(c["max_cols"][q], c["max_tile"][q] // c["max_rows"][q] - 1)])
        nB = np.array([min(c["max_entries"][q], int(I[0]) * int(J[0]))])
        assert 0 <= bench.bin_of(I, J, nB, c)[0] <= q
    I, J = np.array([c["max_rows"][-1] + 1]), np.array([2])
    assert bench.bin_of(I, J, np.array([8]), c)[0] == -1
    rows, cols = np.zeros(1, np.int32), np.zeros(1, np.int32)
    sam.load().sam_limits(rows.ctypes.data_as(sam._i32p), cols.ctypes.data_as(sam._i32p))
    assert rows[0] == c["max_rows"][-1] and cols[0] == c["max_cols"][-1]


def test_adjoint_flops_with_a_factor_tape_drop_only_the_qr():
    """The adjoint's algorithmic work with R from a factor tape is the
    recomputing adjoint's minus the forward's QR of [B c] (the same FP64
    work), for every step count."""
    I = np.array([49, 81, 25], dtype=np.int64)
    J = np.array([25, 49, 9], dtype=np.int64)
    nB = np.array([225, 441, 81], dtype=np.int64)
    m, n = I.astype(float), J.astype(float)
    qr = 2 * n * n * (m - n / 3) + (4 * m * n - 2 * n * n) + n * n
    for steps in (0, 1, 2):
        f32r, f64r = bench.adjoint_algorithmic_flops(I, J, nB, steps)
        f32t, f64t = bench.adjoint_algorithmic_flops(I, J, nB, steps, tape=True)
        assert np.allclose(f32r - f32t, qr)
        assert np.array_equal(f64r, f64t)


def test_kernel_hash_covers_code_not_comments():
    """The recorded ncu traffic is tied to the kernel's code: comments and
    blank lines do not change the hash, code and string literals do."""
    src = b'int a; // note\n/* block\n   comment */\nconst char *s = "x // kept";\n\n  int b;  \n'
    assert bench._code_only(src) == b'int a;\nconst char *s = "x // kept";\n  int b;'
    assert bench._code_only(src.replace(b"note", b"other note")) == bench._code_only(src)
    assert bench._code_only(src.replace(b"int b", b"int c")) != bench._code_only(src)
    assert len(bench.kernel_hash()) == 64
