"""Pins for the FP64 CPU oracle: each check compares the oracle against
something other than itself -- numbers printed in the paper, closed forms,
brute force on tiny graphs, LAPACK least squares, exact recovery and dense
residuals.  A plausible mistake in the oracle (a transposed operand, a
dropped term, a wrong index, a wrong sign in a reflector) fails at least one
of these.  CPU only."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2406_17656_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line)
    return out


def _paper_example():
    rows = _golden_rows("paper_example_n7.txt")
    i0, i1 = rows.index("A_0"), rows.index("A_1")
    a0 = np.array([[int(x) for x in r.split()] for r in rows[i0 + 1: i1]])
    a1 = np.array([[int(x) for x in r.split()] for r in rows[i1 + 1:]])
    return a0, a1


def _cols(colptr, rowidx):
    return [rowidx[colptr[j]: colptr[j + 1]] for j in range(len(colptr) - 1)]


def _reach(adj, level):
    """Brute force: reach[i, j] iff a directed path i -> ... -> j with at most
    `level` edges exists (edge i->j iff adj[i, j])."""
    n = adj.shape[0]
    step = (adj.astype(np.int64) + np.eye(n, dtype=np.int64)) > 0
    r = np.eye(n, dtype=bool)
    for _ in range(level):
        r = (r.astype(np.int64) @ step.astype(np.int64)) > 0
    return r


def _random_csr(n, density, seed, symmetric=False):
    rng = np.random.default_rng(seed)
    p = rng.random((n, n)) < density
    if symmetric:
        p = p | p.T
    a = np.where(p, rng.uniform(0.5, 1.5, (n, n)) * rng.choice([-1.0, 1.0], (n, n)), 0.0)
    np.fill_diagonal(a, 0.0)
    np.fill_diagonal(a, np.abs(a).sum(1) + 1.0)
    return W.CSR.from_dense(a)


# ------------------------------------------------------------- patterns


@pytest.mark.parametrize("line", _golden_rows("cd2d_pattern_nnz.txt"))
def test_pattern_counts_printed_in_paper(line):
    side, power, nnz = (int(x) for x in line.split())
    a = W.poisson5(side)
    cp, ri = oracle.pattern(a, power)
    assert int(cp[-1]) == nnz


def test_pattern_counts_closed_forms():
    nx = 20
    # 5-point: n rows of 5 minus the 4 missing couplings along each side
    cp, _ = oracle.pattern(W.poisson5(nx), 1)
    assert cp[-1] == 5 * nx * nx - 4 * nx
    # 9-point and its square: every offset (dx, dy) in [-r, r]^2 is present
    # (nx-|dx|)(nx-|dy|) times, so the count is (sum_d (nx-|d|))^2
    kap = np.ones((nx + 1, nx + 1))
    a9 = W.q1_diffusion(kap)
    for level, r in ((1, 1), (2, 2), (3, 3)):
        cp, _ = oracle.pattern(a9, level)
        assert cp[-1] == sum(nx - abs(d) for d in range(-r, r + 1)) ** 2
    # 7-point 3-D: offsets with |dx|+|dy|+|dz| <= level
    m = 6
    a7 = W.upwind7(m, 30.0, np.array([1.0, 0.5, 0.25]))
    for level in (1, 2):
        cp, _ = oracle.pattern(a7, level)
        want = 0
        for dx in range(-level, level + 1):
            for dy in range(-level, level + 1):
                for dz in range(-level, level + 1):
                    if abs(dx) + abs(dy) + abs(dz) <= level:
                        want += (m - abs(dx)) * (m - abs(dy)) * (m - abs(dz))
        assert cp[-1] == want


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_pattern_brute_force_nonsymmetric(seed, level):
    n = 14
    a = _random_csr(n, 0.12, seed)
    adj = a.dense() != 0
    np.fill_diagonal(adj, False)
    reach = _reach(adj, level)
    cp, ri = oracle.pattern(a, level)
    for j, col in enumerate(_cols(cp, ri)):
        assert list(col) == list(np.nonzero(reach[:, j])[0])


def test_pattern_symmetric_input_gives_symmetric_pattern():
    a = _random_csr(30, 0.08, 7, symmetric=True)
    for level in (1, 2):
        cp, ri = oracle.pattern(a, level)
        s = sp.csc_matrix((np.ones(len(ri)), ri, cp), shape=(a.n, a.n)).toarray()
        assert np.array_equal(s, s.T)


def test_shadow_rows_brute_force():
    a = _random_csr(16, 0.15, 3)
    adj = a.dense() != 0
    for level in (1, 2):
        cp, ri = oracle.pattern(a, level)
        icp, iri = oracle.shadow(a, cp, ri)
        for j, col in enumerate(_cols(cp, ri)):
            want = np.nonzero(adj[:, col].any(1))[0]
            assert list(iri[icp[j]: icp[j + 1]]) == list(want)


# -------------------------------------------- paper's worked example (Sec. 3)


def test_paper_example_closure_equals_exact_map_pattern():
    b0, b1 = _paper_example()
    assert np.all(b1 >= b0)  # the subset property (Eq. (property)) holds
    rng = np.random.default_rng(11)
    a0 = np.where(b0 > 0, rng.uniform(1.0, 2.0, b0.shape), 0.0)
    a1 = np.where(b1 > 0, rng.uniform(1.0, 2.0, b1.shape), 0.0)
    A1 = W.CSR.from_dense(a1)
    cp, ri = oracle.pattern(A1, 6)  # n-1 steps reach the transitive closure
    closure = sp.csc_matrix((np.ones(len(ri)), ri, cp), shape=(7, 7)).toarray() > 0
    inv = np.linalg.inv(a1)
    exact = inv @ a0
    tol = 1e-12 * np.abs(exact).max()
    assert np.array_equal(np.abs(inv) > tol, closure)
    assert np.array_equal(np.abs(exact) > tol, closure)
    # The full pattern makes the SAM the exact map with a zero residual.
    out = oracle.build(A1, W.CSR.from_dense(a0), cp, ri)
    m = sp.csc_matrix((out["mval"], ri, cp), shape=(7, 7)).toarray()
    assert np.allclose(m, exact, rtol=0, atol=1e-13 * np.abs(exact).max())
    assert np.sum(out["res2"] + out["out2"]) < 1e-26


@pytest.mark.parametrize("seed", range(8))
def test_subset_property_exact_map_inside_closure(seed):
    """Sec. 3: under S(A_0) in S(A_k), S(A_k^{-1} A_0) lies inside G*(A_k)."""
    A0, A1 = W.random_nested_pair(9, 0.15, seed)
    cp, ri = oracle.pattern(A1, 8)
    closure = sp.csc_matrix((np.ones(len(ri)), ri, cp), shape=(9, 9)).toarray() > 0
    exact = np.linalg.solve(A1.dense(), A0.dense())
    big = np.abs(exact) > 1e-12 * np.abs(exact).max()
    assert not np.any(big & ~closure)


# ---------------------------------------------------- least-squares solve


def _map_dense(n, cp, ri, mval):
    return sp.csc_matrix((mval, ri, cp), shape=(n, n)).toarray()


@pytest.mark.parametrize("level", [1, 2])
def test_identity_when_source_equals_target(level):
    a = W.config2(nx=12, nmat=1).mats[0]
    cp, ri = oracle.pattern(a, level)
    out = oracle.build(a, a, cp, ri)
    m = _map_dense(a.n, cp, ri, out["mval"])
    assert np.abs(m - np.eye(a.n)).max() < 1e-13
    assert np.sqrt(np.sum(out["res2"] + out["out2"])) < 1e-12


def test_exact_recovery_of_a_map_inside_the_pattern():
    seq = W.config3(nx=5, nmat=3)
    ak = seq.mats[2]
    cp, ri = oracle.pattern(ak, 1)
    rng = np.random.default_rng(5)
    n_true = sp.csc_matrix((rng.uniform(-1, 1, len(ri)), ri, cp), shape=(ak.n, ak.n))
    a0 = W.CSR.from_scipy(ak.to_scipy() @ n_true)
    out = oracle.build(ak, a0, cp, ri)
    m = _map_dense(ak.n, cp, ri, out["mval"])
    assert np.abs(m - n_true.toarray()).max() < 1e-12
    assert np.sqrt(np.sum(out["res2"] + out["out2"])) < 1e-11


def test_full_pattern_gives_dense_exact_map():
    A0, A1 = W.random_nested_pair(10, 0.2, 42)
    cp = np.arange(0, 101, 10, dtype=np.int32)
    ri = np.tile(np.arange(10, dtype=np.int32), 10)
    out = oracle.build(A1, A0, cp, ri)
    m = _map_dense(10, cp, ri, out["mval"])
    exact = np.linalg.solve(A1.dense(), A0.dense())
    assert np.abs(m - exact).max() < 1e-13 * np.abs(exact).max()


def _ls_problems(ak, a0, cp, ri):
    akc, a0c = ak.to_scipy().tocsc(), a0.to_scipy().tocsc()
    for j in range(ak.n):
        J = ri[cp[j]: cp[j + 1]]
        sub = akc[:, J]
        I = np.unique(sub.indices)
        yield j, J, I, sub[I, :].toarray(), a0c[I, j].toarray().ravel()


@pytest.mark.parametrize("which", ["q1_L1", "q1_L2", "upwind_L2", "fem_L2"])
def test_columns_match_lapack_lstsq(which):
    if which.startswith("q1"):
        seq = W.config2(nx=14, nmat=4)
    elif which.startswith("upwind"):
        seq = W.config3(nx=6, nmat=5)
    else:
        seq = W.config4(ncell=10, nmat=4, flip_frac=0.2)
    level = 1 if which.endswith("L1") else 2
    ak, a0 = seq.mats[-1], seq.mats[0]
    cp, ri = oracle.pattern(ak, level)
    out = oracle.build(ak, a0, cp, ri)
    for j, J, I, B, c in _ls_problems(ak, a0, cp, ri):
        ref = np.linalg.lstsq(B, c, rcond=None)[0]
        got = out["mval"][cp[j]: cp[j + 1]]
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
        r = c - B @ got
        assert abs(np.dot(r, r) - out["res2"][j]) <= 1e-12 * (np.dot(c, c) + 1e-300)


def test_normal_equations_hold_for_every_column():
    seq = W.config2(nx=14, nmat=3)
    ak, a0 = seq.mats[2], seq.mats[0]
    for level in (1, 2):
        cp, ri = oracle.pattern(ak, level)
        out = oracle.build(ak, a0, cp, ri)
        m = sp.csc_matrix((out["mval"], ri, cp), shape=(ak.n, ak.n))
        R = (ak.to_scipy() @ m - a0.to_scipy()).tocsc()
        akc = ak.to_scipy().tocsc()
        for j in range(ak.n):
            J = ri[cp[j]: cp[j + 1]]
            B = akc[:, J].toarray()
            r = R[:, j].toarray().ravel()
            g = B.T @ r
            mj = out["mval"][cp[j]: cp[j + 1]]
            c = a0.to_scipy().tocsc()[:, j].toarray().ravel()
            bound = 1e-14 * np.linalg.norm(B) * (np.linalg.norm(B) * np.linalg.norm(mj) + np.linalg.norm(c))
            assert np.linalg.norm(g) <= bound


def test_residual_matches_dense_product():
    seq = W.config1()
    ak, a0 = seq.mats[1], seq.mats[0]
    cp, ri = oracle.pattern(ak, 1)
    out = oracle.build(ak, a0, cp, ri)
    fro, rel = oracle.residual(ak, cp, ri, out["mval"], a0)
    m = _map_dense(ak.n, cp, ri, out["mval"])
    dense = np.linalg.norm(ak.dense() @ m - a0.dense())
    assert abs(fro - dense) <= 1e-13 * dense
    assert abs(rel - dense / np.linalg.norm(a0.dense())) <= 1e-13 * rel
    assert abs(np.sqrt(np.sum(out["res2"] + out["out2"])) - dense) <= 1e-12 * dense


def test_residual_counts_target_entries_outside_the_shadow():
    """Non-nested patterns (like the NWP sequence, Sec. 5.2): entries of A_0
    in rows outside I_j must enter the residual."""
    seq = W.config4(ncell=8, nmat=6, flip_frac=0.3)
    ak, a0 = seq.mats[5], seq.mats[0]
    # level 0 (the diagonal-only pattern of the tau = 0.6 / 0.7 rows of
    # Table 1): a flipped mesh diagonal leaves A_0(:, j) entries in rows
    # that no column of A_k(:, J_j) reaches
    cp, ri = oracle.pattern(ak, 0)
    out = oracle.build(ak, a0, cp, ri)
    assert np.any(out["out2"] > 0)
    m = _map_dense(ak.n, cp, ri, out["mval"])
    dense = np.linalg.norm(ak.dense() @ m - a0.dense())
    assert abs(np.sqrt(np.sum(out["res2"] + out["out2"])) - dense) <= 1e-12 * dense
    fro, _ = oracle.residual(ak, cp, ri, out["mval"], a0)
    assert abs(fro - dense) <= 1e-12 * dense


@pytest.mark.parametrize("cfg", ["q1", "upwind"])
def test_nested_patterns_do_not_increase_the_residual(cfg):
    """Sec. 5.1: higher-level neighbour patterns give better approximations;
    with nested patterns the minimum cannot increase."""
    seq = W.config2(nx=12, nmat=5) if cfg == "q1" else W.config3(nx=5, nmat=8)
    ak, a0 = seq.mats[-1], seq.mats[0]
    prev = np.inf
    for level in (0, 1, 2, 3):
        cp, ri = oracle.pattern(ak, level)
        out = oracle.build(ak, a0, cp, ri)
        fro, rel = oracle.residual(ak, cp, ri, out["mval"], a0)
        assert fro <= prev * (1 + 1e-12)
        prev = fro


def test_apply_is_the_sparse_product():
    a = W.config1().mats[1]
    cp, ri = oracle.pattern(a, 1)
    out = oracle.build(a, W.config1().mats[0], cp, ri)
    ip, ix, dv = oracle.to_csr(a.n, cp, ri, out["mval"])
    x = np.random.default_rng(0).standard_normal(a.n)
    y = oracle.apply(ip, ix, dv, x)
    m = _map_dense(a.n, cp, ri, out["mval"])
    assert np.allclose(y, m @ x, rtol=1e-14, atol=1e-14)


# ------------------------------------------------------- sparsification


@pytest.mark.parametrize("line", _golden_rows("cd2d_sparsified_nnz.txt"))
def test_sparsified_pattern_counts_printed_in_paper(line):
    """Sec. 4 sparsifications of the 5-point stencil (off-diagonal |A_ij| = 1/4
    of the diagonal: inside 1 - 0.8 of the column maximum, outside 1 - 0.7),
    then the printed power of the pattern."""
    side, mode, param, power, nnz = line.split()
    a = W.poisson5(int(side))
    ip, ix, dv = oracle.sparsify(a, mode, float(param))
    cp, ri = oracle.pattern(W.CSR(a.n, ip, ix, dv), int(power))
    assert int(cp[-1]) == int(nnz)


def _brute_sparsify(d, mode, param):
    """Dense restatement of the Sec. 4 criteria on a small matrix."""
    n = d.shape[0]
    keep = np.zeros_like(d, dtype=bool)
    stored = d != 0
    if mode == "global":
        diag = np.where(np.abs(np.diag(d)) > 0, np.abs(np.diag(d)), 1.0)
        for i in range(n):
            for j in range(n):
                if stored[i, j]:
                    keep[i, j] = i == j or abs(d[i, j]) / np.sqrt(diag[i] * diag[j]) > param
    else:
        for j in range(n):
            rows = np.nonzero(stored[:, j])[0]
            mags = np.abs(d[rows, j])
            if mode == "tau":
                for r, m in zip(rows, mags):
                    keep[r, j] = r == j or m > (1.0 - param) * mags.max()
            else:  # lfil: sort by magnitude descending, then row ascending
                order = sorted(range(len(rows)), key=lambda t: (-mags[t], rows[t]))
                for rank, t in enumerate(order):
                    keep[rows[t], j] = rows[t] == j or rank < int(param)
    return keep


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("mode,param", [("global", 0.05), ("global", 0.3), ("tau", 0.3), ("tau", 0.75),
                                        ("lfil", 1), ("lfil", 3)])
def test_sparsify_brute_force(seed, mode, param):
    rng = np.random.default_rng(700 + seed)
    n = 40
    p = rng.random((n, n)) < 0.15
    d = np.where(p, rng.uniform(-1.0, 1.0, (n, n)), 0.0)
    # ties: a few equal magnitudes inside columns
    d[p & (rng.random((n, n)) < 0.2)] = 0.5
    np.fill_diagonal(d, np.where(rng.random(n) < 0.8, 2.0 + rng.random(n), 0.0))
    a = W.CSR.from_dense(d)
    ip, ix, dv = oracle.sparsify(a, mode, param)
    got = np.zeros((n, n), dtype=bool)
    rows = np.repeat(np.arange(n), np.diff(ip))
    got[rows, ix] = True
    assert np.array_equal(got, _brute_sparsify(d, mode, param))
    # kept values are the source values
    assert np.array_equal(dv, d[rows, ix])


def test_sparsify_extremes():
    """tau = 1 and lfil >= column length keep every entry; tau = 0 and
    lfil = 0 keep the diagonal and, for tau, nothing but it."""
    a = W.config2(nx=12, nmat=1).mats[0]
    for mode, param in (("tau", 1.0), ("lfil", 100)):
        ip, ix, _ = oracle.sparsify(a, mode, param)
        assert np.array_equal(ip, a.indptr) and np.array_equal(ix, a.indices)
    for mode, param in (("tau", 0.0), ("lfil", 0)):
        ip, ix, _ = oracle.sparsify(a, mode, param)
        rows = np.repeat(np.arange(a.n), np.diff(ip))
        assert np.array_equal(rows, ix)


# ------------------------------------------------------------- Krylov


def _small_nonsym(seed, n=60):
    rng = np.random.default_rng(seed)
    p = (rng.random((n, n)) < 0.1) | np.eye(n, dtype=bool)
    a = np.where(p, rng.uniform(-1.0, 1.0, (n, n)), 0.0)
    a[np.arange(n), np.arange(n)] = 3.0 + rng.random(n)
    return a


@pytest.mark.parametrize("seed", range(3))
def test_gmres_solves_small_systems(seed):
    """The exact solution within the error bound: ||x - A^-1 b|| <=
    kappa(A) rtol ||x||, and the true residual meets the tolerance."""
    d = _small_nonsym(seed)
    A = W.CSR.from_dense(d)
    b = np.random.default_rng(seed + 10).standard_normal(d.shape[0])
    x, its, hist = oracle.gmres(A, b, restart=20, rtol=1e-10)
    exact = np.linalg.solve(d, b)
    kappa = np.linalg.cond(d)
    assert np.linalg.norm(x - exact) <= kappa * 2e-10 * np.linalg.norm(exact)
    assert np.linalg.norm(b - d @ x) <= 2e-10 * np.linalg.norm(b)
    # GMRES minimises the residual over growing spaces: the estimates do not
    # increase inside a cycle
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(min(19, len(hist) - 1)))


def test_gmres_exact_preconditioner_converges_in_one_step():
    d = _small_nonsym(5, n=40)
    A = W.CSR.from_dense(d)
    M = W.CSR.from_dense(np.linalg.inv(d))
    b = np.ones(40)
    x, its, hist = oracle.gmres(A, b, M=M, restart=10, rtol=1e-10)
    assert its == 1 and np.allclose(d @ x, b, atol=1e-10)


def test_gmres_diagonal_preconditioner_equals_scaled_system():
    """P_0 = diag(p0): GMRES on A diag(p0) u = b, x = diag(p0) u, written out
    with an explicitly scaled matrix and no preconditioner."""
    d = _small_nonsym(7, n=50)
    p0 = 1.0 / np.diag(d)
    b = np.random.default_rng(3).standard_normal(50)
    x1, it1, h1 = oracle.gmres(W.CSR.from_dense(d), b, p0=p0, restart=15, rtol=1e-9)
    u, it2, h2 = oracle.gmres(W.CSR.from_dense(d * p0[None, :]), b, restart=15, rtol=1e-9)
    assert it1 == it2
    assert np.allclose(x1, p0 * u, rtol=1e-10, atol=1e-14)


def test_gmres_iterations_match_scipy():
    """A library special case: unpreconditioned restarted GMRES in scipy
    stops after as many Arnoldi steps (same criterion ||r|| <= rtol ||b||),
    give or take one at a restart boundary."""
    import scipy.sparse.linalg as spla

    a = W.config2(nx=16, nmat=1).mats[0]
    b = np.random.default_rng(4).standard_normal(a.n)
    x, its, hist = oracle.gmres(a, b, restart=25, rtol=1e-8, maxiter=2000)
    count = [0]
    xs, info = spla.gmres(a.to_scipy(), b, restart=25, rtol=1e-8, atol=0.0, maxiter=200,
                          callback=lambda r: count.__setitem__(0, count[0] + 1), callback_type="pr_norm")
    assert info == 0
    assert abs(count[0] - its) <= 1
    assert np.linalg.norm(x - xs) <= 1e-6 * np.linalg.norm(xs)


def test_gmres_sparse_p0_operator():
    """P_0 given as a sparse operator: a diagonal one reproduces the diagonal
    p0 bit for bit (each product has one term), and an exact inverse of A
    converges in one step, alone or composed with M = I."""
    d = _small_nonsym(11, n=45)
    A = W.CSR.from_dense(d)
    p0 = 1.0 / np.diag(d)
    b = np.random.default_rng(12).standard_normal(45)
    x1, it1, h1 = oracle.gmres(A, b, p0=p0, restart=12, rtol=1e-10)
    x2, it2, h2 = oracle.gmres(A, b, P0=W.CSR.from_dense(np.diag(p0)), restart=12, rtol=1e-10)
    assert it1 == it2 and np.array_equal(x1, x2) and h1 == h2
    inv = W.CSR.from_dense(np.linalg.inv(d))
    for M in (None, W.CSR.from_dense(np.eye(45))):
        x, its, _ = oracle.gmres(A, b, M=M, P0=inv, restart=12, rtol=1e-10)
        assert its == 1 and np.allclose(d @ x, b, atol=1e-10)
