"""Seeded synthetic matrix sequences shaped like the paper's PDE workloads.

This module only assembles matrices (finite-difference and finite-element
stencils with seeded random coefficients).  It holds none of the SAM
arithmetic: no patterns, no least-squares, no residuals.  It is the one
module that both the CUDA path's tests/bench and the CPU oracle's tests
draw their inputs from.

The paper's own matrices (CD2D, Sec. 5.1; NWP, Sec. 5.2; THT, Sec. 4) are
not available, so these stand-ins reproduce their shapes: 2-D/3-D stencil
sequences whose values drift along the sequence while the pattern stays
fixed (the subset property, Eq. (property) in Sec. 3), and a finite-element
sequence whose pattern changes from matrix to matrix (like NWP, which
violates the subset property, Sec. 5.2).

Every matrix is returned as a `CSR` with int32 indices, float64 values,
rows sorted, column indices ascending and unique within a row.  Patterns
are structural: every stencil/mesh coupling is stored even if its value
happens to be tiny.  Seeds follow `numpy.random.default_rng(1000*config+k)`.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class CSR:
    """Square sparse matrix in compressed sparse row form (0-based)."""

    n: int
    indptr: np.ndarray  # int32 [n+1]
    indices: np.ndarray  # int32 [nnz], ascending within each row
    data: np.ndarray  # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def to_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.data, self.indices, self.indptr), shape=(self.n, self.n))

    def dense(self) -> np.ndarray:
        return self.to_scipy().toarray()

    @staticmethod
    def from_scipy(m) -> "CSR":
        m = sp.csr_matrix(m)
        m.sum_duplicates()
        m.sort_indices()
        return CSR(
            int(m.shape[0]),
            np.ascontiguousarray(m.indptr, dtype=np.int32),
            np.ascontiguousarray(m.indices, dtype=np.int32),
            np.ascontiguousarray(m.data, dtype=np.float64),
        )

    @staticmethod
    def from_dense(a: np.ndarray) -> "CSR":
        return CSR.from_scipy(sp.csr_matrix(np.asarray(a, dtype=np.float64)))


@dataclass
class Sequence:
    """A matrix sequence A_0..A_{N-1}; maps are built for every k (incl. k=0)."""

    name: str
    mats: list  # list[CSR]
    level: int  # pattern level used by this workload (1 or 2)
    meta: dict = field(default_factory=dict)


# ---------------------------------------------------------------- stencils


def poisson5(nx: int) -> CSR:
    """5-point Laplacian (4 on the diagonal, -1 to the 4 neighbours) on an
    nx-by-nx interior grid with Dirichlet boundary; lexicographic order."""
    n = nx * nx
    iy, ix = np.divmod(np.arange(n), nx)
    rows, cols, vals = [np.arange(n)], [np.arange(n)], [np.full(n, 4.0)]
    for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        jy, jx = iy + dy, ix + dx
        ok = (jy >= 0) & (jy < nx) & (jx >= 0) & (jx < nx)
        rows.append(np.arange(n)[ok])
        cols.append((jy * nx + jx)[ok])
        vals.append(np.full(int(ok.sum()), -1.0))
    m = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return CSR.from_scipy(m)


def gaussian_random_field(ncell: int, rng: np.random.Generator, ell: float = 0.1) -> np.ndarray:
    """Squared-exponential Gaussian random field on an ncell-by-ncell cell grid
    of the unit square (spacing 1/ncell), correlation length `ell`, by FFT
    spectral synthesis on a 2x periodic embedding; normalised to zero sample
    mean and unit sample variance."""
    m = 2 * ncell
    w = rng.standard_normal((m, m))
    k = np.fft.fftfreq(m, d=1.0 / ncell)
    k2 = k[:, None] ** 2 + k[None, :] ** 2
    amp = np.exp(-np.pi**2 * ell**2 * k2)  # sqrt of the SE spectral density (up to a constant)
    f = np.real(np.fft.ifft2(np.fft.fft2(w) * amp))[:ncell, :ncell]
    f = f - f.mean()
    return f / f.std()


def q1_diffusion(kappa: np.ndarray) -> CSR:
    """Bilinear (Q1) finite-element stiffness of -div(kappa grad u) on the unit
    square, cell-wise constant kappa of shape (ncell, ncell) indexed [cy, cx],
    homogeneous Dirichlet nodes eliminated.  Unknowns are the nx = ncell-1
    interior nodes per direction, lexicographic; 9-point stencil."""
    ncell = kappa.shape[0]
    nx = ncell - 1
    n = nx * nx
    # local Q1 stiffness on a square, corners ordered (0,0),(1,0),(1,1),(0,1)
    ke = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]], dtype=np.float64) / 6.0
    corner = [(0, 0), (1, 0), (1, 1), (0, 1)]
    cy, cx = np.meshgrid(np.arange(ncell), np.arange(ncell), indexing="ij")
    kap = kappa.ravel()
    rows, cols, vals = [], [], []
    for a in range(4):
        ax, ay = cx.ravel() + corner[a][0], cy.ravel() + corner[a][1]
        ina = (ax >= 1) & (ax <= nx) & (ay >= 1) & (ay <= nx)
        ia = (ay - 1) * nx + (ax - 1)
        for b in range(4):
            bx, by = cx.ravel() + corner[b][0], cy.ravel() + corner[b][1]
            inb = (bx >= 1) & (bx <= nx) & (by >= 1) & (by <= nx)
            ib = (by - 1) * nx + (bx - 1)
            keep = ina & inb
            rows.append(ia[keep])
            cols.append(ib[keep])
            vals.append(ke[a, b] * kap[keep])
    m = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return CSR.from_scipy(m)


def upwind7(nx: int, pe: float, w: np.ndarray) -> CSR:
    """-Lap(u) + pe * w.grad(u) on the unit cube, nx^3 interior nodes,
    h = 1/(nx+1), 7-point stencil with first-order upwinding of the
    convection term, Dirichlet boundary, scaled by h^2; lexicographic
    order (x fastest)."""
    h = 1.0 / (nx + 1)
    n = nx**3
    idx = np.arange(n).reshape(nx, nx, nx)  # [iz, iy, ix]
    diag = 6.0 + pe * h * float(np.abs(w).sum())
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [np.full(n, diag)]
    for d in range(3):  # d = 0:x, 1:y, 2:z ; array axis = 2 - d
        ax = 2 - d
        wp, wm = max(w[d], 0.0), min(w[d], 0.0)
        for step, val in ((-1, -1.0 - pe * h * wp), (1, -1.0 + pe * h * wm)):
            sl_src = [slice(None)] * 3
            sl_dst = [slice(None)] * 3
            if step == -1:
                sl_src[ax], sl_dst[ax] = slice(1, None), slice(0, -1)
            else:
                sl_src[ax], sl_dst[ax] = slice(0, -1), slice(1, None)
            src, dst = idx[tuple(sl_src)].ravel(), idx[tuple(sl_dst)].ravel()
            rows.append(src)
            cols.append(dst)
            vals.append(np.full(src.size, val))
    m = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return CSR.from_scipy(m)


def p1_fem(nv: int, xy: np.ndarray, flip: np.ndarray, c_react: float) -> CSR:
    """P1 finite-element Laplacian + c_react * consistent mass on an
    nv-by-nv vertex grid (positions xy[nv*nv, 2]) whose (nv-1)^2 cells are
    split into two triangles along the diagonal chosen by flip[cy, cx]
    (False: (0,0)-(1,1), True: (1,0)-(0,1)).  No Dirichlet nodes; every mesh
    edge is stored structurally."""
    nc = nv - 1
    cy, cx = np.meshgrid(np.arange(nc), np.arange(nc), indexing="ij")
    v00 = (cy * nv + cx).ravel()
    v10, v11, v01 = v00 + 1, v00 + nv + 1, v00 + nv
    f = flip.ravel().astype(bool)
    t1 = np.where(f[:, None], np.stack([v00, v10, v01], 1), np.stack([v00, v10, v11], 1))
    t2 = np.where(f[:, None], np.stack([v10, v11, v01], 1), np.stack([v00, v11, v01], 1))
    tri = np.concatenate([t1, t2])
    p = xy[tri]  # [T, 3, 2]
    d1, d2 = p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]
    det = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    area = 0.5 * np.abs(det)
    # gradients of the barycentric basis functions: grad phi_a = rot(edge opposite a) / (2*signed area)
    e = np.stack([p[:, 2] - p[:, 1], p[:, 0] - p[:, 2], p[:, 1] - p[:, 0]], 1)  # [T,3,2]
    g = np.stack([-e[..., 1], e[..., 0]], -1) / det[:, None, None]
    kloc = area[:, None, None] * np.einsum("tad,tbd->tab", g, g)
    mloc = (area / 12.0)[:, None, None] * (np.ones((3, 3)) + np.eye(3))[None]
    loc = kloc + c_react * mloc
    rows = np.repeat(tri, 3, axis=1).ravel()
    cols = np.tile(tri, (1, 3)).ravel()
    n = nv * nv
    m = sp.coo_matrix((loc.ravel(), (rows, cols)), shape=(n, n))
    return CSR.from_scipy(m)


# --------------------------------------------------------------- sequences


def config1(nx: int = 32) -> Sequence:
    """2-D Poisson 5-point on nx^2 (n=1024 at nx=32); A_1 = A_0 + diag(d),
    d ~ U(0, 0.5); level-1 pattern."""
    a0 = poisson5(nx)
    d = np.random.default_rng(1001).uniform(0.0, 0.5, size=a0.n)
    a1 = CSR.from_scipy(a0.to_scipy() + sp.diags(d))
    return Sequence("poisson5_%dx%d" % (nx, nx), [a0, a1], level=1, meta={"config": 1, "nx": nx})


def config2(nx: int = 256, nmat: int = 10, level: int = 2) -> Sequence:
    """Q1 9-point diffusion on nx^2 with kappa_k = kappa_0 * exp(0.05 k GRF_k),
    kappa_0 = exp(GRF_0), correlation length 0.1, sigma 1."""
    ncell = nx + 1
    g0 = gaussian_random_field(ncell, np.random.default_rng(2000))
    kap0 = np.exp(g0)
    mats = [q1_diffusion(kap0)]
    for k in range(1, nmat):
        gk = gaussian_random_field(ncell, np.random.default_rng(2000 + k))
        mats.append(q1_diffusion(kap0 * np.exp(0.05 * k * gk)))
    return Sequence("q1_diffusion_%dx%d" % (nx, nx), mats, level=level, meta={"config": 2, "nx": nx})


def config3(nx: int = 64, nmat: int = 20) -> Sequence:
    """7-point upwind convection-diffusion on nx^3; Peclet 10 -> 100 linearly,
    velocity (1, 0.5, 0.25) rotated by 5 degrees per step about z."""
    w0 = np.array([1.0, 0.5, 0.25])
    mats = []
    for k in range(nmat):
        pe = 10.0 + 90.0 * k / max(nmat - 1, 1)
        th = np.deg2rad(5.0 * k)
        rz = np.array([[np.cos(th), -np.sin(th), 0.0], [np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]])
        mats.append(upwind7(nx, pe, rz @ w0))
    return Sequence("upwind7_%d^3" % nx, mats, level=2, meta={"config": 3, "nx": nx})


def config4(ncell: int = 512, nmat: int = 16, flip_frac: float = 0.01) -> Sequence:
    """P1 FEM Laplacian + reaction on a jittered, randomly-diagonalised
    ncell^2 cell triangulation ((ncell+1)^2 vertices, no Dirichlet); each step
    re-flips `flip_frac` of the cell diagonals, reaction 0.1 -> 10
    geometrically."""
    nv = ncell + 1
    h = 1.0 / ncell
    rng = np.random.default_rng(4000)
    gy, gx = np.meshgrid(np.arange(nv) * h, np.arange(nv) * h, indexing="ij")
    xy = np.stack([gx.ravel(), gy.ravel()], 1) + rng.uniform(-0.3 * h, 0.3 * h, size=(nv * nv, 2))
    flip = rng.random((ncell, ncell)) < 0.5
    mats = []
    for k in range(nmat):
        if k > 0:
            r = np.random.default_rng(4000 + k)
            sel = r.random((ncell, ncell)) < flip_frac
            flip = flip ^ sel
        c = 0.1 * (100.0 ** (k / max(nmat - 1, 1)))
        mats.append(p1_fem(nv, xy, flip, c))
    return Sequence("p1_fem_%dx%d" % (ncell, ncell), mats, level=2, meta={"config": 4, "ncell": ncell})


def config5_pair(b: int, nx: int = 512):
    """One of the independent (A_0, A_1) Q1 9-point pairs of the adjoint run:
    kappa_0 = exp(GRF), kappa_1 = kappa_0 exp(0.05 GRF')."""
    ncell = nx + 1
    g0 = gaussian_random_field(ncell, np.random.default_rng(5000 + 2 * b + 1))
    g1 = gaussian_random_field(ncell, np.random.default_rng(5000 + 2 * b + 2))
    kap0 = np.exp(g0)
    return q1_diffusion(kap0), q1_diffusion(kap0 * np.exp(0.05 * g1))


def config5_vector(n: int) -> np.ndarray:
    """The seeded probe vector v of the adjoint loss ||M_1 v||^2."""
    return np.random.default_rng(5000).standard_normal(n)


def wide_band(n: int = 500, half: int = 50, keep: float = 0.85, nmat: int = 3, seed: int = 7000) -> Sequence:
    """A sequence of sources with about 85 stored entries per column, the
    density of the paper's NWP matrices (Sec. 5.2: 646,471 entries at
    n = 7700), for column problems past the register tiles at level 1: every
    entry of the band |i - j| <= half is stored with probability `keep`
    (one structure for the whole sequence, plus the diagonal), values
    U(-1, 1) with a dominant diagonal; A_k = A_0 with its off-diagonal
    values scaled by 1 + 0.05 k U(-1, 1)."""
    rng = np.random.default_rng(seed)
    i, j = np.nonzero(np.abs(np.arange(n)[:, None] - np.arange(n)[None, :]) <= half)
    sel = (rng.random(len(i)) < keep) | (i == j)
    i, j = i[sel], j[sel]
    base = rng.uniform(-1.0, 1.0, len(i))
    mats = []
    for k in range(nmat):
        v = base * (1.0 + 0.05 * k * rng.uniform(-1.0, 1.0, len(i)))
        off = np.where(i == j, 0.0, v)
        rowsum = np.bincount(i, weights=np.abs(off), minlength=n)
        v = np.where(i == j, rowsum[i] + 1.0, v)
        mats.append(CSR.from_scipy(sp.csr_matrix((v, (i, j)), shape=(n, n))))
    return Sequence("wide_band_%d_h%d" % (n, half), mats, level=1, meta={"half": half, "keep": keep})


def random_nested_pair(n: int, density: float, seed: int, extra: float = 0.5):
    """Small random diagonally dominant A_0, A_1 with S(A_0) subset of S(A_1)
    (the subset property of Sec. 3); used for brute-force checks."""
    rng = np.random.default_rng(seed)
    p0 = rng.random((n, n)) < density
    p1 = p0 | (rng.random((n, n)) < density * extra)
    np.fill_diagonal(p0, True)
    np.fill_diagonal(p1, True)
    a0 = np.where(p0, rng.uniform(-1.0, 1.0, (n, n)), 0.0)
    a1 = np.where(p1, rng.uniform(-1.0, 1.0, (n, n)), 0.0)
    for a in (a0, a1):
        np.fill_diagonal(a, 0.0)
        np.fill_diagonal(a, np.abs(a).sum(1) + 1.0)
    return CSR.from_dense(a0), CSR.from_dense(a1)


# ------------------------------------------------------------ CD2D stand-in


def _cd2d_residual_jacobian(u: np.ndarray, nx: int, gamma: float, eta: float = 0.1, r: float = 1.0,
                            s: float = 1.0):
    """F(u) and its Jacobian for -div((eta + gamma u^2) grad u) + r u_x + s u_y = 0
    on the unit square, second-order central differences on the nx-by-nx
    interior grid (h = 1/(nx+1)), face coefficients k((u_P + u_Q)/2),
    Dirichlet data u(0, y) = 0.2 + y (1 - y^2) and u = 0 on the other sides
    (Sec. 5.1, Eq. (convDif), t = f = 0).  Unknowns in lexicographic order
    (x fastest)."""
    h = 1.0 / (nx + 1)
    t = np.arange(nx + 2) * h
    U = np.zeros((nx + 2, nx + 2))  # U[j, i] = u(x_i, y_j)
    U[:, 0] = 0.2 + t * (1.0 - t * t)
    U[1:-1, 1:-1] = u.reshape(nx, nx)
    C = U[1:-1, 1:-1]
    nb = {"E": U[1:-1, 2:], "W": U[1:-1, :-2], "N": U[2:, 1:-1], "S": U[:-2, 1:-1]}
    kf = {d: eta + gamma * ((C + v) / 2) ** 2 for d, v in nb.items()}
    dkf = {d: gamma * (C + v) / 2 for d, v in nb.items()}  # d k(face) / d u_P = d k / d u_Q
    F = (-(kf["E"] * (nb["E"] - C) - kf["W"] * (C - nb["W"])) - (kf["N"] * (nb["N"] - C) - kf["S"] * (C - nb["S"]))) / h**2 \
        + r * (nb["E"] - nb["W"]) / (2 * h) + s * (nb["N"] - nb["S"]) / (2 * h)
    diag = (kf["E"] + kf["W"] + kf["N"] + kf["S"] - dkf["E"] * (nb["E"] - C) + dkf["W"] * (C - nb["W"])
            - dkf["N"] * (nb["N"] - C) + dkf["S"] * (C - nb["S"])) / h**2
    off = {"E": (-kf["E"] - dkf["E"] * (nb["E"] - C)) / h**2 + r / (2 * h),
           "W": (-kf["W"] + dkf["W"] * (C - nb["W"])) / h**2 - r / (2 * h),
           "N": (-kf["N"] - dkf["N"] * (nb["N"] - C)) / h**2 + s / (2 * h),
           "S": (-kf["S"] + dkf["S"] * (C - nb["S"])) / h**2 - s / (2 * h)}
    idx = np.arange(nx * nx).reshape(nx, nx)
    jj, ii = np.meshgrid(np.arange(nx), np.arange(nx), indexing="ij")
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [diag.ravel()]
    for d, (dj, di) in (("E", (0, 1)), ("W", (0, -1)), ("N", (1, 0)), ("S", (-1, 0))):
        tj, ti = jj + dj, ii + di
        ok = (tj >= 0) & (tj < nx) & (ti >= 0) & (ti < nx)
        rows.append(idx[jj[ok], ii[ok]])
        cols.append(idx[tj[ok], ti[ok]])
        vals.append(off[d][ok])
    J = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nx * nx, nx * nx))
    return F.ravel(), J


def cd2d(nx: int = 64, nmat: int = 66, stages: int = 24) -> Sequence:
    """Stand-in for the paper's CD2D sequence (Sec. 5.1): the Jacobians met
    by Newton's method with a backtracking line search on the nonlinear
    convection-diffusion problem of `_cd2d_residual_jacobian` (eta = 0.1,
    r = s = 1), n = nx^2 = 4096 at nx = 64.  The paper takes 66 Jacobians
    without saying how they arise (Newton from u = 0 converges in six
    steps), so the nonlinearity is raised by natural-parameter
    continuation: gamma = g / stages for g = 1..stages, each stage solved by
    Newton (Armijo line search, halving) from the previous solution to
    ||F|| <= 1e-9 ||F_stage start||; the first `nmat` Jacobians form the
    sequence.  Every matrix has the 5-point pattern (the subset property
    holds) and off-diagonal magnitudes between 20% and 30% of the diagonal,
    as the paper's Sec. 5.1 reads its Table 1."""
    import scipy.sparse.linalg as spla

    u = np.zeros(nx * nx)
    mats = []
    for g in range(1, stages + 1):
        gamma = g / stages
        F, J = _cd2d_residual_jacobian(u, nx, gamma)
        f0 = np.linalg.norm(F)
        for _ in range(50):
            if np.linalg.norm(F) <= 1e-9 * f0 or len(mats) >= nmat:
                break
            mats.append(CSR.from_scipy(J))
            d = spla.spsolve(J.tocsc(), F)
            nf, a = np.linalg.norm(F), 1.0
            while a > 1e-4:
                Ft, _ = _cd2d_residual_jacobian(u - a * d, nx, gamma)
                if np.linalg.norm(Ft) <= (1.0 - 1e-4 * a) * nf:
                    break
                a /= 2
            u = u - a * d
            F, J = _cd2d_residual_jacobian(u, nx, gamma)
        if len(mats) >= nmat:
            break
    return Sequence("cd2d_%dx%d" % (nx, nx), mats[:nmat], level=1, meta={"nx": nx, "stages": stages})
