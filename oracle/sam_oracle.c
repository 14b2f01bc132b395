/*
 * sam_oracle.c -- plain, slow, FP64 CPU reference for Sparse Approximate Map
 * (SAM) construction.  TEST INFRASTRUCTURE ONLY: it is loaded by the tests,
 * by the package's smoke check and by the benchmark's CPU-baseline leg, never
 * by the product path.  It shares no code with the CUDA library.
 *
 * What it computes (arXiv 2406.17656):
 *   - Sec. 3: the level-L neighbour pattern of column j in the adjacency
 *     graph G(A) (edge i->j iff A(i,j) is stored, i != j): all vertices with
 *     a path of length <= L pointing to j, plus j itself.  Level 1 is the
 *     column pattern of A with the diagonal, level 2 is paths of length <= 2.
 *   - Eq. (approx_map), and the column decomposition that follows it in
 *     Sec. 2: N_k = argmin ||A_k N - A_0||_F over the pattern, solved as n
 *     independent least-squares problems  min_m ||A_k(I_j, J_j) m - A_0(I_j, j)||
 *     where J_j is the pattern of column j and I_j the rows in which the
 *     columns A_k(:, J_j) have stored entries.  Rows outside I_j are zero in
 *     A_k(:, J_j), so they do not change the minimiser; their A_0 entries
 *     enter the residual only.
 *   - Eq. (res): R_k = A_k N_k - A_0 and the relative residual
 *     ||R_k||_F / ||A_0||_F used in Sec. 5.
 *   - Sec. 4: the three sparsifications of A_k whose level-L patterns the
 *     paper compares (global threshold on the diagonally scaled matrix,
 *     column threshold tau, fixed count lfil per column).
 *
 * Each least-squares problem is solved with textbook Householder QR
 * (Golub & Van Loan, Matrix Computations, Sec. 5.1.2 "house" and Sec. 5.2.1
 * Householder QR), applied to the augmented matrix [B c] so that Q^T c comes
 * out of the same sweep, followed by back substitution.  Columns are
 * independent, so an OpenMP loop over them changes no arithmetic.
 *
 * Memory: every array that a function returns through an `int **` /
 * `double **` argument is malloc'ed here and released with so_free().
 * Return value: 0 on success, 1 on allocation failure, 2 on invalid input,
 * 3 when a least-squares matrix is rank deficient (an exact zero pivot).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void so_free(void *p) { free(p); }

int so_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Transpose a CSR matrix: returns the CSR of A^T, i.e. the CSC of A.
 * Entries of each output row come out in ascending column order because the
 * input rows are visited in ascending order. */
static int transpose(int n, const int *rp, const int *ci, const double *v,
                     int **tp_out, int **ti_out, double **tv_out) {
    int nnz = rp[n];
    int *tp = (int *)calloc((size_t)n + 1, sizeof(int));
    int *ti = (int *)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    double *tv = v ? (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1)) : NULL;
    int *fill = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!tp || !ti || (v && !tv) || !fill) {
        free(tp); free(ti); free(tv); free(fill);
        return 1;
    }
    for (int e = 0; e < nnz; ++e) tp[ci[e] + 1]++;
    for (int i = 0; i < n; ++i) tp[i + 1] += tp[i];
    for (int i = 0; i < n; ++i) fill[i] = tp[i];
    for (int i = 0; i < n; ++i)
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            int p = fill[ci[e]]++;
            ti[p] = i;
            if (v) tv[p] = v[e];
        }
    free(fill);
    *tp_out = tp;
    *ti_out = ti;
    if (tv_out) *tv_out = tv;
    return 0;
}

static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* Check that a CSR structure is well formed: monotone row pointers, column
 * indices in range, strictly ascending within each row. */
int so_check_csr(int n, const int *rp, const int *ci) {
    if (n < 0 || rp[0] != 0) return 2;
    for (int i = 0; i < n; ++i) {
        if (rp[i + 1] < rp[i]) return 2;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            if (ci[e] < 0 || ci[e] >= n) return 2;
            if (e > rp[i] && ci[e] <= ci[e - 1]) return 2;
        }
    }
    return 0;
}

/*
 * Level-L pattern (Sec. 3).  Column j of the result lists, ascending, every
 * vertex i with a directed path i -> ... -> j of at most L edges in G(A),
 * and j itself.  Predecessors of vertex l are the rows stored in column l of
 * A, so the set is grown L times by adding the column patterns of the
 * vertices reached so far (a breadth-first search backwards from j).
 * Output: CSC structure colptr[n+1], rowidx[nnz].
 */
int so_pattern(int n, const int *rp, const int *ci, int level, int **colptr_out, int **rowidx_out) {
    if (level < 0 || so_check_csr(n, rp, ci)) return 2;
    int *cp, *cr;
    if (transpose(n, rp, ci, NULL, &cp, &cr, NULL)) return 1;
    char *mark = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    int *set = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *colptr = (int *)calloc((size_t)n + 1, sizeof(int));
    size_t cap = (size_t)rp[n] + (size_t)n + 16, used = 0;
    int *rowidx = (int *)malloc(sizeof(int) * cap);
    if (!mark || !set || !colptr || !rowidx) {
        free(cp); free(cr); free(mark); free(set); free(colptr); free(rowidx);
        return 1;
    }
    for (int j = 0; j < n; ++j) {
        int cnt = 0, frontier_begin = 0;
        set[cnt++] = j;
        mark[j] = 1;
        for (int lev = 0; lev < level; ++lev) {
            int frontier_end = cnt;
            for (int t = frontier_begin; t < frontier_end; ++t) {
                int l = set[t];
                for (int e = cp[l]; e < cp[l + 1]; ++e) {
                    int i = cr[e];
                    if (!mark[i]) {
                        mark[i] = 1;
                        set[cnt++] = i;
                    }
                }
            }
            frontier_begin = frontier_end;
        }
        qsort(set, (size_t)cnt, sizeof(int), cmp_int);
        if (used + (size_t)cnt > cap) {
            while (used + (size_t)cnt > cap) cap *= 2;
            int *tmp = (int *)realloc(rowidx, sizeof(int) * cap);
            if (!tmp) {
                free(cp); free(cr); free(mark); free(set); free(colptr); free(rowidx);
                return 1;
            }
            rowidx = tmp;
        }
        for (int t = 0; t < cnt; ++t) {
            rowidx[used++] = set[t];
            mark[set[t]] = 0;
        }
        colptr[j + 1] = (int)used;
    }
    free(cp); free(cr); free(mark); free(set);
    *colptr_out = colptr;
    *rowidx_out = rowidx;
    return 0;
}

/*
 * Shadow rows: I_j = union over c in J_j of the rows stored in column c of
 * A, ascending.  These are the only rows in which A(:, J_j) is nonzero.
 */
int so_shadow(int n, const int *rp, const int *ci, const int *jcp, const int *jri,
              int **icp_out, int **iri_out) {
    if (so_check_csr(n, rp, ci)) return 2;
    int *cp, *cr;
    if (transpose(n, rp, ci, NULL, &cp, &cr, NULL)) return 1;
    char *mark = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    int *set = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *icp = (int *)calloc((size_t)n + 1, sizeof(int));
    size_t cap = 4 * (size_t)rp[n] + 16, used = 0;
    int *iri = (int *)malloc(sizeof(int) * cap);
    if (!mark || !set || !icp || !iri) {
        free(cp); free(cr); free(mark); free(set); free(icp); free(iri);
        return 1;
    }
    for (int j = 0; j < n; ++j) {
        int cnt = 0;
        for (int t = jcp[j]; t < jcp[j + 1]; ++t) {
            int c = jri[t];
            for (int e = cp[c]; e < cp[c + 1]; ++e)
                if (!mark[cr[e]]) {
                    mark[cr[e]] = 1;
                    set[cnt++] = cr[e];
                }
        }
        qsort(set, (size_t)cnt, sizeof(int), cmp_int);
        if (used + (size_t)cnt > cap) {
            while (used + (size_t)cnt > cap) cap *= 2;
            int *tmp = (int *)realloc(iri, sizeof(int) * cap);
            if (!tmp) {
                free(cp); free(cr); free(mark); free(set); free(icp); free(iri);
                return 1;
            }
            iri = tmp;
        }
        for (int t = 0; t < cnt; ++t) {
            iri[used++] = set[t];
            mark[set[t]] = 0;
        }
        icp[j + 1] = (int)used;
    }
    free(cp); free(cr); free(mark); free(set);
    *icp_out = icp;
    *iri_out = iri;
    return 0;
}

/* position of key in the ascending array a[0..len), or -1 */
static int find_sorted(const int *a, int len, int key) {
    int lo = 0, hi = len - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (a[mid] == key) return mid;
        if (a[mid] < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/*
 * Householder QR of the m-by-(n+1) column-major matrix X = [B c] (leading
 * dimension m), m >= n, in place: on return the upper triangle of the first
 * n columns holds R and column n holds Q^T c.  For each k the reflector
 * P = I - beta v v^T with v(k) = 1 maps X(k:m, k) to mu e_1, mu = its norm
 * (Golub & Van Loan's "house", which avoids cancellation by choosing v(k)
 * = -sigma / (x_k + mu) when x_k > 0).  Returns 3 if a pivot is exactly 0.
 */
static int householder_qr(int m, int n, double *X, double *v) {
    for (int k = 0; k < n; ++k) {
        double *xk = X + (size_t)k * m;
        double sigma = 0.0;
        for (int i = k + 1; i < m; ++i) sigma += xk[i] * xk[i];
        double x1 = xk[k];
        double beta, mu;
        v[k] = 1.0;
        for (int i = k + 1; i < m; ++i) v[i] = xk[i];
        if (sigma == 0.0) {
            /* already triangular in this column: no reflection needed */
            beta = 0.0;
            mu = x1;
        } else {
            mu = sqrt(x1 * x1 + sigma);
            double v1 = (x1 <= 0.0) ? x1 - mu : -sigma / (x1 + mu);
            beta = 2.0 * v1 * v1 / (sigma + v1 * v1);
            for (int i = k + 1; i < m; ++i) v[i] /= v1;
        }
        if (mu == 0.0) return 3;
        /* apply P to columns k+1..n (the last one is the right-hand side) */
        for (int c = k + 1; c <= n; ++c) {
            double *xc = X + (size_t)c * m;
            double w = 0.0;
            for (int i = k; i < m; ++i) w += v[i] * xc[i];
            w *= beta;
            for (int i = k; i < m; ++i) xc[i] -= w * v[i];
        }
        xk[k] = mu;
        for (int i = k + 1; i < m; ++i) xk[i] = 0.0;
    }
    return 0;
}

/*
 * SAM build (Eq. (approx_map) and the column decomposition of Sec. 2).
 * Inputs: A_k and A_0 in CSR, the pattern J in CSC (jcp, jri; every column
 * must be nonempty).  Outputs (caller-allocated):
 *   mval[nnz(J)]  values of N_k in the pattern's CSC order (column j's values
 *                 at jcp[j]..jcp[j+1]-1, matching rows jri[...]),
 *   res2[n]       ||A_k(I_j,J_j) m_j - A_0(I_j,j)||^2, evaluated from the
 *                 original (unfactored) FP64 entries,
 *   out2[n]       sum of A_0(i,j)^2 over stored rows i outside I_j.
 * So ||R_k||_F^2 = sum_j (res2[j] + out2[j]).
 */
static int build_impl(int n, const int *krp, const int *kci, const double *kv,
                      const int *zrp, const int *zci, const double *zv,
                      const int *jcp, const int *jri, int nthreads,
                      const int *cols, int ncols,
                      double *mval, double *res2, double *out2) {
    if (so_check_csr(n, krp, kci) || so_check_csr(n, zrp, zci)) return 2;
    for (int j = 0; j < n; ++j)
        if (jcp[j + 1] <= jcp[j]) return 2;
    for (int t = 0; cols && t < ncols; ++t)
        if (cols[t] < 0 || cols[t] >= n) return 2;
    int *kcp, *kcr, *zcp, *zcr;
    double *kcv, *zcv;
    if (transpose(n, krp, kci, kv, &kcp, &kcr, &kcv)) return 1;
    if (transpose(n, zrp, zci, zv, &zcp, &zcr, &zcv)) {
        free(kcp); free(kcr); free(kcv);
        return 1;
    }
    /* shadow rows of every column */
    int *icp, *iri;
    int st = so_shadow(n, krp, kci, jcp, jri, &icp, &iri);
    if (st) {
        free(kcp); free(kcr); free(kcv); free(zcp); free(zcr); free(zcv);
        return st;
    }
    int maxm = 1, maxn = 1;
    for (int j = 0; j < n; ++j) {
        if (icp[j + 1] - icp[j] > maxm) maxm = icp[j + 1] - icp[j];
        if (jcp[j + 1] - jcp[j] > maxn) maxn = jcp[j + 1] - jcp[j];
    }
    int status = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        double *X = (double *)malloc(sizeof(double) * (size_t)maxm * (size_t)(maxn + 1));
        double *B = (double *)malloc(sizeof(double) * (size_t)maxm * (size_t)maxn);
        double *v = (double *)malloc(sizeof(double) * (size_t)maxm);
        double *m = (double *)malloc(sizeof(double) * (size_t)maxn);
        if (!X || !B || !v || !m) {
#pragma omp atomic write
            status = 1;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int t = 0; t < ncols; ++t) {
                const int j = cols ? cols[t] : t;
                const int *I = iri + icp[j];
                const int *J = jri + jcp[j];
                int mi = icp[j + 1] - icp[j], nj = jcp[j + 1] - jcp[j];
                if (mi < nj) {
#pragma omp atomic write
                    status = 3;
                    continue;
                }
                /* B = A_k(I, J), column major */
                memset(B, 0, sizeof(double) * (size_t)mi * (size_t)nj);
                for (int c = 0; c < nj; ++c) {
                    int col = J[c];
                    for (int e = kcp[col]; e < kcp[col + 1]; ++e) {
                        int p = find_sorted(I, mi, kcr[e]);
                        B[(size_t)c * mi + p] = kcv[e];
                    }
                }
                memcpy(X, B, sizeof(double) * (size_t)mi * (size_t)nj);
                /* right-hand side A_0(I, j); entries of A_0(:, j) outside I */
                double *rhs = X + (size_t)nj * mi;
                memset(rhs, 0, sizeof(double) * (size_t)mi);
                double o2 = 0.0;
                for (int e = zcp[j]; e < zcp[j + 1]; ++e) {
                    int p = find_sorted(I, mi, zcr[e]);
                    if (p >= 0) rhs[p] = zcv[e];
                    else o2 += zcv[e] * zcv[e];
                }
                if (householder_qr(mi, nj, X, v)) {
#pragma omp atomic write
                    status = 3;
                    continue;
                }
                /* back substitution R m = (Q^T c)(1:nj) */
                for (int r = nj - 1; r >= 0; --r) {
                    double s = rhs[r];
                    for (int c = r + 1; c < nj; ++c) s -= X[(size_t)c * mi + r] * m[c];
                    m[r] = s / X[(size_t)r * mi + r];
                }
                /* residual from the original entries: c - B m */
                double r2 = 0.0;
                for (int i = 0; i < mi; ++i) {
                    double ri = 0.0;
                    for (int e = zcp[j]; e < zcp[j + 1]; ++e)
                        if (zcr[e] == I[i]) ri = zcv[e];
                    for (int c = 0; c < nj; ++c) ri -= B[(size_t)c * mi + i] * m[c];
                    r2 += ri * ri;
                }
                for (int c = 0; c < nj; ++c) mval[jcp[j] + c] = m[c];
                res2[j] = r2;
                out2[j] = o2;
            }
        }
        free(X); free(B); free(v); free(m);
    }
    free(kcp); free(kcr); free(kcv); free(zcp); free(zcr); free(zcv);
    free(icp); free(iri);
    return status;
}

int so_build(int n, const int *krp, const int *kci, const double *kv,
             const int *zrp, const int *zci, const double *zv,
             const int *jcp, const int *jri, int nthreads,
             double *mval, double *res2, double *out2) {
    return build_impl(n, krp, kci, kv, zrp, zci, zv, jcp, jri, nthreads, NULL, n, mval, res2, out2);
}

/* The same for the listed columns only (cols[0..ncols)); the outputs of
 * other columns are left untouched.  Used to check sampled columns of large
 * problems. */
int so_build_cols(int n, const int *krp, const int *kci, const double *kv,
                  const int *zrp, const int *zci, const double *zv,
                  const int *jcp, const int *jri, int nthreads, const int *cols, int ncols,
                  double *mval, double *res2, double *out2) {
    return build_impl(n, krp, kci, kv, zrp, zci, zv, jcp, jri, nthreads, cols, ncols, mval, res2, out2);
}

/*
 * Residual of Eq. (res) straight from its definition, one column at a time:
 * R(:, j) = sum_c A_k(:, c) N(c, j) - A_0(:, j) accumulated in a dense
 * length-n vector.  N is given in CSC (ncp, nri, nv).  Returns
 * fro2 = ||R||_F^2 and a02 = ||A_0||_F^2.
 */
int so_residual(int n, const int *krp, const int *kci, const double *kv,
                const int *ncp, const int *nri, const double *nv,
                const int *zrp, const int *zci, const double *zv,
                double *fro2, double *a02) {
    if (so_check_csr(n, krp, kci) || so_check_csr(n, zrp, zci)) return 2;
    int *kcp, *kcr, *zcp, *zcr;
    double *kcv, *zcv;
    if (transpose(n, krp, kci, kv, &kcp, &kcr, &kcv)) return 1;
    if (transpose(n, zrp, zci, zv, &zcp, &zcr, &zcv)) {
        free(kcp); free(kcr); free(kcv);
        return 1;
    }
    /* dense accumulator plus the list of rows it touched in this column */
    double *w = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    char *hit = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    int *rows = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!w || !hit || !rows) {
        free(w); free(hit); free(rows);
        free(kcp); free(kcr); free(kcv); free(zcp); free(zcr); free(zcv);
        return 1;
    }
    double total = 0.0, a0 = 0.0;
    for (int j = 0; j < n; ++j) {
        int nt = 0;
        for (int t = ncp[j]; t < ncp[j + 1]; ++t) {
            int c = nri[t];
            for (int e = kcp[c]; e < kcp[c + 1]; ++e) {
                int i = kcr[e];
                if (!hit[i]) { hit[i] = 1; rows[nt++] = i; }
                w[i] += kcv[e] * nv[t];
            }
        }
        for (int e = zcp[j]; e < zcp[j + 1]; ++e) {
            int i = zcr[e];
            if (!hit[i]) { hit[i] = 1; rows[nt++] = i; }
            w[i] -= zcv[e];
            a0 += zcv[e] * zcv[e];
        }
        for (int t = 0; t < nt; ++t) {
            int i = rows[t];
            total += w[i] * w[i];
            w[i] = 0.0;
            hit[i] = 0;
        }
    }
    free(hit); free(rows);
    free(w);
    free(kcp); free(kcr); free(kcv); free(zcp); free(zcr); free(zcv);
    *fro2 = total;
    *a02 = a0;
    return 0;
}

/*
 * Adjoint of the SAM build on a fixed pattern (reverse-mode derivative of
 * the column least-squares solutions of Sec. 2).  With the loss
 *     L = sum over pattern entries of gbar * N  +  rho * ||A_k N - A_0||_F^2,
 * and, per column j, B = A_k(I_j, J_j), c = A_0(I_j, j), m = N(J_j, j),
 * r = c - B m, g = gbar(J_j, j), lambda = (B^T B)^{-1} g:
 *     dL/dB = r lambda^T - (B lambda) m^T - 2 rho r m^T,
 *     dL/dc = B lambda + 2 rho r,
 *     dL/dA_0(i, j) = 2 rho A_0(i, j) for stored rows i outside I_j,
 * summed over the columns into the stored entries of A_k and A_0 (in CSR
 * order, as the inputs).  lambda is solved with the R factor of B's
 * Householder QR: R^T z = g, R lambda = z.  dmres (nullable, pattern CSC
 * order) receives the direct residual part of dL/dN: -2 rho B^T r.
 * mval and gbar are in the pattern's CSC order; gbar may be NULL (zero).
 * Columns are visited in order and accumulated one after the other.
 */
int so_adjoint(int n, const int *krp, const int *kci, const double *kv,
               const int *zrp, const int *zci, const double *zv,
               const int *jcp, const int *jri, const double *mval, const double *gbar,
               double rho, double *dak, double *da0, double *dmres) {
    if (so_check_csr(n, krp, kci) || so_check_csr(n, zrp, zci)) return 2;
    int *kcp, *kcr, *zcp, *zcr;
    double *kcv, *zcv;
    if (transpose(n, krp, kci, kv, &kcp, &kcr, &kcv)) return 1;
    if (transpose(n, zrp, zci, zv, &zcp, &zcr, &zcv)) {
        free(kcp); free(kcr); free(kcv);
        return 1;
    }
    /* CSR index of every CSC entry (to return gradients in CSR order) */
    int *kperm = (int *)malloc(sizeof(int) * (size_t)(krp[n] > 0 ? krp[n] : 1));
    int *zperm = (int *)malloc(sizeof(int) * (size_t)(zrp[n] > 0 ? zrp[n] : 1));
    int *fill = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    double *dk = (double *)calloc((size_t)(krp[n] > 0 ? krp[n] : 1), sizeof(double));
    double *dz = (double *)calloc((size_t)(zrp[n] > 0 ? zrp[n] : 1), sizeof(double));
    int *icp, *iri;
    int st = so_shadow(n, krp, kci, jcp, jri, &icp, &iri);
    if (st || !kperm || !zperm || !fill || !dk || !dz) {
        free(kcp); free(kcr); free(kcv); free(zcp); free(zcr); free(zcv);
        free(kperm); free(zperm); free(fill); free(dk); free(dz);
        if (!st) { free(icp); free(iri); }
        return st ? st : 1;
    }
    for (int i = 0; i < n; ++i) fill[i] = kcp[i];
    for (int i = 0; i < n; ++i)
        for (int e = krp[i]; e < krp[i + 1]; ++e) kperm[fill[kci[e]]++] = e;
    for (int i = 0; i < n; ++i) fill[i] = zcp[i];
    for (int i = 0; i < n; ++i)
        for (int e = zrp[i]; e < zrp[i + 1]; ++e) zperm[fill[zci[e]]++] = e;
    int maxm = 1, maxn = 1;
    for (int j = 0; j < n; ++j) {
        if (icp[j + 1] - icp[j] > maxm) maxm = icp[j + 1] - icp[j];
        if (jcp[j + 1] - jcp[j] > maxn) maxn = jcp[j + 1] - jcp[j];
    }
    double *B = (double *)malloc(sizeof(double) * (size_t)maxm * (size_t)maxn);
    double *X = (double *)malloc(sizeof(double) * (size_t)maxm * (size_t)(maxn + 1));
    double *v = (double *)malloc(sizeof(double) * (size_t)maxm);
    double *c = (double *)malloc(sizeof(double) * (size_t)maxm);
    double *r = (double *)malloc(sizeof(double) * (size_t)maxm);
    double *w = (double *)malloc(sizeof(double) * (size_t)maxm);
    double *lam = (double *)malloc(sizeof(double) * (size_t)maxn);
    int status = 0;
    if (!B || !X || !v || !c || !r || !w || !lam) status = 1;
    for (int j = 0; j < n && !status; ++j) {
        const int *I = iri + icp[j];
        const int *J = jri + jcp[j];
        const int mi = icp[j + 1] - icp[j], nj = jcp[j + 1] - jcp[j];
        const double *m = mval + jcp[j];
        if (mi < nj) { status = 3; break; }
        memset(B, 0, sizeof(double) * (size_t)mi * (size_t)nj);
        for (int q = 0; q < nj; ++q)
            for (int e = kcp[J[q]]; e < kcp[J[q] + 1]; ++e)
                B[(size_t)q * mi + find_sorted(I, mi, kcr[e])] = kcv[e];
        memset(c, 0, sizeof(double) * (size_t)mi);
        for (int e = zcp[j]; e < zcp[j + 1]; ++e) {
            int p = find_sorted(I, mi, zcr[e]);
            if (p >= 0) c[p] = zcv[e];
            else dz[e] += 2.0 * rho * zcv[e];
        }
        /* r = c - B m */
        for (int i = 0; i < mi; ++i) {
            double s2 = c[i];
            for (int q = 0; q < nj; ++q) s2 -= B[(size_t)q * mi + i] * m[q];
            r[i] = s2;
        }
        /* lambda = (B^T B)^{-1} g through R of B = QR */
        for (int q = 0; q < nj; ++q) lam[q] = gbar ? gbar[jcp[j] + q] : 0.0;
        memcpy(X, B, sizeof(double) * (size_t)mi * (size_t)nj);
        memset(X + (size_t)nj * mi, 0, sizeof(double) * (size_t)mi);
        if (householder_qr(mi, nj, X, v)) { status = 3; break; }
        for (int q = 0; q < nj; ++q) {  /* R^T z = g */
            double s2 = lam[q];
            for (int p = 0; p < q; ++p) s2 -= X[(size_t)q * mi + p] * lam[p];
            lam[q] = s2 / X[(size_t)q * mi + q];
        }
        for (int q = nj - 1; q >= 0; --q) {  /* R lambda = z */
            double s2 = lam[q];
            for (int p = q + 1; p < nj; ++p) s2 -= X[(size_t)p * mi + q] * lam[p];
            lam[q] = s2 / X[(size_t)q * mi + q];
        }
        /* w = B lambda */
        for (int i = 0; i < mi; ++i) {
            double s2 = 0.0;
            for (int q = 0; q < nj; ++q) s2 += B[(size_t)q * mi + i] * lam[q];
            w[i] = s2;
        }
        /* dL/dB on the stored entries of A_k(:, J) */
        for (int q = 0; q < nj; ++q)
            for (int e = kcp[J[q]]; e < kcp[J[q] + 1]; ++e) {
                int i = find_sorted(I, mi, kcr[e]);
                dk[e] += r[i] * lam[q] - w[i] * m[q] - 2.0 * rho * r[i] * m[q];
            }
        /* dL/dc on the stored entries of A_0(I, j) */
        for (int e = zcp[j]; e < zcp[j + 1]; ++e) {
            int p = find_sorted(I, mi, zcr[e]);
            if (p >= 0) dz[e] += w[p] + 2.0 * rho * r[p];
        }
        if (dmres)
            for (int q = 0; q < nj; ++q) {
                double s2 = 0.0;
                for (int i = 0; i < mi; ++i) s2 += B[(size_t)q * mi + i] * r[i];
                dmres[jcp[j] + q] = -2.0 * rho * s2;
            }
    }
    if (!status) {
        for (int p = 0; p < krp[n]; ++p) dak[kperm[p]] = dk[p];
        for (int p = 0; p < zrp[n]; ++p) da0[zperm[p]] = dz[p];
    }
    free(B); free(X); free(v); free(c); free(r); free(w); free(lam);
    free(kcp); free(kcr); free(kcv); free(zcp); free(zcr); free(zcv);
    free(kperm); free(zperm); free(fill); free(dk); free(dz); free(icp); free(iri);
    return status;
}

/*
 * Sec. 4 sparsifications of A (CSR): keep[e] = 1 for every stored entry e
 * that the sparsified matrix keeps, 0 otherwise.  The diagonal is always
 * kept.  Readings of the printed formulas:
 *   mode 0, global threshold `param`: keep (i, j) when
 *           |A_ij| / sqrt(D_ii D_jj) > param, with D_ii = |A_ii| when that is
 *           stored and nonzero, else 1 (the printed D^{1/2} A D^{1/2} read as
 *           the usual symmetric scaling D^{-1/2} A D^{-1/2});
 *   mode 1, column threshold tau = `param` in [0, 1]: keep (i, j) when
 *           |A_ij| > (1 - tau) max_i |A_ij|, the maximum over the stored
 *           entries of column j, as printed;
 *   mode 2, lfil = (int)`param` >= 0: keep the lfil entries of column j of
 *           largest |A_ij| (equal magnitudes: the lower row index first).
 * Plain loops over the columns of the transpose.
 */
int so_sparsify(int n, const int *rp, const int *ci, const double *v, int mode, double param, int *keep) {
    if (n < 0 || !rp || !keep || (rp[n] > 0 && (!ci || !v))) return 2;
    if (mode < 0 || mode > 2) return 2;
    const int nnz = rp[n];
    for (int e = 0; e < nnz; ++e) keep[e] = 0;
    if (mode == 0) {
        double *d = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        if (!d) return 1;
        for (int i = 0; i < n; ++i) {
            d[i] = 1.0;
            for (int e = rp[i]; e < rp[i + 1]; ++e)
                if (ci[e] == i && fabs(v[e]) > 0.0) d[i] = fabs(v[e]);
        }
        for (int i = 0; i < n; ++i)
            for (int e = rp[i]; e < rp[i + 1]; ++e) {
                const int j = ci[e];
                keep[e] = (i == j) || (fabs(v[e]) / sqrt(d[i] * d[j]) > param);
            }
        free(d);
        return 0;
    }
    /* column criteria: walk the columns through the transpose, remembering
     * where each CSC entry sits in the CSR arrays */
    int *tp = NULL, *ti = NULL;
    double *tv = NULL;
    if (transpose(n, rp, ci, v, &tp, &ti, &tv)) return 1;
    int *pos = (int *)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    int *fill = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!pos || !fill) {
        free(tp); free(ti); free(tv); free(pos); free(fill);
        return 1;
    }
    for (int j = 0; j < n; ++j) fill[j] = tp[j];
    for (int i = 0; i < n; ++i)
        for (int e = rp[i]; e < rp[i + 1]; ++e) pos[fill[ci[e]]++] = e;
    for (int j = 0; j < n; ++j) {
        const int b = tp[j], en = tp[j + 1];
        if (mode == 1) {
            double mx = 0.0;
            for (int p = b; p < en; ++p) mx = fabs(tv[p]) > mx ? fabs(tv[p]) : mx;
            for (int p = b; p < en; ++p) keep[pos[p]] = (ti[p] == j) || (fabs(tv[p]) > (1.0 - param) * mx);
        } else {
            const int lfil = (int)param;
            for (int p = b; p < en; ++p) {
                /* rank = entries of the column that come before p in the
                 * order (larger magnitude, then lower row) */
                int rank = 0;
                for (int q = b; q < en; ++q) {
                    if (q == p) continue;
                    const double aq = fabs(tv[q]), ap = fabs(tv[p]);
                    if (aq > ap || (aq == ap && ti[q] < ti[p])) ++rank;
                }
                keep[pos[p]] = (ti[p] == j) || (rank < lfil);
            }
        }
    }
    free(tp); free(ti); free(tv); free(pos); free(fill);
    return 0;
}
