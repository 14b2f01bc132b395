/*
 * sam.h -- C ABI of libsam, a GB300 (sm_103a) library that builds Sparse
 * Approximate Maps (SAMs) as defined in arXiv 2406.17656, "Optimization of
 * Approximate Maps for Linear Systems Arising in Discretized PDEs".
 *
 * Given a sequence of sparse matrices A_0, A_1, ..., the SAM of A_k is
 * (Sec. 2, Eq. (approx_map))
 *
 *     N_k = argmin_N || A_k N - A_0 ||_F   over N with sparsity pattern S,
 *
 * which splits into one small least-squares problem per column j:
 * min_m || A_k(I_j, J_j) m - A_0(I_j, j) ||, with J_j the pattern of column
 * j and I_j the "shadow" rows, the rows in which A_k(:, J_j) has stored
 * entries.  The patterns used here are the level-L neighbourhoods of the
 * adjacency graph G(A_k) (Sec. 3): level 1 is S(A_k) plus the diagonal,
 * level 2 adds every vertex with a path of length <= 2 to j (the pattern of
 * (A_k + I)^2).  The map is returned in CSR and is called M_k below
 * (the paper's N_k).
 *
 * Conventions common to every call
 *  - Indices are 0-based int32; a matrix is square, 1 <= n <= 2^31-1 rows
 *    (an empty matrix is rejected with SAM_ERR_INVALID_ARG), at most
 *    2^31-1 stored entries.  CSR rows list column indices in strictly
 *    ascending order.  Values are IEEE double.
 *  - Pointers in `sam_csr` and the vector/array arguments may point to
 *    device memory (cudaMalloc, managed) or to host memory (pinned or
 *    pageable); the library checks each pointer with
 *    cudaPointerGetAttributes and stages host arrays through its own device
 *    workspace, copying host outputs back before the call returns.  With
 *    device pointers every call is asynchronous on the handle's stream.
 *  - All memory passed in is owned by the caller and never freed by the
 *    library.  Objects returned through `sam_handle*` / `sam_pattern*` are
 *    owned by the library and released with the matching destroy call;
 *    patterns live in their handle's memory pool, so destroy them before
 *    the handle.
 *  - No call aborts, traps or throws.  Each returns a sam_status.  Errors
 *    detected on the device (a rank-deficient or non-finite column, an
 *    unsupported column size) are recorded in a sticky status word that
 *    sam_sync() returns; calls that return host scalars synchronise and
 *    report it themselves.
 */
#ifndef SAM_H
#define SAM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t sam_status;

enum {
    SAM_OK = 0,
    SAM_ERR_INVALID_ARG = 1,    /* null pointer, bad size, level, precision, ... */
    SAM_ERR_BAD_CSR = 2,        /* row pointers not monotone, index out of range, unsorted/duplicate */
    SAM_ERR_RANK_DEFICIENT = 3, /* a column's least-squares matrix has a zero pivot */
    SAM_ERR_NONFINITE = 4,      /* NaN/Inf met in a column's solve */
    SAM_ERR_CUDA = 5,           /* a CUDA runtime call failed */
    SAM_ERR_OOM = 6,            /* device allocation failed */
    SAM_ERR_TIMEOUT = 7,        /* a host-side wait ran out */
    SAM_ERR_UNSUPPORTED = 8     /* a column exceeds the kernels' size limits (see sam_limits) */
};

/* precision of the per-column least-squares solves */
enum {
    SAM_FP64 = 0,        /* Householder QR, triangular solves and residuals in FP64 */
    SAM_FP32_REFINE = 1  /* Householder QR in FP32, then `refine_steps` corrected
                            semi-normal-equation steps with FP64 residuals */
};

/*
 * refine_steps = SAM_REFINE_AUTO (SAM_FP32_REFINE only): one or two steps per
 * column, chosen by a stopping test, with an FP64 re-solve of the columns
 * that miss the target.  A fixed number of steps s >= 1 is guarded the same
 * way; s = 0 (the FP32 solve alone, about 1e-5 relative) is not.
 *
 * Corrected semi-normal-equation steps contract the error by
 * rho ~ u_32 kappa(B)^2 each, so the error after step s is at most
 * rho / (1 - rho) |d_s| for the correction d_s of that step.  rho is
 * estimated as the larger of 8 u_32 kappa^2, with kappa estimated as
 * max |R_kk| / min |R_kk| (a lower bound on kappa(B), hence the factor 8),
 * and 4 |d_1| / |m| after step 1 or
 * |d_s| / |d_{s-1}| after later steps.  Automatic mode takes step 2 when
 * 4 |d_1|^2 > 1e-12 |m|^2 or the prediction after step 1 misses (such a
 * column is solved again with two steps by a launch of its own, so that its
 * result equals the two-step build's and every other column's equals the
 * one-step build's, bit for bit); after the
 * last step (2 in automatic mode, s otherwise) a predicted error above
 * 1e-10 |m|, or rho >= 1/2, sends the column to an FP64 Householder
 * re-solve (the large class's FP64 kernel).  The large class's FP32 tile
 * takes the same steps under the same test.  sam_refine_stats counts the
 * outcomes.
 */
#define SAM_REFINE_AUTO (-1)

/* flag bits for sam_set_flags */
enum {
    SAM_FLAG_TRUSTED = 1 /* skip CSR validation of inputs */
};

/* A square sparse matrix in CSR form. */
typedef struct {
    int32_t n;              /* rows = columns */
    int64_t nnz;            /* stored entries = row_ptr[n] */
    const int32_t *row_ptr; /* [n+1] */
    const int32_t *col_idx; /* [nnz], ascending within each row */
    const double *val;      /* [nnz]; may be NULL for structure-only calls */
} sam_csr;

typedef struct sam_handle_t *sam_handle;   /* stream, device workspace, sticky status */
typedef struct sam_pattern_t *sam_pattern; /* a map sparsity pattern S (device resident) */
typedef struct sam_plan_t *sam_plan;       /* a captured numeric rebuild (sam_plan_create) */

/* Largest column sizes the least-squares kernels accept:
 * |J_j| <= *max_cols and |I_j| <= *max_rows (the large class's limits; it
 * also needs |I_j| (|J_j| + 1) <= 23552 and nnz(B_j) <= 16384). */
void sam_limits(int32_t *max_rows, int32_t *max_cols);

/*
 * Size classes of the column problems (the batching of Sec. 2's column
 * solves by their uneven sizes; no counterpart in the paper).  A column
 * with |I_j| >= |J_j| shadow rows, |J_j| unknowns and nnz(B_j) stored
 * entries goes to the first class b with |I_j| <= max_rows[b],
 * |J_j| <= max_cols[b], nnz(B_j) <= max_entries[b] and
 * |I_j| (|J_j| + 1) <= max_tile[b]; a column that fits none is
 * SAM_ERR_UNSUPPORTED.  Classes 0..4 are register tiles with
 * FP32 or FP64 arithmetic; class 5 (SAM_NUM_SIZE_CLASSES - 1) is one thread
 * block per column with the tile in shared memory (FP64 for SAM_FP64; FP32
 * with the FP64 refinement steps and their guard for SAM_FP32_REFINE); its
 * adjoint (sam_build_backward) runs in FP64 for either precision.  variants[b]: tile shapes of class b
 * (sam_tune, sam_set_tile_variants).  count must be SAM_NUM_SIZE_CLASSES;
 * any output may be NULL.
 */
#define SAM_NUM_SIZE_CLASSES 6
sam_status sam_size_classes(int32_t *max_rows, int32_t *max_cols, int32_t *max_entries, int32_t *max_tile,
                            int32_t *variants, int count);

/* Human-readable text of a status code (static storage). */
const char *sam_status_string(sam_status s);

/* Create a handle bound to the current CUDA device and the given stream
 * (a cudaStream_t, NULL for the legacy default stream). */
sam_status sam_create(sam_handle *h, void *cuda_stream);
sam_status sam_destroy(sam_handle h);
sam_status sam_set_stream(sam_handle h, void *cuda_stream);
sam_status sam_set_flags(sam_handle h, uint32_t flags);
/* Wait for the handle's stream and return (then clear) the sticky status. */
sam_status sam_sync(sam_handle h);

/*
 * sam_pattern_build -- level-`level` neighbour pattern of every column of
 * G(A_k) (Sec. 3): column j holds, ascending, every vertex i with a directed
 * path i -> ... -> j of at most `level` edges (edge i -> j iff A_k(i, j) is
 * stored, i != j) and j itself.  level 0 is the diagonal, 1 is S(A_k) plus
 * the diagonal, 2 the pattern of (A_k + I)^2, 3 of (A_k + I)^3.
 * Only the structure of A_k is read (A_k->val may be NULL).  The pattern is
 * stored on the device in CSC form (= the CSC structure of the map) together
 * with the CSR structure of the map.  Synchronises to validate A_k and to
 * size the output (for level >= 2 also to size the candidate lists; the
 * status word is read with the size).  *out is library-owned: release with
 * sam_pattern_destroy.
 * Limit: a column whose merged candidate lists hold more than 1024 entries
 * and span more than 32768 row indices is SAM_ERR_UNSUPPORTED.
 */
sam_status sam_pattern_build(sam_handle h, const sam_csr *A_k, int level, sam_pattern *out);

/* The same for K matrices at once, with a single synchronisation. */
sam_status sam_pattern_build_batched(sam_handle h, int K, const sam_csr *A_k, int level, sam_pattern *out);

/* Wrap a caller-chosen pattern given in CSC (colptr[n+1], rowidx[nnz], rows
 * ascending within a column, every column nonempty); the arrays are copied.
 * Lets a map use e.g. the target's pattern S(A_0), the choice the paper
 * compares against (Sec. 5). */
sam_status sam_pattern_from_csc(sam_handle h, int32_t n, int64_t nnz, const int32_t *colptr,
                                const int32_t *rowidx, sam_pattern *out);

/* Device views of a pattern: n, nnz, CSC colptr[n+1] and rowidx[nnz] of the
 * map's pattern, valid until sam_pattern_destroy.  Any output may be NULL. */
sam_status sam_pattern_get(sam_pattern S, int32_t *n, int64_t *nnz, const int32_t **colptr,
                           const int32_t **rowidx);
sam_status sam_pattern_destroy(sam_pattern S);

/*
 * sam_sparsify -- the sparsified source A~ of Sec. 4, whose level-L pattern
 * (sam_pattern_build on A~) the paper compares as the map's pattern.  The
 * diagonal is kept whenever it is stored; other stored entries by `mode`:
 *   SAM_SPARSIFY_GLOBAL  |A_ij| / sqrt(D_ii D_jj) > param (the global
 *                        threshold `thresh`), D_ii = |A_ii| if stored and
 *                        nonzero, else 1 (the printed D^{1/2} A D^{1/2} is
 *                        read as the symmetric scaling D^{-1/2} A D^{-1/2});
 *   SAM_SPARSIFY_TAU     |A_ij| > (1 - param) max_i |A_ij| (column threshold
 *                        tau = param in [0, 1], as printed);
 *   SAM_SPARSIFY_LFIL    the (int)param entries of largest |A_ij| in each
 *                        column (equal magnitudes: lower row index first).
 * Outputs (caller-allocated, device or host): S_row_ptr[n+1],
 * S_col_idx[nnz(A)] and S_val[nnz(A)] (nullable) receive the kept entries in
 * CSR order; *S_nnz (host) their number.  Synchronises the handle's stream.
 * Errors: SAM_ERR_INVALID_ARG (bad mode / parameter / pointers),
 * SAM_ERR_BAD_CSR.
 */
enum { SAM_SPARSIFY_GLOBAL = 0, SAM_SPARSIFY_TAU = 1, SAM_SPARSIFY_LFIL = 2 };
sam_status sam_sparsify(sam_handle h, const sam_csr *A, int mode, double param, int32_t *S_row_ptr,
                        int32_t *S_col_idx, double *S_val, int64_t *S_nnz);

/*
 * sam_sparsify_batched -- sam_sparsify of K matrices of the same order n in
 * one pass (one validation, one set of launches, one synchronisation; the
 * sparsifications of Sec. 4 act within one matrix, so the batch is
 * sparsified as its block-diagonal concatenation).  Outputs
 * (caller-allocated, device or host): S_row_ptr[K][n+1], map k's row
 * pointers relative to its own first entry; S_col_idx / S_val (nullable)
 * with room for the sum of nnz(A_k) entries, map k's kept entries at
 * S_offsets[k] .. S_offsets[k+1]; S_offsets (host, int64[K+1]).
 * Synchronises the handle's stream.  Errors: those of sam_sparsify.
 */
sam_status sam_sparsify_batched(sam_handle h, int K, const sam_csr *A, int mode, double param, int32_t *S_row_ptr,
                                int32_t *S_col_idx, double *S_val, int64_t *S_offsets);

/*
 * sam_build -- the SAM M_k = argmin ||A_k M - A_0||_F on the pattern S
 * (Eq. (approx_map), column decomposition of Sec. 2), one least-squares
 * problem per column, written as CSR:
 *   M_row_ptr[n+1], M_col_idx[nnz(S)], M_val[nnz(S)] (caller-allocated,
 *   nnz from sam_pattern_get).  Column indices ascend within each row.
 * precision: SAM_FP64 or SAM_FP32_REFINE; refine_steps (0..4, or
 * SAM_REFINE_AUTO) is used by SAM_FP32_REFINE only.  col_status (nullable, int32[n]) receives 0 or a
 * sam_status per column.  res2 (nullable, double[n]) receives per column
 * ||A_k(I_j,J_j) m_j - A_0(I_j,j)||^2 + sum of A_0(i,j)^2 over rows i
 * outside I_j, so that ||R_k||_F^2 = sum_j res2[j] (Eq. (res)).
 * A_k must have the structure the pattern's shadow rows are taken from
 * (any A_k works: shadows are computed here from A_k and S).
 */
sam_status sam_build(sam_handle h, const sam_csr *A_k, const sam_csr *A_0, sam_pattern S, int precision,
                     int refine_steps, int32_t *M_row_ptr, int32_t *M_col_idx, double *M_val,
                     int32_t *col_status, double *res2);

/*
 * sam_build_batched -- K maps M_k for the sources A_k[0..K-1] against the
 * one target A_0, in one pass: all maps' columns are binned by size and each
 * size class runs as a single persistent launch over every map.
 * M_offsets[K+1] (host, int64) gives each map's offset into M_col_idx /
 * M_val; map k's row pointers go to M_row_ptr + k*(n+1) (relative to its own
 * offset).  col_status and res2 (nullable) are laid out as [K][n].
 * fro (nullable, host double[K]) receives ||A_k M_k - A_0||_F per map and
 * forces a synchronisation.
 * With host arrays the copies overlap the work: input values travel on a
 * library-owned side stream while the structure work runs, the maps' CSR
 * structure is copied out while the solves run, and when every map has one
 * structure the large size classes are solved in chunks of maps, each
 * chunk's values copied out while the next is solved.  The side streams
 * are joined into the handle's stream before the call returns; the results
 * are the same bits as with device arrays.
 */
sam_status sam_build_batched(sam_handle h, int K, const sam_csr *A_k, const sam_csr *A_0,
                             const sam_pattern *S, int precision, int refine_steps,
                             const int64_t *M_offsets, int32_t *M_row_ptr, int32_t *M_col_idx,
                             double *M_val, int32_t *col_status, double *res2, double *fro);

/*
 * sam_build_multi -- as sam_build_batched, but map k has its own target:
 * A_0[0..K-1] (all of order n), M_k = argmin ||A_k M - A_0[k]||_F on S[k].
 * For batches of independent (A_0, A_1) pairs; fro[k] is the residual of
 * map k against A_0[k].  Same outputs, errors and synchronisation.
 */
sam_status sam_build_multi(sam_handle h, int K, const sam_csr *A_k, const sam_csr *A_0,
                           const sam_pattern *S, int precision, int refine_steps,
                           const int64_t *M_offsets, int32_t *M_row_ptr, int32_t *M_col_idx,
                           double *M_val, int32_t *col_status, double *res2, double *fro);

/*
 * sam_plan_create -- the batched build (sam_build_batched when n_targets = 1,
 * sam_build_multi when n_targets = K) split into its value-independent part,
 * done here once, and its value-dependent part, captured once into a CUDA
 * graph that sam_plan_execute replays.  For sequences whose sparsity stays
 * fixed while the values change (the paper's setting of Sec. 2: a sequence
 * A_k of one discretisation), every replay re-reads the values of the A_k
 * and A_0 given here (the val pointers; structure arrays are read only here),
 * gathers them, solves every column and writes M_val, col_status, res2 and
 * fro2 -- the same results, bit for bit, as the corresponding direct call
 * with the handle's tile variants at creation.
 * Done at creation: validation, transposes, shadow rows, size classes, work
 * lists and the map structure (M_row_ptr / M_col_idx are written here and
 * not again).  All arrays must be device memory and stay allocated while
 * the plan lives; the patterns may be destroyed after creation.
 * fro2 (nullable, device double[K]): ||A_k M_k - A_0||_F^2 per map.
 * Synchronises the handle's stream (creation only).  Errors: those of
 * sam_build_batched; SAM_ERR_INVALID_ARG for host pointers.
 */
sam_status sam_plan_create(sam_handle h, int K, const sam_csr *A_k, const sam_csr *A_0, int n_targets,
                           const sam_pattern *S, int precision, int refine_steps,
                           const int64_t *M_offsets, int32_t *M_row_ptr, int32_t *M_col_idx,
                           double *M_val, int32_t *col_status, double *res2, double *fro2,
                           sam_plan *out);
/* Replays the plan on the handle's current stream (asynchronous; a failed
 * column raises the sticky status read by sam_sync). */
sam_status sam_plan_execute(sam_plan p);
/* Kernels one replay launches. */
sam_status sam_plan_launches(sam_plan p, int64_t *launches);
/* Synchronises the handle's stream and frees the plan. */
sam_status sam_plan_destroy(sam_plan p);

/*
 * sam_residual -- ||R_k||_F and ||R_k||_F / ||A_0||_F for R_k = A_k M_k - A_0
 * (Eq. (res); the relative form is the metric of Sec. 5), computed in FP64
 * column by column with a deterministic reduction.  fro and rel are host
 * pointers (either may be NULL); the call synchronises.
 */
sam_status sam_residual(sam_handle h, const sam_csr *A_k, const sam_csr *M_k, const sam_csr *A_0,
                        double *fro, double *rel);

/*
 * sam_apply -- y = M_k x (FP64 CSR product).  Used as the preconditioner
 * update of Sec. 1/2: since A_k M_k ~ A_0, A_k (M_k P_0) ~ A_0 P_0 ~ I for a
 * preconditioner P_0 of A_0, so the right preconditioner applied to v is
 * M_k (P_0 v): apply P_0 first, then this call.  x and y must not overlap.
 */
sam_status sam_apply(sam_handle h, const sam_csr *M_k, const double *x, double *y);

/*
 * sam_apply_grad -- the gradient of a loss through y = M_k x with respect to
 * the stored values of M_k: dM_val[e] = dy[i] x[c] for every stored entry
 * e = (i, c) of M_k (CSR order), given dy = dL/dy.  With sam_apply it makes
 * a loss term such as ||M_k v||^2 differentiable in the map values, as in
 * the sensitivity studies of the map (the paper builds the map for use in
 * M_k (P_0 v), Sec. 1-2).  Only the structure of M_k is read (M_k->val may
 * be NULL).  x[n], dy[n], dM_val[nnz(M_k)] device or host.  Errors:
 * SAM_ERR_INVALID_ARG, SAM_ERR_BAD_CSR.
 */
sam_status sam_apply_grad(sam_handle h, const sam_csr *M_k, const double *x, const double *dy, double *dM_val);

/*
 * sam_gmres -- restarted GMRES(restart) for A x = b with the right
 * preconditioner z = M (P_0 v), the use of a map stated in Sec. 1-2: P_0 is
 * a preconditioner built once for A_0, M = M_k the map of A_k, so that
 * A_k M_k P_0 ~ A_0 P_0 ~ I (the paper builds the maps but does not run
 * this solve).  FP64 throughout; orthogonalisation by classical
 * Gram-Schmidt applied twice, Givens rotations on the Hessenberg matrix.
 *   A       system matrix (values required).
 *   M       nullable: the map M_k (identity when NULL).
 *   P_0     nullable: a preconditioner of A_0 given as a sparse operator
 *           (e.g. a diagonal, or a sparse approximate inverse of A_0 such as
 *           sam_build(A_0, I, S) returns); applied by a product; identity
 *           when NULL.
 *   b[n]    right-hand side; x[n] the initial guess on entry, the solution
 *           on return (x = x0 + M P_0 V y after every cycle).
 *   restart Arnoldi steps per cycle, 1..SAM_GMRES_MAX_RESTART; maxiter the
 *           total number of Arnoldi steps allowed (0: x is left as given).
 *   rtol    stop when the least-squares residual estimate |g_{k+1}| falls
 *           to rtol ||b||, or when the true residual ||b - A x|| computed at
 *           the start of a cycle does.
 *   iters   (host, nullable) Arnoldi steps taken; relres (host, nullable)
 *           the last residual estimate (or cycle-start residual) / ||b||;
 *           history (nullable, device or host double[maxiter]) the estimate
 *           after each step (entries past *iters are left untouched).
 * b = 0 gives x = 0 and 0 steps.  Not converging within maxiter is not an
 * error (check relres).  Arrays may be host or device memory; the call
 * synchronises once per restart cycle and returns when done.  Errors:
 * SAM_ERR_INVALID_ARG, SAM_ERR_BAD_CSR (validated operators),
 * SAM_ERR_NONFINITE (NaN/Inf in b or in the iteration), SAM_ERR_OOM.
 * Workspace (handle's pool): (restart + 3) n + O(restart^2 + n restart / 256)
 * doubles.
 */
#define SAM_GMRES_MAX_RESTART 128
sam_status sam_gmres(sam_handle h, const sam_csr *A, const sam_csr *M, const sam_csr *P_0, const double *b, double *x,
                     int restart, int maxiter, double rtol, int32_t *iters, double *relres, double *history);

/*
 * sam_gmres_batched -- K independent solves A_k x_k = b_k of one order n
 * (a sequence of Sec. 2, each with its own map M_k and the one P_0 built for
 * A_0), by sam_gmres's algorithm, in the same launches: every system keeps
 * its own Krylov basis, Hessenberg matrix, step count and stopping test, and
 * drops out when it stops; the launches of a restart cycle cover all
 * systems.
 *   A[K]       system matrices; M (nullable) K maps; P_0 (nullable) shared.
 *   b, x       [K][n] (system k at k n); x holds x0_k on entry.
 *   iters, relres (host, nullable) [K]; history (nullable, device or host)
 *              [K][maxiter].
 * Same arguments, errors and synchronisation as sam_gmres otherwise.
 */
sam_status sam_gmres_batched(sam_handle h, int K, const sam_csr *A, const sam_csr *M, const sam_csr *P_0,
                             const double *b, double *x, int restart, int maxiter, double rtol, int32_t *iters,
                             double *relres, double *history);

/*
 * sam_build_backward -- adjoint of sam_build on a fixed pattern: gradients
 * with respect to the stored values of A_k and A_0 of
 *     L = <dM, M_k>  +  resid_weight * ||A_k M_k - A_0||_F^2,
 * where the first term stands for any loss whose gradient with respect to the
 * map values is dM_val (CSR order of the map, nnz(S) values; NULL = zero) and
 * the second is the residual of Eq. (res), differentiated directly (its
 * dependence through M_k is returned separately, see dM_resid).
 * Per column, with B = A_k(I_j, J_j), c = A_0(I_j, j), m the column of M_k,
 * r = c - B m, g = dM(J_j, j) and lambda = (B^T B)^{-1} g:
 *     dL/dB += r lambda^T - (B lambda) m^T - 2 w r m^T,
 *     dL/dc += B lambda + 2 w r,   dL/dA_0(i, j) += 2 w A_0(i, j) for rows
 *     i outside I_j  (w = resid_weight).
 * Entries of dL/dB at positions not stored in A_k are dropped; every stored
 * A_k entry receives the sum of its contributions from all columns, added
 * in a fixed order (deterministic).  lambda uses the recomputed QR (FP32 R
 * plus `refine_steps` FP64-residual corrections for SAM_FP32_REFINE), or the
 * forward build's R from a factor tape (sam_set_factor_tape).
 * dA_k_val[nnz(A_k)], dA_0_val[nnz(A_0)]: outputs in the CSR order of A_k
 * and A_0 (overwritten).  dM_resid (nullable, nnz(S), CSR order of the map):
 * receives w * d||A_k M - A_0||_F^2 / dM = -2 w A_k^T R on the pattern (zero
 * up to rounding at the least-squares solution).  M_val must be the map built
 * from the same A_k, A_0 and S.
 */
sam_status sam_build_backward(sam_handle h, const sam_csr *A_k, const sam_csr *A_0, sam_pattern S,
                              int precision, int refine_steps, const double *M_val,
                              const double *dM_val, double resid_weight, double *dA_k_val,
                              double *dA_0_val, double *dM_resid);

/*
 * sam_build_backward_batched -- sam_build_backward for K maps in one pass,
 * map k built from A_k[k] against its own target A_0[k] on S[k] (pass the
 * same A_0 K times for a shared target; its gradient is then returned per
 * map).  M_offsets[K+1] (host): offsets of each map's values in M_val,
 * dM_val and dM_resid (concatenated CSR orders, as sam_build_multi writes
 * them).  dA_k_val: the K gradients concatenated in the order of A_k
 * (sum of nnz(A_k[k]) values); dA_0_val: likewise for A_0.
 */
sam_status sam_build_backward_batched(sam_handle h, int K, const sam_csr *A_k, const sam_csr *A_0,
                                      const sam_pattern *S, int precision, int refine_steps,
                                      const int64_t *M_offsets, const double *M_val,
                                      const double *dM_val, double resid_weight, double *dA_k_val,
                                      double *dA_0_val, double *dM_resid);

/*
 * Factor tape (no counterpart in the paper): the adjoint of a build needs
 * the triangular factor R of every column problem, which it otherwise
 * recomputes (gathering B_j into a tile and running the QR again, about a
 * quarter of an adjoint's time).  A caller that runs the adjoint after the
 * build (reverse-mode training) can keep the build's factors instead:
 *
 *   sam_factor_tape_bytes(h, K, S, precision, &bytes);   allocate bytes
 *   sam_set_factor_tape(h, SAM_TAPE_RECORD, buf, bytes);
 *   sam_build_batched(h, K, A_k, A_0, S, precision, ...);  (writes R)
 *   sam_set_factor_tape(h, SAM_TAPE_REPLAY, buf, bytes);
 *   sam_build_backward_batched(h, K, A_k, A_0s, S, precision, ...);
 *   sam_set_factor_tape(h, SAM_TAPE_OFF, NULL, 0);
 *
 * The tape holds, per column j of the batch with |J_j| <= 27, the packed
 * upper triangle of R in the build's arithmetic type (FP32 for
 * SAM_FP32_REFINE, FP64 for SAM_FP64), rows in order, each from its
 * diagonal, in a slot of |J_j| (|J_j| + 1) / 2 elements rounded up to a
 * multiple of four; slots follow the columns of the batch in order (map k's
 * columns after map k-1's).  Columns with more than 27 unknowns have no slot
 * and columns of the large class (sam_size_classes) write nothing: their
 * adjoint always factors B again (in FP64), as do the two smallest classes,
 * whose QR costs less than reading the tape.
 *
 * sam_factor_tape_bytes -- bytes of the tape of the K maps on patterns S
 * (one slot per column of each pattern) at `precision`.  Synchronises.
 *
 * sam_set_factor_tape -- mode SAM_TAPE_RECORD: later builds on the handle
 * (sam_build, sam_build_batched, sam_build_multi; not captured plans, not
 * sam_tune's trial builds) write their columns' R into buf;
 * SAM_TAPE_REPLAY: later adjoints (sam_build_backward,
 * sam_build_backward_batched) read R from buf instead of recomputing it;
 * SAM_TAPE_OFF: neither (buf and bytes ignored).  buf: device memory of the
 * handle's device, 16-byte aligned, owned by the caller and kept alive while
 * the mode is set.  A replaying adjoint must see the same K, sources,
 * patterns, precision and tile variants as the recording build (as M_val
 * must be the build's map).  The adjoint recomputes R with the default tile
 * shapes (variant 0); for a build with those shapes, replaying the tape
 * gives the recomputing adjoint's results bit for bit, and otherwise
 * results that differ in rounding only.  Errors: SAM_ERR_INVALID_ARG for a bad
 * mode or buffer; a build or adjoint whose tape needs more than `bytes`
 * returns SAM_ERR_INVALID_ARG before launching its solves (each of them
 * synchronises once to size the tape).
 */
enum { SAM_TAPE_OFF = 0, SAM_TAPE_RECORD = 1, SAM_TAPE_REPLAY = 2 };
sam_status sam_factor_tape_bytes(sam_handle h, int K, const sam_pattern *S, int precision, int64_t *bytes);
sam_status sam_set_factor_tape(sam_handle h, int mode, void *buf, int64_t bytes);

/*
 * sam_tune -- autotuner (no counterpart in the paper, which fixes one kernel
 * shape).  It chooses, for SAM_FP32_REFINE builds on this handle:
 *  - the register tile shape of each size class (variant 0: the default;
 *    variant 1: one problem per 8 or 32 lanes with fewer register slots per
 *    lane), and
 *  - the bin schedule: which size class solves the columns of each natural
 *    class (sam_set_bin_schedule); a small class can hand its columns to the
 *    next larger register class, saving its launch and filling the larger
 *    class's persistent wave.
 * The call runs the complete batched build of the given problems (as
 * sam_build_batched, outputs to workspace it frees): once to count the
 * columns of every natural size class, then per variant and per candidate
 * schedule one warm-up and three builds, timing every size class's
 * least-squares launches with CUDA events.  The fastest variant per class
 * is kept; then, from the smallest class up, folding a class into the next
 * is kept when the summed launch time drops by 1% or more.  Results of every
 * choice satisfy the same accuracy bounds (they differ only in rounding).
 * cache_path (nullable): a text file with one line per tuned family, keyed by
 * device name, SM count, K, n, total nnz(S), precision, refine_steps and the
 * histogram of natural size classes (two families of equal sizes but
 * different column sizes get their own lines); a matching line is used
 * without timing, and a new choice is appended.  SAM_FP64 has one shape per
 * class: returns SAM_OK at once.  Synchronises the handle's stream.  Tracing
 * counters of the handle are left as they were.  Errors: those of
 * sam_build_batched; SAM_ERR_INVALID_ARG if cache_path cannot be opened for
 * appending.
 */
sam_status sam_tune(sam_handle h, int K, const sam_csr *A_k, const sam_csr *A_0, const sam_pattern *S,
                    int precision, int refine_steps, const char *cache_path);

/*
 * sam_set_tile_variants / sam_get_tile_variants -- set or read the tile
 * variant per size class (count must be SAM_NUM_SIZE_CLASSES; variant 0 for
 * every class is the default of a new handle; classes 0 and 5 have only
 * variant 0).  Set: returns
 * SAM_ERR_INVALID_ARG, changing nothing, if a value is out of range.
 */
sam_status sam_set_tile_variants(sam_handle h, const int *variants, int count);
sam_status sam_get_tile_variants(sam_handle h, int *variants, int count);

/*
 * sam_set_bin_schedule / sam_get_bin_schedule -- the size class that solves
 * the columns of each natural size class b (the first class they fit, see
 * sam_size_classes): to[b] in [b, 4] for the register classes b = 0..4
 * (a larger register tile always holds a smaller class's columns), to[5] = 5
 * (count must be SAM_NUM_SIZE_CLASSES).  A new handle has to[b] = b;
 * sam_tune chooses one.  Applies to later builds, plans and adjoints on the
 * handle.  Set: returns SAM_ERR_INVALID_ARG, changing nothing, if an entry is
 * out of range.
 */
sam_status sam_set_bin_schedule(sam_handle h, const int *to, int count);
sam_status sam_get_bin_schedule(sam_handle h, int *to, int count);

/*
 * sam_refine_stats -- outcome counts of the last guarded SAM_FP32_REFINE
 * build on this handle (refine_steps = SAM_REFINE_AUTO or >= 1):
 * counts[0] columns that kept their solution after one step, counts[1]
 * after two or more, counts[2] re-solved in FP64 after missing the target
 * (count must be 3).
 * Synchronises the handle's stream.
 */
sam_status sam_refine_stats(sam_handle h, int64_t *counts, int count);

/*
 * sam_profile -- tracing.  enable != 0 starts timing every least-squares
 * launch (one per size class and build call) with CUDA events recorded on
 * the handle's stream; any call resets the counters.
 * sam_profile_read -- launches: kernels this handle launched since the last
 * reset; lsq_ms / lsq_launches (nullable, SAM_NUM_SIZE_CLASSES entries):
 * accumulated event time and launch count of the least-squares kernel of
 * each size class.  Synchronises.
 */
sam_status sam_profile(sam_handle h, int enable);
sam_status sam_profile_read(sam_handle h, int64_t *launches, double *lsq_ms, int64_t *lsq_launches);

/*
 * sam_peak_flops -- measured FP32 and FP64 FMA throughput of this GPU in
 * FLOP/s (2 flops per FMA), from dependent-chain FMA kernels filling every
 * SM for about `ms` milliseconds each.  Used as roofline denominators.
 */
sam_status sam_peak_flops(sam_handle h, double ms, double *fp32_flops, double *fp64_flops);

/*
 * sam_residual_static -- the same two numbers as sam_residual,
 * ||A_k M_k - A_0||_F and ||A_k M_k - A_0||_F / ||A_0||_F, for callers that
 * cannot allocate device memory.  The paper has no counterpart: this is an
 * interface choice of the library.
 *
 * Who needs it: code that may not call cudaMalloc or any allocating routine
 * -- a step running while the device memory budget is already handed out,
 * a caller whose memory belongs to another framework's caching allocator,
 * or an environment that only lends the library device buffers.
 * sam_residual allocates its workspace from a handle's memory pool; this
 * entry point takes no handle and allocates nothing.  Its workspace is one
 * file-scope device array of fixed size (about 4.2 MB: one double per row
 * for up to SAM_STATIC_MAX_ROWS rows, plus reduction partials and a status
 * word) that every GPU which loads the library holds until the process
 * exits.
 *
 * Arguments: cuda_stream (a cudaStream_t, NULL for the legacy stream); A_k,
 * M_k, A_0 square CSR matrices of the same order n, 1 <= n <=
 * SAM_STATIC_MAX_ROWS (n = 0 is SAM_ERR_INVALID_ARG, as for every call);
 * out (device, 2 doubles) receives ||R||_F and ||R||_F / ||A_0||_F; status
 * (device, nullable) receives 0 or a sam_status detected on the device
 * (SAM_ERR_BAD_CSR for a malformed structure, SAM_ERR_UNSUPPORTED for a row
 * of R with more than 1024 candidate entries), in which case both outputs
 * are NaN.  Every array must be device memory of the current device, or
 * managed memory: host arrays and arrays of another device are rejected
 * (SAM_ERR_INVALID_ARG), as are orders above SAM_STATIC_MAX_ROWS.
 * The call is asynchronous on cuda_stream.  It looks up the workspace's
 * device address (cudaGetSymbolAddress, which allocates nothing) on every
 * call made while cuda_stream is not being captured, and reuses the
 * address found last on that device while it is; so make the first call
 * on a device before capturing a stream into a CUDA graph (a first call
 * under capture returns SAM_ERR_CUDA).
 * Every call reuses the same workspace and clears what must start at zero,
 * so a call never depends on an earlier one; calls whose work overlaps on
 * the GPU (other streams or host threads) race on the workspace and must be
 * serialised by the caller.
 */
#define SAM_STATIC_MAX_ROWS (1 << 19)
sam_status sam_residual_static(void *cuda_stream, const sam_csr *A_k, const sam_csr *M_k, const sam_csr *A_0,
                               double *out, int32_t *status);

#ifdef __cplusplus
}
#endif

#endif /* SAM_H */
