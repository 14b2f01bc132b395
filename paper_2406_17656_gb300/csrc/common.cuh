// common.cuh -- internal declarations shared by the libsam translation units.
//
// Layout conventions (device memory):
//   * A batch of K maps of order n is handled as ONE block-diagonal problem
//     of order N = K n: map k's rows and columns are [k n, (k+1) n) of the
//     "big" arrays.  Source matrices enter as CSR and are concatenated into
//     the block-diagonal CSR, then transposed once into CSC
//     (cp i32[N+1], ri i32[nnz], cv f64[nnz]) because the kernels read columns.
//   * A map pattern is stored in CSC: column j has rows J_j (ascending).  The
//     CSR structure of the map (its transpose) is kept alongside, with
//     csr_pos[e] = CSR position of CSC entry e.
//   * Shadow rows I_j are stored padded: ish[j * kICap + t], t < icnt[j].
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/sam.h"

namespace sam {

// Limits of the register-tile least-squares kernels (size classes 0..4).
constexpr int kICap = 64;    // max |I_j| (shadow rows) of one column problem
constexpr int kJCap = 27;    // max |J_j| (unknowns) of one column problem
constexpr int kRegBins = 5;  // register-tile size classes (see lsq.cu)
constexpr int kLCap = 512;   // max stored entries of one column's B (8 per shadow row)
// The large class (lsq_big.cu): one thread block per column, [B c] as a
// dense tile in shared memory (FP64, or FP32 for FP32 + refinement builds).
constexpr int kBinBig = kRegBins;  // its size-class index
constexpr int kNumBins = kRegBins + 1;
constexpr int kBigJCap = 128;                  // max |J_j|
constexpr int kBigICap = 1024;                 // max |I_j|
constexpr int kBigLCap = 16384;                // max stored entries of B_j
constexpr int kBigTileDoubles = 23 * 1024;     // max |I_j| (|J_j| + 1) (184 KB)
constexpr int kZCap = 32;    // target entries per column with a precomputed local row (zloc)
constexpr int kZOutside = 255;  // zloc value of a target entry outside the shadow rows
constexpr int kBinNone = 255;

// Per-column status codes written by the kernels (0 = ok); equal to the
// public sam_status values so the host can return them unchanged.
constexpr int kStOk = SAM_OK;
constexpr int kStRank = SAM_ERR_RANK_DEFICIENT;
constexpr int kStNonfinite = SAM_ERR_NONFINITE;
constexpr int kStUnsupported = SAM_ERR_UNSUPPORTED;
// internal: the FP32 solve missed the accuracy target; the FP64 kernel
// re-solves the column (never left in a status array)
constexpr int kStRefine = 100;
// internal: automatic refinement asks for a second step; a launch with two
// steps solves the column again (never left in a status array)
constexpr int kStStep2 = 101;
// automatic refinement (refine_steps = SAM_REFINE_AUTO)
constexpr int kAutoSteps = 2;
constexpr double kAutoC = 4.0, kAutoTol = 1e-12, kFallbackTol = 1e-10;
constexpr double kU32 = 5.9604644775390625e-8;  // unit roundoff of FP32, 2^-24
// the refinement guard's factor on u_32 kappa^2, kappa estimated from the R
// diagonal (which can fall short of kappa(B) several times on P1 FEM columns)
constexpr double kRhoSafety = 8.0;
constexpr double kNoise2 = 1e-28;  // |d|^2 / |m|^2 below which a correction is rounding noise of the FP64 residual

// Factor tape (sam_set_factor_tape): a build on a recording handle writes
// every register-class column's triangular factor R; an adjoint on a
// replaying handle reads it instead of gathering B into a tile and
// factoring it again.  Column j's R is stored packed (row k from its
// diagonal, rows in order, in the tile's type) at element fac_off[j], in a
// slot of tape_elems(|J_j|) elements (a multiple of four: 16-byte aligned).
constexpr int kTapeOff = 0, kTapeRecord = 1, kTapeReplay = 2;
__host__ __device__ __forceinline__ int64_t tape_elems(int nJ) {
    return (nJ >= 1 && nJ <= kJCap) ? (((int64_t)nJ * (nJ + 1) / 2 + 3) & ~(int64_t)3) : 0;
}

// Source CSR of one map (device pointers) for the batch concatenation.
struct CsrPtrs {
    const int32_t *rp;
    const int32_t *ci;
    const double *v;
};

// Arguments of the least-squares launches (all device pointers, big arrays).
struct LsqArgs {
    int n;                       // order of one map (A_0)
    const int32_t *kcp, *kri;    // CSC of the block-diagonal source
    const double *kcv;
    const float *kcv32;          // the same values rounded to FP32 (FP32 tiles)
    const int32_t *jcp, *jri;    // pattern (CSC, big)
    const int32_t *ish, *icnt;   // shadow rows (padded) and counts
    const uint8_t *lrow;         // local shadow row of every gathered entry (padded [N][kLCap])
    const uint8_t *zloc;         // local shadow row of the first kZCap entries of each column's target
                                 // column ([N][kZCap], kZOutside = not a shadow row); the shadow rows
                                 // (ish) are stored only for columns with more target entries
    const int32_t *zcp, *zri;    // CSC of the target: A_0 (order n, shared by every map; zbig = 0)
                                 // or the block-diagonal of one target per map (order N; zbig = 1)
    const double *zcv;
    const float *zcv32;          // the same values rounded to FP32
    int shadow_shared;           // 1: every map has the same source, target and pattern structure, and
                                 // ish / lrow / zloc hold map 0's columns only (indexed by the column
                                 // within its map); 0: one entry per column of the batch
    int64_t map_nnz_src;         // shadow_shared: stored entries of one source map and of one map
    int64_t map_nnz_pat;         // pattern; map k's pattern and source metadata are map 0's, read
                                 // at the same addresses for every map, plus k times these
    const int32_t *csr_pos;      // pattern CSC entry -> map CSR position
    double *mval;                // map values, CSR order of the block-diagonal map
    double *colres;              // per-column residual^2 (+ out-of-shadow part)
    int32_t *colstat;            // per-column status
    const int32_t *work;         // columns grouped by size class
    const int32_t *bin_off;      // [kNumBins+1] offsets into work
    int item_lo, item_hi;        // item_hi > 0: only items [item_lo, item_hi) of the launched class
    int refine_steps;            // < 0: automatic (up to kAutoSteps, FP64 fallback)
    uint8_t *refine_used;        // automatic mode: steps taken per column, kAutoSteps+1 = FP64 fallback
    int zbig;                    // 1: one target per map, stored block-diagonally
    // adjoint
    const double *dmval;         // dL/dM, CSR order (nullable)
    double resid_weight;         // weight of ||A_k M - A_0||_F^2 in the loss
    double *dB;                  // per-column dL/dB entries (gather order)
    const int64_t *dB_off;       // [N+1] offsets of each column's entries in dB
    double *dzval;               // dL/dA_0 contributions: CSC(A_0) order per map [K][nnz(A_0)] (zbig = 0)
                                 // or the CSC order of the block-diagonal targets (zbig = 1)
    double *dmres;               // dL/dM direct residual part, map CSR order (nullable)
    int64_t *dbase;              // per pattern entry (map CSR order): offset of its column block in dB
    int64_t znnz;                // nnz(A_0)
    // factor tape: kTapeRecord (the least-squares kernels write R) or
    // kTapeReplay (the adjoint reads it); fac holds the tile's type
    void *fac;
    const int64_t *fac_off;      // [N+1] element offsets of the columns' slots
    int fac_mode;
};

// --------------------------------------------------------------- helpers

template <typename T>
__device__ __forceinline__ T shfl_xor(T v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
template <typename T>
__device__ __forceinline__ T shfl(T v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// ------------------------------------------------------- host-side helpers
// (all asynchronous on the handle's stream unless noted)

// Scratch memory from the handle's stream-ordered pool.
void *pool_alloc(sam_handle h, size_t bytes);
void pool_free(sam_handle h, void *p);
cudaStream_t handle_stream(sam_handle h);
int handle_sms(sam_handle h);
int32_t *handle_flag(sam_handle h);  // device int32 error word (sticky)
// tracing: count kernel launches; time least-squares launches when enabled
void count_launch(sam_handle h, int n = 1);
void profile_begin(sam_handle h, int bin);
void profile_end(sam_handle h, int bin);
// FP32 tile shape of a size class chosen by sam_tune (0: two problems per
// warp where the tile allows, 1: the alternative shape)
int handle_variant(sam_handle h, int bin);
// Bin schedule: the size class that solves the columns of each natural size
// class (the first class they fit); a class may hand its columns to a larger
// register-tile class (to[b] in [b, kRegBins - 1]); the large class keeps its own
struct BinSchedule {
    uint8_t to[kNumBins];
};
BinSchedule handle_schedule(sam_handle h);
// number of FP32 tile shapes per size class
constexpr int kTileVariants[kNumBins] = {1, 2, 2, 2, 2, 1};

// out[0..n] = exclusive scan of in[0..n), out[n] = total
cudaError_t exclusive_scan_i32(sam_handle h, const int32_t *in, int32_t *out, int64_t n);
cudaError_t exclusive_scan_i64(sam_handle h, const int64_t *in, int64_t *out, int64_t n);

// CSR structure checks of K matrices of order n; sets *flag to SAM_ERR_BAD_CSR
// on any violation.  mats/nnz are device arrays of K entries; asym[k] and
// maxrow[k] (nullable, zeroed by the caller) receive "not structurally
// symmetric" and the longest row of matrix k.
cudaError_t validate_csr_batch(sam_handle h, int K, int n, const CsrPtrs *mats, const int64_t *nnz, int32_t *flag,
                               int32_t *asym = nullptr, int32_t *maxrow = nullptr);

// Concatenate K CSR matrices of order n into the block-diagonal CSR of order
// K n.  nnz_off (device, [K+1]) = prefix of the nnz; values optional.
cudaError_t concat_block_diag(sam_handle h, int K, int n, const CsrPtrs *mats, const int64_t *nnz_off,
                              int32_t *rp, int32_t *ci, double *v);

// CSR -> CSC transpose with sorted rows per column.  perm (nullable) gets the
// CSR index of every CSC entry; val / cv may be null.  symmetric: the
// structure is known to be structurally symmetric (validated), so the CSC
// structure is a copy and values / perm come from a mirror lookup (no
// atomics, no sort).
cudaError_t csr_to_csc(sam_handle h, int n, int64_t nnz, const int32_t *rp, const int32_t *ci,
                       const double *val, int32_t *cp, int32_t *ri, double *cv, int32_t *perm,
                       bool symmetric = false);

// Level-L pattern (CSC) of the matrix with CSC structure (kcp, kri), order N.
// Allocates *jcp / *jri from the pool; synchronises to size the result (and
// reads the status word with it).  maxcol >= 0: no column of the matrix is
// longer, which bounds the level-2 and level-3 candidate lists and saves the
// synchronisation that sizes them.
sam_status level_pattern(sam_handle h, int N, const int32_t *kcp, const int32_t *kri, int64_t nnz, int level,
                         int32_t **jcp, int32_t **jri, int64_t *nnz_out, int maxcol = -1);

// The target of a shadow pass: zloc (nullable) receives the local row of
// every target entry (see LsqArgs::zloc)
struct ShadowTarget {
    const int32_t *zcp = nullptr, *zri = nullptr;
    int zbig = 0, n = 1;
    uint8_t *zloc = nullptr;
};
// Shadow rows (padded), |I_j| and size class of every column.
// nbcnt (nullable) receives nnz(B_j) = sum of |A(:, c)| over c in J_j;
// lrow (nullable, padded [N][kLCap]) the local shadow row of every entry of
// A(:, J_j) in gather order, for the columns that have a size class.
// With a target (tg.zloc), ish is written only for the columns whose target
// column has more than kZCap entries.
cudaError_t shadow_and_bins(sam_handle h, int N, const int32_t *kcp, const int32_t *kri, const int32_t *jcp,
                            const int32_t *jri, int32_t *ish, int32_t *icnt, uint8_t *bin, int32_t *colstat,
                            int64_t *nbcnt = nullptr, uint8_t *lrow = nullptr, ShadowTarget tg = ShadowTarget());

// Work list: columns grouped by size class; bin_off (device, [kNumBins+1]);
// ws (nullable): int32[2 kNumBins] workspace
cudaError_t build_work_list(sam_handle h, int N, const uint8_t *bin, int32_t *work, int32_t *bin_off,
                            int32_t *ws = nullptr);
// out[j] = bin[j] where colstat[j] == flag, else no size class
cudaError_t flagged_bins(sam_handle h, int N, const uint8_t *bin, const int32_t *colstat, int32_t flag, uint8_t *out);
// automatic refinement's two-step launch (refine_steps < 0): the size class of
// every column (bin), and workspace for the flagged columns' classes (bins2,
// uint8[N]), their work list (work, int32[N]), its offsets (bin_off,
// int32[kNumBins + 1]) and the list's counters (ws, int32[2 kNumBins])
struct RedoLists {
    const uint8_t *bin = nullptr;
    uint8_t *bins2 = nullptr;
    int32_t *work = nullptr, *bin_off = nullptr, *ws = nullptr;
};
// guarded refinement: in the automatic mode, the two-step solve of the columns
// that automatic refinement flagged (redo); then the FP64 re-solve of the
// columns the FP32 kernel flagged (list: int32[N] workspace, list_off:
// int32[2]), then the per-outcome column counts (counts[kAutoSteps + 1], nullable)
cudaError_t launch_refine_fallback(sam_handle h, const LsqArgs &args, int N, int32_t *list, int32_t *list_off,
                                   int64_t *counts, const RedoLists &redo = RedoLists());

// Least-squares launches for every size class.
cudaError_t launch_lsq(sam_handle h, int precision, const LsqArgs &args);
// the large class; profile: time it as size class `bin` with the handle's
// tracing events; fp32: FP32 tile and QR with the refinement steps of
// args.refine_steps (SAM_FP32_REFINE builds), else FP64 throughout
cudaError_t launch_lsq_big(sam_handle h, const LsqArgs &args, int bin, bool profile = true, bool fp32 = false);
// one size class (the items args.item_lo/item_hi select, else all of it)
cudaError_t launch_lsq_bin(sam_handle h, int precision, const LsqArgs &args, int bin);
// the FP64 register tiles of size classes 0-4 (lsq_fp64.cu)
cudaError_t launch_lsq_fp64_bin(sam_handle h, const LsqArgs &args, int bin);
cudaError_t launch_adjoint(sam_handle h, int precision, const LsqArgs &args);
// the adjoint of one register size class: FP32 tiles recomputing R
// (adjoint_f32.cu), and the lean shapes reading the factor tape, classes
// 2-4 (adjoint_tape.cu)
cudaError_t launch_adjoint_f32_bin(sam_handle h, const LsqArgs &args, int bin);
cudaError_t launch_adjoint_tape_bin(sam_handle h, int precision, const LsqArgs &args, int bin);
// the adjoint of the large class's columns (FP64, lsq_big.cu)
cudaError_t launch_adjoint_big(sam_handle h, const LsqArgs &args, int bin);
// dA(e) = sum over map entries t of row c(e): dB[dbase[t] + (e - kcp[c])], CSC order of A
cudaError_t adjoint_reduce(sam_handle h, int N, const int32_t *kcp, const int32_t *mrp, const int64_t *dbase,
                           const double *dB, double *dak_csc);
// out[i] = (float) in[i]
cudaError_t round_to_f32(sam_handle h, int64_t n, const double *in, float *out);
// factor tape slots: off[j] = sum over columns i < j of tape_elems(|J_i|),
// off[N] = the total (sizes: int64[N] workspace)
cudaError_t tape_offsets(sam_handle h, int64_t N, const int32_t *jcp, int64_t *sizes, int64_t *off);
// out[perm[p]] = in[p]
cudaError_t permute_scatter_f64(sam_handle h, int64_t nnz, const int32_t *perm, const double *in, double *out);

// Deterministic sums: out[k] = sum of x[k*seg .. (k+1)*seg) (squares optional).
cudaError_t segmented_sum_f64(sam_handle h, const double *x, int K, int64_t seg, double *out, bool squares,
                              double *work = nullptr);
// pos[q] = position of the mirror entry of CSR position q of a structurally
// symmetric matrix (the CSR position of A(ci[q], row of q))
cudaError_t mirror_positions(sam_handle h, int n, const int32_t *rp, const int32_t *ci, int32_t *pos);
// Sec. 4 sparsification by lfil (mode 2): keep[e] (one byte per stored
// entry); then the kept entries in CSR (cnt: int32[n] workspace).  The
// row-wise criteria (global threshold, column tau) are sparsify_rows_batched;
// mode 0 or 1 here is cudaErrorInvalidValue unless there is nothing to do.
cudaError_t sparsify_keep(sam_handle h, int n, int64_t nnz, const int32_t *rp, const int32_t *ci, const double *v,
                          int mode, double param, uint8_t *keep);
// Global threshold (mode 0) or column tau (mode 1) of K matrices of order n
// given by a device table (map k's entries at off[k] .. of the batch), in one
// pass without concatenating them: keep (tot flags), cnt and orp (K n + 1)
// are workspace; the kept entries of map k go to out_ci / out_v (nullable)
// at koff[k] in its own numbering, its row pointers to out_rp + k (n + 1)
// relative to koff[k]; koff has K + 1 entries.
cudaError_t sparsify_rows_batched(sam_handle h, int K, int n, const CsrPtrs *mats, const int64_t *off, int64_t tot,
                                  int mode, double param, uint8_t *keep, int32_t *cnt, int32_t *orp,
                                  int32_t *out_rp, int32_t *out_ci, double *out_v, int64_t *koff);
cudaError_t compact_kept(sam_handle h, int n, const int32_t *rp, const int32_t *ci, const double *v,
                         const uint8_t *keep, int32_t *cnt, int32_t *orp, int32_t *oci, double *ov);
// doubles of workspace segmented_sum_f64 needs for K segments
size_t segmented_sum_workspace(int K);
// K matrices of one structure: out[k m + q] = vals[k][perm[q]] (vals: device
// array of K value pointers; perm: the common CSC -> CSR positions)
cudaError_t gather_values_shared(sam_handle h, int64_t m, int K, const double *const *vals, const int32_t *perm,
                                 double *out);
// values of K matrices into the CSC order of their block-diagonal (+ FP32 copy)
cudaError_t gather_values(sam_handle h, int64_t tot, int K, const int64_t *off, const double *const *vals,
                          const int32_t *perm, double *v, float *v32);
cudaError_t sum_f64(sam_handle h, const double *x, int64_t n, double *out_dev, bool squares);
cudaError_t csr_spmv(sam_handle h, int n, const int32_t *rp, const int32_t *ci, const double *v, const double *x,
                     double *y);
// g[e] = dy[i] x[c] for every stored entry e = (i, c) of the CSR structure
cudaError_t csr_outer_on_pattern(sam_handle h, int n, const int32_t *rp, const int32_t *ci, const double *dy,
                                 const double *x, double *g);
cudaError_t residual_rows(sam_handle h, int n, const int32_t *krp, const int32_t *kci, const double *kv,
                          const int32_t *mrp, const int32_t *mci, const double *mv, const int32_t *zrp,
                          const int32_t *zci, const double *zv, double *row_r2, int32_t *flag);
cudaError_t status_reduce(sam_handle h, const int32_t *colstat, int64_t n, int32_t *flag);
cudaError_t peak_fma(sam_handle h, double ms, double *f32, double *f64);

// A CSR operator of a Krylov solve (device pointers; rp == nullptr: identity)
struct KryOp {
    int64_t nnz = 0;
    const int32_t *rp = nullptr, *ci = nullptr;
    const double *v = nullptr;
};
// Restarted GMRES(restart) for K systems A_k x_k = b_k of order n with the
// right preconditioners z = M_k (P v) (krylov.cu).  A[K], M[K] (nullable:
// identity) host tables of device operators, P shared (P.rp nullptr:
// identity); b, x device [K][n], x holding x0 on entry.  hist_dev
// (nullable, device double[K][maxiter]) receives the residual estimate /
// ||b_k|| of every step; its_out, rel_out host [K].  Synchronises once per
// restart cycle.
sam_status gmres_solve(sam_handle h, int K, int n, const KryOp *A, const KryOp *M, const KryOp &P, const double *b,
                       double *x, int restart, int maxiter, double rtol, double *hist_dev, int32_t *its_out,
                       double *rel_out, int64_t *launches_out);

// Split the block-diagonal map CSR into per-map CSR arrays (row pointers
// rebased to each map's offset, column indices shifted back by k n).
cudaError_t split_map_structure(sam_handle h, int K, int n, const int32_t *mrp_big, const int32_t *mci_big,
                                int32_t *rp_out, int32_t *ci_out);

}  // namespace sam
