// common.cuh -- internal declarations shared by the libsam translation units.
//
// Layout conventions (device memory):
//   * A matrix enters as CSR (row_ptr i32[n+1], col_idx i32[nnz], val f64[nnz]).
//     The kernels read it by columns, so every source matrix is transposed
//     once per call into CSC (cp i32[n+1], ri i32[nnz], cv f64[nnz]).
//   * A map pattern S is stored in CSC: column j of the map has rows J_j
//     (ascending).  The CSR structure of the map (its transpose) is kept
//     alongside with csr_pos[e] = CSR position of CSC entry e.
//   * Shadow rows I_j are stored padded: ish[j * kICap + t], t < icnt[j].
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/sam.h"

namespace sam {

// Hard limits of the least-squares kernels.
constexpr int kICap = 64;    // max |I_j| (shadow rows) of one column problem
constexpr int kJCap = 27;    // max |J_j| (unknowns) of one column problem
constexpr int kNumBins = 5;  // size classes (see lsq.cu)
constexpr int kBinNone = 255;

// Per-column status codes written by the kernels (0 = ok); equal to the
// public sam_status values so the host can return them unchanged.
constexpr int kStOk = SAM_OK;
constexpr int kStRank = SAM_ERR_RANK_DEFICIENT;
constexpr int kStNonfinite = SAM_ERR_NONFINITE;
constexpr int kStUnsupported = SAM_ERR_UNSUPPORTED;

struct Csc {
    int n = 0;
    int64_t nnz = 0;
    int32_t *cp = nullptr;  // [n+1]
    int32_t *ri = nullptr;  // [nnz]
    double *cv = nullptr;   // [nnz] (may be null for structure-only)
};

// Everything one map's least-squares launch needs (device pointers).
struct MapDev {
    const int32_t *kcp, *kri;  // CSC of A_k
    const double *kcv;
    const int32_t *jcp, *jri;  // pattern J (CSC)
    const int32_t *ish;        // shadow rows, padded [n][kICap]
    const int32_t *icnt;       // |I_j|
    const int32_t *csr_pos;    // CSC entry of the pattern -> CSR position of the map
    double *mval;              // map values, CSR order
    double *colres;            // per-column residual^2 (+ out-of-shadow part)
    int32_t *colstat;          // per-column status
    // adjoint only
    const double *dmval;       // dL/dM in CSR order
    double *dB;                // per-entry contributions (see adjoint.cu)
    const int64_t *dB_off;     // per-column offset into dB
    double *dzval;             // dL/dA_0 values in CSC(A_0) order
};

struct LsqArgs {
    const MapDev *maps;       // [K]
    const int32_t *zcp, *zri; // CSC of A_0 (shared by every map)
    const double *zcv;
    const int2 *work;         // (map, column) items of this size class
    const int32_t *work_count;// device scalar: number of items
    int32_t *ticket;          // device scalar: persistent-loop work counter (zeroed before launch)
    int refine_steps;
    int mode;                 // 0 forward, 1 adjoint
};

// --------------------------------------------------------------- helpers

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

template <typename T>
__device__ __forceinline__ T shfl_xor(T v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
template <typename T>
__device__ __forceinline__ T shfl(T v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// ------------------------------------------------------- host-side helpers
// (implemented in symbolic.cu; all asynchronous on `st`)

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

// out[0..n] = exclusive scan of in[0..n), out[n] = total (int32 and int64 variants)
cudaError_t exclusive_scan_i32(sam_handle h, const int32_t *in, int32_t *out, int64_t n);
cudaError_t exclusive_scan_i64(sam_handle h, const int64_t *in, int64_t *out, int64_t n);

// CSR structure checks; sets *flag to SAM_ERR_BAD_CSR on any violation.
cudaError_t validate_csr(sam_handle h, int n, int64_t nnz, const int32_t *rp, const int32_t *ci, int32_t *flag);

// CSR -> CSC transpose with sorted rows per column.  perm (nullable) gets the
// CSR index of every CSC entry; val / cv may be null.
cudaError_t csr_to_csc(sam_handle h, int n, int64_t nnz, const int32_t *rp, const int32_t *ci,
                       const double *val, int32_t *cp, int32_t *ri, double *cv, int32_t *perm);

// Level pattern (CSC) of A given by its CSC structure (kcp, kri).  Allocates
// *jcp / *jri from the pool; synchronises once to size the result.
sam_status level_pattern(sam_handle h, int n, const int32_t *kcp, const int32_t *kri, int level,
                         int32_t **jcp, int32_t **jri, int64_t *nnz_out);

// Batched variant: K structures, one synchronisation.
sam_status level_pattern_batched(sam_handle h, int K, int n, const int32_t *const *kcp,
                                 const int32_t *const *kri, int level, int32_t **jcp, int32_t **jri,
                                 int64_t *nnz_out);

// Shadow rows (padded) + size class of every column of one map.
cudaError_t shadow_and_bins(sam_handle h, int n, const int32_t *kcp, const int32_t *kri, const int32_t *jcp,
                            const int32_t *jri, int precision, int32_t *ish, int32_t *icnt, uint8_t *bin,
                            int32_t *colstat);

// Work lists: items (map, col) grouped by bin; bin_off (device, [kNumBins+1])
cudaError_t build_work_lists(sam_handle h, int K, int n, const uint8_t *const *bins_dev_of_map,
                             int2 *work, int32_t *bin_off);

// Least-squares launches for every size class over the work lists.
cudaError_t launch_lsq(sam_handle h, int precision, int refine_steps, int mode, const MapDev *maps_dev,
                       const int32_t *zcp, const int32_t *zri, const double *zcv, const int2 *work,
                       const int32_t *bin_off, int32_t *tickets);

// Deterministic sums.
cudaError_t sum_f64(sam_handle h, const double *x, int64_t n, double *out_dev, bool squares);
cudaError_t csr_spmv(sam_handle h, int n, const int32_t *rp, const int32_t *ci, const double *v, const double *x,
                     double *y);
cudaError_t residual_rows(sam_handle h, int n, const int32_t *krp, const int32_t *kci, const double *kv,
                          const int32_t *mrp, const int32_t *mci, const double *mv, const int32_t *zrp,
                          const int32_t *zci, const double *zv, double *row_r2, int32_t *flag);
cudaError_t status_reduce(sam_handle h, const int32_t *colstat, int64_t n, int32_t *flag);
cudaError_t peak_fma(sam_handle h, double ms, double *f32, double *f64);

}  // namespace sam
