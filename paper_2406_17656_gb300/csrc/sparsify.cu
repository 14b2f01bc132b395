// sparsify.cu -- the sparsifications of A_k of arXiv 2406.17656 Sec. 4 that
// produce the matrix A~_k whose level-L pattern serves as the map's pattern:
//   global threshold  keep (i, j) if i = j or |A_ij| / sqrt(D_ii D_jj) > thresh,
//                     D_ii = |A_ii| when stored and nonzero, else 1 (the
//                     printed D^{1/2} A D^{1/2} read as the symmetric scaling
//                     D^{-1/2} A D^{-1/2});
//   column tau        keep (i, j) if i = j or |A_ij| > (1 - tau) max_i |A_ij|;
//   lfil              keep the lfil entries of each column with the largest
//                     |A_ij| (equal magnitudes: lower row first), and i = j.
// Every decision is one FP64 comparison of the same expression on the same
// inputs, so the kept structure is bit-exact.  The kept entries are written
// compactly in CSR order.
#include "common.cuh"

namespace sam {
namespace {

__device__ __forceinline__ int lower_bound_row(const int32_t *a, int len, int key) {
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// one warp per column of the CSC (cp, ri, cv): the rank of an entry is the
// number of entries before it in the order (larger |value|, then lower row)
__global__ void keep_lfil_kernel(int n, const int32_t *cp, const int32_t *ri, const double *cv, const int32_t *perm,
                                 int lfil, uint8_t *keep) {
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    const int b = cp[j], len = cp[j + 1] - b;
    for (int p = lane; p < len; p += 32) {
        const double a = fabs(cv[b + p]);
        const int r = ri[b + p];
        int rank = 0;
        for (int q = 0; q < len && rank < lfil; ++q) {
            const double aq = fabs(cv[b + q]);
            rank += (aq > a || (aq == a && ri[b + q] < r)) ? 1 : 0;
        }
        keep[perm[b + p]] = (uint8_t)((r == (int)j) || rank < lfil);
    }
}

__global__ void count_kept_kernel(int n, const int32_t *rp, const uint8_t *keep, int32_t *cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) c += keep[e];
    cnt[i] = c;
}

__global__ void fill_kept_kernel(int n, const int32_t *rp, const int32_t *ci, const double *v, const uint8_t *keep,
                                 const int32_t *orp, int32_t *oci, double *ov) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int o = orp[i];
    for (int e = rp[i]; e < rp[i + 1]; ++e)
        if (keep[e]) {
            oci[o] = ci[e];
            if (ov) ov[o] = v[e];
            ++o;
        }
}

// ---- row-wise sparsifications of K matrices of order n, read in place
// through a table (map k's entries at offsets off[k] .. of the batch; its
// rows and columns numbered within the map; per-map arrays [K][n])

// D_ii: |A_ii| when the diagonal is stored and nonzero, else 1
__global__ void diag_scale_batch_kernel(const CsrPtrs *mats, int n, double *d) {
    const int k = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t *rp = mats[k].rp, *ci = mats[k].ci;
    const double *v = mats[k].v;
    const int b = rp[i], len = rp[i + 1] - b;
    const int q = lower_bound_row(ci + b, len, i);
    double di = 1.0;
    if (q < len && ci[b + q] == i && fabs(v[b + q]) > 0.0) di = fabs(v[b + q]);
    d[(int64_t)k * n + i] = di;
}

// column maxima of |A| as the bit patterns of non-negative doubles (which
// order like the numbers)
__global__ void col_max_batch_kernel(const CsrPtrs *mats, const int64_t *off, int n, unsigned long long *cmax) {
    const int k = blockIdx.y;
    const int64_t nnz = off[k + 1] - off[k];
    const int32_t *ci = mats[k].ci;
    const double *v = mats[k].v;
    unsigned long long *cm = cmax + (int64_t)k * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicMax(&cm[ci[e]], (unsigned long long)__double_as_longlong(fabs(v[e])));
}

// keep flags (global threshold: i = j or |A_ij| / sqrt(D_ii D_jj) > thresh;
// column tau: i = j or |A_ij| > (1 - tau) max_i |A_ij|) and each row's kept
// count; rows are short, so one thread walks a row
__global__ void keep_count_batch_kernel(const CsrPtrs *mats, const int64_t *off, int n, int mode, double param,
                                        const double *d, const unsigned long long *cmax, uint8_t *keep,
                                        int32_t *cnt) {
    const int k = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t *rp = mats[k].rp, *ci = mats[k].ci;
    const double *v = mats[k].v;
    const int64_t base = (int64_t)k * n;
    uint8_t *kp = keep + off[k];
    int c = 0;
    if (mode == 0) {
        const double di = d[base + i];
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const int j = ci[e];
            const uint8_t f = (uint8_t)((j == i) || (fabs(v[e]) / sqrt(di * d[base + j]) > param));
            kp[e] = f;
            c += f;
        }
    } else {
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const int j = ci[e];
            const double mx = __longlong_as_double((long long)cmax[base + j]);
            const uint8_t f = (uint8_t)((j == i) || (fabs(v[e]) > (1.0 - param) * mx));
            kp[e] = f;
            c += f;
        }
    }
    cnt[base + i] = c;
}

// the kept entries of row i of map k, in order, at orp[k n + i] of the
// batch's output (column indices in the map's own numbering); rows are
// short, so one thread walks a row
__global__ void fill_kept_batch_kernel(const CsrPtrs *mats, const int64_t *off, int n, const uint8_t *keep,
                                       const int32_t *orp, int32_t *oci, double *ov) {
    const int k = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t *rp = mats[k].rp, *ci = mats[k].ci;
    const double *v = mats[k].v;
    const uint8_t *kp = keep + off[k];
    int o = orp[(int64_t)k * n + i];
    for (int e = rp[i]; e < rp[i + 1]; ++e)
        if (kp[e]) {
            oci[o] = ci[e];
            if (ov) ov[o] = v[e];
            ++o;
        }
}

// map k's row pointers relative to its own offset, and the offsets
__global__ void kept_rows_kernel(int K, int n, const int32_t *orp, int32_t *out_rp, int64_t *koff) {
    const int k = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    const int64_t base = (int64_t)k * n;
    const int32_t o0 = orp[base];
    out_rp[(int64_t)k * (n + 1) + i] = orp[base + i] - o0;
    if (i == 0) {
        koff[k] = o0;
        if (k == K - 1) koff[K] = orp[(int64_t)K * n];
    }
}

}  // namespace

cudaError_t sparsify_rows_batched(sam_handle h, int K, int n, const CsrPtrs *mats, const int64_t *off, int64_t tot,
                                  int mode, double param, uint8_t *keep, int32_t *cnt, int32_t *orp,
                                  int32_t *out_rp, int32_t *out_ci, double *out_v, int64_t *koff) {
    cudaStream_t st = handle_stream(h);
    const int64_t N = (int64_t)K * n;
    if (K < 1 || n < 1) return cudaErrorInvalidValue;
    double *d = nullptr;
    unsigned long long *cmax = nullptr;
    if (mode == 0) {
        d = (double *)pool_alloc(h, sizeof(double) * (size_t)N);
        if (!d) return cudaErrorMemoryAllocation;
        diag_scale_batch_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)K), 256, 0, st>>>(mats, n, d);
        count_launch(h);
    } else {
        cmax = (unsigned long long *)pool_alloc(h, sizeof(unsigned long long) * (size_t)N);
        if (!cmax) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaMemsetAsync(cmax, 0, sizeof(unsigned long long) * (size_t)N, st);
        if (e != cudaSuccess) return e;
        int64_t bx = (tot / K + 255) / 256 + 1;
        const int64_t cap = (int64_t)handle_sms(h) * 8 / K + 1;
        if (bx > cap) bx = cap;
        col_max_batch_kernel<<<dim3((unsigned)bx, (unsigned)K), 256, 0, st>>>(mats, off, n, cmax);
        count_launch(h);
    }
    const unsigned rows1 = (unsigned)((n + 255) / 256);
    keep_count_batch_kernel<<<dim3(rows1, (unsigned)K), 256, 0, st>>>(mats, off, n, mode, param, d, cmax, keep, cnt);
    count_launch(h);
    pool_free(h, d);
    pool_free(h, cmax);
    cudaError_t e = exclusive_scan_i32(h, cnt, orp, N);
    if (e != cudaSuccess) return e;
    fill_kept_batch_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)K), 256, 0, st>>>(mats, off, n, keep, orp,
                                                                                           out_ci, out_v);
    kept_rows_kernel<<<dim3((unsigned)((n + 1 + 255) / 256), (unsigned)K), 256, 0, st>>>(K, n, orp, out_rp, koff);
    count_launch(h, 2);
    return cudaGetLastError();
}

cudaError_t sparsify_keep(sam_handle h, int n, int64_t nnz, const int32_t *rp, const int32_t *ci, const double *v,
                          int mode, double param, uint8_t *keep) {
    cudaStream_t st = handle_stream(h);
    if (n == 0 || nnz == 0) return cudaSuccess;
    if (mode != 2) return cudaErrorInvalidValue;  // the row-wise criteria: sparsify_rows_batched
    // lfil: rank within the columns of the transpose
    int32_t *cp = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)n + 1));
    int32_t *ri = (int32_t *)pool_alloc(h, sizeof(int32_t) * (size_t)nnz);
    double *cv = (double *)pool_alloc(h, sizeof(double) * (size_t)nnz);
    int32_t *perm = (int32_t *)pool_alloc(h, sizeof(int32_t) * (size_t)nnz);
    cudaError_t e = cudaErrorMemoryAllocation;
    if (cp && ri && cv && perm) {
        e = csr_to_csc(h, n, nnz, rp, ci, v, cp, ri, cv, perm);
        if (e == cudaSuccess) {
            const int64_t threads = (int64_t)n * 32;
            const int lfil = param < 0.0 ? 0 : (param > 1e9 ? 1000000000 : (int)param);
            keep_lfil_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(n, cp, ri, cv, perm, lfil, keep);
            count_launch(h);
            e = cudaGetLastError();
        }
    }
    pool_free(h, cp);
    pool_free(h, ri);
    pool_free(h, cv);
    pool_free(h, perm);
    return e;
}

cudaError_t compact_kept(sam_handle h, int n, const int32_t *rp, const int32_t *ci, const double *v,
                         const uint8_t *keep, int32_t *cnt, int32_t *orp, int32_t *oci, double *ov) {
    cudaStream_t st = handle_stream(h);
    if (n == 0) return cudaMemsetAsync(orp, 0, sizeof(int32_t), st);
    count_kept_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, rp, keep, cnt);
    count_launch(h);
    cudaError_t e = exclusive_scan_i32(h, cnt, orp, n);
    if (e != cudaSuccess) return e;
    fill_kept_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, rp, ci, v, keep, orp, oci, ov);
    count_launch(h);
    return cudaGetLastError();
}

}  // namespace sam
