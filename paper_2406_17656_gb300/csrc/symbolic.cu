// symbolic.cu -- integer (bit-exact) part of SAM construction:
//   * CSR validation and CSR -> CSC transposition,
//   * the level-L neighbour patterns of G(A) (Sec. 3 of arXiv 2406.17656):
//     level 1 = column pattern of A plus the diagonal, level L+1 = union of
//     the level-1 columns of every vertex in the level-L column (paths of
//     length <= L+1 pointing to j),
//   * shadow rows I_j = union of the row patterns of A(:, c), c in J_j (the
//     rows of the column least-squares problem of Sec. 2), and the size
//     class ("bin") of every column problem,
//   * the (map, column) work lists of each size class,
//   * exclusive scans used by all of the above.
// All kernels are bounded loops over their input; none waits on another
// block.  Errors are reported through an int32 flag word, never by trapping.
#include <climits>
#include <vector>

#include "common.cuh"

namespace sam {

// ------------------------------------------------------------------ scans

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T v, T *warp_tot, T *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : T(0);
        T wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = wi - w;
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    T r = warp_tot[warp] + incl - v;
    __syncthreads();
    return r;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_tile_sums(const T *in, int64_t n, T *sums) {
    __shared__ T wt[32];
    __shared__ T tot;
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q)
        if (base + q < n) s += in[base + q];
    block_exclusive_scan<T>(s, wt, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// single block: exclusive scan of the tile sums in place; total -> *grand
template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_spine(T *sums, int64_t nt, T *grand) {
    __shared__ T wt[32];
    __shared__ T tot;
    T carry = 0;
    for (int64_t b = 0; b < nt; b += kScanTile) {
        int64_t base = b + (int64_t)threadIdx.x * kScanItems;
        T loc[kScanItems];
        T s = 0;
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            loc[q] = (base + q < nt) ? sums[base + q] : T(0);
            s += loc[q];
        }
        T ex = block_exclusive_scan<T>(s, wt, &tot);
        T run = carry + ex;
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            if (base + q < nt) sums[base + q] = run;
            run += loc[q];
        }
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *grand = carry;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_apply(const T *in, T *out, int64_t n, const T *offs) {
    __shared__ T wt[32];
    __shared__ T tot;
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T loc[kScanItems];
    T s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        loc[q] = (base + q < n) ? in[base + q] : T(0);
        s += loc[q];
    }
    T run = block_exclusive_scan<T>(s, wt, &tot) + offs[blockIdx.x];
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        if (base + q < n) out[base + q] = run;
        run += loc[q];
    }
}

template <typename T>
__global__ void copy_scalar(const T *src, T *dst) { *dst = *src; }

template <typename T>
cudaError_t exclusive_scan_impl(sam_handle h, const T *in, T *out, int64_t n) {
    cudaStream_t st = handle_stream(h);
    int64_t nt = (n + kScanTile - 1) / kScanTile;
    if (nt == 0) return cudaMemsetAsync(out, 0, sizeof(T), st);
    T *sums = (T *)pool_alloc(h, sizeof(T) * (size_t)(nt + 1));
    if (!sums) return cudaErrorMemoryAllocation;
    scan_tile_sums<T><<<(unsigned)nt, kScanThreads, 0, st>>>(in, n, sums);
    count_launch(h);
    scan_spine<T><<<1, kScanThreads, 0, st>>>(sums, nt, sums + nt);
    count_launch(h);
    scan_apply<T><<<(unsigned)nt, kScanThreads, 0, st>>>(in, out, n, sums);
    count_launch(h);
    copy_scalar<T><<<1, 1, 0, st>>>(sums + nt, out + n);
    count_launch(h);
    pool_free(h, sums);
    return cudaGetLastError();
}

}  // namespace

cudaError_t exclusive_scan_i32(sam_handle h, const int32_t *in, int32_t *out, int64_t n) {
    return exclusive_scan_impl<int32_t>(h, in, out, n);
}
cudaError_t exclusive_scan_i64(sam_handle h, const int64_t *in, int64_t *out, int64_t n) {
    return exclusive_scan_impl<int64_t>(h, in, out, n);
}

// ------------------------------------------------------------- validation

namespace {
__global__ void validate_csr_kernel(int n, int64_t nnz, const int32_t *rp, const int32_t *ci, int32_t *flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && (rp[0] != 0 || (int64_t)rp[n] != nnz)) atomicCAS(flag, 0, SAM_ERR_BAD_CSR);
    if (i >= n) return;
    int b = rp[i], e = rp[i + 1];
    if (e < b || b < 0 || (int64_t)e > nnz) {
        atomicCAS(flag, 0, SAM_ERR_BAD_CSR);
        return;
    }
    int prev = -1;
    for (int t = b; t < e; ++t) {
        int c = ci[t];
        if (c <= prev || c >= n) {
            atomicCAS(flag, 0, SAM_ERR_BAD_CSR);
            return;
        }
        prev = c;
    }
}
}  // namespace

cudaError_t validate_csr(sam_handle h, int n, int64_t nnz, const int32_t *rp, const int32_t *ci, int32_t *flag) {
    int blocks = (n + 255) / 256;
    validate_csr_kernel<<<blocks > 0 ? blocks : 1, 256, 0, handle_stream(h)>>>(n, nnz, rp, ci, flag);
    count_launch(h);
    return cudaGetLastError();
}

// -------------------------------------------------------------- transpose

namespace {

__global__ void count_cols_kernel(int64_t nnz, const int32_t *ci, int32_t *cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[ci[e]], 1);
}

// one warp per row; positions claimed with atomics, ordered afterwards
__global__ void fill_cols_kernel(int n, const int32_t *rp, const int32_t *ci, const double *val, int32_t *cursor,
                                 int32_t *ri, double *cv, int32_t *perm) {
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= n) return;
    int row = (int)w;
    for (int e = rp[row] + lane; e < rp[row + 1]; e += 32) {
        int p = atomicAdd(&cursor[ci[e]], 1);
        ri[p] = row;
        if (cv) cv[p] = val[e];
        if (perm) perm[p] = e;
    }
}

// insertion sort of each column segment by row index (rows are unique)
__global__ void sort_cols_kernel(int n, const int32_t *cp, int32_t *ri, double *cv, int32_t *perm) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    int b = cp[c], e = cp[c + 1];
    for (int t = b + 1; t < e; ++t) {
        int key = ri[t];
        double kv = cv ? cv[t] : 0.0;
        int kp = perm ? perm[t] : 0;
        int s = t - 1;
        while (s >= b && ri[s] > key) {
            ri[s + 1] = ri[s];
            if (cv) cv[s + 1] = cv[s];
            if (perm) perm[s + 1] = perm[s];
            --s;
        }
        ri[s + 1] = key;
        if (cv) cv[s + 1] = kv;
        if (perm) perm[s + 1] = kp;
    }
}

}  // namespace

cudaError_t csr_to_csc(sam_handle h, int n, int64_t nnz, const int32_t *rp, const int32_t *ci, const double *val,
                       int32_t *cp, int32_t *ri, double *cv, int32_t *perm) {
    cudaStream_t st = handle_stream(h);
    int32_t *cnt = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)n + 1));
    if (!cnt) return cudaErrorMemoryAllocation;
    cudaError_t err = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)n + 1), st);
    if (err != cudaSuccess) return err;
    if (nnz > 0) {
        int64_t blocks = (nnz + 255) / 256;
        if (blocks > 65535 * 4) blocks = 65535 * 4;
        count_cols_kernel<<<(unsigned)blocks, 256, 0, st>>>(nnz, ci, cnt);
        count_launch(h);
    }
    err = exclusive_scan_i32(h, cnt, cp, n);
    if (err != cudaSuccess) return err;
    err = cudaMemcpyAsync(cnt, cp, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    if (err != cudaSuccess) return err;
    if (n > 0) {
        int64_t threads = (int64_t)n * 32;
        fill_cols_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(n, rp, ci, val, cnt, ri, cv, perm);
        count_launch(h);
        sort_cols_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, cp, ri, val ? cv : nullptr, perm);
        count_launch(h);
    }
    pool_free(h, cnt);
    return cudaGetLastError();
}

// ---------------------------------------------------------- level patterns

namespace {

// Level 0/1 columns: J_j = {j} (level 0) or rows of A(:, j) plus j (level 1).
__global__ void level01_count(int n, const int32_t *kcp, const int32_t *kri, int level, int32_t *cnt) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (level == 0) {
        cnt[j] = 1;
        return;
    }
    int b = kcp[j], e = kcp[j + 1], has = 0;
    for (int t = b; t < e; ++t) has |= (kri[t] == j);
    cnt[j] = e - b + (has ? 0 : 1);
}

__global__ void level01_fill(int n, const int32_t *kcp, const int32_t *kri, int level, const int32_t *jcp,
                             int32_t *jri) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int o = jcp[j];
    if (level == 0) {
        jri[o] = j;
        return;
    }
    int b = kcp[j], e = kcp[j + 1];
    bool placed = false;
    for (int t = b; t < e; ++t) {
        int r = kri[t];
        if (!placed && r >= j) {
            if (r != j) jri[o++] = j;
            placed = true;
        }
        jri[o++] = r;
    }
    if (!placed) jri[o++] = j;
}

constexpr int kMergeWarps = 4;
constexpr int kMergeBuf = 2048;  // candidate capacity per column (ints)

// Warp-cooperative sort + unique of buf[0..cnt), cnt <= kMergeBuf.  Returns
// the number of distinct values, left ascending in buf[0..u).
__device__ int warp_sort_unique(int *buf, int cnt) {
    const int lane = threadIdx.x & 31;
    int p2 = 32;
    while (p2 < cnt) p2 <<= 1;
    for (int i = cnt + lane; i < p2; i += 32) buf[i] = INT_MAX;
    __syncwarp();
    for (int k = 2; k <= p2; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = lane; i < p2; i += 32) {
                int ixj = i ^ jj;
                if (ixj > i) {
                    int a = buf[i], b = buf[ixj];
                    bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        buf[i] = b;
                        buf[ixj] = a;
                    }
                }
            }
            __syncwarp();
        }
    }
    int u = 0, prev_last = INT_MIN;
    for (int base = 0; base < cnt; base += 32) {
        int i = base + lane;
        int v = (i < cnt) ? buf[i] : INT_MAX;
        int left = __shfl_up_sync(0xffffffffu, v, 1);
        if (lane == 0) left = prev_last;
        bool first = (i < cnt) && (v != left);
        unsigned bal = __ballot_sync(0xffffffffu, first);
        prev_last = __shfl_sync(0xffffffffu, v, 31);
        __syncwarp();
        if (first) buf[u + __popc(bal & ((1u << lane) - 1u))] = v;
        u += __popc(bal);
        __syncwarp();
    }
    return u;
}

// Gather the candidate rows of column j: the concatenation of X(:, l) for l
// in Y(:, j).  Returns the candidate count (may exceed kMergeBuf, in which
// case the buffer content is incomplete).
__device__ int gather_candidates(int j, const int32_t *xcp, const int32_t *xri, const int32_t *ycp,
                                 const int32_t *yri, int *buf) {
    const int lane = threadIdx.x & 31;
    int yb = ycp[j], ye = ycp[j + 1];
    int total = 0;
    for (int base = yb; base < ye; base += 32) {
        int t = base + lane;
        int xb = 0, len = 0;
        if (t < ye) {
            int l = yri[t];
            xb = xcp[l];
            len = xcp[l + 1] - xb;
        }
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int off = total + incl - len;
        int chunk = __shfl_sync(0xffffffffu, incl, 31);
        if (off + len <= kMergeBuf)
            for (int q = 0; q < len; ++q) buf[off + q] = xri[xb + q];
        total += chunk;
    }
    __syncwarp();
    return total;
}

// mode 0: count distinct rows -> cnt[j] (-1 if the candidates overflow)
// mode 1: write the distinct rows to out[optr[j] ...]
__global__ void __launch_bounds__(kMergeWarps * 32) product_pattern_kernel(
    int n, const int32_t *xcp, const int32_t *xri, const int32_t *ycp, const int32_t *yri, int mode,
    int32_t *cnt, const int32_t *optr, int32_t *out, int32_t *flag) {
    __shared__ int bufs[kMergeWarps][kMergeBuf];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *buf = bufs[warp];
    for (int64_t j = (int64_t)blockIdx.x * kMergeWarps + warp; j < n; j += (int64_t)gridDim.x * kMergeWarps) {
        int total = gather_candidates((int)j, xcp, xri, ycp, yri, buf);
        if (total > kMergeBuf) {
            if (lane == 0) {
                if (mode == 0) cnt[j] = 0;
                atomicCAS(flag, 0, SAM_ERR_UNSUPPORTED);
            }
            continue;
        }
        int u = warp_sort_unique(buf, total);
        if (mode == 0) {
            if (lane == 0) cnt[j] = u;
        } else {
            int o = optr[j];
            for (int i = lane; i < u; i += 32) out[o + i] = buf[i];
        }
        __syncwarp();
    }
}

int merge_grid(sam_handle h, int n) {
    int blocks = (n + kMergeWarps - 1) / kMergeWarps;
    int cap = handle_sms(h) * 16;
    return blocks < cap ? (blocks > 0 ? blocks : 1) : cap;
}

}  // namespace

// Patterns for K structures at once; all count passes run before the single
// synchronisation that sizes the outputs.
sam_status level_pattern_batched(sam_handle h, int K, int n, const int32_t *const *kcp, const int32_t *const *kri,
                                 int level, int32_t **jcp, int32_t **jri, int64_t *nnz_out) {
    cudaStream_t st = handle_stream(h);
    int32_t *flag = handle_flag(h);
    int blocks = (n + 255) / 256;
    if (blocks < 1) blocks = 1;
    // level-1 (or 0) patterns of every map: sizes are bounded by nnz + n, so
    // they need no synchronisation
    std::vector<int32_t *> l1cp(K, nullptr), l1ri(K, nullptr), cnt(K, nullptr);
    for (int k = 0; k < K; ++k) {
        int lv = level == 0 ? 0 : 1;
        l1cp[k] = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)n + 1));
        cnt[k] = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)n + 1));
        if (!l1cp[k] || !cnt[k]) return SAM_ERR_OOM;
        level01_count<<<blocks, 256, 0, st>>>(n, kcp[k], kri[k], lv, cnt[k]);
        count_launch(h);
        if (exclusive_scan_i32(h, cnt[k], l1cp[k], n) != cudaSuccess) return SAM_ERR_CUDA;
    }
    // the level-1 total is needed for its allocation: read all K at once
    std::vector<int32_t> tot(K);
    int32_t *tot_dev = (int32_t *)pool_alloc(h, sizeof(int32_t) * (size_t)K);
    if (!tot_dev) return SAM_ERR_OOM;
    for (int k = 0; k < K; ++k)
        cudaMemcpyAsync(tot_dev + k, l1cp[k] + n, sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (cudaMemcpyAsync(tot.data(), tot_dev, sizeof(int32_t) * (size_t)K, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SAM_ERR_CUDA;
    for (int k = 0; k < K; ++k) {
        l1ri[k] = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)tot[k] + 1));
        if (!l1ri[k]) return SAM_ERR_OOM;
        level01_fill<<<blocks, 256, 0, st>>>(n, kcp[k], kri[k], level == 0 ? 0 : 1, l1cp[k], l1ri[k]);
        count_launch(h);
    }
    if (level <= 1) {
        for (int k = 0; k < K; ++k) {
            jcp[k] = l1cp[k];
            jri[k] = l1ri[k];
            nnz_out[k] = tot[k];
            pool_free(h, cnt[k]);
        }
        pool_free(h, tot_dev);
        return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
    }
    // level L+1 = union of level-1 columns over the level-L column
    std::vector<int32_t *> curcp = l1cp, curri = l1ri;
    for (int lv = 2; lv <= level; ++lv) {
        std::vector<int32_t *> nxcp(K), nxri(K);
        for (int k = 0; k < K; ++k) {
            nxcp[k] = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)n + 1));
            if (!nxcp[k]) return SAM_ERR_OOM;
            product_pattern_kernel<<<merge_grid(h, n), kMergeWarps * 32, 0, st>>>(
                n, l1cp[k], l1ri[k], curcp[k], curri[k], 0, cnt[k], nullptr, nullptr, flag);
            count_launch(h);
            if (exclusive_scan_i32(h, cnt[k], nxcp[k], n) != cudaSuccess) return SAM_ERR_CUDA;
            cudaMemcpyAsync(tot_dev + k, nxcp[k] + n, sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
        }
        if (cudaMemcpyAsync(tot.data(), tot_dev, sizeof(int32_t) * (size_t)K, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SAM_ERR_CUDA;
        for (int k = 0; k < K; ++k) {
            nxri[k] = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)tot[k] + 1));
            if (!nxri[k]) return SAM_ERR_OOM;
            product_pattern_kernel<<<merge_grid(h, n), kMergeWarps * 32, 0, st>>>(
                n, l1cp[k], l1ri[k], curcp[k], curri[k], 1, nullptr, nxcp[k], nxri[k], flag);
            count_launch(h);
            if (curcp[k] != l1cp[k]) {
                pool_free(h, curcp[k]);
                pool_free(h, curri[k]);
            }
        }
        curcp = nxcp;
        curri = nxri;
    }
    for (int k = 0; k < K; ++k) {
        pool_free(h, l1cp[k]);
        pool_free(h, l1ri[k]);
        pool_free(h, cnt[k]);
        jcp[k] = curcp[k];
        jri[k] = curri[k];
        nnz_out[k] = tot[k];
    }
    pool_free(h, tot_dev);
    return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}

sam_status level_pattern(sam_handle h, int n, const int32_t *kcp, const int32_t *kri, int level, int32_t **jcp,
                         int32_t **jri, int64_t *nnz_out) {
    return level_pattern_batched(h, 1, n, &kcp, &kri, level, jcp, jri, nnz_out);
}

// ------------------------------------------------------- shadows and bins

namespace {

// Size classes shared by both precisions: |I| <= bin_maxi, |J| <= bin_maxj,
// nnz(B) <= 8 * bin_maxi.  Must match the tile table in lsq.cu.
__constant__ int c_bin_maxi[kNumBins] = {14, 26, 40, 52, 64};
__constant__ int c_bin_maxj[kNumBins] = {5, 9, 23, 27, 27};

__global__ void __launch_bounds__(kMergeWarps * 32) shadow_kernel(int n, const int32_t *kcp, const int32_t *kri,
                                                                  const int32_t *jcp, const int32_t *jri,
                                                                  int32_t *ish, int32_t *icnt, uint8_t *bin,
                                                                  int32_t *colstat) {
    __shared__ int bufs[kMergeWarps][kMergeBuf];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *buf = bufs[warp];
    for (int64_t j = (int64_t)blockIdx.x * kMergeWarps + warp; j < n; j += (int64_t)gridDim.x * kMergeWarps) {
        int total = gather_candidates((int)j, kcp, kri, jcp, jri, buf);
        int nj = jcp[j + 1] - jcp[j];
        int u = -1;
        if (total <= kMergeBuf) u = warp_sort_unique(buf, total);
        int b = kBinNone;
        if (u >= nj && u >= 0) {
            for (int q = 0; q < kNumBins; ++q)
                if (u <= c_bin_maxi[q] && nj <= c_bin_maxj[q] && total <= 8 * c_bin_maxi[q]) {
                    b = q;
                    break;
                }
        }
        int uc = (u < 0) ? 0 : (u > kICap ? kICap : u);
        for (int i = lane; i < uc; i += 32) ish[j * kICap + i] = buf[i];
        if (lane == 0) {
            icnt[j] = (u < 0) ? -1 : u;
            bin[j] = (uint8_t)b;
            // fewer shadow rows than unknowns means a zero column: rank deficient
            colstat[j] = (b != kBinNone) ? kStOk : ((u >= 0 && u < nj) ? kStRank : kStUnsupported);
        }
        __syncwarp();
    }
}

__global__ void bin_count_kernel(int n, const uint8_t *bin, int32_t *counts /* [kNumBins] */) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int b = (j < n) ? bin[j] : kBinNone;
    // warp-aggregated increments
    for (int q = 0; q < kNumBins; ++q) {
        unsigned m = __ballot_sync(0xffffffffu, b == q);
        if (m && (threadIdx.x & 31) == (__ffs(m) - 1)) atomicAdd(&counts[q], __popc(m));
    }
}

__global__ void bin_scatter_kernel(int n, int map, const uint8_t *bin, int32_t *cursor, int2 *work) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int b = (j < n) ? bin[j] : kBinNone;
    int lane = threadIdx.x & 31;
    for (int q = 0; q < kNumBins; ++q) {
        unsigned m = __ballot_sync(0xffffffffu, b == q);
        if (!m) continue;
        int leader = __ffs(m) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&cursor[q], __popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (b == q) work[base + __popc(m & ((1u << lane) - 1u))] = make_int2(map, j);
    }
}

__global__ void bin_offsets_kernel(const int32_t *counts, int32_t *off, int32_t *cursor) {
    if (threadIdx.x == 0) {
        int s = 0;
        for (int q = 0; q < kNumBins; ++q) {
            off[q] = s;
            cursor[q] = s;
            s += counts[q];
        }
        off[kNumBins] = s;
    }
}

}  // namespace

cudaError_t shadow_and_bins(sam_handle h, int n, const int32_t *kcp, const int32_t *kri, const int32_t *jcp,
                            const int32_t *jri, int precision, int32_t *ish, int32_t *icnt, uint8_t *bin,
                            int32_t *colstat) {
    (void)precision;
    shadow_kernel<<<merge_grid(h, n), kMergeWarps * 32, 0, handle_stream(h)>>>(n, kcp, kri, jcp, jri, ish, icnt,
                                                                              bin, colstat);
    count_launch(h);
    return cudaGetLastError();
}

cudaError_t build_work_lists(sam_handle h, int K, int n, const uint8_t *const *bins, int2 *work, int32_t *bin_off) {
    cudaStream_t st = handle_stream(h);
    int32_t *tmp = (int32_t *)pool_alloc(h, sizeof(int32_t) * 2 * kNumBins);
    if (!tmp) return cudaErrorMemoryAllocation;
    int32_t *counts = tmp, *cursor = tmp + kNumBins;
    cudaMemsetAsync(counts, 0, sizeof(int32_t) * kNumBins, st);
    int blocks = (n + 255) / 256;
    if (blocks < 1) blocks = 1;
    for (int k = 0; k < K; ++k) bin_count_kernel<<<blocks, 256, 0, st>>>(n, bins[k], counts);
    count_launch(h, K);
    bin_offsets_kernel<<<1, 32, 0, st>>>(counts, bin_off, cursor);
    count_launch(h);
    for (int k = 0; k < K; ++k) bin_scatter_kernel<<<blocks, 256, 0, st>>>(n, k, bins[k], cursor, work);
    count_launch(h, K);
    pool_free(h, tmp);
    return cudaGetLastError();
}

}  // namespace sam
