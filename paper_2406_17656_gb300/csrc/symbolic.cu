// symbolic.cu -- integer (bit-exact) part of SAM construction:
//   * CSR validation, block-diagonal concatenation of a batch, CSR -> CSC,
//   * the level-L neighbour patterns of G(A) (Sec. 3 of arXiv 2406.17656):
//     level 1 = column pattern of A plus the diagonal, level L+1 = union of
//     the level-1 columns of every vertex in the level-L column (paths of
//     length <= L+1 pointing to j),
//   * shadow rows I_j = union of the row patterns of A(:, c), c in J_j (the
//     rows of the column least-squares problem of Sec. 2), and the size
//     class ("bin") of every column problem,
//   * the work list of each size class, exclusive scans.
// Column unions are computed by one warp per column with a bitmap over the
// column's index window [lo, hi] in shared memory (atomicOr, then popcount
// prefix sums give the sorted, duplicate-free result); windows wider than
// 65536 fall back to a bitonic sort of the concatenated candidates.  All
// kernels are bounded loops; errors are reported through an int32 flag.
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

// scan of each tile plus its offset; the last block also writes the total
// to out[n]
template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_apply(const T *in, T *out, int64_t n, const T *offs,
                                                           const T *grand) {
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
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = *grand;
}

template <typename T>
cudaError_t exclusive_scan_impl(sam_handle h, const T *in, T *out, int64_t n) {
    cudaStream_t st = handle_stream(h);
    int64_t nt = (n + kScanTile - 1) / kScanTile;
    if (nt == 0) return cudaMemsetAsync(out, 0, sizeof(T), st);
    T *sums = (T *)pool_alloc(h, sizeof(T) * (size_t)(nt + 1));
    if (!sums) return cudaErrorMemoryAllocation;
    scan_tile_sums<T><<<(unsigned)nt, kScanThreads, 0, st>>>(in, n, sums);
    scan_spine<T><<<1, kScanThreads, 0, st>>>(sums, nt, sums + nt);
    scan_apply<T><<<(unsigned)nt, kScanThreads, 0, st>>>(in, out, n, sums, sums + nt);
    count_launch(h, 3);
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

// --------------------------------------------- validation, concatenation

namespace {

__device__ __forceinline__ int lower_bound_i32(const int32_t *a, int len, int key) {
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Row i of a CSR matrix: checks (row pointers inside [0, nz], columns
// strictly ascending and inside [0, n)) and, with sym, whether every (i, c)
// has a stored mirror (c, i).  Returns the row's length, or -1 after
// flagging an error.
__device__ __forceinline__ int check_row(int n, const int32_t *rp, const int32_t *ci, int64_t nz, int64_t i,
                                         int32_t *flag, bool &sym) {
    const int b = rp[i], e = rp[i + 1];
    if (e < b || b < 0 || (int64_t)e > nz) {
        atomicCAS(flag, 0, SAM_ERR_BAD_CSR);
        return -1;
    }
    int prev = -1;
    for (int t = b; t < e; ++t) {
        const int c = ci[t];
        if (c <= prev || c >= n) {
            atomicCAS(flag, 0, SAM_ERR_BAD_CSR);
            return -1;
        }
        prev = c;
        if (sym) {
            // the mirror (c, i) in row c, read only inside row c's valid range
            const int cb = rp[c], ce = rp[c + 1];
            if (cb < 0 || ce < cb || (int64_t)ce > nz) {
                sym = false;
            } else {
                const int q = lower_bound_i32(ci + cb, ce - cb, (int)i);
                sym = q < ce - cb && ci[cb + q] == (int)i;
            }
        }
    }
    return e - b;
}

// Structure checks of K CSR matrices of order n; asym[k] (nullable) is set
// when matrix k is not structurally symmetric (some stored (i, c) without
// a stored (c, i)); maxrow[k] (nullable) receives its longest row.
__global__ void validate_batch_kernel(int n, const CsrPtrs *mats, const int64_t *nnz, int32_t *flag,
                                      int32_t *asym, int32_t *maxrow) {
    __shared__ int smax;
    if (threadIdx.x == 0) smax = 0;
    const int k = blockIdx.y;
    const int32_t *rp = mats[k].rp, *ci = mats[k].ci;
    const int64_t nz = nnz[k];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && (rp[0] != 0 || (int64_t)rp[n] != nz)) atomicCAS(flag, 0, SAM_ERR_BAD_CSR);
    int len = -1;
    if (i < n) {
        bool sym = asym != nullptr;
        len = check_row(n, rp, ci, nz, i, flag, sym);
        if (asym && len >= 0 && !sym) asym[k] = 1;
    }
    if (maxrow) {  // the same for every thread of the launch
        __syncthreads();
        if (len > 0) atomicMax(&smax, len);
        __syncthreads();
        if (threadIdx.x == 0 && smax > 0) atomicMax(&maxrow[k], smax);
    }
}

__global__ void concat_rows_kernel(int K, int n, const CsrPtrs *mats, const int64_t *nnz_off, int32_t *rp) {
    const int k = blockIdx.y;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rp[(int64_t)k * n + i] = mats[k].rp[i] + (int32_t)nnz_off[k];
    if (k == K - 1 && i == n) rp[(int64_t)K * n] = (int32_t)nnz_off[K];
}

__global__ void concat_entries_kernel(int n, const CsrPtrs *mats, const int64_t *nnz_off, int32_t *ci, double *v) {
    const int k = blockIdx.y;
    const int64_t off = nnz_off[k], nz = nnz_off[k + 1] - off;
    const int32_t *src = mats[k].ci;
    const double *sv = mats[k].v;
    const int32_t shift = (int32_t)((int64_t)k * n);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nz; e += (int64_t)gridDim.x * blockDim.x) {
        ci[off + e] = src[e] + shift;
        if (v) v[off + e] = sv[e];
    }
}

}  // namespace

cudaError_t validate_csr_batch(sam_handle h, int K, int n, const CsrPtrs *mats, const int64_t *nnz, int32_t *flag,
                               int32_t *asym, int32_t *maxrow) {
    dim3 grid((unsigned)((n + 1 + 255) / 256), (unsigned)K);
    validate_batch_kernel<<<grid, 256, 0, handle_stream(h)>>>(n, mats, nnz, flag, asym, maxrow);
    count_launch(h);
    return cudaGetLastError();
}

cudaError_t concat_block_diag(sam_handle h, int K, int n, const CsrPtrs *mats, const int64_t *nnz_off, int32_t *rp,
                              int32_t *ci, double *v) {
    cudaStream_t st = handle_stream(h);
    dim3 g1((unsigned)((n + 1 + 255) / 256), (unsigned)K);
    concat_rows_kernel<<<g1, 256, 0, st>>>(K, n, mats, nnz_off, rp);
    dim3 g2((unsigned)(handle_sms(h) * 4 / K + 1), (unsigned)K);
    concat_entries_kernel<<<g2, 256, 0, st>>>(n, mats, nnz_off, ci, v);
    count_launch(h, 2);
    return cudaGetLastError();
}

// -------------------------------------------------------------- transpose

namespace {

__global__ void count_cols_kernel(int64_t nnz, const int32_t *ci, int32_t *cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[ci[e]], 1);
}

// positions claimed with atomics (8 lanes per row), ordered afterwards
__global__ void fill_cols_kernel(int n, const int32_t *rp, const int32_t *ci, const double *val, int32_t *cursor,
                                 int32_t *ri, double *cv, int32_t *perm) {
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    int sub = threadIdx.x & 7;
    if (row >= n) return;
    for (int e = rp[row] + sub; e < rp[row + 1]; e += 8) {
        int p = atomicAdd(&cursor[ci[e]], 1);
        ri[p] = (int)row;
        if (cv) cv[p] = val[e];
        if (perm) perm[p] = e;
    }
}

// one warp per column: bitonic sort of the (row, value, perm) triples of a
// segment of up to 32 entries in registers; longer segments fall back to an
// insertion sort by lane 0
__global__ void sort_cols_kernel(int n, const int32_t *cp, int32_t *ri, double *cv, int32_t *perm) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= n) return;
    const int b = cp[c], e = cp[c + 1], len = e - b;
    if (len <= 1) return;
    if (len <= 32) {
        int key = (lane < len) ? ri[b + lane] : INT_MAX;
        double v = (cv && lane < len) ? cv[b + lane] : 0.0;
        int p = (perm && lane < len) ? perm[b + lane] : 0;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const int ok = __shfl_xor_sync(0xffffffffu, key, j);
                const double ov = __shfl_xor_sync(0xffffffffu, v, j);
                const int op = __shfl_xor_sync(0xffffffffu, p, j);
                const bool up = (lane & k) == 0;
                const bool low = (lane & j) == 0;
                const bool take = low ? (up ? ok < key : ok > key) : (up ? ok > key : ok < key);
                if (take) {
                    key = ok;
                    v = ov;
                    p = op;
                }
            }
        }
        if (lane < len) {
            ri[b + lane] = key;
            if (cv) cv[b + lane] = v;
            if (perm) perm[b + lane] = p;
        }
        return;
    }
    if (lane != 0) return;
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

// Transpose of a structurally symmetric CSR matrix: the CSC structure is the
// CSR structure, and the entry at position q of row c (column r = ci[q]) of
// the CSC is A(r, c), stored at position mirror(q) of row r.  Eight threads
// per row; no atomics, no sort.
__global__ void mirror_lookup_kernel(int n, const int32_t *rp, const int32_t *ci, const double *val, double *cv,
                                     int32_t *perm) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int sub = threadIdx.x & 7;
    if (c >= n) return;
    for (int q = rp[c] + sub; q < rp[c + 1]; q += 8) {
        const int r = ci[q];
        const int rb = rp[r];
        const int e = rb + lower_bound_i32(ci + rb, rp[r + 1] - rb, (int)c);
        if (cv) cv[q] = val[e];
        if (perm) perm[q] = e;
    }
}

}  // namespace

cudaError_t mirror_positions(sam_handle h, int n, const int32_t *rp, const int32_t *ci, int32_t *pos) {
    if (n == 0) return cudaSuccess;
    const int64_t threads = (int64_t)n * 8;
    mirror_lookup_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, handle_stream(h)>>>(n, rp, ci, nullptr,
                                                                                         nullptr, pos);
    count_launch(h);
    return cudaGetLastError();
}

cudaError_t csr_to_csc(sam_handle h, int n, int64_t nnz, const int32_t *rp, const int32_t *ci, const double *val,
                       int32_t *cp, int32_t *ri, double *cv, int32_t *perm, bool symmetric) {
    cudaStream_t st = handle_stream(h);
    if (symmetric) {
        cudaError_t err = cudaMemcpyAsync(cp, rp, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, st);
        if (err == cudaSuccess && nnz > 0)
            err = cudaMemcpyAsync(ri, ci, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToDevice, st);
        if (err != cudaSuccess) return err;
        if (n > 0 && ((val && cv) || perm)) {
            const int64_t threads = (int64_t)n * 8;
            mirror_lookup_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(n, rp, ci, val, val ? cv : nullptr,
                                                                                    perm);
            count_launch(h);
        }
        return cudaGetLastError();
    }
    int32_t *cnt = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)n + 1));
    if (!cnt) return cudaErrorMemoryAllocation;
    cudaError_t err = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)n + 1), st);
    if (err != cudaSuccess) return err;
    if (nnz > 0) {
        int64_t blocks = (nnz + 255) / 256;
        if (blocks > (int64_t)handle_sms(h) * 32) blocks = (int64_t)handle_sms(h) * 32;
        count_cols_kernel<<<(unsigned)blocks, 256, 0, st>>>(nnz, ci, cnt);
        count_launch(h);
    }
    err = exclusive_scan_i32(h, cnt, cp, n);
    if (err != cudaSuccess) return err;
    err = cudaMemcpyAsync(cnt, cp, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    if (err != cudaSuccess) return err;
    if (n > 0) {
        int64_t threads = (int64_t)n * 8;
        fill_cols_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(n, rp, ci, val, cnt, ri, cv, perm);
        int64_t wthreads = (int64_t)n * 32;
        sort_cols_kernel<<<(unsigned)((wthreads + 255) / 256), 256, 0, st>>>(n, cp, ri, val ? cv : nullptr, perm);
        count_launch(h, 2);
    }
    pool_free(h, cnt);
    return cudaGetLastError();
}

// ----------------------------------------------------------- column unions

namespace {

constexpr int kMergeWarps = 4;
constexpr int kBitWords = 1024;  // bitmap window of 32768 indices per warp
constexpr int kMergeBuf = 1024;  // fallback candidate buffer (shares the storage)

// Warp-cooperative sort + unique of buf[0..cnt), cnt <= kMergeBuf (fallback
// path for wide windows).  Returns the number of distinct values, left
// ascending in buf[0..u).
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

struct UnionResult {
    int count;  // distinct entries (-1: too many candidates for the fallback)
    int total;  // candidates, i.e. the sum of the list lengths
    int mode;   // 0: bitmap over [lo, lo + 32 words) left in shared memory, 1: sorted buffer
    int lo;
    int words;
};

// Rank of x among the union left in shared memory by warp_union / union_fast
// (bitmap with word prefixes wpre, or sorted buffer), -1 when absent.
__device__ __forceinline__ int union_rank(int x, const UnionResult &r, const unsigned *bm, const unsigned char *wpre) {
    if (r.count <= 0) return -1;
    if (r.mode == 0) {
        const int64_t d = (int64_t)x - r.lo;
        if (d < 0 || d >= (int64_t)r.words * 32) return -1;
        const unsigned w = bm[d >> 5], bit = 1u << (d & 31);
        if (!(w & bit)) return -1;
        return wpre[d >> 5] + __popc(w & (bit - 1u));
    }
    const int *srt = reinterpret_cast<const int *>(bm);
    int lo = 0, hi = r.count - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int v = srt[mid];
        if (v == x) return mid;
        if (v < x) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// Union of the sorted lists X(:, l), l in Y(:, j).  The distinct values are
// written ascending to out[0..min(count, cap)) when out != nullptr.  Every
// lane returns the same result.
__device__ UnionResult warp_union(int j, const int32_t *xcp, const int32_t *xri, const int32_t *ycp,
                                  const int32_t *yri, unsigned *bm, int32_t *out, int cap,
                                  unsigned char *wpre = nullptr) {
    const int lane = threadIdx.x & 31;
    const int yb = ycp[j], ye = ycp[j + 1];
    int lo = INT_MAX, hi = INT_MIN, total = 0;
    for (int t = yb + lane; t < ye; t += 32) {
        const int l = yri[t];
        const int b = xcp[l], e = xcp[l + 1];
        if (e > b) {
            lo = min(lo, xri[b]);
            hi = max(hi, xri[e - 1]);
            total += e - b;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        total += __shfl_xor_sync(0xffffffffu, total, o);
    }
    UnionResult res{0, total, 0, lo, 0};
    if (total == 0) return res;
    const int64_t span = (int64_t)hi - lo + 1;
    if (span <= (int64_t)kBitWords * 32) {
        const int words = (int)((span + 31) >> 5);
        res.words = words;
        for (int w = lane; w < words; w += 32) bm[w] = 0u;
        __syncwarp();
        for (int t = yb + lane; t < ye; t += 32) {
            const int l = yri[t];
            const int e = xcp[l + 1];
            for (int q = xcp[l]; q < e; ++q) {
                const int x = xri[q] - lo;
                atomicOr(&bm[x >> 5], 1u << (x & 31));
            }
        }
        __syncwarp();
        const int wpl = (words + 31) >> 5;
        const int w0 = lane * wpl, w1 = min(words, w0 + wpl);
        int cnt = 0;
        for (int w = w0; w < w1; ++w) cnt += __popc(bm[w]);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        res.count = __shfl_sync(0xffffffffu, incl, 31);
        if (wpre) {  // rank of the first index of every word (saturating at 255)
            int run = incl - cnt;
            for (int w = w0; w < w1; ++w) {
                wpre[w] = (unsigned char)(run < 255 ? run : 255);
                run += __popc(bm[w]);
            }
        }
        if (out) {
            int pos = incl - cnt;
            for (int w = w0; w < w1 && pos < cap; ++w) {
                unsigned bits = bm[w];
                while (bits && pos < cap) {
                    const int bit = __ffs(bits) - 1;
                    out[pos++] = lo + (w << 5) + bit;
                    bits &= bits - 1u;
                }
            }
        }
        __syncwarp();
        return res;
    }
    // wide window: concatenate the candidates and sort
    if (total > kMergeBuf) {
        res.count = -1;
        return res;
    }
    int *buf = (int *)bm;
    int off = 0;
    for (int base = yb; base < ye; base += 32) {
        const int t = base + lane;
        int xb = 0, len = 0;
        if (t < ye) {
            const int l = yri[t];
            xb = xcp[l];
            len = xcp[l + 1] - xb;
        }
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        for (int q = 0; q < len; ++q) buf[off + incl - len + q] = xri[xb + q];
        off += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    const int u = warp_sort_unique(buf, total);
    res.count = u;
    res.mode = 1;
    if (out)
        for (int i = lane; i < u && i < cap; i += 32) out[i] = buf[i];
    __syncwarp();
    return res;
}

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

// Size classes: |I| <= bin_maxi, |J| <= bin_maxj, nnz(B) <= 8 * bin_maxi
// (the register tiles of lsq.cu, whose table these must match); larger
// columns within the large class's limits go to it (lsq_big.cu).
__constant__ int c_bin_maxi[kRegBins] = {14, 26, 40, 52, 64};
__constant__ int c_bin_maxj[kRegBins] = {5, 9, 23, 27, 27};

__device__ __forceinline__ int size_class(int u, int nj, int total) {
    int b = kBinNone;
    if (u >= nj && u >= 0) {
        for (int q = 0; q < kRegBins; ++q)
            if (u <= c_bin_maxi[q] && nj <= c_bin_maxj[q] && total <= 8 * c_bin_maxi[q]) {
                b = q;
                break;
            }
        if (b == kBinNone && nj <= kBigJCap && u <= kBigICap && total <= kBigLCap &&
            (int64_t)u * (nj + 1) <= kBigTileDoubles)
            b = kBinBig;
    }
    return b;
}

constexpr int kRegRows = 16;  // stored entries per source column held in registers (fast path)

// Fast path of the union of the lists X(:, l), l in Y(:, j), when Y(:, j)
// has at most 32 entries and every list at most kRegRows (every stencil and
// FEM matrix here): lane t holds list Y(:, j)[t] in registers, read in one
// round of independent loads and reused for the bitmap union, the sorted
// output (out[0..min(count, cap)), nullable) and, for the shadow (SHADOW),
// the size class and the local ranks of all entries (lrow_j, nullable).
// Returns false, having written nothing, when the column does not qualify
// or its values span more than the bitmap window.
template <bool SHADOW>
__device__ bool union_fast(int j, const int32_t *kcp, const int32_t *kri, const int32_t *jcp, const int32_t *jri,
                           unsigned *bm, unsigned char *wpre, unsigned char *stage, int32_t *ish_j, int cap,
                           uint8_t *lrow_j, UnionResult &r, int &bsz) {
    const int lane = threadIdx.x & 31;
    const int yb = jcp[j], nj = jcp[j + 1] - yb;
    if (nj > 32) return false;
    int cb = 0, len = 0;
    if (lane < nj) {
        const int l = jri[yb + lane];
        cb = kcp[l];
        len = kcp[l + 1] - cb;
    }
    int mx = len;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (mx > kRegRows) return false;
    int v[kRegRows];
#pragma unroll
    for (int u = 0; u < kRegRows; ++u) {
        if (u >= mx) break;  // warp-uniform: no predicated-off tail iterations
        v[u] = (u < len) ? __ldg(kri + cb + u) : 0;
    }
    int lo = INT_MAX, hi = INT_MIN;
#pragma unroll
    for (int u = 0; u < kRegRows; ++u) {
        if (u >= mx) break;
        if (u < len) {
            lo = min(lo, v[u]);
            hi = max(hi, v[u]);
        }
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int off = incl - len;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (total == 0) {
        r = UnionResult{0, 0, 0, lo, 0};
        if (SHADOW) bsz = size_class(0, nj, 0);
        return true;
    }
    const int64_t span = (int64_t)hi - lo + 1;
    if (span > (int64_t)kBitWords * 32) return false;
    const int words = (int)((span + 31) >> 5);
    for (int w = lane; w < words; w += 32) bm[w] = 0u;
    __syncwarp();
#pragma unroll
    for (int u = 0; u < kRegRows; ++u) {
        if (u >= mx) break;
        if (u < len) {
            const int x = v[u] - lo;
            atomicOr(&bm[x >> 5], 1u << (x & 31));
        }
    }
    __syncwarp();
    const int wpl = (words + 31) >> 5;
    const int w0 = lane * wpl, w1 = min(words, w0 + wpl);
    int cnt = 0;
    for (int w = w0; w < w1; ++w) cnt += __popc(bm[w]);
    int winc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, winc, o);
        if (lane >= o) winc += y;
    }
    const int count = __shfl_sync(0xffffffffu, winc, 31);
    {
        int run = winc - cnt;
        int pos = run;
        for (int w = w0; w < w1; ++w) {
            if (SHADOW) wpre[w] = (unsigned char)(run < 255 ? run : 255);
            unsigned bits = bm[w];
            run += __popc(bits);
            if (!ish_j) continue;
            while (bits && pos < cap) {
                const int bit = __ffs(bits) - 1;
                ish_j[pos++] = lo + (w << 5) + bit;
                bits &= bits - 1u;
            }
        }
    }
    __syncwarp();
    if (SHADOW) bsz = size_class(count, nj, total);
    if (SHADOW && lrow_j && bsz < kRegBins) {
        // rank of every entry among the shadow rows, in gather order
#pragma unroll
        for (int u = 0; u < kRegRows; ++u) {
            if (u >= mx) break;
            if (u < len) {
                const int d = v[u] - lo;
                stage[off + u] = (unsigned char)(wpre[d >> 5] + __popc(bm[d >> 5] & ((1u << (d & 31)) - 1u)));
            }
        }
        __syncwarp();
        const unsigned *src = reinterpret_cast<const unsigned *>(stage);
        unsigned *dst = reinterpret_cast<unsigned *>(lrow_j);
        for (int w = lane; w < (total + 3) / 4; w += 32) dst[w] = src[w];
    }
    __syncwarp();
    r = UnionResult{count, total, 0, lo, words};
    return true;
}

// Distinct rows of the union of X(:, l), l in Y(:, j): cnt[j] receives their
// number and, with out != nullptr, they are written ascending to
// out + ooff[j] (ooff: room for every candidate of column j).
__global__ void __launch_bounds__(kMergeWarps * 32) product_pattern_kernel(
    int n, const int32_t *xcp, const int32_t *xri, const int32_t *ycp, const int32_t *yri, int32_t *cnt,
    const int64_t *ooff, int32_t *out, int32_t *flag) {
    __shared__ unsigned bms[kMergeWarps][kBitWords];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned *bm = bms[warp];
    for (int64_t j = (int64_t)blockIdx.x * kMergeWarps + warp; j < n; j += (int64_t)gridDim.x * kMergeWarps) {
        int32_t *dst = out ? out + ooff[j] : nullptr;
        UnionResult r;
        int unused = 0;
        if (!union_fast<false>((int)j, xcp, xri, ycp, yri, bm, nullptr, nullptr, dst, INT_MAX, nullptr, r, unused))
            r = warp_union((int)j, xcp, xri, ycp, yri, bm, dst, INT_MAX);
        if (lane == 0) {
            if (r.count < 0) {
                cnt[j] = 0;
                atomicCAS(flag, 0, SAM_ERR_UNSUPPORTED);
            } else {
                cnt[j] = r.count;
            }
        }
    }
}

// candidates of column j: sum of |X(:, l)| over l in Y(:, j)
__global__ void candidate_count_kernel(int n, const int32_t *xcp, const int32_t *ycp, const int32_t *yri,
                                       int64_t *cand) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int64_t c = 0;
    for (int t = ycp[j]; t < ycp[j + 1]; ++t) {
        const int l = yri[t];
        c += xcp[l + 1] - xcp[l];
    }
    cand[j] = c;
}

// column j of the union result: from its padded slot to its final place
__global__ void compact_columns_kernel(int n, const int64_t *ooff, const int32_t *pad, const int32_t *cp,
                                       int32_t *ri) {
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int sub = threadIdx.x & 7;
    if (j >= n) return;
    const int32_t *src = pad + ooff[j];
    const int b = cp[j], len = cp[j + 1] - b;
    for (int t = sub; t < len; t += 8) ri[b + t] = src[t];
}

// One resident wave of a grid-stride union kernel: blocks beyond what the
// SMs hold at once would run as a second wave with the same per-block work.
template <typename Kernel>
int merge_grid(sam_handle h, int n, Kernel kernel) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kMergeWarps * 32, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int blocks = (n + kMergeWarps - 1) / kMergeWarps;
    const int cap = handle_sms(h) * per_sm;
    return blocks < cap ? (blocks > 0 ? blocks : 1) : cap;
}


__global__ void __launch_bounds__(kMergeWarps * 32) shadow_kernel(int n, const int32_t *kcp, const int32_t *kri,
                                                                  const int32_t *jcp, const int32_t *jri,
                                                                  int32_t *ish, int32_t *icnt, uint8_t *bin,
                                                                  int32_t *colstat, int64_t *nbcnt, uint8_t *lrow,
                                                                  ShadowTarget tg, BinSchedule sched) {
    __shared__ unsigned bms[kMergeWarps][kBitWords];
    __shared__ unsigned char pres[kMergeWarps][kBitWords];
    __shared__ __align__(16) unsigned char stg[kMergeWarps][kLCap];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned *bm = bms[warp];
    unsigned char *wpre = pres[warp];
    unsigned char *stage = stg[warp];
    for (int64_t j = (int64_t)blockIdx.x * kMergeWarps + warp; j < n; j += (int64_t)gridDim.x * kMergeWarps) {
        const int nj = jcp[j + 1] - jcp[j];
        // the target column of this map column: local rows go to zloc; the
        // sorted shadow rows themselves are only stored when some target
        // entries lie beyond zloc's capacity (or no target is given)
        int zb = 0, zlen = 0, zro = 0;
        if (tg.zloc) {
            const int kmap = (int)((uint32_t)j / (uint32_t)tg.n);  // j < 2^31: 32-bit division
            const int zc = tg.zbig ? (int)j : (int)(j - (int64_t)kmap * tg.n);
            zro = tg.zbig ? 0 : kmap * tg.n;
            zb = tg.zcp[zc];
            zlen = tg.zcp[zc + 1] - zb;
        }
        int32_t *ish_j = (!tg.zloc || zlen > kZCap) ? ish + j * kICap : nullptr;
        UnionResult r;
        int b = kBinNone;
        if (!union_fast<true>((int)j, kcp, kri, jcp, jri, bm, wpre, stage, ish_j, kICap,
                              lrow ? lrow + j * kLCap : nullptr, r, b)) {
            r = warp_union((int)j, kcp, kri, jcp, jri, bm, ish_j, kICap, wpre);
            b = size_class(r.count, nj, r.total);
            // local shadow row of every entry of A(:, J_j), in gather order (the
            // columns of J_j in order, each in CSC order): its rank in I_j,
            // staged in shared memory and written out as 32-bit words
            if (lrow && b < kRegBins) {
                const int yb = jcp[j], ye = jcp[j + 1];
                const int u = r.count;
                int off = 0;
                for (int base = yb; base < ye; base += 32) {
                    const int t = base + lane;
                    int xb = 0, len = 0;
                    if (t < ye) {
                        const int l = jri[t];
                        xb = kcp[l];
                        len = kcp[l + 1] - xb;
                    }
                    int incl = len;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += y;
                    }
                    unsigned char *dst = stage + off + incl - len;
                    for (int q = 0; q < len; ++q) {
                        const int x = kri[xb + q];
                        int rank;
                        if (r.mode == 0) {
                            const int d = x - r.lo;
                            rank = wpre[d >> 5] + __popc(bm[d >> 5] & ((1u << (d & 31)) - 1u));
                        } else {
                            const int *srt = (const int *)bm;
                            int lo = 0, hi = u - 1;
                            rank = 0;
                            while (lo <= hi) {
                                const int mid = (lo + hi) >> 1;
                                if (srt[mid] < x) lo = mid + 1; else if (srt[mid] > x) hi = mid - 1; else { rank = mid; break; }
                            }
                        }
                        dst[q] = (unsigned char)rank;
                    }
                    off += __shfl_sync(0xffffffffu, incl, 31);
                }
                __syncwarp();
                const unsigned *src = reinterpret_cast<const unsigned *>(stage);
                unsigned *out = reinterpret_cast<unsigned *>(lrow + j * kLCap);
                for (int w = lane; w < (r.total + 3) / 4; w += 32) out[w] = src[w];
            }
            __syncwarp();
        }
        if (tg.zloc && b < kRegBins) {
            uint8_t *zl = tg.zloc + j * kZCap;
            for (int t = lane; t < zlen && t < kZCap; t += 32) {
                const int rk = union_rank(tg.zri[zb + t] + zro, r, bm, wpre);
                zl[t] = (uint8_t)(rk < 0 ? kZOutside : rk);
            }
        }
        __syncwarp();
        if (lane == 0) {
            const int u = r.count;
            icnt[j] = u;
            bin[j] = (uint8_t)(b != kBinNone ? sched.to[b] : b);  // the class that solves it
            if (nbcnt) nbcnt[j] = r.total;
            // fewer shadow rows than unknowns means a zero column: rank deficient
            colstat[j] = (b != kBinNone) ? kStOk : ((u >= 0 && u < nj) ? kStRank : kStUnsupported);
        }
    }
}

__global__ void flagged_bins_kernel(int n, const uint8_t *bin, const int32_t *colstat, int32_t flag, uint8_t *out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = (colstat[j] == flag) ? bin[j] : (uint8_t)kBinNone;
}

__global__ void bin_count_kernel(int n, const uint8_t *bin, int32_t *counts /* [kNumBins] */) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int b = (j < n) ? bin[j] : kBinNone;
    for (int q = 0; q < kNumBins; ++q) {
        unsigned m = __ballot_sync(0xffffffffu, b == q);
        if (m && (threadIdx.x & 31) == (__ffs(m) - 1)) atomicAdd(&counts[q], __popc(m));
    }
}

__global__ void bin_scatter_kernel(int n, const uint8_t *bin, int32_t *cursor, int32_t *work) {
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
        if (b == q) work[base + __popc(m & ((1u << lane) - 1u))] = j;
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

// a known bound sizes the candidate buffer only up to 2^28 entries (1 GiB);
// past that the exact total is read back
constexpr int64_t kCandidateBoundCap = int64_t(1) << 28;

sam_status level_pattern(sam_handle h, int N, const int32_t *kcp, const int32_t *kri, int64_t nnz, int level,
                         int32_t **jcp_out, int32_t **jri_out, int64_t *nnz_out, int maxcol) {
    cudaStream_t st = handle_stream(h);
    int32_t *flag = handle_flag(h);
    const int blocks = (N + 255) / 256 > 0 ? (N + 255) / 256 : 1;
    const int lv1 = level == 0 ? 0 : 1;
    // level 1 (or 0): size bounded by nnz + N, no synchronisation needed
    int32_t *cnt = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)N + 1));
    int32_t *l1cp = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)N + 1));
    int32_t *l1ri = (int32_t *)pool_alloc(h, sizeof(int32_t) * (size_t)(nnz + N + 1));
    if (!cnt || !l1cp || !l1ri) return SAM_ERR_OOM;
    level01_count<<<blocks, 256, 0, st>>>(N, kcp, kri, lv1, cnt);
    count_launch(h);
    if (exclusive_scan_i32(h, cnt, l1cp, N) != cudaSuccess) return SAM_ERR_CUDA;
    level01_fill<<<blocks, 256, 0, st>>>(N, kcp, kri, lv1, l1cp, l1ri);
    count_launch(h);
    int32_t *curcp = l1cp, *curri = l1ri;
    int32_t tot = -1;  // entries of the current pattern, once read back
    for (int lv = 2; lv <= level; ++lv) {
        // one union pass: rows go to a slot per column sized by its candidate
        // count, then are compacted once the counts are known
        int32_t *nxcp = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)N + 1));
        int64_t *cand = (int64_t *)pool_alloc(h, sizeof(int64_t) * ((size_t)N + 1));
        int64_t *coff = (int64_t *)pool_alloc(h, sizeof(int64_t) * ((size_t)N + 1));
        if (!nxcp || !cand || !coff) return SAM_ERR_OOM;
        candidate_count_kernel<<<blocks, 256, 0, st>>>(N, l1cp, curcp, curri, cand);
        count_launch(h);
        if (exclusive_scan_i64(h, cand, coff, N) != cudaSuccess) return SAM_ERR_CUDA;
        // candidates of column j: sum over l in the previous pattern's column j
        // of |L1(l)| <= maxcol + 1, so in all at most (entries of the previous
        // pattern) (maxcol + 1); entries: nnz + N for level 1, tot after that
        int64_t ctot = -1;
        if (maxcol >= 0) {
            const int64_t prev = tot >= 0 ? (int64_t)tot : nnz + N;
            const int64_t bound = prev * ((int64_t)maxcol + 1);
            if (bound <= kCandidateBoundCap) ctot = bound;
        }
        if (ctot < 0 && (cudaMemcpyAsync(&ctot, coff + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                         cudaStreamSynchronize(st) != cudaSuccess))
            return SAM_ERR_CUDA;
        int32_t *pad = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)ctot + 1));
        if (!pad) return SAM_ERR_OOM;
        product_pattern_kernel<<<merge_grid(h, N, product_pattern_kernel), kMergeWarps * 32, 0, st>>>(
            N, l1cp, l1ri, curcp, curri, cnt, coff, pad, flag);
        count_launch(h);
        if (exclusive_scan_i32(h, cnt, nxcp, N) != cudaSuccess) return SAM_ERR_CUDA;
        // the size and the status word in one synchronisation (the union
        // flags a column it cannot hold; the word is sticky, so an earlier
        // asynchronous call's error is reported here too)
        int32_t fl = 0;
        if (cudaMemcpyAsync(&tot, nxcp + N, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&fl, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SAM_ERR_CUDA;
        if (fl != SAM_OK) {
            cudaMemsetAsync(flag, 0, sizeof(int32_t), st);
            return (sam_status)fl;
        }
        int32_t *nxri = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)tot + 1));
        if (!nxri) return SAM_ERR_OOM;
        const int64_t cthreads = (int64_t)N * 8;
        compact_columns_kernel<<<(unsigned)((cthreads + 255) / 256), 256, 0, st>>>(N, coff, pad, nxcp, nxri);
        count_launch(h);
        pool_free(h, pad);
        pool_free(h, cand);
        pool_free(h, coff);
        if (curcp != l1cp) {
            pool_free(h, curcp);
            pool_free(h, curri);
        }
        curcp = nxcp;
        curri = nxri;
    }
    if (tot < 0) {
        int32_t fl = 0;
        if (cudaMemcpyAsync(&tot, curcp + N, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&fl, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SAM_ERR_CUDA;
        if (fl != SAM_OK) {
            cudaMemsetAsync(flag, 0, sizeof(int32_t), st);
            return (sam_status)fl;
        }
    }
    if (curcp != l1cp) {
        pool_free(h, l1cp);
        pool_free(h, l1ri);
    }
    pool_free(h, cnt);
    *jcp_out = curcp;
    *jri_out = curri;
    *nnz_out = tot;
    return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}

cudaError_t shadow_and_bins(sam_handle h, int N, const int32_t *kcp, const int32_t *kri, const int32_t *jcp,
                            const int32_t *jri, int32_t *ish, int32_t *icnt, uint8_t *bin, int32_t *colstat,
                            int64_t *nbcnt, uint8_t *lrow, ShadowTarget tg) {
    shadow_kernel<<<merge_grid(h, N, shadow_kernel), kMergeWarps * 32, 0, handle_stream(h)>>>(N, kcp, kri, jcp, jri, ish, icnt, bin,
                                                                              colstat, nbcnt, lrow, tg, handle_schedule(h));
    count_launch(h);
    return cudaGetLastError();
}

cudaError_t build_work_list(sam_handle h, int N, const uint8_t *bin, int32_t *work, int32_t *bin_off,
                            int32_t *ws) {
    cudaStream_t st = handle_stream(h);
    int32_t *tmp = ws ? ws : (int32_t *)pool_alloc(h, sizeof(int32_t) * 2 * kNumBins);
    if (!tmp) return cudaErrorMemoryAllocation;
    int32_t *counts = tmp, *cursor = tmp + kNumBins;
    cudaMemsetAsync(counts, 0, sizeof(int32_t) * kNumBins, st);
    const int blocks = (N + 255) / 256 > 0 ? (N + 255) / 256 : 1;
    bin_count_kernel<<<blocks, 256, 0, st>>>(N, bin, counts);
    bin_offsets_kernel<<<1, 32, 0, st>>>(counts, bin_off, cursor);
    bin_scatter_kernel<<<blocks, 256, 0, st>>>(N, bin, cursor, work);
    count_launch(h, 3);
    if (!ws) pool_free(h, tmp);
    return cudaGetLastError();
}

cudaError_t flagged_bins(sam_handle h, int N, const uint8_t *bin, const int32_t *colstat, int32_t flag,
                         uint8_t *out) {
    if (N == 0) return cudaSuccess;
    flagged_bins_kernel<<<(N + 255) / 256, 256, 0, handle_stream(h)>>>(N, bin, colstat, flag, out);
    count_launch(h);
    return cudaGetLastError();
}

// ------------------------------------------------- per-map map structure

namespace {
__global__ void split_rows_kernel(int K, int n, const int32_t *mrp, int32_t *rp_out) {
    const int k = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    rp_out[(int64_t)k * (n + 1) + i] = mrp[(int64_t)k * n + i] - mrp[(int64_t)k * n];
}

__global__ void split_cols_kernel(int n, int64_t N, const int32_t *mrp, const int32_t *mci, int32_t *ci_out) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int sub = threadIdx.x & 7;
    if (row >= N) return;
    const int32_t shift = (int32_t)((row / n) * n);
    for (int e = mrp[row] + sub; e < mrp[row + 1]; e += 8) ci_out[e] = mci[e] - shift;
}
}  // namespace

cudaError_t split_map_structure(sam_handle h, int K, int n, const int32_t *mrp_big, const int32_t *mci_big,
                                int32_t *rp_out, int32_t *ci_out) {
    cudaStream_t st = handle_stream(h);
    dim3 g1((unsigned)((n + 1 + 255) / 256), (unsigned)K);
    split_rows_kernel<<<g1, 256, 0, st>>>(K, n, mrp_big, rp_out);
    const int64_t N = (int64_t)K * n;
    if (N > 0) split_cols_kernel<<<(unsigned)((N * 8 + 255) / 256), 256, 0, st>>>(n, N, mrp_big, mci_big, ci_out);
    count_launch(h, 2);
    return cudaGetLastError();
}

}  // namespace sam
