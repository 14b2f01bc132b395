// misc.cu -- deterministic FP64 reductions, the residual of Eq. (res) for an
// arbitrary map, the map application y = M x, the status reduction and the
// FMA-throughput probes used as roofline denominators.
#include <climits>

#include "common.cuh"
#include "residual_row.cuh"

namespace sam {
namespace {

constexpr int kSumBlocks = 256;
constexpr int kSumThreads = 256;

// Fixed grid and fixed per-thread strides: the summation order does not
// depend on scheduling, so results are bit-reproducible.
__global__ void __launch_bounds__(kSumThreads) sum_partial_kernel(const double *x, int64_t n, bool squares,
                                                                  double *part) {
    __shared__ double sh[kSumThreads];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kSumThreads + threadIdx.x; i < n; i += (int64_t)kSumBlocks * kSumThreads) {
        double v = x[i];
        s += squares ? v * v : v;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kSumThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// segment k of length seg: blocks (b, k) sum fixed strided parts, then one
// block per segment adds the partials in index order
constexpr int kSegBlocks = 16;
__global__ void __launch_bounds__(kSumThreads) seg_partial_kernel(const double *x, int64_t seg, bool squares,
                                                                  double *part) {
    __shared__ double sh[kSumThreads];
    const int k = blockIdx.y;
    const double *xs = x + (int64_t)k * seg;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kSumThreads + threadIdx.x; i < seg; i += (int64_t)kSegBlocks * kSumThreads) {
        double v = xs[i];
        s += squares ? v * v : v;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kSumThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[k * kSegBlocks + blockIdx.x] = sh[0];
}

__global__ void seg_final_kernel(const double *part, int K, double *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    double s = 0.0;
    for (int b = 0; b < kSegBlocks; ++b) s += part[k * kSegBlocks + b];
    out[k] = s;
}

__global__ void __launch_bounds__(kSumBlocks) sum_final_kernel(const double *part, double *out) {
    __shared__ double sh[kSumBlocks];
    sh[threadIdx.x] = part[threadIdx.x];
    __syncthreads();
    for (int o = kSumBlocks / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// y = M x, one warp per row, fixed shuffle tree
__global__ void spmv_kernel(int n, const int32_t *rp, const int32_t *ci, const double *v, const double *x,
                            double *y) {
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= n) return;
    double s = 0.0;
    for (int e = rp[w] + lane; e < rp[w + 1]; e += 32) s = fma(v[e], x[ci[e]], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[w] = s;
}

// g[e] = dy[i] x[c] for every stored entry e = (i, c) of M: the gradient of
// <dy, M x> with respect to M's values, one warp per row
__global__ void outer_on_pattern_kernel(int n, const int32_t *rp, const int32_t *ci, const double *dy,
                                        const double *x, double *g) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const double d = dy[w];
    for (int e = rp[w] + lane; e < rp[w + 1]; e += 32) g[e] = d * x[ci[e]];
}

// Row i of R = A_k M - A_0 into row_r2[i] (residual_row_sq: products
// gathered as (column, value) pairs, sorted by column, summed and squared).
constexpr int kResWarps = 2;

__global__ void __launch_bounds__(kResWarps * 32) residual_rows_kernel(
    int n, const int32_t *krp, const int32_t *kci, const double *kv, const int32_t *mrp, const int32_t *mci,
    const double *mv, const int32_t *zrp, const int32_t *zci, const double *zv, double *row_r2, int32_t *flag) {
    __shared__ int keys[kResWarps][kResRowBuf];
    __shared__ double vals[kResWarps][kResRowBuf];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t i = (int64_t)blockIdx.x * kResWarps + warp; i < n; i += (int64_t)gridDim.x * kResWarps) {
        const double r2 = residual_row_sq(i, lane, krp, kci, kv, mrp, mci, mv, zrp, zci, zv, keys[warp], vals[warp]);
        if (lane == 0) {
            row_r2[i] = r2 < 0.0 ? 0.0 : r2;
            if (r2 < 0.0) atomicCAS(flag, 0, SAM_ERR_UNSUPPORTED);
        }
    }
}

__global__ void round_f32_kernel(int64_t n, const double *in, float *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

__global__ void status_max_kernel(const int32_t *st, int64_t n, int32_t *flag) {
    int m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, st[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m != 0) atomicMax(flag, m);
}

// ------------------------------------------------------- throughput probes

constexpr int kChains = 8;

template <typename T>
__global__ void fma_probe_kernel(int iters, T seed, T *sink) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = seed + T(threadIdx.x + c);
    const T m = T(0.999999), a = T(1e-7);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], m, a);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == T(-1.2345)) sink[threadIdx.x] = s;  // never true; keeps the chains live
}

template <typename T>
double probe(sam_handle h, double ms, int blocks, int threads) {
    cudaStream_t st = handle_stream(h);
    T *sink = (T *)pool_alloc(h, sizeof(T) * 1024);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int iters = 64;
    double flops = 0.0;
    for (int rep = 0; rep < 8; ++rep) {
        cudaEventRecord(e0, st);
        fma_probe_kernel<T><<<blocks, threads, 0, st>>>(iters, T(1), sink);
        count_launch(h);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        flops = 2.0 * kChains * 16.0 * (double)iters * blocks * threads / (t * 1e-3);
        if (t >= 0.8 * ms) break;
        double scale = ms / (t > 1e-3 ? t : 1e-3);
        if (scale > 64) scale = 64;
        iters = (int)(iters * scale) + 1;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pool_free(h, sink);
    return flops;
}

}  // namespace

cudaError_t sum_f64(sam_handle h, const double *x, int64_t n, double *out_dev, bool squares) {
    cudaStream_t st = handle_stream(h);
    double *part = (double *)pool_alloc(h, sizeof(double) * kSumBlocks);
    if (!part) return cudaErrorMemoryAllocation;
    sum_partial_kernel<<<kSumBlocks, kSumThreads, 0, st>>>(x, n, squares, part);
    count_launch(h);
    sum_final_kernel<<<1, kSumBlocks, 0, st>>>(part, out_dev);
    count_launch(h);
    pool_free(h, part);
    return cudaGetLastError();
}

size_t segmented_sum_workspace(int K) { return (size_t)K * kSegBlocks; }

cudaError_t segmented_sum_f64(sam_handle h, const double *x, int K, int64_t seg, double *out, bool squares,
                              double *work) {
    cudaStream_t st = handle_stream(h);
    double *part = work ? work : (double *)pool_alloc(h, sizeof(double) * segmented_sum_workspace(K));
    if (!part) return cudaErrorMemoryAllocation;
    seg_partial_kernel<<<dim3(kSegBlocks, (unsigned)K), kSumThreads, 0, st>>>(x, seg, squares, part);
    seg_final_kernel<<<(K + 127) / 128, 128, 0, st>>>(part, K, out);
    count_launch(h, 2);
    if (!work) pool_free(h, part);
    return cudaGetLastError();
}

// values of K matrices gathered into the CSC order of their block-diagonal
// (and rounded to FP32 when v32 != nullptr): entry p of the CSC belongs to
// matrix k with off[k] <= p < off[k+1] and is entry perm[p] - off[k] of it
__global__ void gather_values_kernel(int64_t tot, int K, const int64_t *off, const double *const *vals,
                                     const int32_t *perm, double *v, float *v32) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < tot; p += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = K - 1;
        while (lo < hi) {  // last k with off[k] <= p
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= p) lo = mid; else hi = mid - 1;
        }
        const double x = vals[lo][perm[p] - off[lo]];
        v[p] = x;
        if (v32) v32[p] = (float)x;
    }
}

// K matrices of one structure: out[k m + q] = vals[k][perm[q]] (perm: the
// common CSC -> CSR positions of m entries)
__global__ void gather_values_shared_kernel(int64_t m, const double *const *vals, const int32_t *perm, double *out) {
    const int k = blockIdx.y;
    const double *v = vals[k];
    double *o = out + (int64_t)k * m;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x)
        o[q] = v[perm[q]];
}

cudaError_t gather_values_shared(sam_handle h, int64_t m, int K, const double *const *vals, const int32_t *perm,
                                 double *out) {
    if (m == 0 || K == 0) return cudaSuccess;
    int64_t bx = (m + 255) / 256;
    const int64_t cap = (int64_t)handle_sms(h) * 8 / K + 1;  // about one resident wave over all maps
    if (bx > cap) bx = cap;
    gather_values_shared_kernel<<<dim3((unsigned)bx, (unsigned)K), 256, 0, handle_stream(h)>>>(m, vals, perm, out);
    count_launch(h);
    return cudaGetLastError();
}

cudaError_t gather_values(sam_handle h, int64_t tot, int K, const int64_t *off, const double *const *vals,
                          const int32_t *perm, double *v, float *v32) {
    if (tot == 0) return cudaSuccess;
    int64_t blocks = (tot + 255) / 256;
    if (blocks > (int64_t)handle_sms(h) * 8) blocks = (int64_t)handle_sms(h) * 8;  // one resident wave
    gather_values_kernel<<<(unsigned)blocks, 256, 0, handle_stream(h)>>>(tot, K, off, vals, perm, v, v32);
    count_launch(h);
    return cudaGetLastError();
}

cudaError_t csr_spmv(sam_handle h, int n, const int32_t *rp, const int32_t *ci, const double *v, const double *x,
                     double *y) {
    if (n == 0) return cudaSuccess;
    int64_t threads = (int64_t)n * 32;
    spmv_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, handle_stream(h)>>>(n, rp, ci, v, x, y);
    count_launch(h);
    return cudaGetLastError();
}

cudaError_t csr_outer_on_pattern(sam_handle h, int n, const int32_t *rp, const int32_t *ci, const double *dy,
                                 const double *x, double *g) {
    if (n <= 0) return cudaSuccess;
    const int64_t threads = (int64_t)n * 32;
    outer_on_pattern_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, handle_stream(h)>>>(n, rp, ci, dy, x, g);
    count_launch(h);
    return cudaGetLastError();
}

cudaError_t residual_rows(sam_handle h, int n, const int32_t *krp, const int32_t *kci, const double *kv,
                          const int32_t *mrp, const int32_t *mci, const double *mv, const int32_t *zrp,
                          const int32_t *zci, const double *zv, double *row_r2, int32_t *flag) {
    if (n == 0) return cudaSuccess;
    int blocks = (n + kResWarps - 1) / kResWarps;
    int cap = handle_sms(h) * 32;
    if (blocks > cap) blocks = cap;
    residual_rows_kernel<<<blocks, kResWarps * 32, 0, handle_stream(h)>>>(n, krp, kci, kv, mrp, mci, mv, zrp, zci,
                                                                          zv, row_r2, flag);
    count_launch(h);
    return cudaGetLastError();
}

cudaError_t round_to_f32(sam_handle h, int64_t n, const double *in, float *out) {
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)handle_sms(h) * 8) blocks = (int64_t)handle_sms(h) * 8;  // one resident wave
    round_f32_kernel<<<(unsigned)blocks, 256, 0, handle_stream(h)>>>(n, in, out);
    count_launch(h);
    return cudaGetLastError();
}

namespace {
__global__ void tape_sizes_kernel(int64_t N, const int32_t *jcp, int64_t *sizes) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x)
        sizes[j] = tape_elems(jcp[j + 1] - jcp[j]);
}
}  // namespace

cudaError_t tape_offsets(sam_handle h, int64_t N, const int32_t *jcp, int64_t *sizes, int64_t *off) {
    if (N > 0) {
        int64_t blocks = (N + 255) / 256;
        if (blocks > (int64_t)handle_sms(h) * 8) blocks = (int64_t)handle_sms(h) * 8;
        tape_sizes_kernel<<<(unsigned)blocks, 256, 0, handle_stream(h)>>>(N, jcp, sizes);
        count_launch(h);
        if (cudaGetLastError() != cudaSuccess) return cudaErrorLaunchFailure;
    }
    return exclusive_scan_i64(h, sizes, off, N);
}

cudaError_t status_reduce(sam_handle h, const int32_t *colstat, int64_t n, int32_t *flag) {
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    status_max_kernel<<<(unsigned)blocks, 256, 0, handle_stream(h)>>>(colstat, n, flag);
    count_launch(h);
    return cudaGetLastError();
}

cudaError_t peak_fma(sam_handle h, double ms, double *f32, double *f64) {
    int blocks = handle_sms(h) * 8, threads = 256;
    probe<float>(h, ms * 0.25, blocks, threads);  // warm-up / clock ramp
    if (f32) *f32 = probe<float>(h, ms, blocks, threads);
    if (f64) *f64 = probe<double>(h, ms, blocks, threads);
    return cudaGetLastError();
}

}  // namespace sam
