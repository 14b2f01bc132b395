// noalloc.cu -- sam_residual_static: the residual of Eq. (res) for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or any allocating routine at all: code
// that runs while a memory budget is already fully handed out, code that
// must never touch the allocator (for instance a step that runs between
// allocations of a framework's caching allocator it does not own), or a
// host that gives the library device pointers only.  This entry point keeps
// its working memory in one file-scope device array of fixed size instead:
// per-row partial sums, per-block partial sums and a status word.  Its cost
// is that every GPU which loads the library holds the array until the
// process exits, and that the problem size it accepts is bounded.
//
// The array is shared by every call: a call overwrites all of it that it
// reads (the status word is cleared at the start of each call), so results
// never depend on an earlier call; two calls whose work overlaps on the GPU
// (different streams, or different host threads) race on it and must be
// ordered by the caller.
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kStaticMaxRows = SAM_STATIC_MAX_ROWS;
constexpr int kBlocks = 256;  // fixed reduction grid: deterministic sums
constexpr int kThreads = 256;
constexpr int kWarps = 2;     // row kernel: warps per block
constexpr int kBuf = 1024;    // candidate entries per row

// [0, kStaticMaxRows): squared residual of every row
// [kStaticMaxRows, +kBlocks): block partials of sum ||R(i,:)||^2
// [.., +kBlocks): block partials of ||A_0||_F^2
// [.., +1): status word (as a 64-bit slot; only its low 32 bits are used)
constexpr size_t kWords = (size_t)kStaticMaxRows + 2 * kBlocks + 1;
static __device__ __align__(256) double g_static_scratch[kWords];

struct Slots {
    double *rows, *part_r, *part_a;
    int32_t *flag;
};

Slots slots_of(double *base) {
    Slots s;
    s.rows = base;
    s.part_r = base + kStaticMaxRows;
    s.part_a = s.part_r + kBlocks;
    s.flag = reinterpret_cast<int32_t *>(s.part_a + kBlocks);
    return s;
}

// CSR checks of the three inputs (blockIdx.y selects the matrix)
__global__ void static_validate_kernel(int n, const int32_t *rp0, const int32_t *ci0, int64_t nz0,
                                       const int32_t *rp1, const int32_t *ci1, int64_t nz1, const int32_t *rp2,
                                       const int32_t *ci2, int64_t nz2, int32_t *flag) {
    const int32_t *rp = blockIdx.y == 0 ? rp0 : (blockIdx.y == 1 ? rp1 : rp2);
    const int32_t *ci = blockIdx.y == 0 ? ci0 : (blockIdx.y == 1 ? ci1 : ci2);
    const int64_t nz = blockIdx.y == 0 ? nz0 : (blockIdx.y == 1 ? nz1 : nz2);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && (rp[0] != 0 || (int64_t)rp[n] != nz)) atomicCAS(flag, 0, SAM_ERR_BAD_CSR);
    if (i >= n) return;
    const int b = rp[i], e = rp[i + 1];
    if (e < b || b < 0 || (int64_t)e > nz) {
        atomicCAS(flag, 0, SAM_ERR_BAD_CSR);
        return;
    }
    int prev = -1;
    for (int t = b; t < e; ++t) {
        const int c = ci[t];
        if (c <= prev || c >= n) {
            atomicCAS(flag, 0, SAM_ERR_BAD_CSR);
            return;
        }
        prev = c;
    }
}

// Row i of R = A_k M - A_0 into rows[i] = ||R(i, :)||^2: the products
// A_k(i, c) M(c, :) and -A_0(i, :) as (column, value) pairs, sorted by column
// with a fixed bitonic network, summed per column, squared.  Does nothing
// when the validation kernel flagged an input.
__global__ void __launch_bounds__(kWarps * 32) static_rows_kernel(
    int n, const int32_t *krp, const int32_t *kci, const double *kv, const int32_t *mrp, const int32_t *mci,
    const double *mv, const int32_t *zrp, const int32_t *zci, const double *zv, double *rows, int32_t *flag) {
    __shared__ int keys[kWarps][kBuf];
    __shared__ double vals[kWarps][kBuf];
    if (*((volatile int32_t *)flag) != 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *K = keys[warp];
    double *V = vals[warp];
    for (int64_t i = (int64_t)blockIdx.x * kWarps + warp; i < n; i += (int64_t)gridDim.x * kWarps) {
        int cnt = zrp[i + 1] - zrp[i];
        for (int base = krp[i]; base < krp[i + 1]; base += 32) {
            const int e = base + lane;
            int len = (e < krp[i + 1]) ? mrp[kci[e] + 1] - mrp[kci[e]] : 0;
            for (int o = 16; o > 0; o >>= 1) len += __shfl_xor_sync(0xffffffffu, len, o);
            cnt += len;
        }
        if (cnt > kBuf) {
            if (lane == 0) {
                rows[i] = 0.0;
                atomicCAS(flag, 0, SAM_ERR_UNSUPPORTED);
            }
            continue;
        }
        const int zb = zrp[i], ze = zrp[i + 1];
        for (int t = zb + lane; t < ze; t += 32) {
            K[t - zb] = zci[t];
            V[t - zb] = -zv[t];
        }
        int off = ze - zb;
        for (int e = krp[i]; e < krp[i + 1]; ++e) {
            const int c = kci[e];
            const double a = kv[e];
            const int mb = mrp[c], me = mrp[c + 1];
            for (int t = mb + lane; t < me; t += 32) {
                K[off + t - mb] = mci[t];
                V[off + t - mb] = a * mv[t];
            }
            off += me - mb;
        }
        __syncwarp();
        int p2 = 32;
        while (p2 < cnt) p2 <<= 1;
        for (int t = cnt + lane; t < p2; t += 32) {
            K[t] = 0x7fffffff;
            V[t] = 0.0;
        }
        __syncwarp();
        for (int k = 2; k <= p2; k <<= 1)
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int t = lane; t < p2; t += 32) {
                    const int u = t ^ jj;
                    if (u > t) {
                        const bool up = (t & k) == 0;
                        const int a = K[t], b = K[u];
                        if ((a > b) == up) {
                            K[t] = b;
                            K[u] = a;
                            const double va = V[t];
                            V[t] = V[u];
                            V[u] = va;
                        }
                    }
                }
                __syncwarp();
            }
        double r2 = 0.0;
        for (int t = lane; t < cnt; t += 32) {
            if (t == 0 || K[t - 1] != K[t]) {
                double s = 0.0;
                for (int q = t; q < cnt && K[q] == K[t]; ++q) s += V[q];
                r2 = fma(s, s, r2);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
        if (lane == 0) rows[i] = r2;
        __syncwarp();
    }
}

// fixed-grid partial sums (blockIdx.y = 0: rows; 1: squares of A_0's values)
__global__ void __launch_bounds__(kThreads) static_partial_kernel(const double *rows, int64_t n, const double *zv,
                                                                  int64_t znnz, double *part_r, double *part_a,
                                                                  const int32_t *flag) {
    __shared__ double sh[kThreads];
    const bool first = blockIdx.y == 0;
    const double *x = first ? rows : zv;
    const int64_t len = first ? n : znnz;
    double s = 0.0;
    if (*((volatile const int32_t *)flag) == 0)
        for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < len; i += (int64_t)kBlocks * kThreads) {
            const double v = x[i];
            s += first ? v : v * v;
        }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) (first ? part_r : part_a)[blockIdx.x] = sh[0];
}

// out[0] = ||R||_F, out[1] = ||R||_F / ||A_0||_F, *status = the flag
__global__ void __launch_bounds__(kBlocks) static_final_kernel(const double *part_r, const double *part_a,
                                                               const int32_t *flag, double *out, int32_t *status) {
    __shared__ double sr[kBlocks], sa[kBlocks];
    sr[threadIdx.x] = part_r[threadIdx.x];
    sa[threadIdx.x] = part_a[threadIdx.x];
    __syncthreads();
    for (int o = kBlocks / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sr[threadIdx.x] += sr[threadIdx.x + o];
            sa[threadIdx.x] += sa[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int32_t st = *flag;
        const double fro = sqrt(sr[0]);
        out[0] = st ? 0.0 : fro;
        out[1] = (st || sa[0] <= 0.0) ? 0.0 : fro / sqrt(sa[0]);
        if (status) *status = st;
    }
}

// Device address of the static array, looked up once per device with that
// device current.
constexpr int kMaxDevices = 64;
std::mutex g_lock;
double *g_addr[kMaxDevices] = {nullptr};

cudaError_t scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

bool bad_csr(const sam_csr *A) {
    return !A || A->n < 0 || A->nnz < 0 || A->nnz > INT32_MAX || !A->row_ptr || (A->nnz > 0 && (!A->col_idx || !A->val));
}

// Every array must already be reachable from the device: this entry point
// cannot stage host memory (staging would need a device buffer).
bool on_device(const void *p) {
    if (!p) return true;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool csr_on_device(const sam_csr *A) { return on_device(A->row_ptr) && on_device(A->col_idx) && on_device(A->val); }

}  // namespace

extern "C" sam_status sam_residual_static(void *cuda_stream, const sam_csr *A_k, const sam_csr *M_k,
                                          const sam_csr *A_0, double *out, int32_t *status) {
    if (bad_csr(A_k) || bad_csr(M_k) || bad_csr(A_0) || !out) return SAM_ERR_INVALID_ARG;
    const int n = A_k->n;
    if (M_k->n != n || A_0->n != n) return SAM_ERR_INVALID_ARG;
    if (n > kStaticMaxRows) return SAM_ERR_INVALID_ARG;  // beyond the fixed workspace
    if (!csr_on_device(A_k) || !csr_on_device(M_k) || !csr_on_device(A_0) || !on_device(out) || !on_device(status))
        return SAM_ERR_INVALID_ARG;
    double *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return SAM_ERR_CUDA;
    const Slots s = slots_of(base);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (cudaMemsetAsync(s.flag, 0, sizeof(int32_t), st) != cudaSuccess) return SAM_ERR_CUDA;
    if (n > 0) {
        dim3 vg((unsigned)((n + 1 + 255) / 256), 3);
        static_validate_kernel<<<vg, 256, 0, st>>>(n, A_k->row_ptr, A_k->col_idx, A_k->nnz, M_k->row_ptr,
                                                   M_k->col_idx, M_k->nnz, A_0->row_ptr, A_0->col_idx, A_0->nnz,
                                                   s.flag);
        int blocks = (n + kWarps - 1) / kWarps;
        if (blocks > 4096) blocks = 4096;
        static_rows_kernel<<<blocks, kWarps * 32, 0, st>>>(n, A_k->row_ptr, A_k->col_idx, A_k->val, M_k->row_ptr,
                                                           M_k->col_idx, M_k->val, A_0->row_ptr, A_0->col_idx,
                                                           A_0->val, s.rows, s.flag);
    }
    static_partial_kernel<<<dim3(kBlocks, 2), kThreads, 0, st>>>(s.rows, n, A_0->val, A_0->nnz, s.part_r, s.part_a,
                                                                 s.flag);
    static_final_kernel<<<1, kBlocks, 0, st>>>(s.part_r, s.part_a, s.flag, out, status);
    return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}
