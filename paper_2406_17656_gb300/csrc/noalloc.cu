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
#include "residual_row.cuh"

namespace {

constexpr int kStaticMaxRows = SAM_STATIC_MAX_ROWS;
constexpr int kBlocks = 256;  // fixed reduction grid: deterministic sums
constexpr int kThreads = 256;
constexpr int kWarps = 2;     // row kernel: warps per block

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

// Row i of R = A_k M - A_0 into rows[i] = ||R(i, :)||^2 (residual_row_sq,
// the routine sam_residual uses).  Does nothing when the validation kernel
// flagged an input.
__global__ void __launch_bounds__(kWarps * 32) static_rows_kernel(
    int n, const int32_t *krp, const int32_t *kci, const double *kv, const int32_t *mrp, const int32_t *mci,
    const double *mv, const int32_t *zrp, const int32_t *zci, const double *zv, double *rows, int32_t *flag) {
    __shared__ int keys[kWarps][sam::kResRowBuf];
    __shared__ double vals[kWarps][sam::kResRowBuf];
    if (*((volatile int32_t *)flag) != 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t i = (int64_t)blockIdx.x * kWarps + warp; i < n; i += (int64_t)gridDim.x * kWarps) {
        const double r2 =
            sam::residual_row_sq(i, lane, krp, kci, kv, mrp, mci, mv, zrp, zci, zv, keys[warp], vals[warp]);
        if (lane == 0) {
            rows[i] = r2 < 0.0 ? 0.0 : r2;
            if (r2 < 0.0) atomicCAS(flag, 0, SAM_ERR_UNSUPPORTED);
        }
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

// out[0] = ||R||_F, out[1] = ||R||_F / ||A_0||_F, *status = the flag; a
// flagged input gives NaN in both outputs, so that a caller who passes no
// status word cannot mistake the failure for an exact map
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
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        out[0] = st ? nan : fro;
        out[1] = st ? nan : (sa[0] <= 0.0 ? 0.0 : fro / sqrt(sa[0]));
        if (status) *status = st;
    }
}

// Device address of the static array for the current device.  It is looked
// up (cudaGetSymbolAddress, which allocates nothing) on every call made
// while the stream is not being captured, so that a device reset or a new
// primary context never leaves a stale address behind; a call made while
// the stream is being captured uses the address its device's last
// uncaptured call found (the first call on a device must therefore come
// before any capture).
constexpr int kMaxDevices = 64;
std::mutex g_lock;
double *g_addr[kMaxDevices] = {nullptr};

cudaError_t scratch_address(cudaStream_t st, int dev, double **out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;  // unknown: do not call into the runtime's loader
    }
    std::lock_guard<std::mutex> guard(g_lock);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double *>(p);
    }
    if (!g_addr[dev]) return cudaErrorStreamCaptureUnsupported;  // first call made under capture
    *out = g_addr[dev];
    return cudaSuccess;
}

// A matrix of order n >= 1 (the library's convention: an empty matrix is
// an invalid argument) with consistent sizes and pointers.
bool bad_csr(const sam_csr *A) {
    return !A || A->n < 1 || A->nnz < 0 || A->nnz > INT32_MAX || !A->row_ptr ||
           (A->nnz > 0 && (!A->col_idx || !A->val));
}

// Every array must already be reachable from the current device: this entry
// point cannot stage host memory (staging would need a device buffer), and
// memory of another device would be read by kernels launched on this one.
bool on_device(const void *p, int dev) {
    if (!p) return true;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

bool csr_on_device(const sam_csr *A, int dev) {
    return on_device(A->row_ptr, dev) && on_device(A->col_idx, dev) && on_device(A->val, dev);
}

}  // namespace

extern "C" sam_status sam_residual_static(void *cuda_stream, const sam_csr *A_k, const sam_csr *M_k,
                                          const sam_csr *A_0, double *out, int32_t *status) {
    if (bad_csr(A_k) || bad_csr(M_k) || bad_csr(A_0) || !out) return SAM_ERR_INVALID_ARG;
    const int n = A_k->n;
    if (M_k->n != n || A_0->n != n) return SAM_ERR_INVALID_ARG;
    if (n > kStaticMaxRows) return SAM_ERR_INVALID_ARG;  // beyond the fixed workspace
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SAM_ERR_CUDA;
    if (!csr_on_device(A_k, dev) || !csr_on_device(M_k, dev) || !csr_on_device(A_0, dev) || !on_device(out, dev) ||
        !on_device(status, dev))
        return SAM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double *base = nullptr;
    if (scratch_address(st, dev, &base) != cudaSuccess) return SAM_ERR_CUDA;
    const Slots s = slots_of(base);
    if (cudaMemsetAsync(s.flag, 0, sizeof(int32_t), st) != cudaSuccess) return SAM_ERR_CUDA;
    dim3 vg((unsigned)((n + 1 + 255) / 256), 3);
    static_validate_kernel<<<vg, 256, 0, st>>>(n, A_k->row_ptr, A_k->col_idx, A_k->nnz, M_k->row_ptr, M_k->col_idx,
                                               M_k->nnz, A_0->row_ptr, A_0->col_idx, A_0->nnz, s.flag);
    int blocks = (n + kWarps - 1) / kWarps;
    if (blocks > 4096) blocks = 4096;
    static_rows_kernel<<<blocks, kWarps * 32, 0, st>>>(n, A_k->row_ptr, A_k->col_idx, A_k->val, M_k->row_ptr,
                                                       M_k->col_idx, M_k->val, A_0->row_ptr, A_0->col_idx, A_0->val,
                                                       s.rows, s.flag);
    static_partial_kernel<<<dim3(kBlocks, 2), kThreads, 0, st>>>(s.rows, n, A_0->val, A_0->nnz, s.part_r, s.part_a,
                                                                 s.flag);
    static_final_kernel<<<1, kBlocks, 0, st>>>(s.part_r, s.part_a, s.flag, out, status);
    return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}
