// lsq.cu -- the batched column least-squares solves of SAM construction
// (arXiv 2406.17656, Sec. 2), FP32 register tiles with FP64 refinement, the
// dispatch over the size classes, and the refinement guard's FP64 re-solve
// and outcome counts.  The kernel is described in lsq_kernel.cuh.
#include "lsq_kernel.cuh"

namespace sam {

cudaError_t launch_lsq_bin(sam_handle h, int precision, const LsqArgs &args, int bin) {
    if (bin == kBinBig) return launch_lsq_big(h, args, bin, true, precision == SAM_FP32_REFINE);
    if (precision == SAM_FP64) return launch_lsq_fp64_bin(h, args, bin);
    // FP32 tiles: the shape of each size class comes from the handle (sam_tune)
    const bool b = handle_variant(h, bin) != 0;
    switch (bin) {
        case 0: return launch_one<F0, false>(h, args, 0);
        case 1: return b ? launch_one<F1b, false>(h, args, 1) : launch_one<F1, false>(h, args, 1);
        case 2: return b ? launch_one<F2b, false>(h, args, 2) : launch_one<F2, false>(h, args, 2);
        case 3: return b ? launch_one<F3b, false>(h, args, 3) : launch_one<F3, false>(h, args, 3);
        default: return b ? launch_one<F4b, false>(h, args, 4) : launch_one<F4, false>(h, args, 4);
    }
}

cudaError_t launch_lsq(sam_handle h, int precision, const LsqArgs &args) {
    for (int b = 0; b < kNumBins; ++b) {
        cudaError_t e = launch_lsq_bin(h, precision, args, b);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

namespace {
// columns that took s = 1..kAutoSteps steps, and FP64 re-solves: per-thread
// counts, summed over the warp by shuffles, one shared atomic per warp
__global__ void refine_count_kernel(int64_t N, const uint8_t *used, unsigned long long *counts) {
    __shared__ unsigned long long sh[kAutoSteps + 1];
    if (threadIdx.x <= kAutoSteps) sh[threadIdx.x] = 0ull;
    __syncthreads();
    unsigned c[kAutoSteps + 1] = {};
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const int u = used[j];
#pragma unroll
        for (int v = 0; v <= kAutoSteps; ++v) c[v] += (u == v + 1) ? 1u : 0u;
    }
#pragma unroll
    for (int v = 0; v <= kAutoSteps; ++v) {
        unsigned t = c[v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0 && t) atomicAdd(&sh[v], (unsigned long long)t);
    }
    __syncthreads();
    if (threadIdx.x <= kAutoSteps && sh[threadIdx.x]) atomicAdd(&counts[threadIdx.x], sh[threadIdx.x]);
}

// the columns flagged for the FP64 re-solve, in any order, into list;
// off[1] receives their number (off[0] = 0: the list as a work-list range)
__global__ void flag_list_kernel(int N, const int32_t *colstat, int32_t *list, int32_t *off) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool f = j < N && colstat[j] == kStRefine;
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&off[1], __popc(m));
    base = __shfl_sync(m, base, leader);
    if (f) list[base + __popc(m & ((1u << lane) - 1u))] = j;
}
}  // namespace

cudaError_t launch_refine_fallback(sam_handle h, const LsqArgs &args, int N, int32_t *list, int32_t *list_off,
                                   int64_t *counts, const RedoLists &redo) {
    cudaStream_t st = handle_stream(h);
    cudaError_t e;
    if (args.refine_steps < 0) {
        // automatic refinement: the columns whose first step asked for a
        // second, solved again from the start with two steps, by their size
        // classes' kernels (the guard after the second step sends a miss to
        // the FP64 re-solve below)
        if (!redo.bin || !redo.bins2 || !redo.work || !redo.bin_off || !redo.ws) return cudaErrorInvalidValue;
        if ((e = flagged_bins(h, N, redo.bin, args.colstat, kStStep2, redo.bins2)) != cudaSuccess ||
            (e = build_work_list(h, N, redo.bins2, redo.work, redo.bin_off, redo.ws)) != cudaSuccess)
            return e;
        LsqArgs a2 = args;
        a2.work = redo.work;
        a2.bin_off = redo.bin_off;
        a2.item_lo = a2.item_hi = 0;
        a2.refine_steps = kAutoSteps;
        // (the large class never flags a column: its kernel takes its own steps)
        for (int b = 0; b < kBinBig; ++b)
            if ((e = launch_lsq_bin(h, SAM_FP32_REFINE, a2, b)) != cudaSuccess) return e;
    }
    if ((e = cudaMemsetAsync(list_off, 0, sizeof(int32_t) * 2, st)) != cudaSuccess) return e;
    if (N > 0) {
        flag_list_kernel<<<(N + 255) / 256, 256, 0, st>>>(N, args.colstat, list, list_off);
        count_launch(h);
    }
    // every flagged column, whatever its size class, by the FP64 kernel of
    // the large class (results do not depend on the order of the list)
    LsqArgs a = args;
    a.work = list;
    a.bin_off = list_off;
    a.item_lo = a.item_hi = 0;
    if ((e = launch_lsq_big(h, a, 0, false)) != cudaSuccess) return e;
    if (counts) {
        if ((e = cudaMemsetAsync(counts, 0, sizeof(int64_t) * (kAutoSteps + 1), st)) != cudaSuccess) return e;
        int blocks = (N + 255) / 256;
        if (blocks > handle_sms(h) * 4) blocks = handle_sms(h) * 4;
        if (blocks < 1) blocks = 1;
        refine_count_kernel<<<blocks, 256, 0, st>>>(N, args.refine_used, reinterpret_cast<unsigned long long *>(counts));
        count_launch(h);
    }
    return cudaGetLastError();
}

}  // namespace sam
