// adjoint.cu -- the adjoint of the column least-squares solves (kernel in
// adjoint_core.cuh): the dispatch over the size classes, the FP64 tiles, and
// the deterministic reduction of the per-column dL/dB blocks into dL/dA_k.
#include "adjoint_core.cuh"

namespace sam {
namespace {

constexpr int kReduceThreads = 256;

// dA(e) for the stored entries e of column c (one warp per column).  The
// contributions come from the map columns whose patterns hold c (map CSR
// row c: mrp[c] .. mrp[c+1]), each a block of the column's len entries in
// dB at dbase[t] (< 0: none).  The warp splits into G = 32 / len lane
// groups; group g sums blocks g, g + G, g + 2G, ... in that order, two loads
// in flight, and the groups' sums are added in group order, so the result
// is fixed by the inputs.
__global__ void __launch_bounds__(kReduceThreads) adjoint_reduce_kernel(int N, const int32_t *kcp, const int32_t *mrp,
                                                                       const int64_t *dbase, const double *dB,
                                                                       double *dak) {
    __shared__ double part[kReduceThreads / 32][32];
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (c >= N) return;  // whole warps
    const int b = kcp[c], e = kcp[c + 1], len = e - b;
    const int tb = mrp[c], te = mrp[c + 1];
    if (len <= 0) return;
    if (len > 32) {
        for (int p = lane; p < len; p += 32) {
            double acc = 0.0;
            for (int t = tb; t < te; ++t) {
                const int64_t base = dbase[t];
                if (base >= 0) acc += dB[base + p];
            }
            dak[b + p] = acc;
        }
        return;
    }
    const int G = 32 / len;
    const int g = lane / len, p = lane - g * len;
    // the column's block offsets are read a chunk of W = G floor(32 / G)
    // pattern entries at a time, one per lane, and handed to the groups by
    // shuffles: group g's entries in the chunk are t0 + g + k G (k < W / G),
    // the same sequence as a stride-G walk, so the sums keep their order;
    // their dL/dB values are loaded kLoads at a time, all before the adds
    constexpr int kLoads = 4;
    const int W = G * (32 / G), KC = W / G;
    double acc = 0.0;
    for (int t0 = tb; t0 < te; t0 += W) {
        const int64_t mine = (lane < W && t0 + lane < te) ? dbase[t0 + lane] : -1;
        const int kc = min(KC, (te - t0 + G - 1) / G);  // the most entries a group has in this chunk
        for (int k0 = 0; k0 < kc; k0 += kLoads) {
            int64_t b[kLoads];
            double v[kLoads];
#pragma unroll
            for (int u = 0; u < kLoads; ++u) {
                const int src = g + (k0 + u) * G;
                b[u] = shfl(mine, src & 31);
                if (!(g < G && k0 + u < KC && t0 + src < te)) b[u] = -1;
            }
#pragma unroll
            for (int u = 0; u < kLoads; ++u) v[u] = b[u] >= 0 ? dB[b[u] + p] : 0.0;
#pragma unroll
            for (int u = 0; u < kLoads; ++u) acc += v[u];
        }
    }
    part[warp][lane] = acc;
    __syncwarp();
    if (lane < len) {
        double sum = part[warp][lane];
        for (int q = 1; q < G; ++q) sum += part[warp][q * len + lane];
        dak[b + lane] = sum;
    }
}

__global__ void permute_scatter_kernel(int64_t nnz, const int32_t *perm, const double *in, double *out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nnz) out[perm[p]] = in[p];
}

}  // namespace

cudaError_t launch_adjoint(sam_handle h, int precision, const LsqArgs &args) {
    cudaError_t e;
    const bool tape = args.fac_mode == kTapeReplay;
    for (int b = 0; b < kRegBins; ++b) {
        // with a tape the two smallest classes still recompute R: their QR
        // (at most 9 unknowns) costs less than reading and unpacking the tape
        if (tape && b >= 2) e = launch_adjoint_tape_bin(h, precision, args, b);
        else if (precision == SAM_FP32_REFINE) e = launch_adjoint_f32_bin(h, args, b);
        else {
            switch (b) {
                case 0: e = launch_one<D0, true>(h, args, 0); break;
                case 1: e = launch_one<D1, true>(h, args, 1); break;
                case 2: e = launch_one<D2, true>(h, args, 2); break;
                case 3: e = launch_one<D3, true>(h, args, 3); break;
                default: e = launch_one<D4, true>(h, args, 4); break;
            }
        }
        if (e != cudaSuccess) return e;
    }
    return launch_adjoint_big(h, args, kBinBig);
}

cudaError_t adjoint_reduce(sam_handle h, int N, const int32_t *kcp, const int32_t *mrp, const int64_t *dbase,
                           const double *dB, double *dak_csc) {
    if (N == 0) return cudaSuccess;
    const int64_t threads = (int64_t)N * 32;
    adjoint_reduce_kernel<<<(unsigned)((threads + kReduceThreads - 1) / kReduceThreads), kReduceThreads, 0,
                            handle_stream(h)>>>(N, kcp, mrp, dbase, dB, dak_csc);
    count_launch(h);
    return cudaGetLastError();
}

cudaError_t permute_scatter_f64(sam_handle h, int64_t nnz, const int32_t *perm, const double *in, double *out) {
    if (nnz == 0) return cudaSuccess;
    permute_scatter_kernel<<<(unsigned)((nnz + 255) / 256), 256, 0, handle_stream(h)>>>(nnz, perm, in, out);
    count_launch(h);
    return cudaGetLastError();
}

}  // namespace sam
