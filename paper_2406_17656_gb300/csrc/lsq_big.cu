// lsq_big.cu -- the column problems of SAM construction (arXiv 2406.17656,
// Sec. 2: min_m || A_k(I_j, J_j) m - A_0(I_j, j) ||) that exceed the
// register tiles of lsq.cu: more than 64 shadow rows, more than 27 unknowns
// or more than 512 stored entries, as met by level-3 patterns of 9-point and
// 7-point stencils (the paper's "level 2", Sec. 5.1) or by sources with many
// entries per column (the NWP matrices of Sec. 5.2 have about 85).
//
// One thread block per column (a persistent grid over the class's work
// list), everything in shared memory:
//   * J_j from the pattern; I_j = the union of the rows of A_k(:, J_j),
//     gathered, sorted by a block-wide bitonic network and made unique;
//   * [B c] as a dense FP64 tile (column-major, leading dimension |I_j|):
//     B from A_k's CSC values, c from the target column, whose entries
//     outside I_j go to the residual only;
//   * textbook Householder QR of [B c] (Golub & Van Loan, Matrix
//     Computations, Alg. 5.2.1, with the right-hand side as the last
//     column): one warp forms reflector k, the block's warps apply it to
//     the remaining columns, one column per warp, the dot products summed
//     lane-wise then by a fixed xor tree (deterministic);
//   * back substitution R m = (Q^T c)(1:|J_j|) by one warp;
//   * the residual r = c - B m from its definition in FP64 (the stored
//     entries of B, column by column), ||r||^2 plus the target's entries
//     outside I_j.
// The class is solved in FP64 whatever precision the build asks for: these
// columns are rare, and the FP64 solve meets both accuracy bars.
#include <climits>

#include "common.cuh"

namespace sam {
namespace {

constexpr int kBigThreads = 512;
constexpr int kBigWarps = kBigThreads / 32;

enum { kSUk = 0, kSTau, kSBeta, kSOut2, kSRes2, kSNum };

struct BigHdr {
    long long colA[kBigJCap];  // value offset of column c of B (this map's values)
    int J[kBigJCap];
    int kcol[kBigJCap];        // structure offset of column c (kcp of the source column)
    int clen[kBigJCap + 1];
    int cb[kBigJCap + 1];      // prefix of clen: gather order of the candidates
    int I[kBigICap];           // shadow rows, ascending
    double r[kBigICap];        // c, then the residual
    double y[kBigJCap];        // (Q^T c)(1:|J|)
    double m[kBigJCap];        // the solution
    int wsum[kBigWarps];
    double scal[kSNum];
    int status;                // of the current column (uniform after a barrier)
    int nI;
    int pad_;
};
static_assert(sizeof(BigHdr) % 16 == 0, "the tile after the header must stay 16-byte aligned");

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int search_rows(const int *I, int nI, int key) {
    int lo = 0, hi = nI - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int v = I[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

__device__ __forceinline__ void set_status(BigHdr &H, int st) {
    atomicMax(&H.status, st);
}

__global__ void __launch_bounds__(kBigThreads, 1) lsq_big_kernel(LsqArgs args, int bin) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BigHdr &H = *reinterpret_cast<BigHdr *>(smem_raw);
    double *T = reinterpret_cast<double *>(smem_raw + sizeof(BigHdr));
    int *keys = reinterpret_cast<int *>(T);  // the candidate rows, before the tile exists
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    const int w0 = args.bin_off[bin] + (args.item_hi > 0 ? args.item_lo : 0);
    const int items = args.item_hi > 0 ? args.item_hi - args.item_lo : args.bin_off[bin + 1] - w0;
    const bool sh = args.shadow_shared != 0;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int jj = args.work[w0 + item];
        const int kmap = jj / args.n;
        const int jl = jj - kmap * args.n;
        const int js = sh ? jl : jj;  // column of the pattern data
        const int64_t aoff = sh ? (int64_t)kmap * args.map_nnz_src : 0;
        const int64_t poff = sh ? (int64_t)kmap * args.map_nnz_pat : 0;
        const int roff = kmap * args.n;
        const int zc = args.zbig ? jj : jl;
        const int zro = (sh ? 0 : roff) - (args.zbig ? roff : 0);  // target rows -> source row numbering
        const int jb = args.jcp[js];
        const int nJ = args.jcp[js + 1] - jb;
        if (tid == 0) {
            H.status = nJ > kBigJCap ? kStUnsupported : kStOk;
            H.nI = 0;
        }
        __syncthreads();
        // ---- the columns of J_j
        if (H.status == kStOk) {
            for (int c = tid; c < nJ; c += kBigThreads) {
                const int col = args.jri[jb + c];
                const int a0 = args.kcp[col];
                H.J[c] = col;
                H.kcol[c] = a0;
                H.clen[c] = args.kcp[col + 1] - a0;
                H.colA[c] = (long long)a0 + aoff;
            }
        }
        __syncthreads();
        if (tid == 0 && H.status == kStOk) {
            int s = 0;
            for (int c = 0; c < nJ; ++c) {
                H.cb[c] = s;
                s += H.clen[c];
            }
            H.cb[nJ] = s;
            if (s > kBigLCap) H.status = kStUnsupported;
        }
        __syncthreads();
        // ---- I_j: candidates sorted (bitonic, padded to a power of two), unique
        if (H.status == kStOk) {
            const int ntot = H.cb[nJ];
            int p2 = 1;
            while (p2 < ntot) p2 <<= 1;
            for (int q = tid; q < p2; q += kBigThreads) {
                int v = INT_MAX;
                if (q < ntot) {
                    int lo = 0, hi = nJ - 1;  // the column holding candidate q
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (H.cb[mid] <= q) lo = mid; else hi = mid - 1;
                    }
                    v = args.kri[H.kcol[lo] + (q - H.cb[lo])];
                }
                keys[q] = v;
            }
            __syncthreads();
            for (int k = 2; k <= p2; k <<= 1)
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int q = tid; q < p2; q += kBigThreads) {
                        const int u = q ^ j;
                        if (u > q) {
                            const int a = keys[q], b = keys[u];
                            if ((a > b) == ((q & k) == 0)) {
                                keys[q] = b;
                                keys[u] = a;
                            }
                        }
                    }
                    __syncthreads();
                }
            // distinct values, in order: each thread counts its contiguous chunk
            const int chunk = (p2 + kBigThreads - 1) / kBigThreads;
            const int q0 = tid * chunk, q1 = min(p2, q0 + chunk);
            int cnt = 0;
            for (int q = q0; q < q1; ++q)
                cnt += (keys[q] != INT_MAX && (q == 0 || keys[q] != keys[q - 1])) ? 1 : 0;
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) H.wsum[warp] = incl;
            __syncthreads();
            if (tid == 0) {
                int s = 0;
                for (int w = 0; w < kBigWarps; ++w) {
                    const int t = H.wsum[w];
                    H.wsum[w] = s;
                    s += t;
                }
                H.nI = s;
                if (s > kBigICap || (int64_t)s * (nJ + 1) > kBigTileDoubles) H.status = kStUnsupported;
                else if (s < nJ) H.status = kStRank;  // a column of B without entries
            }
            __syncthreads();
            if (H.status == kStOk) {
                int pos = H.wsum[warp] + incl - cnt;
                for (int q = q0; q < q1; ++q)
                    if (keys[q] != INT_MAX && (q == 0 || keys[q] != keys[q - 1])) H.I[pos++] = keys[q];
            }
        }
        __syncthreads();
        const int nI = H.nI;
        const int ld = nI;
        // ---- the tile [B c] and the target column
        if (H.status == kStOk) {
            for (int q = tid; q < ld * (nJ + 1); q += kBigThreads) T[q] = 0.0;
            for (int i = tid; i < nI; i += kBigThreads) H.r[i] = 0.0;
        }
        __syncthreads();
        if (H.status == kStOk) {
            for (int c = warp; c < nJ; c += kBigWarps)
                for (int e = lane; e < H.clen[c]; e += 32) {
                    const int p = search_rows(H.I, nI, args.kri[H.kcol[c] + e]);
                    if (p >= 0) T[p + ld * c] = args.kcv[H.colA[c] + e];
                    else set_status(H, kStUnsupported);  // impossible: every row of B is in I_j
                }
            if (warp == kBigWarps - 1) {
                const int zb = args.zcp[zc], ze = args.zcp[zc + 1];
                double o2 = 0.0;
                for (int t = zb + lane; t < ze; t += 32) {
                    const double v = args.zcv[t];
                    const int p = search_rows(H.I, nI, args.zri[t] + zro);
                    if (p >= 0) {
                        T[p + ld * nJ] = v;
                        H.r[p] = v;
                    } else {
                        o2 = fma(v, v, o2);
                    }
                }
                o2 = warp_sum_f64(o2);
                if (lane == 0) H.scal[kSOut2] = o2;
            }
        }
        __syncthreads();
        // ---- Householder QR of [B c]
        if (H.status == kStOk) {
            for (int k = 0; k < nJ; ++k) {
                if (warp == 0) {
                    double s = 0.0;
                    for (int i = k + 1 + lane; i < nI; i += 32) {
                        const double x = T[i + ld * k];
                        s = fma(x, x, s);
                    }
                    s = warp_sum_f64(s);
                    if (lane == 0) {
                        const double alpha = T[k + ld * k];
                        const double nrm = sqrt(fma(alpha, alpha, s));
                        const double beta = (s == 0.0) ? alpha : ((alpha >= 0.0) ? -nrm : nrm);
                        const double uk = alpha - beta;
                        H.scal[kSUk] = uk;
                        H.scal[kSTau] = (s == 0.0) ? 0.0 : -1.0 / (beta * uk);
                        H.scal[kSBeta] = beta;
                    }
                }
                __syncthreads();
                const double uk = H.scal[kSUk], taup = H.scal[kSTau];
                if (taup != 0.0) {
                    for (int t = k + 1 + warp; t <= nJ; t += kBigWarps) {
                        double w = 0.0;
                        for (int i = k + 1 + lane; i < nI; i += 32) w = fma(T[i + ld * k], T[i + ld * t], w);
                        w = warp_sum_f64(w);
                        w = fma(uk, T[k + ld * t], w);
                        const double coef = taup * w;
                        __syncwarp();
                        if (lane == 0) T[k + ld * t] = fma(-coef, uk, T[k + ld * t]);
                        for (int i = k + 1 + lane; i < nI; i += 32) T[i + ld * t] = fma(-coef, T[i + ld * k], T[i + ld * t]);
                    }
                }
                __syncthreads();
                if (tid == 0) T[k + ld * k] = H.scal[kSBeta];
            }
        }
        __syncthreads();
        // ---- pivots, back substitution R m = (Q^T c)(1:|J|), residual
        if (H.status == kStOk && warp == 0) {
            int st = kStOk;
            for (int k = lane; k < nJ; k += 32) {
                const double d = T[k + ld * k];
                if (!isfinite(d)) st = max(st, (int)kStNonfinite);
                else if (d == 0.0) st = max(st, (int)kStRank);
                H.y[k] = T[k + ld * nJ];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) st = max(st, __shfl_xor_sync(0xffffffffu, st, o));
            __syncwarp();
            if (st == kStOk) {
                for (int k = nJ - 1; k >= 0; --k) {
                    const double mk = H.y[k] / T[k + ld * k];
                    __syncwarp();
                    for (int i = lane; i < k; i += 32) H.y[i] = fma(-T[i + ld * k], mk, H.y[i]);
                    if (lane == 0) H.m[k] = mk;
                    __syncwarp();
                }
                int nf = 0;
                for (int c = 0; c < nJ; ++c) {
                    const double mc = H.m[c];
                    nf |= !isfinite(mc);
                    for (int e = lane; e < H.clen[c]; e += 32) {
                        const int p = search_rows(H.I, nI, args.kri[H.kcol[c] + e]);
                        if (p >= 0) H.r[p] = fma(-args.kcv[H.colA[c] + e], mc, H.r[p]);
                    }
                    __syncwarp();
                }
                double s = 0.0;
                for (int i = lane; i < nI; i += 32) s = fma(H.r[i], H.r[i], s);
                s = warp_sum_f64(s);
                if (nf || !isfinite(s)) st = kStNonfinite;
                if (lane == 0) H.scal[kSRes2] = s;
            }
            if (lane == 0 && st != kStOk) set_status(H, st);
        }
        __syncthreads();
        // ---- outputs
        if (warp == 0) {
            const int status = H.status;
            const bool ok = status == kStOk;
            for (int c = lane; c < nJ; c += 32)
                args.mval[(int64_t)args.csr_pos[jb + c] + poff] = ok ? H.m[c] : 0.0;
            if (lane == 0) {
                const double r2 = H.scal[kSRes2];
                args.colres[jj] = ok ? (r2 > 0.0 ? r2 : 0.0) + H.scal[kSOut2] : 0.0;
                args.colstat[jj] = status;
                if (args.refine_used) args.refine_used[jj] = (uint8_t)(kAutoSteps + 1);  // solved in FP64
            }
        }
        __syncthreads();  // the next column reuses the shared memory
    }
}

}  // namespace

cudaError_t launch_lsq_big(sam_handle h, const LsqArgs &args, int bin, bool profile) {
    const size_t smem = sizeof(BigHdr) + sizeof(double) * (size_t)kBigTileDoubles;
    const cudaError_t e = cudaFuncSetAttribute(lsq_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (profile) profile_begin(h, bin);
    lsq_big_kernel<<<handle_sms(h), kBigThreads, smem, handle_stream(h)>>>(args, bin);
    count_launch(h);
    if (profile) profile_end(h, bin);
    return cudaGetLastError();
}

}  // namespace sam
