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
//     column): the block's warps apply reflector k to the remaining
//     columns, one column per warp, the dot products summed lane-wise then
//     by a fixed xor tree (deterministic); the warp that updates column
//     k + 1 forms reflector k + 1 at once (one barrier per reflector);
//   * back substitution R m = (Q^T c)(1:|J_j|) by one warp;
//   * the residual r = c - B m from its definition in FP64 (the stored
//     entries of B, column by column), ||r||^2 plus the target's entries
//     outside I_j.
// Two arithmetic types.  FP64 (SAM_FP64 builds, and the re-solve of every
// column that the refinement's guard flags): tile, QR and solves in FP64.
// FP32 (SAM_FP32_REFINE builds): the tile, the QR and the triangular solves
// in FP32 (half the shared memory: two blocks per SM), then the corrected
// semi-normal-equation steps of the register classes, g = B^T r in FP64,
// R^T R d = g in FP32, m += d, r -= B d in FP64, under the same accuracy
// guard; a column that misses it is re-solved by the FP64 kernel.
#include <cfloat>
#include <climits>

#include "common.cuh"

namespace sam {
namespace {

constexpr int kBigThreads = 512;
constexpr int kBigWarps = kBigThreads / 32;

enum { kSOut2 = 0, kSRes2, kSKap2, kSMsq, kSDprev, kSNum };
enum { kRStop = 0, kRMiss, kRUsed, kRNum };

struct __align__(16) BigHdr {
    long long colA[kBigJCap];  // value offset of column c of B (this map's values)
    int J[kBigJCap];
    int kcol[kBigJCap];        // structure offset of column c (kcp of the source column)
    int clen[kBigJCap + 1];
    int cb[kBigJCap + 1];      // prefix of clen: gather order of the candidates
    // the QR's band: rband[k] = 1 + the last row holding an entry of columns
    // 0..k (at least k + 1), cband[k] = 1 + the last column whose first row
    // is below rband[k] (at least k + 1); built from each column's last and
    // first rows
    short rband[kBigJCap];
    short cband[kBigJCap];
    short cfirst[kBigJCap];    // first row of column c, then the suffix minimum
    int I[kBigICap];           // shadow rows, ascending
    double r[kBigICap];        // c, then the residual
    double y[kBigJCap];        // (Q^T c)(1:|J|), in the tile's type
    double m[kBigJCap];        // the solution
    double g[kBigJCap];        // refinement: B^T r (rounded to FP32)
    float dv[kBigJCap];        // refinement: the correction d
    int wsum[kBigWarps];
    int rstate[kRNum];         // refinement: stop, guard missed, steps taken
    double qp[2][4];           // reflectors k and k + 1: u_k, tau', beta (in the tile's type)
    double scal[kSNum];
    int status;                // of the current column (uniform after a barrier)
    int nI;
    int pad_;
};
static_assert(sizeof(BigHdr) % 16 == 0, "the tile after the header must stay 16-byte aligned");

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_f64(double v) { return warp_sum<double>(v); }

// a value of [B c] in the tile's type: FP64 as stored, FP32 from the rounded
// copy the build made for the FP32 tiles
template <typename TT>
__device__ __forceinline__ TT big_value(const double *v, const float *v32, int64_t i) {
    if constexpr (sizeof(TT) == 4) return v32[i];
    else return v[i];
}

// blocks per SM: the FP64 tile fills the shared memory of one, the FP32 tile
// half of it
template <typename TT>
struct BigBlocks {
    static constexpr int value = sizeof(TT) == 4 ? 2 : 1;
};

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

// Reflector k (u_k, tau') applied by one warp to the NQ columns tq[] of the
// tile, rows k..re-1 (the rows after re are zero in column k): each column's
// dot product summed lane-wise then by a fixed xor tree, as one column at a
// time would
template <typename TT, int NQ>
__device__ __forceinline__ void apply_cols(TT *T, int ld, int re, int k, const int (&tq)[4], int lane, TT uk,
                                           TT taup) {
    TT w[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) w[q] = TT(0);
    for (int i = k + 1 + lane; i < re; i += 32) {
        const TT v = T[i + ld * k];
#pragma unroll
        for (int q = 0; q < NQ; ++q) w[q] = fma(v, T[i + ld * tq[q]], w[q]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < NQ; ++q) w[q] += __shfl_xor_sync(0xffffffffu, w[q], o);
    TT coef[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) coef[q] = taup * fma(uk, T[k + ld * tq[q]], w[q]);
    __syncwarp();
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) T[k + ld * tq[q]] = fma(-coef[q], uk, T[k + ld * tq[q]]);
    }
    for (int i = k + 1 + lane; i < re; i += 32) {
        const TT v = T[i + ld * k];
#pragma unroll
        for (int q = 0; q < NQ; ++q) T[i + ld * tq[q]] = fma(-coef[q], v, T[i + ld * tq[q]]);
    }
}

// Householder reflector of column k of the tile (rows k..re-1; the rows
// after re are zero in column k), by one warp: out = {u_k, tau', beta} with
// beta = -sign(alpha) ||x||, u_k = alpha - beta and tau' = -1 / (beta u_k)
// (0 when the column is already zero below the diagonal); the sum of
// squares lane-wise, then by a fixed xor tree
template <typename TT>
__device__ __forceinline__ void reflector(const TT *T, int ld, int re, int k, int lane, TT *out) {
    TT s = TT(0);
    for (int i = k + 1 + lane; i < re; i += 32) {
        const TT x = T[i + ld * k];
        s = fma(x, x, s);
    }
    s = warp_sum<TT>(s);
    if (lane == 0) {
        const TT alpha = T[k + ld * k];
        const TT nrm = sqrt(fma(alpha, alpha, s));
        const TT beta = (s == TT(0)) ? alpha : ((alpha >= TT(0)) ? -nrm : nrm);
        const TT uk = alpha - beta;
        out[0] = uk;
        out[1] = (s == TT(0)) ? TT(0) : TT(-1) / (beta * uk);
        out[2] = beta;
    }
}

// The adjoint of one large column (FP64; R in the tile's upper triangle, r =
// c - B m in H.r): lambda = (R^T R)^{-1} g, w = B lambda (after the tile),
// dL/dB(i, c) = r_i (lambda_c - 2 rho m_c) - w_i m_c into the column's
// block (gather order) with the block offsets of its pattern entries,
// dL/dM's direct residual part -2 rho (B^T r), dL/dA_0 of the target column.
__device__ __forceinline__ void big_adjoint(const LsqArgs &args, BigHdr &H, double *T, int ld, int nI, int nJ,
                                            int jj, int jb, int64_t poff, int zc, int zro, int64_t zoff, int tid,
                                            int lane, int warp) {
    double *wv = T + (size_t)ld * (nJ + 1);
    if (tid == 0 && H.status == kStOk && (int64_t)ld * (nJ + 2) > kBigTileDoubles) H.status = kStUnsupported;
    __syncthreads();
    const double rho = args.resid_weight;
    if (H.status == kStOk && warp == 0) {
        for (int k = 0; k < nJ; ++k) {  // R^T y = g
            double sk = 0.0;
            for (int i = lane; i < k; i += 32) sk = fma(T[i + ld * k], H.y[i], sk);
            sk = warp_sum_f64(sk);
            if (lane == 0) H.y[k] = (H.g[k] - sk) / T[k + ld * k];
            __syncwarp();
        }
        for (int k = nJ - 1; k >= 0; --k) {  // R lambda = y
            const double lk = H.y[k] / T[k + ld * k];
            __syncwarp();
            for (int i = lane; i < k; i += 32) H.y[i] = fma(-T[i + ld * k], lk, H.y[i]);
            if (lane == 0) H.y[k] = lk;
            __syncwarp();
        }
        for (int i = lane; i < nI; i += 32) wv[i] = 0.0;
        __syncwarp();
        for (int c = 0; c < nJ; ++c) {  // w = B lambda, column by column
            const double lc = H.y[c];
            for (int e = lane; e < H.clen[c]; e += 32) {
                const int p = search_rows(H.I, nI, args.kri[H.kcol[c] + e]);
                if (p >= 0) wv[p] = fma(args.kcv[H.colA[c] + e], lc, wv[p]);
            }
            __syncwarp();
        }
    }
    __syncthreads();
    if (H.status == kStOk) {
        const int64_t blk = args.dB_off[jj];
        for (int c = warp; c < nJ; c += kBigWarps) {
            const double ac = fma(-2.0 * rho, H.m[c], H.y[c]), nm = -H.m[c];
            double bt = 0.0;
            for (int e = lane; e < H.clen[c]; e += 32) {
                const int p = search_rows(H.I, nI, args.kri[H.kcol[c] + e]);
                const double rp = p >= 0 ? H.r[p] : 0.0, wp = p >= 0 ? wv[p] : 0.0;
                args.dB[blk + H.cb[c] + e] = fma(rp, ac, wp * nm);
                bt = fma(args.kcv[H.colA[c] + e], rp, bt);
            }
            bt = warp_sum_f64(bt);
            if (lane == 0) {
                const int64_t t = (int64_t)args.csr_pos[jb + c] + poff;
                args.dbase[t] = blk + H.cb[c];
                if (args.dmres) args.dmres[t] = -2.0 * rho * bt;
            }
        }
        const int zb = args.zcp[zc], ze = args.zcp[zc + 1];
        for (int t = zb + tid; t < ze; t += kBigThreads) {
            const int p = search_rows(H.I, nI, args.zri[t] + zro);
            args.dzval[zoff + t] = (p >= 0) ? wv[p] + 2.0 * rho * H.r[p] : 2.0 * rho * args.zcv[t];
        }
    }
    if (tid == 0) args.colstat[jj] = H.status;
}

// ADJ: the adjoint of the column solves (as adjoint.cu for the register
// classes) instead of the solve: m and dL/dm from the map, lambda by the FP64
// triangular solves with R, dL/dB blocks, dL/dc, and the residual's direct
// partials.
template <typename TT, bool ADJ = false>
__global__ void __launch_bounds__(kBigThreads, BigBlocks<TT>::value) lsq_big_kernel(LsqArgs args, int bin) {
    constexpr bool F32 = sizeof(TT) == 4;
    static_assert(!(ADJ && F32), "the large class's adjoint runs in FP64");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BigHdr &H = *reinterpret_cast<BigHdr *>(smem_raw);
    TT *T = reinterpret_cast<TT *>(smem_raw + sizeof(BigHdr));
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
        TT *yT = reinterpret_cast<TT *>(H.y);
        // FP32 tile: the local row of every stored entry of B, kept after the
        // tile when it fits there (the refinement passes then skip the row
        // searches); lr[H.cb[c] + e] for entry e of column c
        // and their FP64 values after those (8-byte aligned): no global loads
        // in the passes
        int *lr = reinterpret_cast<int *>(T + (size_t)ld * (nJ + 1));
        const bool keep_lr = F32 && H.status == kStOk && 3 * (int64_t)H.cb[nJ] + 1 + (int64_t)ld * (nJ + 1) <= kBigTileDoubles;
        double *bv = reinterpret_cast<double *>(lr + ((ld * (nJ + 1) + (keep_lr ? H.cb[nJ] : 0)) & 1) + (keep_lr ? H.cb[nJ] : 0));
        // ---- the tile [B c] and the target column
        if (H.status == kStOk) {
            for (int q = tid; q < ld * (nJ + 1); q += kBigThreads) T[q] = TT(0);
            for (int i = tid; i < nI; i += kBigThreads) H.r[i] = 0.0;
        }
        __syncthreads();
        if (H.status == kStOk) {
            for (int c = warp; c < nJ; c += kBigWarps) {
                int plo = INT_MAX, phi = -1;  // first and last row of column c
                for (int e = lane; e < H.clen[c]; e += 32) {
                    const int p = search_rows(H.I, nI, args.kri[H.kcol[c] + e]);
                    if (p >= 0) {
                        T[p + ld * c] = big_value<TT>(args.kcv, args.kcv32, H.colA[c] + e);
                        plo = min(plo, p);
                        phi = max(phi, p);
                    } else {
                        set_status(H, kStUnsupported);  // impossible: every row of B is in I_j
                    }
                    if (keep_lr) {
                        lr[H.cb[c] + e] = p;
                        bv[H.cb[c] + e] = args.kcv[H.colA[c] + e];
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    plo = min(plo, __shfl_xor_sync(0xffffffffu, plo, o));
                    phi = max(phi, __shfl_xor_sync(0xffffffffu, phi, o));
                }
                if (lane == 0) {
                    H.cfirst[c] = (short)min(plo, kBigICap);
                    H.rband[c] = (short)phi;
                }
            }
            if (warp == kBigWarps - 1) {
                const int zb = args.zcp[zc], ze = args.zcp[zc + 1];
                double o2 = 0.0;
                for (int t = zb + lane; t < ze; t += 32) {
                    const double v = args.zcv[t];
                    const int p = search_rows(H.I, nI, args.zri[t] + zro);
                    if (p >= 0) {
                        T[p + ld * nJ] = big_value<TT>(args.zcv, args.zcv32, t);
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
        // ---- the QR's band.  Rows are in ascending order of the source's
        // numbering, so B has a staircase profile: Householder reflectors
        // 0..k leave every row after the last row holding an entry of
        // columns 0..k as it was (by induction: such a row is zero in those
        // columns, so the reflectors' vectors are zero there), and a column
        // whose first row is after that row is zero in all the rows they
        // touch (its dot products vanish): reflector k acts on rows
        // k..rband[k]-1 of columns k+1..cband[k]-1 and of c.
        if (tid == 0 && H.status == kStOk) {
            int mx = -1;
            for (int k = 0; k < nJ; ++k) {
                mx = max(mx, (int)H.rband[k]);
                H.rband[k] = (short)(max(mx, k) + 1);
            }
            int mn = INT_MAX;
            for (int t = nJ - 1; t >= 0; --t) {
                mn = min(mn, (int)H.cfirst[t]);
                H.cfirst[t] = (short)mn;
            }
            // the suffix minimum is ascending: the last column with a first
            // row below the band's end moves forward with k
            int t = -1;
            for (int k = 0; k < nJ; ++k) {
                while (t + 1 < nJ && H.cfirst[t + 1] < H.rband[k]) ++t;
                H.cband[k] = (short)(max(t, k) + 1);
            }
        }
        __syncthreads();
        // ---- Householder QR of [B c].  Reflector k + 1 is formed by warp 0
        // right after it applied reflector k to column k + 1 (its parameters
        // double-buffered), so each reflector costs one block barrier.
        if (H.status == kStOk) {
            TT *qp = reinterpret_cast<TT *>(&H.qp[0][0]);  // qp[4 b + q], b = reflector parity
            if (warp == 0) reflector<TT>(T, ld, H.rband[0], 0, lane, qp);
            __syncthreads();
            for (int k = 0; k < nJ; ++k) {
                const TT *qk = qp + 4 * (k & 1);
                const TT uk = qk[0], taup = qk[1];
                const int re = H.rband[k];
                if (taup != TT(0)) {
                    // the band's columns after k, then c: nv columns, v = 0
                    // being column k + 1 (or c).  FP32: a warp's columns v,
                    // v + 16, v + 32, v + 48 at once (independent dot products
                    // and updates; the FP64 pipe gains nothing from it and
                    // pays for idle slots)
                    constexpr int G = F32 ? 4 : 1;
                    const int nb = H.cband[k] - (k + 1), nv = nb + 1;
                    for (int v0 = warp; v0 < nv; v0 += G * kBigWarps) {
                        const int nq = min(G, (nv - 1 - v0) / kBigWarps + 1);
                        int tq[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int v = v0 + q * kBigWarps;
                            tq[q] = v < nb ? k + 1 + v : nJ;
                        }
                        if (nq >= 4) apply_cols<TT, 4>(T, ld, re, k, tq, lane, uk, taup);
                        else if (nq == 3) apply_cols<TT, 3>(T, ld, re, k, tq, lane, uk, taup);
                        else if (nq == 2) apply_cols<TT, 2>(T, ld, re, k, tq, lane, uk, taup);
                        else apply_cols<TT, 1>(T, ld, re, k, tq, lane, uk, taup);
                        if (v0 == 0 && k + 1 < nJ) {  // warp 0: column k + 1 is final below row k
                            __syncwarp();
                            reflector<TT>(T, ld, H.rband[k + 1], k + 1, lane, qp + 4 * ((k + 1) & 1));
                        }
                    }
                } else if (warp == 0 && k + 1 < nJ) {
                    reflector<TT>(T, ld, H.rband[k + 1], k + 1, lane, qp + 4 * ((k + 1) & 1));
                }
                if (tid == 0) T[k + ld * k] = qk[2];
                __syncthreads();
            }
        }
        __syncthreads();
        // ---- pivots, back substitution R m = (Q^T c)(1:|J|), residual
        if (H.status == kStOk && warp == 0) {
            int st = kStOk;
            for (int k = lane; k < nJ; k += 32) {
                const double d = (double)T[k + ld * k];
                if (!isfinite(d)) st = max(st, (int)kStNonfinite);
                else if (d == 0.0) st = max(st, (int)kStRank);
                yT[k] = T[k + ld * nJ];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) st = max(st, __shfl_xor_sync(0xffffffffu, st, o));
            __syncwarp();
            if (st == kStOk) {
                if constexpr (ADJ) {  // the forward map's column and the incoming gradient
                    for (int c = lane; c < nJ; c += 32) {
                        const int64_t t = (int64_t)args.csr_pos[jb + c] + poff;
                        H.m[c] = args.mval[t];
                        H.g[c] = args.dmval ? args.dmval[t] : 0.0;
                    }
                    __syncwarp();
                } else {
                    for (int k = nJ - 1; k >= 0; --k) {
                        const TT mk = yT[k] / T[k + ld * k];
                        __syncwarp();
                        for (int i = lane; i < k; i += 32) yT[i] = fma(-T[i + ld * k], mk, yT[i]);
                        if (lane == 0) H.m[k] = (double)mk;
                        __syncwarp();
                    }
                }
                int nf = 0;
                for (int c = 0; c < nJ; ++c) {
                    const double mc = H.m[c];
                    nf |= !isfinite(mc);
                    for (int e = lane; e < H.clen[c]; e += 32) {
                        const int p = keep_lr ? lr[H.cb[c] + e] : search_rows(H.I, nI, args.kri[H.kcol[c] + e]);
                        const double b = keep_lr ? bv[H.cb[c] + e] : args.kcv[H.colA[c] + e];
                        if (p >= 0) H.r[p] = fma(-b, mc, H.r[p]);
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
        if (tid == 0) {
            H.rstate[kRMiss] = 0;
            H.rstate[kRUsed] = kAutoSteps + 1;  // solved in FP64
        }
        __syncthreads();
        if constexpr (ADJ) {
            big_adjoint(args, H, reinterpret_cast<double *>(T), ld, nI, nJ, jj, jb, poff, args.zbig ? jj : jl,
                        zro, args.zbig ? 0 : (int64_t)kmap * args.znnz, tid, lane, warp);
            __syncthreads();  // the next column reuses the shared memory
            continue;
        }
        // ---- FP32 tile: corrected semi-normal-equation steps, r = c - B m0 above
        if constexpr (F32) {
            const bool autoref = args.refine_steps < 0;
            const int steps = autoref ? kAutoSteps : args.refine_steps;
            if (H.status == kStOk && steps > 0) {
                float *gf = reinterpret_cast<float *>(H.g);
                if (tid == 0) {  // the guard's kappa estimate (|R_kk| range) and |m_0|^2
                    float rmax = 0.f, rmin = FLT_MAX;
                    double m2 = 0.0;
                    for (int k = 0; k < nJ; ++k) {
                        const float a = fabsf((float)T[k + ld * k]);
                        rmax = fmaxf(rmax, a);
                        rmin = fminf(rmin, a);
                        m2 = fma(H.m[k], H.m[k], m2);
                    }
                    const float kap = rmax / rmin;
                    H.scal[kSKap2] = kap * kap;
                    H.scal[kSMsq] = m2;
                    H.rstate[kRStop] = 0;
                }
                __syncthreads();
                for (int step = 0; step < steps; ++step) {
                    // g = B^T r (FP64), a warp per column
                    for (int c = warp; c < nJ; c += kBigWarps) {
                        double acc = 0.0;
                        for (int e = lane; e < H.clen[c]; e += 32) {
                            const int p = keep_lr ? lr[H.cb[c] + e] : search_rows(H.I, nI, args.kri[H.kcol[c] + e]);
                            const double b = keep_lr ? bv[H.cb[c] + e] : args.kcv[H.colA[c] + e];
                            if (p >= 0) acc = fma(b, H.r[p], acc);
                        }
                        acc = warp_sum_f64(acc);
                        if (lane == 0) gf[c] = (float)acc;  // the FP32 solve's right-hand side
                    }
                    __syncthreads();
                    if (warp == 0) {
                        // R^T y = g, then R d = y (FP32; R in the tile's upper triangle)
                        for (int k = 0; k < nJ; ++k) {
                            float sk = 0.f;
                            for (int i = lane; i < k; i += 32) sk = fmaf((float)T[i + ld * k], H.dv[i], sk);
                            sk = warp_sum<float>(sk);
                            if (lane == 0) H.dv[k] = (gf[k] - sk) / (float)T[k + ld * k];
                            __syncwarp();
                        }
                        for (int k = nJ - 1; k >= 0; --k) {
                            const float dk = H.dv[k] / (float)T[k + ld * k];
                            __syncwarp();
                            for (int i = lane; i < k; i += 32) H.dv[i] = fmaf(-(float)T[i + ld * k], dk, H.dv[i]);
                            if (lane == 0) H.dv[k] = dk;
                            __syncwarp();
                        }
                        // m += d (FP64), r -= B d (FP64, column by column)
                        float dsq = 0.f;
                        for (int c = lane; c < nJ; c += 32) {
                            const float d = H.dv[c];
                            const double dd = (double)d;
                            H.m[c] += dd;
                            H.y[c] = dd;  // d in FP64 for r -= B d
                            dsq = fmaf(d, d, dsq);
                        }
                        __syncwarp();
                        dsq = warp_sum<float>(dsq);
                        for (int c = 0; c < nJ; ++c) {
                            const double dc = H.y[c];
                            for (int e = lane; e < H.clen[c]; e += 32) {
                                const int p = keep_lr ? lr[H.cb[c] + e] : search_rows(H.I, nI, args.kri[H.kcol[c] + e]);
                                const double b = keep_lr ? bv[H.cb[c] + e] : args.kcv[H.colA[c] + e];
                                if (p >= 0) H.r[p] = fma(-b, dc, H.r[p]);
                            }
                            __syncwarp();
                        }
                        if (lane == 0) {
                            // the register classes' accuracy guard (lsq.cu), on the whole column
                            constexpr float kTol = (float)kFallbackTol, kTol2 = kTol * kTol, kC = (float)kAutoC;
                            const float msq = (float)H.scal[kSMsq];
                            const float rk = (float)(kRhoSafety * kU32) * (float)H.scal[kSKap2];
                            bool miss = !(rk < 0.5f) || rk * rk * dsq > kTol2 * (1.f - rk) * (1.f - rk) * msq;
                            if (step == 0) {
                                miss = miss || 4.f * kC * kC * dsq >= msq || 2.f * kC * dsq > kTol * msq;
                            } else if (dsq > (float)kNoise2 * msq) {
                                const float dprev2 = (float)H.scal[kSDprev];
                                miss = miss || 4.f * dsq >= dprev2 || 4.f * dsq * dsq > kTol2 * msq * dprev2;
                            }
                            H.scal[kSDprev] = dsq;
                            H.rstate[kRUsed] = step + 1;
                            if (autoref) {
                                if (step == 0 && !(kC * dsq > (float)kAutoTol * msq || miss)) H.rstate[kRStop] = 1;
                                if (step == steps - 1) H.rstate[kRMiss] = miss ? 1 : 0;
                            } else if (step == steps - 1) {
                                H.rstate[kRMiss] = miss ? 1 : 0;
                            }
                        }
                    }
                    __syncthreads();
                    if (H.rstate[kRStop]) break;
                }
                // the final residual and the solution's finiteness
                if (warp == 0) {
                    double s2 = 0.0;
                    int nf = 0;
                    for (int i = lane; i < nI; i += 32) s2 = fma(H.r[i], H.r[i], s2);
                    for (int c = lane; c < nJ; c += 32) nf |= !isfinite(H.m[c]);
                    s2 = warp_sum_f64(s2);
                    nf = __any_sync(0xffffffffu, nf);
                    if (lane == 0) {
                        H.scal[kSRes2] = s2;
                        if (nf || !isfinite(s2)) set_status(H, kStNonfinite);
                        else if (H.rstate[kRMiss]) set_status(H, kStRefine);  // re-solved by the FP64 kernel
                    }
                }
                __syncthreads();
            }
        }
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
                if (args.refine_used)
                    args.refine_used[jj] = (uint8_t)(status == kStRefine ? kAutoSteps + 1 : H.rstate[kRUsed]);
            }
        }
        __syncthreads();  // the next column reuses the shared memory
    }
}

}  // namespace

cudaError_t launch_adjoint_big(sam_handle h, const LsqArgs &args, int bin) {
    const size_t smem = sizeof(BigHdr) + sizeof(double) * (size_t)kBigTileDoubles;
    auto kern = lsq_big_kernel<double, true>;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<handle_sms(h), kBigThreads, smem, handle_stream(h)>>>(args, bin);
    count_launch(h);
    return cudaGetLastError();
}

cudaError_t launch_lsq_big(sam_handle h, const LsqArgs &args, int bin, bool profile, bool fp32) {
    const size_t smem = sizeof(BigHdr) + (fp32 ? sizeof(float) : sizeof(double)) * (size_t)kBigTileDoubles;
    auto kern = fp32 ? lsq_big_kernel<float> : lsq_big_kernel<double>;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (profile) profile_begin(h, bin);
    kern<<<handle_sms(h) * (fp32 ? BigBlocks<float>::value : 1), kBigThreads, smem, handle_stream(h)>>>(args, bin);
    count_launch(h);
    if (profile) profile_end(h, bin);
    return cudaGetLastError();
}

}  // namespace sam
