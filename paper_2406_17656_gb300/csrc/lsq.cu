// lsq.cu -- the batched column least-squares solves of SAM construction
// (arXiv 2406.17656, Sec. 2: Eq. (approx_map) splits into one problem per
// column, min_m || A_k(I_j, J_j) m - A_0(I_j, j) ||).
//
// One launch per size class covers the columns of every map in the batch: a
// persistent grid pulls (map, column) items from a work list with an atomic
// ticket (a bounded loop: it ends when the ticket passes the item count).
//
// Register-tiled Householder QR.  A column problem is owned by a group of
// P = RG x CG lanes (several groups per warp).  The dense augmented matrix
// [B c] (|I| x (|J|+1), padded to MAXI x NCOL with zeros, c in the last
// column) is distributed over the group as a 2-D grid: element (i, col)
// lives on lane (rg = i % RG, cg = col % CG) in register slot
// (s = i / RG, t = col / CG).  Reflector k needs
//   * the norm of column k below the diagonal: an FMA chain per lane plus a
//     log2(RG)-step shuffle reduction over the column's RG lanes,
//   * the Householder vector on every lane: one shuffle per live row slot
//     from the lanes that own column k,
//   * per live column slot a dot product (FMA chain + log2(RG) shuffles)
//     and a rank-1 update (FMA chain).
// The k loop is split into phases of L = min(RG, CG) steps; within a phase
// the first live row slot and column slot are compile-time constants, so
// register slots holding only finished rows/columns drop out of the code.
// The right-hand side is the last column, so Q^T c falls out of the sweep.
//
// Precision.  SAM_FP64: the tile, the solves and the residual are FP64.
// SAM_FP32_REFINE: the QR and triangular solves run in FP32; accuracy is won
// back by corrected semi-normal-equation steps with FP64 residuals
//   r = c - B m (FP64),  g = B^T r (FP64),  R^T R d = g (FP32),  m += d,
// which converge at a rate ~ u_32 kappa(B)^2 to the FP64 least-squares
// solution (plain "solve with Q^T r" refinement stalls at
// ~u_32 kappa^2 ||r||/(||B|| ||m||) for problems with a nonzero residual, as
// every SAM column has).  The FP64 products use the sparse B straight from
// A_k's CSC values, in a fixed order, so results are deterministic.
// Finally r = c - B m is recomputed in FP64 for the per-column residual.
#include <cfloat>
#include <climits>

#include "common.cuh"

namespace sam {
namespace {

constexpr int kWarpsPerBlock = 4;

template <int RG_, int CG_, int RS_, int CS_, typename T_, int MAXI_BIN_>
struct Tile {
    static constexpr int RG = RG_, CG = CG_, RS = RS_, CS = CS_;
    static constexpr int P = RG * CG;    // lanes per column problem
    static constexpr int PPW = 32 / P;   // problems per warp
    static constexpr int MAXI = RG * RS; // padded rows
    static constexpr int NCOL = CG * CS; // padded columns incl. right-hand side
    static constexpr int MAXJ = NCOL - 1;
    static constexpr int L = RG < CG ? RG : CG;  // phase length
    static constexpr int NBCAP = 8 * MAXI_BIN_; // max stored entries of B
    static constexpr int JQ = (MAXJ + P - 1) / P; // unknowns per lane (solves)
    static constexpr int IQ = (MAXI + P - 1) / P; // rows per lane (residuals)
    using T = T_;
    static_assert(32 % P == 0, "group size must divide the warp");
    static_assert(MAXJ <= 31, "column masks are 32-bit");
    static_assert(MAXI <= 255, "local row indices are 8-bit");
};

template <class TL>
struct ProbSmem {
    using T = typename TL::T;
    int I[TL::MAXI];
    int J[TL::MAXJ];
    int colA[TL::MAXJ];
    int colB[TL::MAXJ + 1];
    unsigned mask[TL::MAXI];
    double c[TL::MAXI];
    unsigned char locr[TL::NBCAP];
    union U {
        T tile[TL::NCOL][TL::MAXI];  // [B c] column-major, only until registers are loaded
        struct S {
            int rowstart[TL::MAXI + 1];
            int rowent[TL::NBCAP];
            unsigned char rowcol[TL::NBCAP];
            double r[TL::MAXI];
            double m[TL::MAXJ];
            double g[TL::MAXJ];
            T y[TL::MAXJ];
            T R[TL::MAXJ][TL::MAXJ + 1];
        } s;
    } u;
};

__device__ __forceinline__ int find_sorted(const int *a, int len, int key) {
    int lo = 0, hi = len - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int v = a[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// column c of entry e: colB[c] <= e < colB[c+1]
__device__ __forceinline__ int entry_col(const int *colB, int nJ, int e) {
    int lo = 0, hi = nJ - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (colB[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__device__ __forceinline__ T group_sum(T v, int P) {
    for (int o = 1; o < P; o <<= 1) v += shfl_xor(v, o);
    return v;
}

// ---------------------------------------------------------- Householder QR

template <class TL, int PH>
struct QRPhase {
    using T = typename TL::T;
    static constexpr int RG = TL::RG, CG = TL::CG, RS = TL::RS, CS = TL::CS, L = TL::L;
    static constexpr int K0 = PH * L;
    static constexpr int SK = K0 / RG;  // row slot of this phase's pivots
    static constexpr int TK = K0 / CG;  // column slot of this phase's pivots
    static constexpr int NPH = (TL::MAXJ + L - 1) / L;

    static __device__ __forceinline__ void run(T (&a)[RS][CS], int rg, int cg, int gbase, int nJ, int kmax) {
        if constexpr (PH < NPH) {
            if (K0 >= kmax) return;
            const int kend = (K0 + L < kmax) ? K0 + L : kmax;
            for (int k = K0; k < kend; ++k) {
                const int ck = k - TK * CG;  // column group owning column k
                const int rk = k - SK * RG;  // row group of row k inside slot SK
                const bool active = k < nJ;
                // squared norm of column k below the diagonal
                T sig = T(0);
#pragma unroll
                for (int s = SK; s < RS; ++s) {
                    T x = a[s][TK];
                    if (s == SK) x = (rg > rk) ? x : T(0);
                    sig = fma(x, x, sig);
                }
#pragma unroll
                for (int o = 1; o < RG; o <<= 1) sig += shfl_xor(sig, o);
                const T alpha = shfl(a[SK][TK], gbase + ck * RG + rk);
                const T sigma = shfl(sig, gbase + ck * RG);
                // reflector H = I - taup u u^T, u = x with u_k = alpha - beta
                const T nrm = sqrt(fma(alpha, alpha, sigma));
                const T beta = (sigma == T(0)) ? alpha : ((alpha >= T(0)) ? -nrm : nrm);
                const T uk = alpha - beta;
                const T taup = (sigma == T(0) || !active) ? T(0) : T(-1) / (beta * uk);
                T u[RS - SK];
#pragma unroll
                for (int s = SK; s < RS; ++s) {
                    T x = shfl(a[s][TK], gbase + ck * RG + rg);
                    if (s == SK) x = (rg > rk) ? x : ((rg == rk) ? uk : T(0));
                    u[s - SK] = x;
                }
#pragma unroll
                for (int t = TK; t < CS; ++t) {
                    T w = T(0);
#pragma unroll
                    for (int s = SK; s < RS; ++s) w = fma(u[s - SK], a[s][t], w);
#pragma unroll
                    for (int o = 1; o < RG; o <<= 1) w += shfl_xor(w, o);
                    const int col = t * CG + cg;
                    const T coef = (col > k) ? taup * w : T(0);
#pragma unroll
                    for (int s = SK; s < RS; ++s) a[s][t] = fma(-coef, u[s - SK], a[s][t]);
                }
                if (active && cg == ck && rg == rk) a[SK][TK] = beta;
            }
            QRPhase<TL, PH + 1>::run(a, rg, cg, gbase, nJ, kmax);
        }
    }
};

// ------------------------------------------------ triangular solves (smem)
// Upper triangular R (R[i][c], i <= c < n) held in shared memory; lanes of
// the group own entries i = ll + P*q.  All groups of the warp step together
// (k runs to the warp's largest n), each only acting while k < its own n.

template <class TL, typename V>
__device__ __forceinline__ void back_solve(const typename TL::T (*R)[TL::MAXJ + 1], V *x, int n, int kmax, int ll) {
    // solve R x = x in place (x holds the right-hand side on entry)
    for (int k = kmax - 1; k >= 0; --k) {
        const bool act = k < n;
        V xk = V(0);
        if (act) xk = x[k] / V(R[k][k]);
        __syncwarp();
        if (act) {
            if (ll == 0) x[k] = xk;
#pragma unroll
            for (int q = 0; q < TL::JQ; ++q) {
                int i = ll + q * TL::P;
                if (i < k) x[i] -= V(R[i][k]) * xk;
            }
        }
        __syncwarp();
    }
}

template <class TL, typename V>
__device__ __forceinline__ void forward_solve_t(const typename TL::T (*R)[TL::MAXJ + 1], V *x, int n, int kmax,
                                                int ll) {
    // solve R^T x = x in place
    for (int k = 0; k < kmax; ++k) {
        const bool act = k < n;
        V xk = V(0);
        if (act) xk = x[k] / V(R[k][k]);
        __syncwarp();
        if (act) {
            if (ll == 0) x[k] = xk;
#pragma unroll
            for (int q = 0; q < TL::JQ; ++q) {
                int i = ll + q * TL::P;
                if (i > k && i < n) x[i] -= V(R[k][i]) * xk;
            }
        }
        __syncwarp();
    }
}

// r = c - B m in FP64 over the row-major entry lists; returns this lane's
// partial sum of r_i^2
template <class TL>
__device__ __forceinline__ double residual_rows(ProbSmem<TL> &S, const double *kcv, int nI, int ll) {
    double r2 = 0.0;
#pragma unroll
    for (int q = 0; q < TL::IQ; ++q) {
        int i = ll + q * TL::P;
        if (i < nI) {
            double ri = S.c[i];
            for (int p = S.u.s.rowstart[i]; p < S.u.s.rowstart[i + 1]; ++p)
                ri = fma(-kcv[S.u.s.rowent[p]], S.u.s.m[S.u.s.rowcol[p]], ri);
            S.u.s.r[i] = ri;
            r2 = fma(ri, ri, r2);
        }
    }
    return r2;
}

// g = B^T r in FP64, column by column (entries of a column in CSC order)
template <class TL>
__device__ __forceinline__ void normal_rhs(ProbSmem<TL> &S, const double *kcv, int nJ, int ll) {
#pragma unroll
    for (int q = 0; q < TL::JQ; ++q) {
        int c = ll + q * TL::P;
        if (c < nJ) {
            double g = 0.0;
            int a0 = S.colA[c], b0 = S.colB[c], len = S.colB[c + 1] - b0;
            for (int p = 0; p < len; ++p) g = fma(kcv[a0 + p], S.u.s.r[S.locr[b0 + p]], g);
            S.u.s.g[c] = g;
        }
    }
}

template <class TL, bool FP64>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) lsq_kernel(LsqArgs args, int bin) {
    using T = typename TL::T;
    constexpr int P = TL::P, PPW = TL::PPW, RG = TL::RG, CG = TL::CG, RS = TL::RS, CS = TL::CS;
    constexpr int MAXI = TL::MAXI, NCOL = TL::NCOL, MAXJ = TL::MAXJ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ProbSmem<TL> *probs = reinterpret_cast<ProbSmem<TL> *>(smem_raw);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / P, ll = lane % P, gbase = grp * P;
    const int rg = ll % RG, cg = ll / RG;
    ProbSmem<TL> &S = probs[warp * PPW + grp];

    const int w0 = args.work_count[bin];
    const int total = args.work_count[bin + 1] - w0;
    const int2 *work = args.work + w0;
    int32_t *ticket = args.ticket + bin;

    for (int iter = 0; iter < (1 << 30); ++iter) {
        int base = 0;
        if (lane == 0) base = atomicAdd(ticket, PPW);
        base = shfl(base, 0);
        if (base >= total) break;
        const int item = base + grp;
        const bool valid = item < total;
        int map = 0, j = 0, nJ = 0, nI = 0;
        const MapDev *md = nullptr;
        if (valid) {
            int2 wv = work[item];
            map = wv.x;
            j = wv.y;
            md = args.maps + map;
            nJ = md->jcp[j + 1] - md->jcp[j];
            nI = md->icnt[j];
        }
        int status = kStOk;

        // ---- gather: J, I, A_k column extents, zero the tile and c
        if (valid) {
            const int jb = md->jcp[j];
            for (int c = ll; c < nJ; c += P) {
                int col = md->jri[jb + c];
                S.J[c] = col;
                int a0 = md->kcp[col];
                S.colA[c] = a0;
                S.colB[c + 1] = md->kcp[col + 1] - a0;  // length for now
            }
            for (int i = ll; i < MAXI; i += P) {
                S.I[i] = (i < nI) ? md->ish[(int64_t)j * kICap + i] : INT_MAX;
                S.mask[i] = 0u;
                S.c[i] = 0.0;
            }
        }
        {
            T *tl = &S.u.tile[0][0];
            for (int e = ll; e < NCOL * MAXI; e += P) tl[e] = T(0);
        }
        __syncwarp();
        if (valid && ll == 0) {
            int acc = 0;
            S.colB[0] = 0;
            for (int c = 0; c < nJ; ++c) {
                acc += S.colB[c + 1];
                S.colB[c + 1] = acc;
            }
        }
        __syncwarp();
        const int nB = valid ? S.colB[nJ] : 0;
        // ---- gather the stored entries of A_k(:, J) into the dense tile
        if (valid) {
            const int32_t *kri = md->kri;
            const double *kcv = md->kcv;
            for (int e = ll; e < nB; e += P) {
                int c = entry_col(S.colB, nJ, e);
                int g = S.colA[c] + (e - S.colB[c]);
                int i = find_sorted(S.I, nI, kri[g]);
                if (i < 0) {  // cannot happen for a consistent shadow; never write out of bounds
                    status = kStUnsupported;
                    i = 0;
                }
                S.locr[e] = (unsigned char)i;
                S.u.tile[c][i] = T(kcv[g]);
                atomicOr(&S.mask[i], 1u << c);
            }
        }
        // ---- right-hand side A_0(I, j); entries outside I go to the residual
        double out2 = 0.0;
        if (valid) {
            for (int t = args.zcp[j] + ll; t < args.zcp[j + 1]; t += P) {
                int i = find_sorted(S.I, nI, args.zri[t]);
                double v = args.zcv[t];
                if (i >= 0) {
                    S.c[i] = v;
                    S.u.tile[NCOL - 1][i] = T(v);
                } else {
                    out2 = fma(v, v, out2);
                }
            }
        }
        out2 = group_sum(out2, P);
        __syncwarp();
        // ---- load the register tile
        T a[RS][CS];
#pragma unroll
        for (int s = 0; s < RS; ++s)
#pragma unroll
            for (int t = 0; t < CS; ++t) a[s][t] = S.u.tile[t * CG + cg][s * RG + rg];
        __syncwarp();
        // ---- row-major entry lists for the FP64 residual r = c - B m
        if (valid && ll == 0) {
            int acc = 0;
            for (int i = 0; i < nI; ++i) {
                S.u.s.rowstart[i] = acc;
                acc += __popc(S.mask[i]);
            }
            S.u.s.rowstart[nI] = acc;
        }
        __syncwarp();
        if (valid) {
            for (int e = ll; e < nB; e += P) {
                int c = entry_col(S.colB, nJ, e);
                int i = S.locr[e];
                int pos = S.u.s.rowstart[i] + __popc(S.mask[i] & ((1u << c) - 1u));
                S.u.s.rowent[pos] = S.colA[c] + (e - S.colB[c]);
                S.u.s.rowcol[pos] = (unsigned char)c;
            }
        }
        // ---- QR of [B c]
        int kmax = nJ;
#pragma unroll
        for (int o = P; o < 32; o <<= 1) kmax = max(kmax, shfl_xor(kmax, o));
        QRPhase<TL, 0>::run(a, rg, cg, gbase, nJ, kmax);
        // ---- R and Q^T c to shared memory
#pragma unroll
        for (int s = 0; s < RS; ++s)
#pragma unroll
            for (int t = 0; t < CS; ++t) {
                int i = s * RG + rg, col = t * CG + cg;
                if (col < MAXJ && i <= col && col < nJ) S.u.s.R[i][col] = a[s][t];
                if (col == NCOL - 1 && i < nJ) S.u.s.y[i] = a[s][t];
            }
        __syncwarp();
        // pivots: zero -> rank deficient, non-finite -> nonfinite
        {
            int st_piv = kStOk;
            if (valid)
                for (int k = ll; k < nJ; k += P) {
                    T d = S.u.s.R[k][k];
                    if (!isfinite((double)d)) st_piv = max(st_piv, (int)kStNonfinite);
                    else if (d == T(0)) st_piv = max(st_piv, (int)kStRank);
                }
            status = max(status, st_piv);
        }
        // combine the group's statuses (largest code wins)
        for (int o = 1; o < P; o <<= 1) status = max(status, shfl_xor(status, o));
        __syncwarp();
        // ---- initial solve R m = (Q^T c)(1:nJ)
        const int kmx = kmax;
        if (status != kStOk) nJ = 0;  // skip numeric work of a failed column
        back_solve<TL, T>(S.u.s.R, S.u.s.y, nJ, kmx, ll);
        for (int c = ll; c < nJ; c += P) S.u.s.m[c] = (double)S.u.s.y[c];
        __syncwarp();
        const double *kcv = valid ? md->kcv : nullptr;
        if constexpr (!FP64) {
            for (int step = 0; step < args.refine_steps; ++step) {
                if (valid && nJ > 0) residual_rows<TL>(S, kcv, nI, ll);
                __syncwarp();
                if (valid && nJ > 0) normal_rhs<TL>(S, kcv, nJ, ll);
                __syncwarp();
                for (int c = ll; c < nJ; c += P) S.u.s.y[c] = (T)S.u.s.g[c];
                __syncwarp();
                forward_solve_t<TL, T>(S.u.s.R, S.u.s.y, nJ, kmx, ll);
                back_solve<TL, T>(S.u.s.R, S.u.s.y, nJ, kmx, ll);
                for (int c = ll; c < nJ; c += P) S.u.s.m[c] += (double)S.u.s.y[c];
                __syncwarp();
            }
        }
        // ---- final FP64 residual and outputs
        double r2 = 0.0;
        if (valid && nJ > 0) r2 = residual_rows<TL>(S, kcv, nI, ll);
        r2 = group_sum(r2, P);
        int nf = 0;
        if (valid)
            for (int c = ll; c < nJ; c += P) nf |= !isfinite(S.u.s.m[c]);
        for (int o = 1; o < P; o <<= 1) nf |= shfl_xor(nf, o);
        if (valid) {
            if (status == kStOk && (nf || !isfinite(r2))) status = kStNonfinite;
            const int jb = md->jcp[j];
            const int njo = md->jcp[j + 1] - jb;
            for (int c = ll; c < njo; c += P)
                md->mval[md->csr_pos[jb + c]] = (status == kStOk) ? S.u.s.m[c] : 0.0;
            if (ll == 0) {
                md->colres[j] = (status == kStOk) ? r2 + out2 : 0.0;
                md->colstat[j] = status;
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------ dispatch

// FP32 tiles per size class (bins: |I| <= 14/26/40/52/64, |J| <= 5/9/23/27/27)
using F0 = Tile<2, 2, 7, 3, float, 14>;
using F1 = Tile<2, 2, 13, 5, float, 26>;
using F2 = Tile<4, 4, 10, 6, float, 40>;
using F3 = Tile<4, 4, 13, 7, float, 52>;
using F4 = Tile<4, 4, 16, 7, float, 64>;
// FP64 tiles
using D0 = Tile<2, 2, 7, 3, double, 14>;
using D1 = Tile<2, 4, 13, 3, double, 26>;
using D2 = Tile<4, 8, 10, 3, double, 40>;
using D3 = Tile<4, 8, 13, 4, double, 52>;
using D4 = Tile<4, 8, 16, 4, double, 64>;

static_assert(F0::MAXI >= 14 && F0::MAXJ >= 5, "bin 0");
static_assert(F1::MAXI >= 26 && F1::MAXJ >= 9, "bin 1");
static_assert(F2::MAXI >= 40 && F2::MAXJ >= 23, "bin 2");
static_assert(F3::MAXI >= 52 && F3::MAXJ >= 27, "bin 3");
static_assert(F4::MAXI >= 64 && F4::MAXJ >= 27, "bin 4");
static_assert(D1::MAXJ >= 9 && D2::MAXJ >= 23 && D3::MAXJ >= 27 && D4::MAXJ >= 27, "fp64 bins");

template <class TL, bool FP64>
cudaError_t launch_one(sam_handle h, const LsqArgs &a, int bin) {
    const size_t smem = sizeof(ProbSmem<TL>) * TL::PPW * kWarpsPerBlock;
    auto kern = lsq_kernel<TL, FP64>;
    static thread_local int configured_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured_dev = dev;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarpsPerBlock * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = per_sm * handle_sms(h);
    profile_begin(h, bin);
    kern<<<grid, kWarpsPerBlock * 32, smem, handle_stream(h)>>>(a, bin);
    count_launch(h);
    profile_end(h, bin);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_lsq(sam_handle h, int precision, int refine_steps, int mode, const MapDev *maps_dev,
                       const int32_t *zcp, const int32_t *zri, const double *zcv, const int2 *work,
                       const int32_t *bin_off, int32_t *tickets) {
    LsqArgs a;
    a.maps = maps_dev;
    a.zcp = zcp;
    a.zri = zri;
    a.zcv = zcv;
    a.work = work;
    a.work_count = bin_off;
    a.ticket = tickets;
    a.refine_steps = refine_steps;
    a.mode = mode;
    cudaError_t e = cudaMemsetAsync(tickets, 0, sizeof(int32_t) * kNumBins, handle_stream(h));
    if (e != cudaSuccess) return e;
    if (precision == SAM_FP64) {
        if ((e = launch_one<D0, true>(h, a, 0)) != cudaSuccess) return e;
        if ((e = launch_one<D1, true>(h, a, 1)) != cudaSuccess) return e;
        if ((e = launch_one<D2, true>(h, a, 2)) != cudaSuccess) return e;
        if ((e = launch_one<D3, true>(h, a, 3)) != cudaSuccess) return e;
        if ((e = launch_one<D4, true>(h, a, 4)) != cudaSuccess) return e;
    } else {
        if ((e = launch_one<F0, false>(h, a, 0)) != cudaSuccess) return e;
        if ((e = launch_one<F1, false>(h, a, 1)) != cudaSuccess) return e;
        if ((e = launch_one<F2, false>(h, a, 2)) != cudaSuccess) return e;
        if ((e = launch_one<F3, false>(h, a, 3)) != cudaSuccess) return e;
        if ((e = launch_one<F4, false>(h, a, 4)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sam
