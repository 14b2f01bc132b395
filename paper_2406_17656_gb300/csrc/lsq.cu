// lsq.cu -- the batched column least-squares solves of SAM construction
// (arXiv 2406.17656, Sec. 2: Eq. (approx_map) splits into one problem per
// column, min_m || A_k(I_j, J_j) m - A_0(I_j, j) ||).
//
// A batch of K maps is one block-diagonal problem: source matrices, patterns
// and shadow rows of map k occupy rows/columns [k n, (k+1) n) of "big"
// arrays, so one launch per size class covers every map.  A persistent grid
// pulls column indices from the size class's work list with an atomic
// ticket (a bounded loop that ends when the ticket passes the item count).
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
// Triangular solves with R run in registers (unknown c on lane c % P) with
// one shuffle per step; R sits in shared memory with an odd row stride.
//
// Precision.  SAM_FP64: tile, solves and residual are FP64.
// SAM_FP32_REFINE: QR and triangular solves in FP32; accuracy is won back by
// corrected semi-normal-equation (CSNE) steps with FP64 residuals
//   r = c - B m (FP64),  g = B^T r (FP64),  R^T R d = g (FP32),  m += d,
// which converge at a rate ~ u_32 kappa(B)^2 to the FP64 least-squares
// solution (plain "solve with Q^T r" refinement stalls at
// ~u_32 kappa^2 ||r||/(||B|| ||m||) for problems with a nonzero residual, as
// SAM columns have).  The FP64 products use the sparse B straight from
// A_k's CSC values in a fixed order, so results are deterministic.  After
// the last step the residual is r - B d with the small product B d taken in
// FP32 and the subtraction and squares in FP64, so no further FP64 pass over
// B is needed.  FP64->FP32
// conversions of the factorisation inputs truncate with integer operations,
// leaving GB300's narrow FP64 pipe to the residual arithmetic.
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
    static constexpr int L = RG < CG ? RG : CG;    // QR phase length
    static constexpr int NBCAP = 8 * MAXI_BIN_;     // max stored entries of B
    static constexpr int JQ = (MAXJ + P - 1) / P;  // unknowns per lane (solves)
    static constexpr int IQ = (MAXI + P - 1) / P;  // rows per lane (residuals)
    static constexpr int RSTR = (MAXJ % 2) ? MAXJ : MAXJ + 1;  // odd row stride of R
    using T = T_;
    static_assert(32 % P == 0, "group size must divide the warp");
    static_assert(MAXJ <= 31, "column masks are 32-bit");
    static_assert(MAXI <= 255, "local row indices are 8-bit");
};

template <class TL>
struct ProbSmem {
    using T = typename TL::T;
    int I[TL::MAXI];
    int colA[TL::MAXJ];
    int colB[TL::MAXJ + 1];
    unsigned mask[TL::MAXI];
    double c[TL::MAXI];
    double m[TL::MAXJ];
    unsigned char locr[TL::NBCAP];
    union U {
        T tile[TL::NCOL][TL::MAXI];  // [B c] column-major, only until registers are loaded
        struct S {
            int rowstart[TL::MAXI + 1];
            int rowent[TL::NBCAP];
            unsigned char rowcol[TL::NBCAP];
            double r[TL::MAXI];
            T y[TL::MAXJ];
            T dinv[TL::MAXJ];
            T R[TL::MAXJ * TL::RSTR];
        } s;
    } u;
};

// ------------------------------------------------------------- utilities

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

// FP64 -> FP32 by truncation of the mantissa, with integer operations only.
// Used for the inputs of the FP32 factorisation, whose rounding the FP64
// refinement removes.  Overflow -> +-inf, NaN -> NaN, below FP32's normal
// range -> +-0.
__device__ __forceinline__ float narrow_trunc(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
    if (e >= 255) {
        const bool nan = ((hi >> 20) & 0x7ffu) == 0x7ffu && ((hi & 0xfffffu) | lo) != 0u;
        return __int_as_float((int)(sign | 0x7f800000u | (nan ? 0x400000u : 0u)));
    }
    if (e <= 0) return __int_as_float((int)sign);
    return __int_as_float((int)(sign | ((unsigned)e << 23) | mant));
}

// FP32 -> FP64 exactly, with integer operations (normal numbers and zeros;
// FP32 subnormals widen to zero, infinities and NaN keep their class).
__device__ __forceinline__ double widen(float x) {
    const unsigned u = (unsigned)__float_as_int(x);
    const unsigned sign = u & 0x80000000u;
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned mant = u & 0x7fffffu;
    unsigned hi, lo;
    if (e == 0u) {
        hi = sign;
        lo = 0u;
    } else if (e == 0xffu) {
        hi = sign | 0x7ff00000u | (mant >> 3);
        lo = mant << 29;
    } else {
        hi = sign | ((e + 896u) << 20) | (mant >> 3);
        lo = mant << 29;
    }
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

template <typename T>
__device__ __forceinline__ T to_tile(double x);
template <>
__device__ __forceinline__ float to_tile<float>(double x) { return narrow_trunc(x); }
template <>
__device__ __forceinline__ double to_tile<double>(double x) { return x; }

template <typename T>
__device__ __forceinline__ double to_f64(T x);
template <>
__device__ __forceinline__ double to_f64<float>(float x) { return widen(x); }
template <>
__device__ __forceinline__ double to_f64<double>(double x) { return x; }

__device__ __forceinline__ bool finite64(double x) {
    return ((unsigned)(__double_as_longlong(x) >> 52) & 0x7ffu) != 0x7ffu;
}

// sum over the P lanes of a group (xor tree inside the aligned group)
template <int P, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int o = 1; o < P; o <<= 1) v += shfl_xor(v, o);
    return v;
}

// exclusive prefix over the P lanes of a group; *total gets the group sum
template <int P>
__device__ __forceinline__ int group_excl_scan(int v, int ll, int *total) {
    int incl = v;
#pragma unroll
    for (int o = 1; o < P; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (ll >= o) incl += y;
    }
    *total = __shfl_sync(0xffffffffu, incl, (int)(threadIdx.x & 31) | (P - 1));
    return incl - v;
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
                // squared norm of column k below the diagonal (two chains)
                T sig0 = T(0), sig1 = T(0);
#pragma unroll
                for (int s = SK; s < RS; ++s) {
                    T x = a[s][TK];
                    if (s == SK) x = (rg > rk) ? x : T(0);
                    if ((s - SK) & 1) sig1 = fma(x, x, sig1); else sig0 = fma(x, x, sig0);
                }
                T sig = sig0 + sig1;
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
                    T w0 = T(0), w1 = T(0);
#pragma unroll
                    for (int s = SK; s < RS; ++s) {
                        if ((s - SK) & 1) w1 = fma(u[s - SK], a[s][t], w1); else w0 = fma(u[s - SK], a[s][t], w0);
                    }
                    T w = w0 + w1;
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

// ----------------------------------------------------- triangular solves
// x[q] holds entry c = ll + P*q of the right-hand side (and the solution on
// return).  Steps run in phases of P with the owning register slot fixed at
// compile time; each step costs one shuffle.  Entries c >= n are untouched.

template <class TL, int Q>
struct SolveUpper {  // R x = y, k from high to low
    using T = typename TL::T;
    static __device__ __forceinline__ void run(const T *R, const T *dinv, T (&x)[TL::JQ], int n, int ll, int gbase) {
        if constexpr (Q >= 0) {
            constexpr int P = TL::P;
            constexpr int KHI = (Q * P + P < TL::MAXJ) ? Q * P + P : TL::MAXJ;
            for (int k = KHI - 1; k >= Q * P; --k) {
                const int owner = k - Q * P;
                T xk = x[Q] * dinv[k];
                xk = shfl(xk, gbase + owner);
                if (k >= n) xk = T(0);
                if (ll == owner && k < n) x[Q] = xk;
#pragma unroll
                for (int q = 0; q <= Q; ++q) {
                    const int i = ll + q * P;
                    // rows of R at k >= n were never written: do not touch them
                    if (i < k && k < n) x[q] = fma(-R[i * TL::RSTR + k], xk, x[q]);
                }
            }
            SolveUpper<TL, Q - 1>::run(R, dinv, x, n, ll, gbase);
        }
    }
};

template <class TL, int Q>
struct SolveUpperT {  // R^T x = y, k from low to high
    using T = typename TL::T;
    static __device__ __forceinline__ void run(const T *R, const T *dinv, T (&x)[TL::JQ], int n, int ll, int gbase) {
        if constexpr (Q < TL::JQ) {
            constexpr int P = TL::P;
            constexpr int KHI = (Q * P + P < TL::MAXJ) ? Q * P + P : TL::MAXJ;
            for (int k = Q * P; k < KHI; ++k) {
                const int owner = k - Q * P;
                T xk = x[Q] * dinv[k];
                xk = shfl(xk, gbase + owner);
                if (k >= n) xk = T(0);
                if (ll == owner && k < n) x[Q] = xk;
#pragma unroll
                for (int q = Q; q < TL::JQ; ++q) {
                    const int i = ll + q * P;
                    if (i > k && i < n) x[q] = fma(-R[k * TL::RSTR + i], xk, x[q]);
                }
            }
            SolveUpperT<TL, Q + 1>::run(R, dinv, x, n, ll, gbase);
        }
    }
};

// r = c - B m in FP64 over the row-major entry lists; returns this lane's
// partial sum of r_i^2
template <class TL, bool SQUARES = true>
__device__ __forceinline__ double residual_rows(ProbSmem<TL> &S, const double *kcv, int nI, int ll) {
    double r2 = 0.0;
#pragma unroll
    for (int q = 0; q < TL::IQ; ++q) {
        const int i = ll + q * TL::P;
        if (i < nI) {
            double ri = S.c[i];
            const int pe = S.u.s.rowstart[i + 1];
            for (int p = S.u.s.rowstart[i]; p < pe; ++p) ri = fma(-kcv[S.u.s.rowent[p]], S.m[S.u.s.rowcol[p]], ri);
            S.u.s.r[i] = ri;
            if (SQUARES) r2 = fma(ri, ri, r2);
        }
    }
    return r2;
}

template <class TL, bool FP64>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) lsq_kernel(LsqArgs args, int bin) {
    using T = typename TL::T;
    constexpr int P = TL::P, PPW = TL::PPW, RG = TL::RG, CG = TL::CG, RS = TL::RS, CS = TL::CS;
    constexpr int MAXI = TL::MAXI, NCOL = TL::NCOL, MAXJ = TL::MAXJ, JQ = TL::JQ;
    constexpr int RPL = (MAXI + P - 1) / P;  // contiguous rows per lane (row prefix sums)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ProbSmem<TL> *probs = reinterpret_cast<ProbSmem<TL> *>(smem_raw);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / P, ll = lane % P, gbase = grp * P;
    const int rg = ll % RG, cg = ll / RG;
    ProbSmem<TL> &S = probs[warp * PPW + grp];

    const int w0 = args.bin_off[bin];
    const int total = args.bin_off[bin + 1] - w0;
    const int32_t *work = args.work + w0;
    int32_t *ticket = args.ticket + bin;
    const int n = args.n;

    for (int iter = 0; iter < (1 << 30); ++iter) {
        int base = 0;
        if (lane == 0) base = atomicAdd(ticket, PPW);
        base = shfl(base, 0);
        if (base >= total) break;
        const int item = base + grp;
        const bool valid = item < total;
        const int jj = valid ? work[item] : 0;   // column of the block-diagonal batch
        const int kmap = jj / n;                 // which map
        const int jl = jj - kmap * n;            // column of A_0
        const int roff = kmap * n;               // row offset of this map
        int jb = 0, nJ = 0, nI = 0, zb = 0, ze = 0;
        if (valid) {
            jb = args.jcp[jj];
            nJ = args.jcp[jj + 1] - jb;
            nI = args.icnt[jj];
            zb = args.zcp[jl];
            ze = args.zcp[jl + 1];
        }
        int status = kStOk;

        // ---- columns of J: lane owns c = ll + P q
        int colA[JQ], clen[JQ], colB[JQ];
#pragma unroll
        for (int q = 0; q < JQ; ++q) {
            const int c = ll + q * P;
            colA[q] = 0;
            clen[q] = 0;
            if (c < nJ) {
                const int col = args.jri[jb + c];
                colA[q] = args.kcp[col];
                clen[q] = args.kcp[col + 1] - colA[q];
            }
        }
        int nB = 0;
#pragma unroll
        for (int q = 0; q < JQ; ++q) {
            int tot;
            colB[q] = nB + group_excl_scan<P>(clen[q], ll, &tot);
            nB += tot;
        }
        // ---- shadow rows, zero masks / c / tile
        for (int i = ll; i < MAXI; i += P) {
            S.I[i] = (i < nI) ? args.ish[(int64_t)jj * kICap + i] : INT_MAX;
            S.mask[i] = 0u;
            S.c[i] = 0.0;
        }
#pragma unroll
        for (int q = 0; q < JQ; ++q) {
            const int c = ll + q * P;
            if (c < MAXJ) {
                S.colA[c] = colA[q];
                S.colB[c] = colB[q];
            }
        }
        if (ll == 0) S.colB[nJ < MAXJ ? nJ : MAXJ] = nB;
        {
            T *tl = &S.u.tile[0][0];
            for (int e = ll; e < NCOL * MAXI; e += P) tl[e] = T(0);
        }
        __syncwarp();
        // ---- gather A_k(I, J): each lane walks its own columns
        const int32_t *kri = args.kri;
        const double *kcv = args.kcv;
#pragma unroll
        for (int q = 0; q < JQ; ++q) {
            const int c = ll + q * P;
            const int len = clen[q];
            for (int p0 = 0; p0 < len; p0 += 4) {
                int rows[4];
                double vals[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    rows[u] = (p0 + u < len) ? kri[colA[q] + p0 + u] : -1;
                    vals[u] = (p0 + u < len) ? kcv[colA[q] + p0 + u] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (rows[u] < 0) continue;
                    int i = find_sorted(S.I, nI, rows[u]);
                    if (i < 0) {  // impossible for a consistent shadow: never write out of bounds
                        status = kStUnsupported;
                        i = 0;
                    }
                    S.locr[colB[q] + p0 + u] = (unsigned char)i;
                    S.u.tile[c][i] = to_tile<T>(vals[u]);
                    atomicOr(&S.mask[i], 1u << c);
                }
            }
        }
        // ---- right-hand side A_0(I, j); entries outside I go to the residual
        double out2 = 0.0;
        for (int t = zb + ll; t < ze; t += P) {
            const int i = find_sorted(S.I, nI, args.zri[t] + roff);
            const double v = args.zcv[t];
            if (i >= 0) {
                S.c[i] = v;
                S.u.tile[NCOL - 1][i] = to_tile<T>(v);
            } else {
                out2 = fma(v, v, out2);
            }
        }
        out2 = group_sum<P>(out2);
        __syncwarp();
        // ---- load the register tile
        T a[RS][CS];
#pragma unroll
        for (int s = 0; s < RS; ++s)
#pragma unroll
            for (int t = 0; t < CS; ++t) a[s][t] = S.u.tile[t * CG + cg][s * RG + rg];
        __syncwarp();
        // ---- row-major entry lists for r = c - B m: row prefix over lanes
        {
            int cnt = 0;
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const int i = ll * RPL + r;
                if (i < nI) cnt += __popc(S.mask[i]);
            }
            int tot;
            int run = group_excl_scan<P>(cnt, ll, &tot);
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const int i = ll * RPL + r;
                if (i < nI) {
                    S.u.s.rowstart[i] = run;
                    run += __popc(S.mask[i]);
                }
            }
            if (ll == 0) S.u.s.rowstart[nI] = tot;
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < JQ; ++q) {
            const int c = ll + q * P;
            for (int p = 0; p < clen[q]; ++p) {
                const int i = S.locr[colB[q] + p];
                const int pos = S.u.s.rowstart[i] + __popc(S.mask[i] & ((1u << c) - 1u));
                S.u.s.rowent[pos] = colA[q] + p;
                S.u.s.rowcol[pos] = (unsigned char)c;
            }
        }
        // ---- QR of [B c]
        int kmax = nJ;
#pragma unroll
        for (int o = P; o < 32; o <<= 1) kmax = max(kmax, shfl_xor(kmax, o));
        QRPhase<TL, 0>::run(a, rg, cg, gbase, nJ, kmax);
        // ---- R (odd stride), 1/R_kk and Q^T c to shared memory
#pragma unroll
        for (int s = 0; s < RS; ++s)
#pragma unroll
            for (int t = 0; t < CS; ++t) {
                const int i = s * RG + rg, col = t * CG + cg;
                if (col < MAXJ && i <= col && col < nJ) {
                    S.u.s.R[i * TL::RSTR + col] = a[s][t];
                    if (i == col) S.u.s.dinv[i] = T(1) / a[s][t];
                }
                if (col == NCOL - 1 && i < nJ) S.u.s.y[i] = a[s][t];
            }
        __syncwarp();
        // pivots: zero -> rank deficient, non-finite -> nonfinite
        {
            int st = kStOk;
            for (int k = ll; k < nJ; k += P) {
                const double d = to_f64<T>(S.u.s.R[k * TL::RSTR + k]);
                if (!finite64(d)) st = max(st, (int)kStNonfinite);
                else if (d == 0.0) st = max(st, (int)kStRank);
            }
            status = max(status, st);
        }
#pragma unroll
        for (int o = 1; o < P; o <<= 1) status = max(status, shfl_xor(status, o));
        if (status != kStOk) nJ = 0;  // skip the numeric work of a failed column
        // ---- m0 = R^{-1} (Q^T c)(1:nJ)
        T x[JQ];
#pragma unroll
        for (int q = 0; q < JQ; ++q) {
            const int c = ll + q * P;
            x[q] = (c < nJ) ? S.u.s.y[c] : T(0);
        }
        SolveUpper<TL, JQ - 1>::run(S.u.s.R, S.u.s.dinv, x, nJ, ll, gbase);
        double mq[JQ];
#pragma unroll
        for (int q = 0; q < JQ; ++q) {
            const int c = ll + q * P;
            mq[q] = to_f64<T>(x[q]);
            if (c < nJ) S.m[c] = mq[q];
        }
        __syncwarp();
        double r2 = 0.0;
        bool need_final = true;
        if constexpr (!FP64) {
            const int steps = args.refine_steps;
            for (int step = 0; step < steps; ++step) {
                // r = c - B m (FP64)
                residual_rows<TL, false>(S, kcv, nI, ll);
                __syncwarp();
                // g = B^T r (FP64), own columns
#pragma unroll
                for (int q = 0; q < JQ; ++q) {
                    double acc = 0.0;
                    for (int p = 0; p < clen[q]; ++p) acc = fma(kcv[colA[q] + p], S.u.s.r[S.locr[colB[q] + p]], acc);
                    x[q] = to_tile<T>(acc);
                }
                // d = (R^T R)^{-1} g in FP32
                SolveUpperT<TL, 0>::run(S.u.s.R, S.u.s.dinv, x, nJ, ll, gbase);
                SolveUpper<TL, JQ - 1>::run(S.u.s.R, S.u.s.dinv, x, nJ, ll, gbase);
#pragma unroll
                for (int q = 0; q < JQ; ++q) {
                    const int c = ll + q * P;
                    if (c < nJ) {
                        const double d = to_f64<T>(x[q]);
                        mq[q] += d;
                        S.m[c] = mq[q];
                        S.u.s.y[c] = x[q];
                    }
                }
                __syncwarp();
                // final residual r - B d: B d in FP32 from the truncated
                // entries (its error, ~1e-7 |B d|, multiplies a correction
                // that is already ~1e-6 of |c|), subtracted and squared in FP64
                double rf2 = 0.0;
#pragma unroll
                for (int q = 0; q < TL::IQ; ++q) {
                    const int i = ll + q * P;
                    if (i < nI) {
                        float v = 0.f;
                        const int pe = S.u.s.rowstart[i + 1];
                        for (int p = S.u.s.rowstart[i]; p < pe; ++p)
                            v = fmaf(narrow_trunc(kcv[S.u.s.rowent[p]]), (float)S.u.s.y[S.u.s.rowcol[p]], v);
                        const double rfi = S.u.s.r[i] - to_f64<float>(v);
                        rf2 = fma(rfi, rfi, rf2);
                    }
                }
                rf2 = group_sum<P>(rf2);
                __syncwarp();
                r2 = rf2;
                need_final = false;
            }
        }
        if (need_final) {
            r2 = residual_rows<TL>(S, kcv, nI, ll);
            r2 = group_sum<P>(r2);
        }
        // ---- outputs
        int nf = 0;
#pragma unroll
        for (int q = 0; q < JQ; ++q)
            if (ll + q * P < nJ) nf |= !finite64(mq[q]);
#pragma unroll
        for (int o = 1; o < P; o <<= 1) nf |= shfl_xor(nf, o);
        if (valid) {
            if (status == kStOk && (nf || !finite64(r2))) status = kStNonfinite;
            const int njo = args.jcp[jj + 1] - jb;
#pragma unroll
            for (int q = 0; q < JQ; ++q) {
                const int c = ll + q * P;
                if (c < njo) args.mval[args.csr_pos[jb + c]] = (status == kStOk) ? mq[q] : 0.0;
            }
            if (ll == 0) {
                args.colres[jj] = (status == kStOk) ? (r2 > 0.0 ? r2 : 0.0) + out2 : 0.0;
                args.colstat[jj] = status;
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
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarpsPerBlock * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = per_sm * handle_sms(h);
    profile_begin(h, bin);
    kern<<<grid, kWarpsPerBlock * 32, smem, handle_stream(h)>>>(a, bin);
    count_launch(h);
    profile_end(h, bin);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_lsq(sam_handle h, int precision, const LsqArgs &args) {
    cudaError_t e = cudaMemsetAsync(args.ticket, 0, sizeof(int32_t) * kNumBins, handle_stream(h));
    if (e != cudaSuccess) return e;
    if (precision == SAM_FP64) {
        if ((e = launch_one<D0, true>(h, args, 0)) != cudaSuccess) return e;
        if ((e = launch_one<D1, true>(h, args, 1)) != cudaSuccess) return e;
        if ((e = launch_one<D2, true>(h, args, 2)) != cudaSuccess) return e;
        if ((e = launch_one<D3, true>(h, args, 3)) != cudaSuccess) return e;
        if ((e = launch_one<D4, true>(h, args, 4)) != cudaSuccess) return e;
    } else {
        if ((e = launch_one<F0, false>(h, args, 0)) != cudaSuccess) return e;
        if ((e = launch_one<F1, false>(h, args, 1)) != cudaSuccess) return e;
        if ((e = launch_one<F2, false>(h, args, 2)) != cudaSuccess) return e;
        if ((e = launch_one<F3, false>(h, args, 3)) != cudaSuccess) return e;
        if ((e = launch_one<F4, false>(h, args, 4)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sam
