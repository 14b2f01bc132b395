// lsq_core.cuh -- device building blocks shared by the forward least-squares
// kernel (lsq.cu) and its adjoint (adjoint.cu): the register-tile
// descriptor, the per-problem shared-memory layout, FP64<->FP32 conversions
// done with integer operations, group reductions, the phased Householder QR
// of [B c] and the register triangular solves with R.  See lsq.cu for the
// method.
#pragma once

#include <cfloat>
#include <climits>

#include "common.cuh"

namespace sam {
namespace {

constexpr int kWarpsPerBlock = 4;
constexpr int kGatherRegs = 12;  // entries per source column gathered with one round of loads
constexpr int kRowRegs = 10;     // entries per row of B loaded with one round in the residual passes
constexpr int kColRegs = 10;     // entries per column of B loaded with one round in the B^T v passes

// LEAN_: the shape of an adjoint that reads R from a factor tape: no
// register tile and no staging buffer for it (more problems per SM).
// BAND_: the QR keeps to the row band of each reflector (QRPhase); on for the
// size classes of 2-D level-2 columns, whose band spans a third to a half of
// the rows (measured: the class-3 launch of the 10-map Q1 level-2 build 7%
// faster), off where the band spans nearly every row and its branches only
// cost (level-1 columns of classes 0-1, 3-D level-2 columns of class 4:
// measured about 5% slower with it).
template <int RG_, int CG_, int RS_, int CS_, typename T_, int MAXI_BIN_, bool LEAN_ = false, bool BAND_ = false>
struct Tile {
    static constexpr bool LEAN = LEAN_;
    static constexpr bool BAND = BAND_ && !LEAN_;
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
    static constexpr int RELEMS = MAXJ * (MAXJ + 1) / 2;  // R's shared-memory elements
    // position of R(i, k), i <= k: packed rows of MAXJ - i elements from the
    // diagonal
    static __device__ __forceinline__ int rpos(int i, int k) { return i * MAXJ - (i * (i - 1)) / 2 + (k - i); }
    // column slots staged per gather pass: the wide tiles stage [B c] in two
    // passes of half the columns (half the staging buffer: more problems
    // per SM); the narrow ones in one
    static constexpr int CSH = (MAXJ >= 20 && CS >= 2) ? (CS + 1) / 2 : CS;
    static constexpr int VEC = 16 / (int)sizeof(T_);            // elements per 16-byte chunk
    static constexpr int NCH0 = (RS + VEC - 1) / VEC;
    static constexpr int NCH = NCH0 <= 1 ? 1 : NCH0 <= 2 ? 2 : NCH0 <= 4 ? 4 : NCH0 <= 8 ? 8 : 16;  // chunks per lane row
    static constexpr int RSP = NCH * VEC;                      // padded row slots per lane
    static constexpr int SWZ = (NCH < 4 ? NCH : 4) - 1;        // chunk swizzle mask
    using T = T_;
    static_assert(32 % P == 0, "group size must divide the warp");
    static_assert(MAXJ <= 31, "column masks are 32-bit");
    static_assert(MAXI <= 255, "local row indices are 8-bit");
};

template <class TL>
struct ProbSmem {
    using T = typename TL::T;
    int I[TL::MAXI];
    // column state parked across the QR (Column::park): every lane's colA and
    // (colB << 16 | clen), and the group's scalars
    int park[TL::LEAN ? 1 : 2 * TL::P * TL::JQ];
    int park_i[8];
    long long park_l[2];
    unsigned mask[TL::MAXI];
    double c[TL::MAXI];
    double m[TL::MAXJ];
    double lam[TL::MAXJ];  // adjoint multipliers (adjoint only)
    float kap2;            // max R_kk^2 / min R_kk^2 (Column::factor): a cheap lower bound on kappa(B)^2
    float dprev2;          // |d|^2 of the previous refinement step (accuracy guard)
    float msq;             // |m|^2 of the FP32 solution (accuracy guard)
    unsigned char locr[TL::NBCAP];
    union U {
        // [B c], only until registers are loaded (see tile_pos)
        __align__(16) T tile[TL::LEAN ? 16 / sizeof(T) : TL::CSH * TL::CG * TL::RG * TL::RSP];
        struct S {
            int rowstart[TL::MAXI + 1];
            int rowent[TL::NBCAP];
            unsigned char rowcol[TL::NBCAP];
            double r[TL::MAXI];
            double w[TL::MAXI];  // B lambda (adjoint only)
            T y[TL::MAXJ];
            T dinv[TL::MAXJ];
            T R[TL::RELEMS];
        } s;
    } u;
};

// ------------------------------------------------------------- utilities

// Position of element (i, col) of [B c] in the shared tile.  The lane that
// owns it (rg = i % RG, cg = col % CG) reads all its row slots of a column
// as one contiguous "lane row" r = col RG + rg of RSP elements, in 16-byte
// chunks; the chunk index is XOR-swizzled with (r >> 1) so that the eight
// lanes of a quarter-warp hit eight different bank groups.
template <class TL>
__device__ __forceinline__ int tile_pos(int i, int col) {
    const int r = col * TL::RG + (i % TL::RG);
    const int s = i / TL::RG;
    const int v = s / TL::VEC, q = s % TL::VEC;
    return r * TL::RSP + (v ^ ((r >> 1) & TL::SWZ)) * TL::VEC + q;
}

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

// value e of a source array as a tile element: the pre-rounded FP32 copy for
// FP32 tiles, the FP64 value itself for FP64 tiles
template <typename T>
__device__ __forceinline__ T tile_value(const double *v64, const float *v32, int64_t e);
template <>
__device__ __forceinline__ float tile_value<float>(const double *, const float *v32, int64_t e) { return v32[e]; }
template <>
__device__ __forceinline__ double tile_value<double>(const double *v64, const float *, int64_t e) { return v64[e]; }

// reflector arithmetic: hardware approximations suffice for the FP32
// factorisation (its rounding is removed by the FP64 refinement); FP64
// tiles keep correctly rounded sqrt and division
__device__ __forceinline__ float refl_sqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
__device__ __forceinline__ double refl_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float refl_neg_rcp(float x) { return -__frcp_rn(x); }
__device__ __forceinline__ double refl_neg_rcp(double x) { return -1.0 / x; }

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
    static constexpr int RG = TL::RG, CG = TL::CG, RS = TL::RS, CS = TL::CS, L = TL::L, P = TL::P;
    static constexpr int K0 = PH * L;
    static constexpr int SK = K0 / RG;  // row slot of this phase's pivots
    static constexpr int TK = K0 / CG;  // column slot of this phase's pivots
    static constexpr int NPH = (TL::MAXJ + L - 1) / L;
    // every reflector takes the row slots SK..SE-1 (the head); the slots
    // after it (the tail) only when its row band reaches them (tiles
    // without BAND: the head is every slot, and no band is read)
    static constexpr int SE = TL::BAND && SK + (RS + 1) / 2 < RS ? SK + (RS + 1) / 2 : RS;

    // band[k]: the row slot of the last row that holds an entry of columns
    // 0..k of B (Column::build_rows).  Householder reflectors 0..k leave
    // every later row as it was (by induction: such a row is zero in
    // columns 0..k, so reflector k's vector is zero there), so reflector k
    // acts on the row slots SK..band[k] only.  Rows are in the order of the
    // source's numbering, where a stencil's or mesh's band keeps most
    // reflectors inside the head.  The bound is the largest over the warp's
    // problems: the tail's branches are warp-uniform.
    static __device__ __forceinline__ void run(T (&a)[RS][CS], int rg, int cg, int gbase, int nJ, int kmax,
                                               const unsigned char *band) {
        if constexpr (PH < NPH) {
            if (K0 >= kmax) return;
            const int kend = (K0 + L < kmax) ? K0 + L : kmax;
            for (int k = K0; k < kend; ++k) {
                const int ck = k - TK * CG;  // column group owning column k
                const int rk = k - SK * RG;  // row group of row k inside slot SK
                const int own = gbase + ck * RG + rg;  // owner of this lane's rows of column k
                const bool active = k < nJ;
                bool tail = false;
                if constexpr (SE < RS) {
                    int sh = band[k];
#pragma unroll
                    for (int o = P; o < 32; o <<= 1) sh = max(sh, shfl_xor(sh, o));
                    tail = sh >= SE;
                }
                // squared norm of column k below the diagonal (two chains)
                T sig0 = T(0), sig1 = T(0);
#pragma unroll
                for (int s = SK; s < SE; ++s) {
                    T x = a[s][TK];
                    if (s == SK) x = (rg > rk) ? x : T(0);
                    if ((s - SK) & 1) sig1 = fma(x, x, sig1); else sig0 = fma(x, x, sig0);
                }
                if (tail) {
#pragma unroll
                    for (int s = SE; s < RS; ++s) {
                        if ((s - SK) & 1) sig1 = fma(a[s][TK], a[s][TK], sig1); else sig0 = fma(a[s][TK], a[s][TK], sig0);
                    }
                }
                T sig = sig0 + sig1;
#pragma unroll
                for (int o = 1; o < RG; o <<= 1) sig += shfl_xor(sig, o);
                // column k of the rows below the pivot slot, from its owners,
                // and their part of the dot products: independent of the
                // reflector's norm, so they overlap its reductions and square
                // root; the pivot slot's part follows once u_k is known
                T u[SE - SK];
                T w[CS - TK];
#pragma unroll
                for (int t = TK; t < CS; ++t) w[t - TK] = T(0);
#pragma unroll
                for (int s = SK + 1; s < SE; ++s) {
                    const T x = shfl(a[s][TK], own);
                    u[s - SK] = x;
#pragma unroll
                    for (int t = TK; t < CS; ++t) w[t - TK] = fma(x, a[s][t], w[t - TK]);
                }
                if (tail) {
#pragma unroll
                    for (int s = SE; s < RS; ++s) {
                        const T x = shfl(a[s][TK], own);
#pragma unroll
                        for (int t = TK; t < CS; ++t) w[t - TK] = fma(x, a[s][t], w[t - TK]);
                    }
                }
                const T alpha = shfl(a[SK][TK], gbase + ck * RG + rk);
                const T sigma = shfl(sig, gbase + ck * RG);
                // reflector H = I - taup u u^T, u = x with u_k = alpha - beta
                const T nrm = refl_sqrt(fma(alpha, alpha, sigma));
                const T beta = (sigma == T(0)) ? alpha : ((alpha >= T(0)) ? -nrm : nrm);
                const T uk = alpha - beta;
                const T taup = (sigma == T(0) || !active) ? T(0) : refl_neg_rcp(beta * uk);
                {
                    T x = shfl(a[SK][TK], own);
                    x = (rg > rk) ? x : ((rg == rk) ? uk : T(0));
                    u[0] = x;
#pragma unroll
                    for (int t = TK; t < CS; ++t) w[t - TK] = fma(x, a[SK][t], w[t - TK]);
                }
                // reductions interleaved (independent shuffles in flight
                // together), then the updates
#pragma unroll
                for (int o = 1; o < RG; o <<= 1)
#pragma unroll
                    for (int t = TK; t < CS; ++t) w[t - TK] += shfl_xor(w[t - TK], o);
#pragma unroll
                for (int t = TK; t < CS; ++t) {
                    // columns of slots after TK are all > k (L divides CG)
                    w[t - TK] = (t > TK || t * CG + cg > k) ? taup * w[t - TK] : T(0);
                }
#pragma unroll
                for (int s = SK; s < SE; ++s)
#pragma unroll
                    for (int t = TK; t < CS; ++t) a[s][t] = fma(-w[t - TK], u[s - SK], a[s][t]);
                if (tail) {
                    // (the owners' column k is left as it was by the update:
                    // its coefficient is zero)
#pragma unroll
                    for (int s = SE; s < RS; ++s) {
                        const T x = shfl(a[s][TK], own);
#pragma unroll
                        for (int t = TK; t < CS; ++t) a[s][t] = fma(-w[t - TK], x, a[s][t]);
                    }
                }
                if (active && cg == ck && rg == rk) a[SK][TK] = beta;
            }
            QRPhase<TL, PH + 1>::run(a, rg, cg, gbase, nJ, kmax, band);
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
                    if (i < k && k < n) x[q] = fma(-R[TL::rpos(i, k)], xk, x[q]);
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
                    if (i > k && i < n) x[q] = fma(-R[TL::rpos(k, i)], xk, x[q]);
                }
            }
            SolveUpperT<TL, Q + 1>::run(R, dinv, x, n, ll, gbase);
        }
    }
};

// r = c - B m in FP64 over the row-major entry lists; returns this lane's
// partial sum of r_i^2.  The lane's rows are taken in groups of up to four:
// every load of a group (the first kRowRegs entries of each row) is issued
// before the first FMA, so a group costs one round of L2 latency, not one
// per row (the registers of the QR tile are free by now).  The FMAs of a
// row run in the same order as a row-at-a-time loop.
template <class TL, bool SQUARES = true>
__device__ __forceinline__ double residual_rows(ProbSmem<TL> &S, const double *kcv, int nI, int ll) {
    constexpr int IQ = TL::IQ, QMAX = TL::P >= 16 ? 4 : 2, QG = IQ < QMAX ? IQ : QMAX;
    double r2 = 0.0;
#pragma unroll
    for (int q0 = 0; q0 < IQ; q0 += QG) {
        int pb[QG], len[QG];
#pragma unroll
        for (int g = 0; g < QG; ++g) {
            const int i = ll + (q0 + g) * TL::P;
            const bool live = q0 + g < IQ && i < nI;
            pb[g] = live ? S.u.s.rowstart[i] : 0;
            len[g] = live ? S.u.s.rowstart[i + 1] - pb[g] : 0;
        }
        double bv[QG][kRowRegs];
#pragma unroll
        for (int g = 0; g < QG; ++g)
#pragma unroll
            for (int u = 0; u < kRowRegs; ++u) bv[g][u] = (u < len[g]) ? kcv[S.u.s.rowent[pb[g] + u]] : 0.0;
#pragma unroll
        for (int g = 0; g < QG; ++g) {
            const int i = ll + (q0 + g) * TL::P;
            if (q0 + g < IQ && i < nI) {
                double ri = S.c[i];
#pragma unroll
                for (int u = 0; u < kRowRegs; ++u)
                    if (u < len[g]) ri = fma(-bv[g][u], S.m[S.u.s.rowcol[pb[g] + u]], ri);
                for (int p = kRowRegs; p < len[g]; ++p)
                    ri = fma(-kcv[S.u.s.rowent[pb[g] + p]], S.m[S.u.s.rowcol[pb[g] + p]], ri);
                S.u.s.r[i] = ri;
                if (SQUARES) r2 = fma(ri, ri, r2);
            }
        }
    }
    return r2;
}


// --------------------------------------------------- size-class tile table
// FP32 tiles per size class (bins: |I| <= 14/26/40/52/64, |J| <= 5/9/23/27/27)
using F0 = Tile<2, 2, 7, 3, float, 14>;
using F1 = Tile<2, 2, 13, 5, float, 26>;
using F2 = Tile<4, 4, 10, 6, float, 40, false, true>;
using F3 = Tile<4, 4, 13, 7, float, 52, false, true>;
using F4 = Tile<4, 4, 16, 7, float, 64>;
// FP64 tiles
using D0 = Tile<2, 2, 7, 3, double, 14>;
using D1 = Tile<2, 4, 13, 3, double, 26>;
using D2 = Tile<4, 8, 10, 3, double, 40, false, true>;
using D3 = Tile<4, 8, 13, 4, double, 52, false, true>;
using D4 = Tile<4, 8, 16, 4, double, 64>;

// alternative shapes for the autotuner: one problem per 8 or 32 lanes
using F1b = Tile<2, 4, 13, 3, float, 26>;
using F2b = Tile<4, 8, 10, 3, float, 40, false, true>;
using F3b = Tile<4, 8, 13, 4, float, 52, false, true>;
using F4b = Tile<4, 8, 16, 4, float, 64>;
// the adjoint's shapes when R comes from a factor tape (size classes 2-4;
// the two smallest recompute their small QR)
using F2L = Tile<4, 4, 10, 6, float, 40, true>;
using F3L = Tile<4, 4, 13, 7, float, 52, true>;
using F4L = Tile<4, 4, 16, 7, float, 64, true>;
using D2L = Tile<4, 8, 10, 3, double, 40, true>;
using D3L = Tile<4, 8, 13, 4, double, 52, true>;
using D4L = Tile<4, 8, 16, 4, double, 64, true>;

static_assert(F0::MAXI >= 14 && F0::MAXJ >= 5, "bin 0");
static_assert(F1b::MAXI >= 26 && F1b::MAXJ >= 9 && F2b::MAXI >= 40 && F2b::MAXJ >= 23, "variants");
static_assert(F3b::MAXI >= 52 && F3b::MAXJ >= 27 && F4b::MAXI >= 64 && F4b::MAXJ >= 27, "variants");
static_assert(F1::MAXI >= 26 && F1::MAXJ >= 9, "bin 1");
static_assert(F2::MAXI >= 40 && F2::MAXJ >= 23, "bin 2");
static_assert(F3::MAXI >= 52 && F3::MAXJ >= 27, "bin 3");
static_assert(F4::MAXI >= 64 && F4::MAXJ >= 27, "bin 4");
static_assert(D1::MAXJ >= 9 && D2::MAXJ >= 23 && D3::MAXJ >= 27 && D4::MAXJ >= 27, "fp64 bins");

// ----------------------------------------------------- one column problem
// Per-lane state of the column problem owned by this lane's group, and the
// stages shared by the forward build and its adjoint: gather of
// A_k(I_j, J_j) and A_0(I_j, j) into the dense tile, the register tile, the
// row-major entry lists, and the QR with its pivot checks.
template <class TL>
struct Column {
    using T = typename TL::T;
    static constexpr int P = TL::P, RG = TL::RG, CG = TL::CG, RS = TL::RS, CS = TL::CS;
    static constexpr int MAXI = TL::MAXI, NCOL = TL::NCOL, MAXJ = TL::MAXJ, JQ = TL::JQ;
    static constexpr int RPL = (MAXI + P - 1) / P;  // contiguous rows per lane (row prefix sums)

    int ll, rg, cg, gbase;
    bool valid;
    int jj, jl, js, roff, zro, jb, nJ, nI, zb, ze, nB, kmax;  // js: column of the shadow data
    // jb: start of the column in the pattern arrays, read at column js (map
    // 0's copy when the batch shares one structure); aoff / poff: this map's
    // offsets into the source values and the map positions
    int64_t aoff, poff;
    int status;
    int colA[JQ], clen[JQ], colB[JQ];
    double out2;

    __device__ __forceinline__ void begin(const LsqArgs &args, int item, int total, const int32_t *work) {
        begin_at(args, item, total, item < total ? work[item] : 0);
    }

    // as begin, with the work item's column (jj_item) already loaded
    __device__ __forceinline__ void begin_at(const LsqArgs &args, int item, int total, int jj_item) {
        const int lane = threadIdx.x & 31;
        ll = lane % P;
        gbase = lane - ll;
        rg = ll % RG;
        cg = ll / RG;
        valid = item < total;
        jj = valid ? jj_item : 0;  // column of the block-diagonal batch
        const int kmap = jj / args.n;
        jl = jj - kmap * args.n;  // column of A_0
        js = args.shadow_shared ? jl : jj;
        aoff = args.shadow_shared ? (int64_t)kmap * args.map_nnz_src : 0;
        poff = args.shadow_shared ? (int64_t)kmap * args.map_nnz_pat : 0;
        roff = kmap * args.n;     // row offset of this map
        // target column: A_0(:, jl) shifted by roff, or column jj of the
        // block-diagonal targets (rows already global)
        const int zc = args.zbig ? jj : jl;
        // shift of the target's row indices into the numbering of the source
        // rows (and so of the shadow rows): the sources' rows are global, or
        // map 0's when the shadow data is shared; the target's rows are
        // A_0's own (one shared target), or global (one target per map)
        zro = (args.shadow_shared ? 0 : roff) - (args.zbig ? roff : 0);
        jb = nJ = nI = zb = ze = 0;
        if (valid) {
            jb = args.jcp[js];
            nJ = args.jcp[js + 1] - jb;
            nI = args.icnt[js];
            zb = args.zcp[zc];
            ze = args.zcp[zc + 1];
        }
        status = kStOk;
    }

    // J columns (value offsets, lengths, gather offsets), shadow rows when
    // needed, cleared row masks and c
    __device__ __forceinline__ void gather_begin(const LsqArgs &args, ProbSmem<TL> &S) {
#pragma unroll
        for (int q = 0; q < JQ; ++q) {
            const int c = ll + q * P;
            colA[q] = 0;
            clen[q] = 0;
            if (c < nJ) {
                const int col = args.jri[jb + c];
                const int a0 = args.kcp[col];
                clen[q] = args.kcp[col + 1] - a0;
                colA[q] = (int)(a0 + aoff);
            }
        }
        nB = 0;
#pragma unroll
        for (int q = 0; q < JQ; ++q) {
            int tot;
            colB[q] = nB + group_excl_scan<P>(clen[q], ll, &tot);
            nB += tot;
        }
        // the sorted shadow rows are needed only for target entries beyond
        // the precomputed local rows
        const bool need_I = !args.zloc || ze - zb > kZCap;
        for (int i = ll; i < MAXI; i += P) {
            if (need_I) S.I[i] = (i < nI) ? args.ish[(int64_t)js * kICap + i] : INT_MAX;
            S.mask[i] = 0u;
            S.c[i] = 0.0;
        }
    }

    __device__ __forceinline__ void zero_stage(ProbSmem<TL> &S) {
        uint4 *tl = reinterpret_cast<uint4 *>(&S.u.tile[0]);
        constexpr int NV = (int)(sizeof(S.u.tile) / sizeof(uint4));
        for (int e = ll; e < NV; e += P) tl[e] = make_uint4(0u, 0u, 0u, 0u);
    }

    // the entries of the lane's columns c in [c_lo, c_hi): local rows, row
    // masks and (TILE) the values at column c - c_lo of the staging tile
    // (compile-time bounds: a column slot q outside them costs nothing)
    template <bool TILE, int c_lo, int c_hi>
    __device__ __forceinline__ void gather_entries(const LsqArgs &args, ProbSmem<TL> &S) {
#pragma unroll
        for (int q = 0; q < JQ; ++q) {
            if (q * P + P <= c_lo || q * P >= c_hi) continue;
            const int c = ll + q * P;
            const int len = (c >= c_lo && c < c_hi) ? clen[q] : 0;
            const int cs = c - c_lo;
            // local shadow rows of the entries, computed with the shadow rows
            // (read straight from global memory: staging them through shared
            // memory first measured 2x slower in the FP64 kernel)
            const uint8_t *lr = args.lrow + (int64_t)js * kLCap + colB[q];
            // the first kGatherRegs entries: all loads issued before any use
            {
                int rows[kGatherRegs];
                T vals[kGatherRegs];
#pragma unroll
                for (int u = 0; u < kGatherRegs; ++u) {
                    rows[u] = (u < len) ? (int)lr[u] : -1;
                    if constexpr (TILE) vals[u] = (u < len) ? tile_value<T>(args.kcv, args.kcv32, colA[q] + u) : T(0);
                }
#pragma unroll
                for (int u = 0; u < kGatherRegs; ++u) {
                    if (rows[u] < 0) continue;
                    int i = rows[u];
                    if (i >= nI) {  // impossible for a consistent shadow: never write out of bounds
                        status = kStUnsupported;
                        i = 0;
                    }
                    S.locr[colB[q] + u] = (unsigned char)i;
                    if constexpr (TILE) S.u.tile[tile_pos<TL>(i, cs)] = vals[u];
                    atomicOr(&S.mask[i], 1u << c);
                }
            }
            for (int p0 = kGatherRegs; p0 < len; p0 += 4) {
                int rows[4];
                T vals[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    rows[u] = (p0 + u < len) ? (int)lr[p0 + u] : -1;
                    if constexpr (TILE)
                        vals[u] = (p0 + u < len) ? tile_value<T>(args.kcv, args.kcv32, colA[q] + p0 + u) : T(0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (rows[u] < 0) continue;
                    int i = rows[u];
                    if (i >= nI) {  // impossible for a consistent shadow: never write out of bounds
                        status = kStUnsupported;
                        i = 0;
                    }
                    S.locr[colB[q] + p0 + u] = (unsigned char)i;
                    if constexpr (TILE) S.u.tile[tile_pos<TL>(i, cs)] = vals[u];
                    atomicOr(&S.mask[i], 1u << c);
                }
            }
        }
    }

    // the target column: c in FP64, out-of-shadow ||A_0(., j)||^2, and (TILE)
    // the right-hand side at column NCOL - 1 - c_lo of the staging tile
    template <bool TILE>
    __device__ __forceinline__ void gather_target(const LsqArgs &args, ProbSmem<TL> &S, int c_lo) {
        out2 = 0.0;
        for (int t = zb + ll; t < ze; t += P) {
            const int i = target_row(args, S, t - zb, t);
            const double v = args.zcv[t];
            if (i >= 0) {
                S.c[i] = v;
                if constexpr (TILE) S.u.tile[tile_pos<TL>(i, NCOL - 1 - c_lo)] = tile_value<T>(args.zcv, args.zcv32, t);
            } else {
                out2 = fma(v, v, out2);
            }
        }
        out2 = group_sum<P>(out2);
    }

    // everything but the tile, for an adjoint that reads R from a factor
    // tape: local rows, row masks, c, out-of-shadow ||A_0(., j)||^2
    __device__ __forceinline__ void gather_sparse(const LsqArgs &args, ProbSmem<TL> &S) {
        gather_begin(args, S);
        __syncwarp();
        gather_entries<false, 0, NCOL>(args, S);
        gather_target<false>(args, S, 0);
        __syncwarp();
    }

    // [B c] into the register tile a: in passes of CSH column slots, each
    // staged (zeroed, scattered) in shared memory in the chunk-swizzled
    // layout of tile_pos and loaded into its slots; plus everything
    // gather_sparse provides
    __device__ __forceinline__ void gather_tile(const LsqArgs &args, ProbSmem<TL> &S, T (&a)[RS][CS]) {
        constexpr int CSH = TL::CSH, NST = CSH * CG;
        gather_begin(args, S);
        zero_stage(S);
        __syncwarp();
        gather_entries<true, 0, NST>(args, S);
        if constexpr (CSH == CS) gather_target<true>(args, S, 0);
        __syncwarp();
        load_slots<0>(S, a);
        if constexpr (CSH < CS) {
            zero_stage(S);
            __syncwarp();
            gather_entries<true, NST, NCOL>(args, S);
            gather_target<true>(args, S, NST);
            __syncwarp();
            load_slots<1>(S, a);
        }
    }

    // The column's state that the QR does not use, parked in shared memory
    // while the QR tile holds the registers, and taken back after it.
    __device__ __forceinline__ void park(ProbSmem<TL> &S) {
#pragma unroll
        for (int q = 0; q < JQ; ++q) {
            S.park[ll + q * P] = colA[q];
            S.park[P * JQ + ll + q * P] = (colB[q] << 16) | clen[q];
        }
        if (ll == 0) {
            S.park_i[0] = jj;
            S.park_i[1] = js;
            S.park_i[2] = jb;
            S.park_i[3] = nI;
            S.park_i[4] = zb;
            S.park_i[5] = ze;
            S.park_i[6] = zro;
            S.park_i[7] = roff;
            S.park_l[0] = poff;
            S.park_l[1] = __double_as_longlong(out2);
        }
    }
    __device__ __forceinline__ void unpark(ProbSmem<TL> &S) {
        __syncwarp();
#pragma unroll
        for (int q = 0; q < JQ; ++q) {
            colA[q] = S.park[ll + q * P];
            const int w = S.park[P * JQ + ll + q * P];
            colB[q] = w >> 16;
            clen[q] = w & 0xffff;
        }
        jj = S.park_i[0];
        js = S.park_i[1];
        jb = S.park_i[2];
        nI = S.park_i[3];
        zb = S.park_i[4];
        ze = S.park_i[5];
        zro = S.park_i[6];
        roff = S.park_i[7];
        poff = S.park_l[0];
        out2 = __longlong_as_double(S.park_l[1]);
    }

    // position in the map (CSR order of the batch) of pattern entry c
    __device__ __forceinline__ int map_pos(const LsqArgs &args, int c) const {
        return (int)(args.csr_pos[jb + c] + poff);
    }

    // local shadow row of entry t (offset tz in the column) of the target
    // column, -1 outside the shadow
    __device__ __forceinline__ int target_row(const LsqArgs &args, const ProbSmem<TL> &S, int tz, int t) {
        if (args.zloc && tz < kZCap) {
            const int z = args.zloc[(int64_t)js * kZCap + tz];
            if (z == kZOutside) return -1;
            if (z >= nI) {  // impossible for a consistent shadow: never index out of bounds
                status = kStUnsupported;
                return -1;
            }
            return z;
        }
        return find_sorted(S.I, nI, args.zri[t] + zro);
    }

    // the register slots t of staging pass H from the staging tile
    template <int H>
    __device__ __forceinline__ void load_slots(ProbSmem<TL> &S, T (&a)[RS][CS]) {
        constexpr int VEC = TL::VEC, CSH = TL::CSH;
#pragma unroll
        for (int t = H * CSH; t < CS && t < (H + 1) * CSH; ++t) {
            const int r = ((t - H * CSH) * CG + cg) * RG + rg;
            const uint4 *row = reinterpret_cast<const uint4 *>(&S.u.tile[r * TL::RSP]);
            const int swz = (r >> 1) & TL::SWZ;
#pragma unroll
            for (int v = 0; v < TL::NCH; ++v) {
                if (v * VEC >= RS) break;
                union {
                    uint4 u;
                    T e[VEC];
                } w;
                w.u = row[v ^ swz];
#pragma unroll
                for (int q = 0; q < VEC; ++q)
                    if (v * VEC + q < RS) a[v * VEC + q][t] = w.e[q];
            }
        }
        __syncwarp();
    }

    // row-major entry lists (rowstart / rowent / rowcol) for products B x
    __device__ __forceinline__ void build_rows(ProbSmem<TL> &S) {
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
        __syncwarp();
        int last[JQ];  // last local row holding an entry of column c
#pragma unroll
        for (int q = 0; q < JQ; ++q) {
            const int c = ll + q * P;
            last[q] = -1;
            for (int p = 0; p < clen[q]; ++p) {
                const int i = S.locr[colB[q] + p];
                const int pos = S.u.s.rowstart[i] + __popc(S.mask[i] & ((1u << c) - 1u));
                S.u.s.rowent[pos] = colA[q] + p;
                S.u.s.rowcol[pos] = (unsigned char)c;
                last[q] = max(last[q], i);
            }
        }
        if constexpr (TL::BAND) {
            // the QR's row band (QRPhase): the row slot of the last row with
            // an entry in columns 0..c, at least the slot of row c, as a
            // prefix maximum over the columns (c = ll + q P); kept in the
            // bytes of dinv, which the QR does not use before its pivots
            unsigned char *band = reinterpret_cast<unsigned char *>(S.u.s.dinv);
            int carry = -1;
#pragma unroll
            for (int q = 0; q < JQ; ++q) {
                const int c = ll + q * P;
                int v = last[q];
#pragma unroll
                for (int o = 1; o < P; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, v, o);
                    if (ll >= o) v = max(v, y);
                }
                v = max(v, carry);
                carry = __shfl_sync(0xffffffffu, v, (int)(threadIdx.x & 31) | (P - 1));
                if (c < MAXJ) band[c] = (unsigned char)((c < nJ ? max(v, c) : 0) / RG);
            }
        }
    }

    // QR of [B c]; R (packed rows), 1/R_kk and Q^T c to shared memory; a zero
    // or non-finite pivot sets the status and clears nJ (no further work)
    __device__ __forceinline__ void factor(ProbSmem<TL> &S, T (&a)[RS][CS]) {
        __syncwarp();  // the row band (build_rows) is read by every lane of the group
        kmax = nJ;
#pragma unroll
        for (int o = P; o < 32; o <<= 1) kmax = max(kmax, shfl_xor(kmax, o));
        QRPhase<TL, 0>::run(a, rg, cg, gbase, nJ, kmax, reinterpret_cast<const unsigned char *>(S.u.s.dinv));
#pragma unroll
        for (int s = 0; s < RS; ++s)
#pragma unroll
            for (int t = 0; t < CS; ++t) {
                const int i = s * RG + rg, col = t * CG + cg;
                if (col < MAXJ && i <= col && col < nJ) S.u.s.R[TL::rpos(i, col)] = a[s][t];
                if (col == NCOL - 1 && i < nJ) S.u.s.y[i] = a[s][t];
            }
        __syncwarp();
        pivots(S);
    }

    // the diagonal of R in shared memory: 1/R_kk, the status (zero or
    // non-finite pivots clear nJ: no further work) and the kappa estimate
    __device__ __forceinline__ void pivots(ProbSmem<TL> &S) {
        int st = kStOk;
        float rmax = 0.f, rmin = FLT_MAX;  // |R_kk| range, in FP32 (an estimate only)
        for (int k = ll; k < nJ; k += P) {
            const T rkk = S.u.s.R[TL::rpos(k, k)];
            const double d = to_f64<T>(rkk);
            if (!finite64(d)) st = max(st, (int)kStNonfinite);
            else if (d == 0.0) st = max(st, (int)kStRank);
            const float a = fabsf((float)rkk);
            rmax = fmaxf(rmax, a);
            rmin = fminf(rmin, a);
            S.u.s.dinv[k] = T(1) / rkk;
        }
        status = max(status, st);
#pragma unroll
        for (int o = 1; o < P; o <<= 1) {
            status = max(status, shfl_xor(status, o));
            rmax = fmaxf(rmax, shfl_xor(rmax, o));
            rmin = fminf(rmin, shfl_xor(rmin, o));
        }
        if (ll == 0) {  // kept in shared memory: no register across the solves
            const float kap = rmax / rmin;
            S.kap2 = kap * kap;
        }
        if (status != kStOk) nJ = 0;
    }

    // factor tape: R (from shared memory, after factor) to the column's slot,
    // packed (row k from its diagonal, rows in order).  n: the column's
    // unknowns, also when a zero or non-finite pivot cleared nJ, so that a
    // replaying adjoint meets the same pivots and reports the same status
    __device__ __forceinline__ void tape_store(const LsqArgs &args, const ProbSmem<TL> &S, int n) const {
        T *dst = reinterpret_cast<T *>(args.fac) + args.fac_off[jj];
        int base = 0;
        for (int k = 0; k < n; ++k) {
            for (int c = k + ll; c < n; c += P) dst[base + c - k] = S.u.s.R[TL::rpos(k, c)];
            base += n - k;
        }
    }

    // factor tape: the column's R from its slot into shared memory (in place
    // of factor).  The packed rows are copied as 16-byte vectors to the start
    // of R's array, then moved to their rows from the last one down: row k's
    // packed start k nJ - k (k - 1) / 2 is at most its place rpos(k, k)
    // (k MAXJ - k (k - 1) / 2, rows of MAXJ - k), so no row overwrites
    // one that has not moved yet.
    __device__ __forceinline__ void tape_load(const LsqArgs &args, ProbSmem<TL> &S) {
        kmax = nJ;
#pragma unroll
        for (int o = P; o < 32; o <<= 1) kmax = max(kmax, shfl_xor(kmax, o));
        constexpr int EV = 16 / (int)sizeof(T);                          // elements per vector
        constexpr int NVMAX = ((MAXJ * (MAXJ + 1) / 2 + EV - 1) / EV + P - 1) / P;  // vectors per lane
        const int nel = nJ * (nJ + 1) / 2, nvec = (nel + EV - 1) / EV;
        const uint4 *src = reinterpret_cast<const uint4 *>(reinterpret_cast<const T *>(args.fac) +
                                                           (valid ? args.fac_off[jj] : 0));
        uint4 v[NVMAX];
#pragma unroll
        for (int u = 0; u < NVMAX; ++u)
            if (ll + u * P < nvec) v[u] = src[ll + u * P];
#pragma unroll
        for (int u = 0; u < NVMAX; ++u) {
            const int e0 = (ll + u * P) * EV;
            if (ll + u * P < nvec) {
                union {
                    uint4 w;
                    T e[EV];
                } x;
                x.w = v[u];
#pragma unroll
                for (int q = 0; q < EV; ++q)
                    if (e0 + q < nel) S.u.s.R[e0 + q] = x.e[q];
            }
        }
        __syncwarp();
        constexpr int RQ = (MAXJ + P - 1) / P;
        for (int k = kmax - 1; k >= 1; --k) {  // warp-uniform bounds: the moves need the whole warp's barriers
            const int ps = k * nJ - k * (k - 1) / 2;
            T t[RQ];
#pragma unroll
            for (int q = 0; q < RQ; ++q) {
                const int c = k + ll + q * P;
                if (k < nJ && c < nJ) t[q] = S.u.s.R[ps + c - k];
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < RQ; ++q) {
                const int c = k + ll + q * P;
                if (k < nJ && c < nJ) S.u.s.R[TL::rpos(k, c)] = t[q];
            }
            __syncwarp();
        }
        pivots(S);
        __syncwarp();
    }

    // (R^T R)^{-1} applied in place to x (layout c = ll + P q)
    __device__ __forceinline__ void normal_solve(ProbSmem<TL> &S, T (&x)[JQ]) {
        SolveUpperT<TL, 0>::run(S.u.s.R, S.u.s.dinv, x, nJ, ll, gbase);
        SolveUpper<TL, JQ - 1>::run(S.u.s.R, S.u.s.dinv, x, nJ, ll, gbase);
    }

    // (B^T v)_c in FP64 for all of the lane's columns, two at a time with
    // every load of the pair issued before the first FMA (same FMA order as
    // bt_times)
    __device__ __forceinline__ void bt_times_all(const LsqArgs &args, ProbSmem<TL> &S, const double *v,
                                                 double (&out)[JQ]) {
        constexpr int JG = JQ < 2 ? JQ : 2;
#pragma unroll
        for (int q0 = 0; q0 < JQ; q0 += JG) {
            double bv[JG][kColRegs];
#pragma unroll
            for (int g = 0; g < JG; ++g) {
                const int q = q0 + g < JQ ? q0 + g : JQ - 1;
                const int len = q0 + g < JQ ? clen[q] : 0;
#pragma unroll
                for (int u = 0; u < kColRegs; ++u) bv[g][u] = (u < len) ? args.kcv[colA[q] + u] : 0.0;
            }
#pragma unroll
            for (int g = 0; g < JG; ++g) {
                if (q0 + g < JQ) {
                    const int q = q0 + g, len = clen[q];
                    double acc = 0.0;
#pragma unroll
                    for (int u = 0; u < kColRegs; ++u)
                        if (u < len) acc = fma(bv[g][u], v[S.locr[colB[q] + u]], acc);
                    for (int p = kColRegs; p < len; ++p) acc = fma(args.kcv[colA[q] + p], v[S.locr[colB[q] + p]], acc);
                    out[q] = acc;
                }
            }
        }
    }

    // (B^T v)_c in FP64 for the lane's own columns; v indexed by local row
    __device__ __forceinline__ double bt_times(const LsqArgs &args, ProbSmem<TL> &S, const double *v, int q) {
        double acc = 0.0;
        const int len = clen[q];
        double bv[kColRegs];
#pragma unroll
        for (int u = 0; u < kColRegs; ++u) bv[u] = (u < len) ? args.kcv[colA[q] + u] : 0.0;
#pragma unroll
        for (int u = 0; u < kColRegs; ++u)
            if (u < len) acc = fma(bv[u], v[S.locr[colB[q] + u]], acc);
        for (int p = kColRegs; p < len; ++p) acc = fma(args.kcv[colA[q] + p], v[S.locr[colB[q] + p]], acc);
        return acc;
    }
};

}  // namespace
}  // namespace sam
