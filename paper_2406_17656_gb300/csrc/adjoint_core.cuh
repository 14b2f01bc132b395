// adjoint_core.cuh -- the adjoint kernel of the register size classes and
// its launcher, shared by the translation units that instantiate it
// (adjoint.cu: FP64 tiles; adjoint_f32.cu: FP32 tiles; adjoint_tape.cu: the
// factor-tape shapes), so that they compile in parallel.
//
// The hand-written adjoint of the column least-squares solves of
// SAM construction (reverse mode of Sec. 2's column problems
// m_j = argmin ||B_j m - c_j||, B_j = A_k(I_j, J_j), c_j = A_0(I_j, j)).
//
// For the loss L = <dM, M> + w ||A_k M - A_0||_F^2 and one column, with
// r = c - B m, g = dM(J_j, j) and lambda = (B^T B)^{-1} g:
//   dL/dB = r lambda^T - (B lambda) m^T - 2 w r m^T   (stored entries only)
//   dL/dc = B lambda + 2 w r,   dL/dA_0(i, j) = 2 w A_0(i, j) outside I_j.
// The QR is recomputed, or R is read from the forward build's factor tape
// (sam_set_factor_tape): lambda comes from the FP32 R with `refine_steps`
// corrections whose residuals g - B^T (B lambda) are FP64 (or from the FP64
// R in FP64 mode).
//
// Deterministic reduction.  Column problem j writes its dL/dB entries, in
// the gather order (columns c of J_j, each in A_k's CSC order), to its own
// block of dB and records, for every pattern entry (c, j) (map CSR order),
// where the block of column c starts (dbase).  A stored entry e of A_k in
// column c then receives sum over the map's CSR row c (all j with c in J_j)
// of dB[dbase[t] + (e - kcp[c])], added in a fixed order.  dL/dA_0(:, j) is
// written by problem j alone.

#pragma once

#include "lsq_core.cuh"

namespace sam {
namespace {

// blocks per SM that a shape's shared memory allows (1..4); the register
// budget of the FP32 shapes is held to it, so registers never lower the
// occupancy that shared memory permits (the FP64 shapes keep the compiler's
// choice: at 128 registers they spill)
template <class TL>
struct AdjBlocks {
    static constexpr int bytes = (int)sizeof(ProbSmem<TL>) * TL::PPW * kWarpsPerBlock + 1024;
    static constexpr int raw = 233472 / bytes;
    static constexpr int value = raw < 1 ? 1 : (raw > 4 ? 4 : raw);
};

// TL::LEAN: R comes from the forward build's factor tape
template <class TL, bool FP64>
__device__ __forceinline__ void adjoint_body(const LsqArgs &args, int bin) {
    constexpr bool TAPE = TL::LEAN;
    using T = typename TL::T;
    constexpr int P = TL::P, PPW = TL::PPW, RS = TL::RS, CS = TL::CS, JQ = TL::JQ, IQ = TL::IQ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ProbSmem<TL> *probs = reinterpret_cast<ProbSmem<TL> *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ProbSmem<TL> &S = probs[warp * PPW + lane / P];

    const int w0 = args.bin_off[bin];
    const int total = args.bin_off[bin + 1] - w0;
    const int32_t *work = args.work + w0;
    const double *kcv = args.kcv;
    const double rho = args.resid_weight;

    // static round-robin over the resident warps, next column index loaded
    // one iteration ahead (as in the forward kernel)
    const int64_t stride = (int64_t)gridDim.x * kWarpsPerBlock * PPW;
    int64_t base = ((int64_t)blockIdx.x * kWarpsPerBlock + warp) * PPW;
    int jj_next = (base + lane / P < total) ? work[base + lane / P] : 0;
    for (int iter = 0; iter < (1 << 30); ++iter) {
        if (base >= total) break;
        const int item = (int)(base + lane / P);
        const int jj_cur = jj_next;
        base += stride;
        jj_next = (base + lane / P < total) ? work[base + lane / P] : 0;
        Column<TL> C;
        C.begin_at(args, item, total, jj_cur);
        const int ll = C.ll;
        if constexpr (TAPE) {
            // R from the forward build's factor tape: no tile, no QR
            C.gather_sparse(args, S);
            C.build_rows(S);
            C.tape_load(args, S);
        } else {
            T a[RS][CS];
            C.gather_tile(args, S, a);
            C.build_rows(S);
            C.park(S);
            C.factor(S, a);
            C.unpark(S);
        }
        const int nJ = C.nJ, nI = C.nI;
        // ---- m (the forward map) and the incoming gradient g
        double mq[JQ], gq[JQ];
#pragma unroll
        for (int q = 0; q < JQ; ++q) {
            const int c = ll + q * P;
            mq[q] = 0.0;
            gq[q] = 0.0;
            if (c < nJ) {
                const int t = C.map_pos(args, c);
                mq[q] = args.mval[t];
                gq[q] = args.dmval ? args.dmval[t] : 0.0;
                S.m[c] = mq[q];
            }
        }
        __syncwarp();
        // ---- r = c - B m (FP64)
        residual_rows<TL, false>(S, kcv, nI, ll);
        __syncwarp();
        // ---- lambda = (B^T B)^{-1} g
        T x[JQ];
        double lq[JQ];
#pragma unroll
        for (int q = 0; q < JQ; ++q) x[q] = to_tile<T>(gq[q]);
        C.normal_solve(S, x);
#pragma unroll
        for (int q = 0; q < JQ; ++q) lq[q] = to_f64<T>(x[q]);
        const int steps = FP64 ? 0 : args.refine_steps;
        for (int step = 0; step <= steps; ++step) {
            if (step == 0 || step < steps) {
                // w = B lambda (FP64) over the row-major entry lists
#pragma unroll
                for (int q = 0; q < JQ; ++q) {
                    const int c = ll + q * P;
                    if (c < nJ) S.lam[c] = lq[q];
                }
                __syncwarp();
#pragma unroll
                for (int q = 0; q < IQ; ++q) {
                    const int i = ll + q * P;
                    if (i < nI) {
                        double wi = 0.0;
                        const int pe = S.u.s.rowstart[i + 1];
                        for (int p = S.u.s.rowstart[i]; p < pe; ++p)
                            wi = fma(kcv[S.u.s.rowent[p]], S.lam[S.u.s.rowcol[p]], wi);
                        S.u.s.w[i] = wi;
                    }
                }
                __syncwarp();
            } else if constexpr (!FP64) {
                // after the last correction d: w += B d with the small product
                // B d in FP32 from the rounded entries (its error, ~1e-7 |B d|,
                // multiplies a correction already ~1e-6 of |lambda|), added in
                // FP64, as the forward kernel forms its final residual
#pragma unroll
                for (int q = 0; q < IQ; ++q) {
                    const int i = ll + q * P;
                    if (i < nI) {
                        float v = 0.f;
                        const int pe = S.u.s.rowstart[i + 1];
                        for (int p = S.u.s.rowstart[i]; p < pe; ++p)
                            v = fmaf(args.kcv32[S.u.s.rowent[p]], (float)S.u.s.y[S.u.s.rowcol[p]], v);
                        S.u.s.w[i] += to_f64<float>(v);
                    }
                }
                __syncwarp();
            }
            if (step == steps) break;
            // correction: lambda += d = (R^T R)^{-1} (g - B^T w)
#pragma unroll
            for (int q = 0; q < JQ; ++q) x[q] = to_tile<T>(gq[q] - C.bt_times(args, S, S.u.s.w, q));
            C.normal_solve(S, x);
#pragma unroll
            for (int q = 0; q < JQ; ++q) {
                const int c = ll + q * P;
                lq[q] += to_f64<T>(x[q]);
                if (c < nJ) S.u.s.y[c] = x[q];
            }
            __syncwarp();
        }
        if (C.valid && C.status == kStOk) {
            // ---- dL/dB entries of this column's block, and where each block starts
            // dL/dB(i, c) = r_i lambda_c - w_i m_c - 2 rho r_i m_c
            //            = r_i (lambda_c - 2 rho m_c) - w_i m_c: two FP64
            // operations per entry, the column factor formed once
            const int64_t blk = args.dB_off[C.jj];
#pragma unroll
            for (int q = 0; q < JQ; ++q) {
                const int c = ll + q * P;
                if (c < nJ) {
                    const double ac = fma(-2.0 * rho, mq[q], lq[q]);
                    const double nm = -mq[q];
                    for (int p = 0; p < C.clen[q]; ++p) {
                        const int i = S.locr[C.colB[q] + p];
                        args.dB[blk + C.colB[q] + p] = fma(S.u.s.r[i], ac, S.u.s.w[i] * nm);
                    }
                    const int t = C.map_pos(args, c);
                    args.dbase[t] = blk + C.colB[q];
                    if (args.dmres) args.dmres[t] = -2.0 * rho * C.bt_times(args, S, S.u.s.r, q);
                }
            }
            // ---- dL/dA_0(:, j)
            const int64_t zoff = args.zbig ? 0 : (int64_t)(C.roff / args.n) * args.znnz;
            for (int t = C.zb + ll; t < C.ze; t += P) {
                const int i = C.target_row(args, S, t - C.zb, t);
                args.dzval[zoff + t] = (i >= 0) ? S.u.s.w[i] + 2.0 * rho * S.u.s.r[i] : 2.0 * rho * args.zcv[t];
            }
        }
        if (C.valid && ll == 0) args.colstat[C.jj] = C.status;
        __syncwarp();
    }
}

template <class TL, bool FP64>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) adjoint_kernel(LsqArgs args, int bin) {
    adjoint_body<TL, FP64>(args, bin);
}

template <class TL, bool FP64>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, AdjBlocks<TL>::value) adjoint_f32_kernel(LsqArgs args,
                                                                                                int bin) {
    adjoint_body<TL, FP64>(args, bin);
}

template <class TL, bool FP64>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, AdjBlocks<TL>::value) adjoint_tape_kernel(LsqArgs args,
                                                                                                 int bin) {
    adjoint_body<TL, FP64>(args, bin);
}

template <class TL, bool FP64>
cudaError_t launch_one(sam_handle h, const LsqArgs &a, int bin) {
    const size_t smem = sizeof(ProbSmem<TL>) * TL::PPW * kWarpsPerBlock;
    void (*kern)(LsqArgs, int);
    if constexpr (TL::LEAN) kern = adjoint_tape_kernel<TL, FP64>;
    else if constexpr (FP64) kern = adjoint_kernel<TL, FP64>;
    else kern = adjoint_f32_kernel<TL, FP64>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarpsPerBlock * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    kern<<<per_sm * handle_sms(h), kWarpsPerBlock * 32, smem, handle_stream(h)>>>(a, bin);
    count_launch(h);
    return cudaGetLastError();
}

}  // namespace
}  // namespace sam
