// lsq_kernel.cuh -- the register-tile least-squares kernel of the size
// classes 0-4 and its launcher, shared by the FP32 (lsq.cu) and FP64
// (lsq_fp64.cu) translation units, which instantiate it for their tile
// shapes.
//
// The batched column least-squares solves of SAM construction
// (arXiv 2406.17656, Sec. 2: Eq. (approx_map) splits into one problem per
// column, min_m || A_k(I_j, J_j) m - A_0(I_j, j) ||).
//
// A batch of K maps is one block-diagonal problem: source matrices, patterns
// and shadow rows of map k occupy rows/columns [k n, (k+1) n) of "big"
// arrays, so one launch per size class covers every map.  A persistent grid
// (one resident wave) walks the size class's work list round-robin, each
// warp loading its next column index one iteration ahead (a bounded loop
// that ends past the item count).
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
// Rows follow the source's numbering, so B has a staircase profile: in the
// size classes of 2-D level-2 columns each reflector takes a fixed head of
// row slots and the rest only when the rows holding entries of columns
// 0..k reach them (QRPhase).
// The right-hand side is the last column, so Q^T c falls out of the sweep.
// Triangular solves with R run in registers (unknown c on lane c % P) with
// one shuffle per step; R sits in shared memory, packed by rows.
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
#pragma once

#include "lsq_core.cuh"


namespace sam {
namespace {

// blocks per SM that the shared memory of a tile allows (1..4; 1..3 for the
// FP64 tiles, whose registers do not fit 128 per thread without spilling):
// the register budget is held to the same count, so registers never lower
// the occupancy that shared memory permits
template <class TL>
struct MinBlocks {
    static constexpr int bytes = (int)sizeof(ProbSmem<TL>) * TL::PPW * kWarpsPerBlock + 1024;
    static constexpr int raw = 233472 / bytes;
    static constexpr int cap = sizeof(typename TL::T) == 8 ? 3 : 4;
    static constexpr int value = raw < 1 ? 1 : (raw > cap ? cap : raw);
};

template <class TL, bool FP64>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, MinBlocks<TL>::value) lsq_kernel(LsqArgs args, int bin) {
    using T = typename TL::T;
    constexpr int P = TL::P, PPW = TL::PPW, RS = TL::RS, CS = TL::CS, JQ = TL::JQ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ProbSmem<TL> *probs = reinterpret_cast<ProbSmem<TL> *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ProbSmem<TL> &S = probs[warp * PPW + lane / P];

    const int w0 = args.bin_off[bin] + (args.item_hi > 0 ? args.item_lo : 0);
    const int total = args.item_hi > 0 ? args.item_hi - args.item_lo : args.bin_off[bin + 1] - w0;
    const int32_t *work = args.work + w0;

    // static round-robin over the resident warps (columns of a size class
    // cost about the same): the next work item is known, and its column
    // index is loaded one iteration ahead, so no atomic counter and no work
    // lookup sit at the head of an iteration's dependent loads (32-bit
    // indices: a class holds fewer than 2^31 - one wave of items)
    const int stride = gridDim.x * kWarpsPerBlock * PPW;
    int base = (blockIdx.x * kWarpsPerBlock + warp) * PPW;
    int jj_next = (base + lane / P < total) ? work[base + lane / P] : 0;
    for (int iter = 0; iter < (1 << 30); ++iter) {
        if (base >= total) break;
        const int item = base + lane / P;
        const int jj_cur = jj_next;
        base += stride;
        jj_next = (base + lane / P < total) ? work[base + lane / P] : 0;
        Column<TL> C;
        C.begin_at(args, item, total, jj_cur);
        const int ll = C.ll;
        T a[RS][CS];
        C.gather_tile(args, S, a);
        C.build_rows(S);
        C.park(S);
        C.factor(S, a);
        C.unpark(S);
        const int nJ = C.nJ, nI = C.nI;
        if (args.fac_mode == kTapeRecord && C.valid && (C.status == kStOk || C.status == kStRank ||
                                                        C.status == kStNonfinite))
            C.tape_store(args, S, args.jcp[C.js + 1] - C.jb);
        // ---- m0 = R^{-1} (Q^T c)(1:nJ)
        T x[JQ];
#pragma unroll
        for (int q = 0; q < JQ; ++q) {
            const int c = ll + q * P;
            x[q] = (c < nJ) ? S.u.s.y[c] : T(0);
        }
        SolveUpper<TL, JQ - 1>::run(S.u.s.R, S.u.s.dinv, x, nJ, ll, C.gbase);
        double mq[JQ];
#pragma unroll
        for (int q = 0; q < JQ; ++q) {
            const int c = ll + q * P;
            mq[q] = to_f64<T>(x[q]);
            if (c < nJ) S.m[c] = mq[q];
        }
        if constexpr (!FP64) {
            // |m|^2 of the FP32 solution: the scale of the refinement's
            // accuracy guard (kept in shared memory, not in a register)
            float m2 = 0.f;
#pragma unroll
            for (int q = 0; q < JQ; ++q)
                if (ll + q * P < nJ) m2 = fmaf(x[q], x[q], m2);
            m2 = group_sum<P>(m2);
            if (ll == 0) S.msq = m2;
        }
        __syncwarp();
        double r2 = 0.0;
        bool need_final = true;
        bool fallback = false;
        bool redo = false;  // automatic refinement: solved again with two steps
        if constexpr (!FP64) {
            // A fixed number of steps, or (refine_steps < 0, automatic) one
            // step and the stopping test below.  A column whose test asks
            // for a second step leaves with status kStStep2, and a launch of
            // its own solves it again with kAutoSteps steps
            // (launch_refine_fallback).  Taking the second step in place, in
            // the warps that hold such a column, was slower by far more than
            // the step's own work: those warps' code runs apart from the
            // others' and instruction fetch stalls every warp of the SM
            const bool autoref = args.refine_steps < 0;
            const int steps = autoref ? 1 : args.refine_steps;
            for (int step = 0; step < steps; ++step) {
                // r = c - B m (FP64), g = B^T r (FP64), d = (R^T R)^{-1} g (FP32)
                residual_rows<TL, false>(S, args.kcv, nI, ll);
                __syncwarp();
                {
                    double g[JQ];
                    C.bt_times_all(args, S, S.u.s.r, g);
#pragma unroll
                    for (int q = 0; q < JQ; ++q) x[q] = to_tile<T>(g[q]);
                }
                C.normal_solve(S, x);
                float dsq = 0.f;
#pragma unroll
                for (int q = 0; q < JQ; ++q) {
                    const int c = ll + q * P;
                    if (c < nJ) {
                        mq[q] += to_f64<T>(x[q]);
                        S.m[c] = mq[q];
                        S.u.s.y[c] = x[q];
                        dsq = fmaf(x[q], x[q], dsq);
                    }
                }
                __syncwarp();
                dsq = group_sum<P>(dsq);
                const float msq = S.msq;
                // Accuracy guard.  CSNE contracts the error e_s by a factor
                // rho ~ u_32 kappa(B)^2 per step, so e_s <= rho / (1 - rho) |d_s|
                // for rho < 1.  rho is estimated as the larger of
                // kRhoSafety u_32 kappa^2, with kappa estimated by
                // max |R_kk| / min |R_kk| (a lower bound on kappa(B), hence the
                // safety factor), and, after step 1, kAutoC |d_1| / |m|
                // (the correction itself is ~ u_32 kappa |m|), after later
                // steps |d_s| / |d_{s-1}|.  A column whose predicted error is
                // above kFallbackTol |m| (or whose rho is 1/2 or more) is
                // re-solved in FP64.  The test is monotone in rho, so it is
                // applied to each estimate in turn; it runs in FP32 on squared
                // norms, with products only (estimates need no more, and FP64
                // arithmetic costs GB300's narrow FP64 pipe dearly), |m| taken
                // from the FP32 solution, and 1 - rho >= 1/2 used for the ratio
                // estimates (conservative)
                constexpr float kTol = (float)kFallbackTol, kTol2 = kTol * kTol, kC = (float)kAutoC;
                const float rk = (float)(kRhoSafety * kU32) * S.kap2;  // u_32 kappa^2, with a safety factor
                bool miss = !(rk < 0.5f) || rk * rk * dsq > kTol2 * (1.f - rk) * (1.f - rk) * msq;
                if (step == 0) {  // rho = kAutoC |d_1| / |m|
                    miss = miss || 4.f * kC * kC * dsq >= msq || 2.f * kC * dsq > kTol * msq;
                } else if (dsq > (float)kNoise2 * msq) {
                    // rho = |d_s| / |d_{s-1}|, unless the corrections are at the
                    // rounding level of the FP64 residual (their ratio is noise)
                    const float dprev2 = S.dprev2;
                    miss = miss || 4.f * dsq >= dprev2 || 4.f * dsq * dsq > kTol2 * msq * dprev2;
                }
                __syncwarp();
                if (C.ll == 0) S.dprev2 = dsq;  // (shared memory: no register across the next step)
                if (step == steps - 1) {
                    // automatic: a second step when step 1 left the column
                    // above kAutoTol (kAutoC |d_1|^2 > kAutoTol |m|^2) or
                    // predicted above the target; with a fixed number of
                    // steps, a miss after the last falls back to FP64
                    if (autoref)
                        redo = kC * dsq > (float)kAutoTol * msq || miss;
                    else
                        fallback = miss;
                }
            }
            if (steps > 0) {
                // final residual r - B d: B d in FP32 from the rounded
                // entries (its error, ~1e-7 |B d|, multiplies a correction
                // that is already ~1e-6 of |c|), subtracted and squared in FP64
                // (rows in groups of up to four, all loads of a group first)
                double rf2 = 0.0;
                constexpr int IQ = TL::IQ, QMAX = P >= 16 ? 4 : 2, QG = IQ < QMAX ? IQ : QMAX;
#pragma unroll
                for (int q0 = 0; q0 < IQ; q0 += QG) {
                    int pb[QG], len[QG];
#pragma unroll
                    for (int g = 0; g < QG; ++g) {
                        const int i = ll + (q0 + g) * P;
                        const bool live = q0 + g < IQ && i < nI;
                        pb[g] = live ? S.u.s.rowstart[i] : 0;
                        len[g] = live ? S.u.s.rowstart[i + 1] - pb[g] : 0;
                    }
                    float bv[QG][kRowRegs];
#pragma unroll
                    for (int g = 0; g < QG; ++g)
#pragma unroll
                        for (int u = 0; u < kRowRegs; ++u)
                            bv[g][u] = (u < len[g]) ? args.kcv32[S.u.s.rowent[pb[g] + u]] : 0.f;
#pragma unroll
                    for (int g = 0; g < QG; ++g) {
                        const int i = ll + (q0 + g) * P;
                        if (q0 + g < IQ && i < nI) {
                            float v = 0.f;
#pragma unroll
                            for (int u = 0; u < kRowRegs; ++u)
                                if (u < len[g]) v = fmaf(bv[g][u], (float)S.u.s.y[S.u.s.rowcol[pb[g] + u]], v);
                            for (int p = kRowRegs; p < len[g]; ++p)
                                v = fmaf(args.kcv32[S.u.s.rowent[pb[g] + p]], (float)S.u.s.y[S.u.s.rowcol[pb[g] + p]], v);
                            const double rfi = S.u.s.r[i] - to_f64<float>(v);
                            rf2 = fma(rfi, rfi, rf2);
                        }
                    }
                }
                rf2 = group_sum<P>(rf2);
                __syncwarp();
                r2 = rf2;
                need_final = false;
            }
            if (C.valid && ll == 0 && args.refine_used)
                args.refine_used[C.jj] = (uint8_t)((fallback && C.status == kStOk)
                                                       ? kAutoSteps + 1
                                                       : (steps < 2 ? steps : 2));
        }
        if (need_final) {
            r2 = residual_rows<TL>(S, args.kcv, nI, ll);
            r2 = group_sum<P>(r2);
        }
        // ---- outputs
        int nf = 0;
#pragma unroll
        for (int q = 0; q < JQ; ++q)
            if (ll + q * P < nJ) nf |= !finite64(mq[q]);
#pragma unroll
        for (int o = 1; o < P; o <<= 1) nf |= shfl_xor(nf, o);
        if (C.valid) {
            int status = C.status;
            if (status == kStOk && (nf || !finite64(r2))) status = kStNonfinite;
            if (status == kStOk && fallback) status = kStRefine;  // re-solved by the FP64 kernel
            if (status == kStOk && redo) status = kStStep2;       // solved again with two steps
            const int njo = args.jcp[C.js + 1] - C.jb;
#pragma unroll
            for (int q = 0; q < JQ; ++q) {
                const int c = ll + q * P;
                if (c < njo) args.mval[C.map_pos(args, c)] = (status == kStOk) ? mq[q] : 0.0;
            }
            if (ll == 0) {
                args.colres[C.jj] = (status == kStOk) ? (r2 > 0.0 ? r2 : 0.0) + C.out2 : 0.0;
                args.colstat[C.jj] = status;
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------ dispatch

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
}  // namespace sam
