// krylov.cu -- restarted GMRES(m) with the right preconditioner z = M (P_0 v)
// (the use of a map named in Sec. 1-2: since A_k M_k ~ A_0 and P_0 is a
// preconditioner of A_0, A_k M_k P_0 ~ A_0 P_0 ~ I).  FP64 throughout.
//
// K independent systems A_k x_k = b_k (a sequence, each with its own map
// M_k and the shared P_0) are solved in the same launches: the grid's y
// index is the system, every system has its own control word, Hessenberg
// matrix, rotations and reductions, and stops on its own.
//
// Everything stays on the device.  One Arnoldi step is at most six launches:
//   [P_0 product] -> [M product] -> A product (w written into V_{j+1})
//   -> orth pass 0 (h = V^T w) -> pass 1 (w -= V h; h' = V^T w)
//   -> pass 2 (w -= V h'; ||w||, Givens rotations, convergence test).
// Orthogonalisation is classical Gram-Schmidt applied twice ("twice is
// enough", Giraud, Langou and Rozloznik 2005), which is as stable as the
// textbook modified Gram-Schmidt and reads the basis once per pass instead
// of once per vector.  Basis vectors are stored unnormalised with a scale
// s_l (the normalised vector is s_l V_l), which saves a normalisation pass.
// Multi-block reductions write per-block partials in a fixed order; the
// last block to finish (atomic ticket, no waiting) sums them in a fixed
// order, so every result is bit-reproducible.
//
// Control lives in a device struct (KryCtl): every kernel of a step returns
// at once when the iteration has stopped, so a whole restart cycle is
// captured once into a CUDA graph and replayed, and the host reads the
// control word once per cycle.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace sam {

namespace {

constexpr int kKryThreads = 256;
constexpr int kMaxRestart = SAM_GMRES_MAX_RESTART;

struct KryCtl {
    int run;          // Arnoldi steps may execute
    int k;            // steps taken in the current cycle
    int its;          // steps taken in total
    int maxiter;
    unsigned ticket;  // last-block-done counter (0 between kernels)
    int pad;
    double rtol, bnorm, rel;
};

struct KryArgs {
    int n, m, nblk, K;  // rows and blocks per system, restart length, systems
    int64_t N;          // K n
    int hstride;        // history entries per system (maxiter)
    KryCtl *ctl;   // [K]
    double *V;     // (m+1) vectors of K n: basis vector l of system k at V + l N + k n (unnormalised)
    double *H;     // [K][(m+1) x m] column-major, rotated in place
    double *cs, *sn;
    double *g;     // [K][m+1] rotated right-hand side
    double *s;     // [K][m+1] scales: the basis vector l is s[l] V_l
    double *h;     // [K][m+1] this pass's projections / the cycle's y
    double *coef;  // [K][m+1] coefficients of the next subtraction / combination
    double *hist;  // [K][hstride] residual estimates / ||b||
    double *part;  // [K][m+1][nblk] block partials (vector-major)
};

// one system's slices of the arguments
struct KrySys {
    KryCtl *c;
    double *H, *cs, *sn, *g, *s, *h, *coef, *hist, *part;
    int64_t base;  // k n: offset of the system's rows in every vector
};

__device__ __forceinline__ KrySys kry_sys(const KryArgs &a, int k) {
    const size_t m1 = (size_t)a.m + 1;
    KrySys y;
    y.c = a.ctl + k;
    y.H = a.H + (size_t)k * m1 * a.m;
    y.cs = a.cs + k * m1;
    y.sn = a.sn + k * m1;
    y.g = a.g + k * m1;
    y.s = a.s + k * m1;
    y.h = a.h + k * m1;
    y.coef = a.coef + k * m1;
    y.hist = a.hist + (size_t)k * a.hstride;
    y.part = a.part + (size_t)k * m1 * a.nblk;
    y.base = (int64_t)k * a.n;
    return y;
}

// gates of the launches of a cycle
enum { kGateAlways = 0, kGateRun = 1, kGateCycle = 2 };

// The kernels of a cycle are launched with programmatic stream
// serialisation, so that a kernel's launch is prepared while its predecessor
// runs; each waits here (griddepcontrol.wait: until the predecessor grid has
// completed and its memory is visible) before reading anything.  No early
// trigger: the successor is released as the blocks exit (triggering at the
// start let waiting successor blocks take scheduling slots, 56 -> 73 us per
// Arnoldi step).  Without the launch attribute the wait returns at once.
__device__ __forceinline__ void after_predecessor() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ bool gate_open(const KryCtl *c, int gate) {
    if (gate == kGateRun) return c->run != 0;
    if (gate == kGateCycle) return c->k > 0;
    return true;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Each block has written its partials; returns true in the one block that
// finishes last, after which all partials are visible to it.  No block waits.
__device__ bool last_block(KryCtl *c, int nblk) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(&c->ticket, 1u);
        last = (t == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        if (threadIdx.x == 0) c->ticket = 0;
    }
    return last;
}

// Fixed-order sum over blocks of part[l][b] for l < cnt (called by the last
// block): out[l] = total.  Warp w sums the vectors l = w, w + 8, ...; its
// lanes read the blocks' partials of a vector, stored contiguously, in one
// round of independent coalesced loads.
__device__ void reduce_partials(const double *part, int nblk, int cnt, double *out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int l = warp; l < cnt; l += kKryThreads / 32) {
        double a = 0.0;
        for (int b = lane; b < nblk; b += 32) a += __ldcg(part + (size_t)l * nblk + b);
        a = warp_sum(a);
        if (lane == 0) out[l] = a;
    }
    __syncthreads();
}

// y = s (Op x), y = b - Op x, or y += Op x for a CSR operator, L lanes per
// row.  s (nullable) is a device scalar.  GB300 runs FP64 at 1/64 of the
// FP32 rate, and the product is bound by FP64 warp instructions rather than
// by memory, so a lane takes a dozen entries of its row: one FMA per entry
// (two accumulators, loads issued four entries ahead) and log2(L)
// shuffle-adds per row, instead of padding lanes and reduction trees.
// System k = blockIdx.y uses ops[per_system ? k : 0]; x, b, y are [K][n]
// and s (nullable) is s[k s_stride].
template <int L>
__global__ void __launch_bounds__(kKryThreads) kry_spmv_kernel(const KryCtl *ctls, int gate, int n,
                                                               const KryOp *ops, int per_system, const double *x,
                                                               const double *s, int s_stride, const double *b,
                                                               double *y, int mode) {
    after_predecessor();
    const int k = blockIdx.y;
    if (!gate_open(ctls + k, gate)) return;
    const KryOp op = ops[per_system ? k : 0];
    const int32_t *rp = op.rp, *ci = op.ci;
    const double *v = op.v;
    const int64_t base = (int64_t)k * n;
    x += base;
    y += base;
    if (b) b += base;
    if (s) s += (size_t)k * s_stride;
    const int lane = threadIdx.x % L;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / L;
    const bool live = row < n;  // every lane reaches the shuffles below
    double a0 = 0.0, a1 = 0.0;
    if (live) {
        const int e1 = rp[row + 1];
        int e = rp[row] + lane;
        for (; e + 3 * L < e1; e += 4 * L) {
            const int c0 = ci[e], c1 = ci[e + L], c2 = ci[e + 2 * L], c3 = ci[e + 3 * L];
            const double v0 = v[e], v1 = v[e + L], v2 = v[e + 2 * L], v3 = v[e + 3 * L];
            const double x0 = __ldg(x + c0), x1 = __ldg(x + c1), x2 = __ldg(x + c2), x3 = __ldg(x + c3);
            a0 = fma(v0, x0, a0);
            a1 = fma(v1, x1, a1);
            a0 = fma(v2, x2, a0);
            a1 = fma(v3, x3, a1);
        }
        for (; e < e1; e += L) a0 = fma(v[e], __ldg(x + ci[e]), a0);
    }
    double acc = a0 + a1;
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, L);
    if (live && lane == 0) {
        if (mode == 0)
            y[row] = s ? acc * *s : acc;
        else if (mode == 1)
            y[row] = b[row] - acc;
        else
            y[row] += acc;
    }
}

// ||x||^2 over blocks; the last block stores ||b|| (what = 0) or starts a
// cycle from the residual in V_0 (what = 1 between cycles, skipped once the
// iteration has stopped; what = 2 for the first cycle, always: beta, g_0,
// s_0, k = 0, and the stopping tests beta <= rtol ||b|| and its >= maxiter).
__global__ void __launch_bounds__(kKryThreads) kry_norm_kernel(KryArgs a, const double *x, int what) {
    after_predecessor();
    __shared__ double red[kKryThreads / 32];
    __shared__ double tot;
    const KrySys S = kry_sys(a, blockIdx.y);
    KryCtl *c = S.c;
    if (what == 1 && !c->run) {
        if (blockIdx.x == 0 && threadIdx.x == 0) c->k = 0;
        return;
    }
    x += S.base;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double t = 0.0;
    if (i < a.n) t = x[i] * x[i];
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int w = 0; w < kKryThreads / 32; ++w) u += red[w];
        S.part[blockIdx.x] = u;
    }
    if (!last_block(c, a.nblk)) return;
    reduce_partials(S.part, a.nblk, 1, &tot);
    if (threadIdx.x == 0) {
        const double nrm = sqrt(tot);
        if (what == 0) {
            c->bnorm = nrm;
        } else {
            c->k = 0;
            S.g[0] = nrm;
            S.s[0] = nrm > 0.0 ? 1.0 / nrm : 0.0;
            c->rel = c->bnorm > 0.0 ? nrm / c->bnorm : 0.0;
            if (nrm <= c->rtol * c->bnorm || c->its >= c->maxiter) c->run = 0;
        }
    }
}

// One classical Gram-Schmidt pass on w = V_{j+1} against V_0..V_j.
//   pass 0: h = V^T w (normalised basis);                 H(:, j)  = h
//   pass 1: w -= sum coef_l V_l; h = V^T w;                H(:, j) += h
//   pass 2: w -= sum coef_l V_l; ||w||, Givens rotations, residual estimate,
//           stopping test.
// A block owns 256 consecutive rows.  In pass 0, op (when given) computes
// w = s (Op z) itself, one row per thread (rows short enough for one lane),
// which fuses the product with A into the first pass.  The subtraction
// takes one row per thread and loads 32 basis values before its FMAs; the
// projections take four vectors per warp at a time, each lane reading 8 of
// the block's rows of each (32 independent loads), against w staged in
// shared memory, with the four shuffle reductions interleaved.
__global__ void __launch_bounds__(kKryThreads) kry_orth_kernel(KryArgs a, int j, int pass, const KryOp *ops,
                                                               const double *z, const double *zs, int zs_stride) {
    after_predecessor();
    __shared__ double ws[2 * (kMaxRestart + 2) > kKryThreads ? 2 * (kMaxRestart + 2) : kKryThreads];
    __shared__ double cf[kMaxRestart + 1];
    __shared__ double red[kKryThreads / 32];
    __shared__ double tot;
    const KrySys S = kry_sys(a, blockIdx.y);
    KryCtl *c = S.c;
    if (!c->run) return;
    const int n = a.n;
    const int64_t N = a.N;
    const int nv = j + 1;
    double *w = a.V + (size_t)(j + 1) * N + S.base;
    const double *V0 = a.V + S.base;  // this system's basis vector l at V0 + l N
    const int64_t row0 = (int64_t)blockIdx.x * kKryThreads;
    const int64_t i = row0 + threadIdx.x;
    const bool in = i < n;
    if (pass > 0)
        for (int l = threadIdx.x; l < nv; l += blockDim.x) cf[l] = S.coef[l];
    __syncthreads();
    double wi = 0.0;
    KryOp op;
    if (pass == 0 && ops) {
        op = ops[blockIdx.y];
        z += S.base;
        if (zs) zs += (size_t)blockIdx.y * zs_stride;
    }
    if (in) {
        if (pass == 0 && ops) {
            double a0 = 0.0, a1 = 0.0;
            const int e1 = op.rp[i + 1];
            int e = op.rp[i];
            for (; e + 3 < e1; e += 4) {
                const int c0 = op.ci[e], c1 = op.ci[e + 1], c2 = op.ci[e + 2], c3 = op.ci[e + 3];
                const double v0 = op.v[e], v1 = op.v[e + 1], v2 = op.v[e + 2], v3 = op.v[e + 3];
                const double x0 = __ldg(z + c0), x1 = __ldg(z + c1), x2 = __ldg(z + c2), x3 = __ldg(z + c3);
                a0 = fma(v0, x0, a0);
                a1 = fma(v1, x1, a1);
                a0 = fma(v2, x2, a0);
                a1 = fma(v3, x3, a1);
            }
            for (; e < e1; ++e) a0 = fma(op.v[e], __ldg(z + op.ci[e]), a0);
            wi = a0 + a1;
            if (zs) wi *= *zs;
            w[i] = wi;
        } else {
            wi = w[i];
        }
    }
    if (pass > 0 && in) {
        // full chunks of 8 basis values: the next chunk's loads are issued
        // before this chunk's FMAs; no FP64 instruction is issued for absent
        // vectors (GB300's narrow FP64 pipe is the bound here)
        const double *vi = V0 + i;
        double s0 = 0.0, s1 = 0.0;
        const int full = nv & ~7;
        double cur[8], nxt[8];
        if (full > 0) {
#pragma unroll
            for (int t = 0; t < 8; ++t) cur[t] = __ldg(vi + (size_t)t * N);
        }
        for (int l0 = 0; l0 < full; l0 += 8) {
            if (l0 + 8 < full) {
#pragma unroll
                for (int t = 0; t < 8; ++t) nxt[t] = __ldg(vi + (size_t)(l0 + 8 + t) * N);
            }
#pragma unroll
            for (int t = 0; t < 8; t += 2) {
                s0 = fma(cf[l0 + t], cur[t], s0);
                s1 = fma(cf[l0 + t + 1], cur[t + 1], s1);
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) cur[t] = nxt[t];
        }
        for (int l = full; l < nv; ++l) s0 = fma(cf[l], __ldg(vi + (size_t)l * N), s0);
        wi -= s0 + s1;
        w[i] = wi;
    }
    ws[threadIdx.x] = wi;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int W8 = kKryThreads / 32;
    if (pass < 2) {
        double wl[W8];
#pragma unroll
        for (int t = 0; t < W8; ++t) wl[t] = ws[lane + 32 * t];  // rows past n hold 0
        for (int q0 = warp; q0 < nv; q0 += 4 * W8) {
            if (q0 + 3 * W8 < nv) {
                // four vectors: 32 independent loads, interleaved reductions
                double d[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const double *vq = V0 + (size_t)(q0 + u * W8) * N + row0;
                    d[u] = 0.0;
#pragma unroll
                    for (int t = 0; t < W8; ++t) {
                        const int r = lane + 32 * t;
                        if (row0 + r < n) d[u] = fma(__ldg(vq + r), wl[t], d[u]);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) d[u] += __shfl_xor_sync(0xffffffffu, d[u], o);
                }
                if (lane == 0) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) S.part[(size_t)(q0 + u * W8) * a.nblk + blockIdx.x] = d[u];
                }
            } else {
                for (int q = q0; q < nv; q += W8) {
                    const double *vq = V0 + (size_t)q * N + row0;
                    double d = 0.0;
#pragma unroll
                    for (int t = 0; t < W8; ++t) {
                        const int r = lane + 32 * t;
                        if (row0 + r < n) d = fma(__ldg(vq + r), wl[t], d);
                    }
                    d = warp_sum(d);
                    if (lane == 0) S.part[(size_t)q * a.nblk + blockIdx.x] = d;
                }
            }
        }
    } else {
        double d = warp_sum(wi * wi);
        if (lane == 0) red[warp] = d;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int ww = 0; ww < W8; ++ww) t += red[ww];
            S.part[blockIdx.x] = t;
        }
    }
    if (!last_block(c, a.nblk)) return;
    const int m = a.m;
    double *Hj = S.H + (size_t)j * (m + 1);
    if (pass < 2) {
        reduce_partials(S.part, a.nblk, nv, S.h);
        for (int l = threadIdx.x; l < nv; l += blockDim.x) {
            const double hl = S.s[l] * S.h[l];  // projection on the normalised s_l V_l
            Hj[l] = pass == 0 ? hl : Hj[l] + hl;
            S.coef[l] = hl * S.s[l];            // subtract hl (s_l V_l)
        }
        return;
    }
    // stage the new column and the earlier rotations in shared memory (one
    // round of loads); the rotations are a serial chain
    double *col = ws, *rc = ws + kMaxRestart + 2, *rs = cf;
    for (int l = threadIdx.x; l <= j; l += blockDim.x) {
        col[l] = Hj[l];
        rc[l] = S.cs[l];
        rs[l] = S.sn[l];
    }
    reduce_partials(S.part, a.nblk, 1, &tot);
    if (threadIdx.x != 0) return;
    const double hn = sqrt(tot);
    col[j + 1] = hn;
    S.s[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
    // earlier rotations on the new column, then the one that zeroes H(j+1, j)
    for (int l = 0; l < j; ++l) {
        const double t = rc[l] * col[l] + rs[l] * col[l + 1];
        col[l + 1] = -rs[l] * col[l] + rc[l] * col[l + 1];
        col[l] = t;
    }
    const double den = hypot(col[j], col[j + 1]);
    const double cj = den == 0.0 ? 1.0 : col[j] / den, sj = den == 0.0 ? 0.0 : col[j + 1] / den;
    S.cs[j] = cj;
    S.sn[j] = sj;
    col[j] = cj * col[j] + sj * col[j + 1];
    for (int l = 0; l <= j; ++l) Hj[l] = col[l];
    Hj[j + 1] = 0.0;
    const double gj = S.g[j];
    S.g[j + 1] = -sj * gj;
    S.g[j] = cj * gj;
    c->its += 1;
    c->k = j + 1;
    const double est = fabs(S.g[j + 1]) / c->bnorm;
    S.hist[c->its - 1] = est;
    c->rel = est;
    if (est <= c->rtol || c->its >= c->maxiter) c->run = 0;
}

// End of a cycle: y = R^{-1} g (back substitution on the rotated H), then
// coef_l = y_l s_l so that the update is sum coef_l V_l.  One block: R and g
// are staged in shared memory, and each column step updates the remaining
// right-hand side in parallel (column-oriented back substitution).
__global__ void __launch_bounds__(kKryThreads) kry_backsolve_kernel(KryArgs a) {
    after_predecessor();
    __shared__ double R[kMaxRestart * (kMaxRestart + 1) / 2 > 0 ? 64 * 65 : 1];
    __shared__ double rhs[kMaxRestart + 1];
    const KrySys S = kry_sys(a, blockIdx.y);
    KryCtl *c = S.c;
    const int k = c->k, m = a.m;
    if (k <= 0) return;
    // R(i, l) for i <= l < k; columns of up to 64 rows fit the tile, longer
    // cycles read R from global memory
    const bool staged = k <= 64;
    for (int e = threadIdx.x; e < k * k && staged; e += blockDim.x) {
        const int i = e % k, l = e / k;
        R[i * 65 + l] = i <= l ? S.H[(size_t)l * (m + 1) + i] : 0.0;
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) rhs[i] = S.g[i];
    __syncthreads();
    for (int i = k - 1; i >= 0; --i) {
        const double rii = staged ? R[i * 65 + i] : S.H[(size_t)i * (m + 1) + i];
        const double yi = rhs[i] / rii;  // every thread reads the finished rhs[i]
        __syncthreads();
        if (threadIdx.x == 0) rhs[i] = yi;
        for (int l = threadIdx.x; l < i; l += blockDim.x)
            rhs[l] -= (staged ? R[l * 65 + i] : S.H[(size_t)i * (m + 1) + l]) * yi;
        __syncthreads();
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        S.h[i] = rhs[i];
        S.coef[i] = rhs[i] * S.s[i];
    }
}

// t = sum_{l<k} coef_l V_l (accumulate = 1: t += that sum)
__global__ void __launch_bounds__(kKryThreads) kry_combine_kernel(KryArgs a, double *t, int accumulate) {
    after_predecessor();
    __shared__ double cf[kMaxRestart + 1];
    const KrySys S = kry_sys(a, blockIdx.y);
    const int k = S.c->k;
    if (k <= 0) return;
    for (int l = threadIdx.x; l < k; l += blockDim.x) cf[l] = S.coef[l];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const double *V0 = a.V + S.base + i;
    t += S.base;
    double u0 = 0.0, u1 = 0.0;
    int l = 0;
    for (; l + 2 <= k; l += 2) {
        u0 = fma(cf[l], __ldg(V0 + (size_t)l * a.N), u0);
        u1 = fma(cf[l + 1], __ldg(V0 + (size_t)(l + 1) * a.N), u1);
    }
    if (l < k) u0 = fma(cf[l], __ldg(V0 + (size_t)l * a.N), u0);
    const double u = u0 + u1;
    if (accumulate)
        t[i] += u;
    else
        t[i] = u;
}

__global__ void kry_init_kernel(KryCtl *ctls, int K, int maxiter, double rtol) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    KryCtl *c = ctls + k;
    c->run = maxiter > 0;
    c->k = 0;
    c->its = 0;
    c->maxiter = maxiter;
    c->ticket = 0;
    c->rtol = rtol;
    c->bnorm = 0.0;
    c->rel = 0.0;
}

// lanes per row: the smallest power of two (1..32) that leaves a lane at
// most 13 entries of an average row
int lanes_for(int n, int64_t nnz) {
    const double mean = n > 0 ? (double)nnz / n : 0.0;
    int L = 1;
    while (L < 32 && 13 * L < mean) L *= 2;
    return L;
}

// Operators of a solve: device tables (A and M one entry per system, P one
// shared entry; M / P nullptr for the identity) and the largest row mean of
// each (lanes per row).
struct KryOps {
    const KryOp *A = nullptr, *M = nullptr, *P = nullptr;
    int64_t a_nnz = 0, m_nnz = 0, p_nnz = 0;  // largest nnz over the systems
};

// a cycle kernel, launched so that it may be scheduled while its
// predecessor finishes (it waits for it on the device: after_predecessor)
template <typename... KArgs, typename... Args>
cudaError_t launch_dep(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

cudaError_t spmv(cudaStream_t st, const KryArgs &a, int gate, const KryOp *ops, int per_system, int64_t nnz,
                 const double *x, const double *s, int s_stride, const double *b, double *y, int mode) {
    const int n = a.n;
    const int L = lanes_for(n, nnz);
    const int64_t threads = (int64_t)n * L;
    const dim3 grid((unsigned)((threads + kKryThreads - 1) / kKryThreads), (unsigned)a.K);
#define SAM_KRY_SPMV(LL)                                                                                        \
    return launch_dep(kry_spmv_kernel<LL>, grid, dim3(kKryThreads), st, a.ctl, gate, n, ops, per_system, x, s, \
                      s_stride, b, y, mode);
    switch (L) {
        case 1: SAM_KRY_SPMV(1)
        case 2: SAM_KRY_SPMV(2)
        case 4: SAM_KRY_SPMV(4)
        case 8: SAM_KRY_SPMV(8)
        case 16: SAM_KRY_SPMV(16)
        default: SAM_KRY_SPMV(32)
    }
#undef SAM_KRY_SPMV
    return cudaGetLastError();
}

// The launches of one restart cycle (all gated on the systems' control
// words): m Arnoldi steps, the update of x, and the residual of the next
// cycle.  Returns the number of kernels enqueued, or -1 on a launch error.
int enqueue_cycle(cudaStream_t st, const KryArgs &a, const KryOps &op, const double *b, double *x, double *t,
                  double *u) {
    int launches = 0;
    const dim3 gb((unsigned)a.nblk, (unsigned)a.K);
    const int ss = a.m + 1;  // stride of the per-system scales
    auto ok = [&](cudaError_t e) { return e == cudaSuccess; };
    // w = A z fused into the first Gram-Schmidt pass when a row of A fits one
    // lane, a separate product otherwise
    const bool fuse = lanes_for(a.n, op.a_nnz) == 1;
    for (int j = 0; j < a.m; ++j) {
        // z = M (P_0 (s_j V_j)), the identity where an operator is absent
        const double *z = a.V + (size_t)j * a.N;
        const double *zs = a.s + j;
        if (op.P) {
            if (!ok(spmv(st, a, kGateRun, op.P, 0, op.p_nnz, z, zs, ss, nullptr, t, 0))) return -1;
            ++launches;
            z = t;
            zs = nullptr;
        }
        if (op.M) {
            if (!ok(spmv(st, a, kGateRun, op.M, 1, op.m_nnz, z, zs, ss, nullptr, u, 0))) return -1;
            ++launches;
            z = u;
            zs = nullptr;
        }
        if (!fuse) {
            if (!ok(spmv(st, a, kGateRun, op.A, 1, op.a_nnz, z, zs, ss, nullptr, a.V + (size_t)(j + 1) * a.N, 0)))
                return -1;
            ++launches;
        }
        for (int pass = 0; pass < 3; ++pass) {
            const bool f0 = pass == 0 && fuse;
            if (!ok(launch_dep(kry_orth_kernel, gb, dim3(kKryThreads), st, a, j, pass, f0 ? op.A : (const KryOp *)nullptr,
                               f0 ? z : (const double *)nullptr, f0 ? zs : (const double *)nullptr, f0 ? ss : 0)))
                return -1;
            ++launches;
        }
    }
    // x += M (P_0 (sum_l y_l s_l V_l))
    if (!ok(launch_dep(kry_backsolve_kernel, dim3(1, (unsigned)a.K), dim3(kKryThreads), st, a))) return -1;
    ++launches;
    if (!op.P && !op.M) {
        if (!ok(launch_dep(kry_combine_kernel, gb, dim3(kKryThreads), st, a, x, 1))) return -1;
        ++launches;
    } else {
        // the sum goes to the temporary the first operator does not write
        double *sum = op.P ? u : t;
        if (!ok(launch_dep(kry_combine_kernel, gb, dim3(kKryThreads), st, a, sum, 0))) return -1;
        ++launches;
        const double *cur = sum;
        if (op.P && op.M) {
            if (!ok(spmv(st, a, kGateCycle, op.P, 0, op.p_nnz, cur, nullptr, 0, nullptr, t, 0))) return -1;
            ++launches;
            cur = t;
        }
        const bool last_m = op.M != nullptr;
        if (!ok(spmv(st, a, kGateCycle, last_m ? op.M : op.P, last_m ? 1 : 0, last_m ? op.m_nnz : op.p_nnz, cur,
                     nullptr, 0, nullptr, x, 2)))
            return -1;
        ++launches;
    }
    if (!ok(cudaGetLastError())) return -1;
    // next cycle: V_0 = b - A x, beta, stopping test
    if (!ok(spmv(st, a, kGateRun, op.A, 1, op.a_nnz, x, nullptr, 0, b, a.V, 1))) return -1;
    if (!ok(launch_dep(kry_norm_kernel, gb, dim3(kKryThreads), st, a, (const double *)a.V, 1))) return -1;
    launches += 2;
    if (!ok(cudaGetLastError())) return -1;
    return launches;
}

}  // namespace

sam_status gmres_solve(sam_handle h, int K, int n, const KryOp *A, const KryOp *M, const KryOp &P, const double *b,
                       double *x, int restart, int maxiter, double rtol, double *hist_dev, int32_t *its_out,
                       double *rel_out, int64_t *launches_out) {
    cudaStream_t st = handle_stream(h);
    const int m = restart;
    const int nblk = (int)((n + kKryThreads - 1) / kKryThreads);
    const int64_t N = (int64_t)K * n;
    const size_t m1 = (size_t)m + 1;
    std::vector<void *> mem;
    bool oom = false;
    auto get = [&](size_t bytes) {
        void *p = pool_alloc(h, bytes);
        if (p)
            mem.push_back(p);
        else
            oom = true;
        return p;
    };
    auto release = [&](sam_status s) {
        for (void *p : mem) pool_free(h, p);
        return s;
    };
    KryArgs a;
    a.n = n;
    a.m = m;
    a.nblk = nblk;
    a.K = K;
    a.N = N;
    a.hstride = maxiter > 0 ? maxiter : 1;
    a.ctl = (KryCtl *)get(sizeof(KryCtl) * K);
    a.V = (double *)get(sizeof(double) * (size_t)N * m1);
    a.H = (double *)get(sizeof(double) * K * m1 * m);
    a.cs = (double *)get(sizeof(double) * K * m1);
    a.sn = (double *)get(sizeof(double) * K * m1);
    a.g = (double *)get(sizeof(double) * K * m1);
    a.s = (double *)get(sizeof(double) * K * m1);
    a.h = (double *)get(sizeof(double) * K * m1);
    a.coef = (double *)get(sizeof(double) * K * m1);
    a.hist = hist_dev ? hist_dev : (double *)get(sizeof(double) * (size_t)K * a.hstride);
    a.part = (double *)get(sizeof(double) * K * m1 * nblk);
    double *t = (double *)get(sizeof(double) * (size_t)N);
    double *u = (double *)get(sizeof(double) * (size_t)N);
    // operator tables
    KryOps op;
    KryOp *dA = (KryOp *)get(sizeof(KryOp) * K);
    KryOp *dM = M ? (KryOp *)get(sizeof(KryOp) * K) : nullptr;
    KryOp *dP = P.rp ? (KryOp *)get(sizeof(KryOp)) : nullptr;
    if (oom) return release(SAM_ERR_OOM);
    cudaMemcpyAsync(dA, A, sizeof(KryOp) * K, cudaMemcpyHostToDevice, st);
    if (dM) cudaMemcpyAsync(dM, M, sizeof(KryOp) * K, cudaMemcpyHostToDevice, st);
    if (dP) cudaMemcpyAsync(dP, &P, sizeof(KryOp), cudaMemcpyHostToDevice, st);
    op.A = dA;
    op.M = dM;
    op.P = dP;
    for (int k = 0; k < K; ++k) {
        op.a_nnz = std::max(op.a_nnz, A[k].nnz);
        if (M) op.m_nnz = std::max(op.m_nnz, M[k].nnz);
    }
    op.p_nnz = P.nnz;
    const dim3 gb((unsigned)nblk, (unsigned)K);
    int64_t launches = 0;
    std::vector<KryCtl> hc((size_t)K);
    auto read_ctl = [&]() {
        return cudaMemcpyAsync(hc.data(), a.ctl, sizeof(KryCtl) * K, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
               cudaStreamSynchronize(st) == cudaSuccess;
    };
    // ||b_k||, then the first residuals (b_k - A_k x0_k) and their norms
    kry_init_kernel<<<(K + 127) / 128, 128, 0, st>>>(a.ctl, K, maxiter, rtol);
    kry_norm_kernel<<<gb, kKryThreads, 0, st>>>(a, b, 0);
    launches += 2;
    if (!read_ctl()) return release(SAM_ERR_CUDA);
    bool any_zero = false;
    for (int k = 0; k < K; ++k) {
        if (!std::isfinite(hc[k].bnorm)) return release(SAM_ERR_NONFINITE);
        any_zero = any_zero || hc[k].bnorm == 0.0;
    }
    if (any_zero) {
        // b_k = 0: x_k = 0 and no steps for that system
        for (int k = 0; k < K; ++k)
            if (hc[k].bnorm == 0.0) {
                cudaMemsetAsync(x + (size_t)k * n, 0, sizeof(double) * n, st);
                cudaMemsetAsync(&a.ctl[k].run, 0, sizeof(int), st);
            }
    }
    if (spmv(st, a, kGateRun, op.A, 1, op.a_nnz, x, nullptr, 0, b, a.V, 1) != cudaSuccess) return release(SAM_ERR_CUDA);
    kry_norm_kernel<<<gb, kKryThreads, 0, st>>>(a, a.V, 2);
    launches += 2;
    // one restart cycle, captured once and replayed while any system runs
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto drop_graph = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
    };
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return release(SAM_ERR_CUDA);
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        drop_graph();
        return release(SAM_ERR_CUDA);
    }
    const int per_cycle = enqueue_cycle(cap, a, op, b, x, t, u);
    cudaError_t ce = cudaStreamEndCapture(cap, &graph);
    if (per_cycle < 0 || ce != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        drop_graph();
        return release(SAM_ERR_CUDA);
    }
    sam_status status = SAM_OK;
    for (;;) {
        if (!read_ctl()) {
            status = SAM_ERR_CUDA;
            break;
        }
        bool any_run = false, bad = false;
        for (int k = 0; k < K; ++k) {
            any_run = any_run || hc[k].run;
            bad = bad || !std::isfinite(hc[k].rel);
        }
        if (bad) {
            status = SAM_ERR_NONFINITE;
            break;
        }
        if (!any_run) break;
        if (cudaGraphLaunch(exec, st) != cudaSuccess) {
            status = SAM_ERR_CUDA;
            break;
        }
        launches += per_cycle;
    }
    drop_graph();
    count_launch(h, (int)launches);
    for (int k = 0; k < K; ++k) {
        if (its_out) its_out[k] = hc[k].bnorm == 0.0 ? 0 : hc[k].its;
        if (rel_out) rel_out[k] = hc[k].bnorm == 0.0 ? 0.0 : hc[k].rel;
    }
    if (launches_out) *launches_out = launches;
    return release(status);
}

}  // namespace sam
