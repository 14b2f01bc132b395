// residual_row.cuh -- one row of R = A_k M - A_0 (Eq. (res)), summed in a
// fixed order by one warp.  Shared by sam_residual (misc.cu) and the
// allocation-free sam_residual_static (noalloc.cu), so that both compute
// the same bits.
#pragma once

#include <climits>

#include "common.cuh"

namespace sam {

constexpr int kResRowBuf = 1024;  // candidate entries of one row of R a warp can hold

// ||R(i, :)||^2 for R = A_k M - A_0, computed by the calling warp: the
// products A_k(i, c) M(c, :) and the entries -A_0(i, :) are collected as
// (column, value) pairs in K / V (kResRowBuf entries of the warp's own
// shared memory), sorted by column with a fixed bitonic network, summed per
// column and squared.  Every lane returns the same value.  Returns a
// negative value, having written nothing, when the row has more than
// kResRowBuf candidate entries.
__device__ __forceinline__ double residual_row_sq(int64_t i, int lane, const int32_t *krp, const int32_t *kci,
                                                  const double *kv, const int32_t *mrp, const int32_t *mci,
                                                  const double *mv, const int32_t *zrp, const int32_t *zci,
                                                  const double *zv, int *K, double *V) {
    // count the candidates
    int cnt = zrp[i + 1] - zrp[i];
    for (int base = krp[i]; base < krp[i + 1]; base += 32) {
        const int e = base + lane;
        int len = (e < krp[i + 1]) ? mrp[kci[e] + 1] - mrp[kci[e]] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) len += __shfl_xor_sync(0xffffffffu, len, o);
        cnt += len;
    }
    if (cnt > kResRowBuf) return -1.0;
    // target entries first, then the products, in a fixed order
    const int zb = zrp[i], ze = zrp[i + 1];
    for (int t = zb + lane; t < ze; t += 32) {
        K[t - zb] = zci[t];
        V[t - zb] = -zv[t];
    }
    int off = ze - zb;
    for (int e = krp[i]; e < krp[i + 1]; ++e) {
        const int c = kci[e];
        const double a = kv[e];
        const int mb = mrp[c], me = mrp[c + 1];
        for (int t = mb + lane; t < me; t += 32) {
            K[off + t - mb] = mci[t];
            V[off + t - mb] = a * mv[t];
        }
        off += me - mb;
    }
    __syncwarp();
    int p2 = 32;
    while (p2 < cnt) p2 <<= 1;
    for (int t = cnt + lane; t < p2; t += 32) {
        K[t] = INT_MAX;
        V[t] = 0.0;
    }
    __syncwarp();
    for (int k = 2; k <= p2; k <<= 1)
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int t = lane; t < p2; t += 32) {
                const int u = t ^ jj;
                if (u > t) {
                    const bool up = (t & k) == 0;
                    const int a = K[t], b = K[u];
                    if ((a > b) == up) {
                        K[t] = b;
                        K[u] = a;
                        const double va = V[t];
                        V[t] = V[u];
                        V[u] = va;
                    }
                }
            }
            __syncwarp();
        }
    // segmented sums: the lane holding the first entry of a column sums it
    double r2 = 0.0;
    for (int t = lane; t < cnt; t += 32) {
        if (t == 0 || K[t - 1] != K[t]) {
            double s = 0.0;
            for (int q = t; q < cnt && K[q] == K[t]; ++q) s += V[q];
            r2 = fma(s, s, r2);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    __syncwarp();
    return r2;
}

}  // namespace sam
