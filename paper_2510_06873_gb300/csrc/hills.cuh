// The FP64 hill sum of one system (Methods, Eqs. 2-3, a per-dimension sigma)
// and the well-tempered deposit, shared by the hill kernels and the fused
// small-system step.  Include only from files compiled with -fmad=false, so
// every instantiation rounds every operation alike.
#pragma once

#include "metad_impl.cuh"

namespace metad {

// V and dV/ds at xin into out (V, then dV/ds_d, kMaxCv of them); with
// deposit, also appends the well-tempered hill there as hill s.K.  s.D
// dimensions (at most kMaxCv).  Every block sums its chunk of the hills; the
// last block to finish adds the block partials in block order and its
// thread 0 writes out.  Returns true in every thread of that last block.
static __device__ __forceinline__ bool hill_sum(const Sys &s, Blk blk, const double *xin, double *out, int deposit)
{
    const int K = s.K, D = s.D, hs = s.hstride;
    double x[kMaxCv], inv2v[kMaxCv], g[kMaxCv];
#pragma unroll
    for (int d = 0; d < kMaxCv; ++d) {
        x[d] = d < D ? xin[d] : 0.0;
        inv2v[d] = d < D ? s.inv2v[d] : 0.0;  // 0.5 / sigma_d^2, formed on the host
        g[d] = 0.0;
    }
    double V = 0.0;
    // block b takes the contiguous chunk [b chunk, (b + 1) chunk) of the hills
    const int chunk = (K + blk.nb - 1) / blk.nb;
    const int k1 = min(K, (blk.b + 1) * chunk);
    for (int k = blk.b * chunk + threadIdx.x; k < k1; k += blockDim.x) {
        const double *c = s.hc + (size_t)hs * k;
        double dd[kMaxCv];
        double e = 0.0;
#pragma unroll
        for (int d = 0; d < kMaxCv; ++d) {
            if (d >= D) break;
            dd[d] = hill_diff(s, d, x[d] - c[d]);
            e = d == 0 ? dd[d] * dd[d] * inv2v[d] : e + dd[d] * dd[d] * inv2v[d];
        }
        const double gk = s.hw[k] * exp(-e);
        V += gk;
#pragma unroll
        for (int d = 0; d < kMaxCv; ++d) {
            if (d >= D) break;
            g[d] -= gk * dd[d] * (2.0 * inv2v[d]);
        }
    }
    // block sums in a fixed order: V, then dV/ds_d
    constexpr int kW = kBlockBias / 32;
    __shared__ double sh[kMaxCv + 1][kW];
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        V += __shfl_down_sync(0xffffffffu, V, o);
#pragma unroll
        for (int d = 0; d < kMaxCv; ++d)
            if (d < D) g[d] += __shfl_down_sync(0xffffffffu, g[d], o);
    }
    if (lane == 0) {
        sh[0][wid] = V;
#pragma unroll
        for (int d = 0; d < kMaxCv; ++d) sh[1 + d][wid] = g[d];
    }
    __syncthreads();
    double *part = s.part + 2 * (size_t)s.part_stride;
    if (threadIdx.x <= D) {  // thread q sums value q over the warps, in warp order
        const int q = threadIdx.x;
        double a = 0.0;
        for (int w = 0; w < kW; ++w) a += sh[q][w];
        part[(D + 1) * blk.b + q] = a;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(&s.ticket[2], 1u);
        am_last = (prev == (unsigned)blk.nb - 1u);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    // the last block adds the partials: thread t takes blocks t, t + blockDim,
    // ... in order, then the same fixed tree as above
    double a[kMaxCv + 1];
#pragma unroll
    for (int q = 0; q <= kMaxCv; ++q) a[q] = 0.0;
    for (int b = threadIdx.x; b < blk.nb; b += blockDim.x) {
#pragma unroll
        for (int q = 0; q <= kMaxCv; ++q)
            if (q <= D) a[q] += __ldcg(part + (D + 1) * b + q);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int q = 0; q <= kMaxCv; ++q)
            if (q <= D) a[q] += __shfl_down_sync(0xffffffffu, a[q], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q <= kMaxCv; ++q) sh[q][wid] = a[q];
    }
    __syncthreads();
    __shared__ double tot[kMaxCv + 1];
    if (threadIdx.x <= kMaxCv) {  // thread q: value q over the warps, in warp order
        const int q = threadIdx.x;
        double t = 0.0;
        if (q <= D)
            for (int w = 0; w < kW; ++w) t += sh[q][w];
        tot[q] = t;
    }
    __syncthreads();
    if (threadIdx.x != 0) return true;
    double out_v[kMaxCv + 1];
    for (int q = 0; q <= kMaxCv; ++q) out_v[q] = tot[q];
    if (s.ncv == 2 && D == 2) {
        double gv, gg0, gg1;
        grid_value(s, x[0], x[1], gv, gg0, gg1);
        out_v[0] += gv;
        out_v[1] += gg0;
        out_v[2] += gg1;
    }
    for (int q = 0; q <= kMaxCv; ++q) out[q] = out_v[q];
    s.ticket[2] = 0u;
    if (deposit) {
        const double w = s.w0 * exp(-out_v[0] / s.kbdt);
        for (int d = 0; d < hs; ++d) s.hc[(size_t)hs * K + d] = x[d];
        s.hw[K] = w;
        s.scal[kDepW] = w;
    }
    return true;
}

}  // namespace metad
