// Steps a6 and a9: the Gaussian-hill bias (Methods, Eqs. 2-3, a per-dimension
// sigma), its gradient, well-tempered deposition and the bias grid, all FP64.
//
//   V(s) = grid(s) + sum_k w_k exp(-sum_d (s_d - c_kd)^2 / (2 sigma_d^2))
//   w_new = w0 exp(-V(c_new) / (kB T (gamma - 1)))
//
// A periodic CV (a torsion angle) sees s_d - c_kd wrapped into [-pi, pi].
//
// The hill sum is spread over many blocks (FP64 throughput per SM is low on
// this part) and finished by the last block to arrive, which adds the
// partials in block order, so the result is independent of scheduling.
// This file is compiled with -fmad=false: no multiply-add contraction, so
// the single-system and batched kernels round every operation alike.
#include "metad_impl.cuh"

namespace metad {

namespace {

// V and dV/ds at s.bias_x into s.bias_out; with s.deposit, also appends the
// well-tempered hill there as hill s.K.
__device__ __forceinline__ void bias(const Sys &s, Blk blk)
{
    const int K = s.K;
    const double x0 = s.bias_x[0];
    const double x1 = s.ncv == 2 ? s.bias_x[1] : 0.0;
    const double inv2v0 = 0.5 / (s.sigma[0] * s.sigma[0]), inv2v1 = 0.5 / (s.sigma[1] * s.sigma[1]);
    double V = 0.0, g0 = 0.0, g1 = 0.0;
    for (int k = blk.b * blockDim.x + threadIdx.x; k < K; k += blk.nb * blockDim.x) {
        const double d0 = hill_diff(s, 0, x0 - s.hc[2 * (size_t)k]);
        double e = d0 * d0 * inv2v0;
        double d1 = 0.0;
        if (s.ncv == 2) {
            d1 = hill_diff(s, 1, x1 - s.hc[2 * (size_t)k + 1]);
            e += d1 * d1 * inv2v1;
        }
        const double gk = s.hw[k] * exp(-e);
        V += gk;
        g0 -= gk * d0 * (2.0 * inv2v0);
        g1 -= gk * d1 * (2.0 * inv2v1);
    }
    // block sums in a fixed order
    __shared__ double sh[3][kBlockBias / 32];
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        V += __shfl_down_sync(0xffffffffu, V, o);
        g0 += __shfl_down_sync(0xffffffffu, g0, o);
        g1 += __shfl_down_sync(0xffffffffu, g1, o);
    }
    if (lane == 0) { sh[0][wid] = V; sh[1][wid] = g0; sh[2][wid] = g1; }
    __syncthreads();
    double *part = s.part + 2 * (size_t)s.part_stride;
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int w = 0; w < kBlockBias / 32; ++w) { a += sh[0][w]; b += sh[1][w]; c += sh[2][w]; }
        part[3 * blk.b + 0] = a;
        part[3 * blk.b + 1] = b;
        part[3 * blk.b + 2] = c;
        __threadfence();
        unsigned prev = atomicAdd(&s.ticket[2], 1u);
        am_last = (prev == (unsigned)blk.nb - 1u);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // the last block adds the partials: thread t takes blocks t, t + blockDim,
    // ... in order, then the same fixed tree as above
    double a = 0.0, b = 0.0, c = 0.0;
    for (int q = threadIdx.x; q < blk.nb; q += blockDim.x) {
        a += __ldcg(part + 3 * q);
        b += __ldcg(part + 3 * q + 1);
        c += __ldcg(part + 3 * q + 2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if (lane == 0) { sh[0][wid] = a; sh[1][wid] = b; sh[2][wid] = c; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    a = b = c = 0.0;
    for (int w = 0; w < kBlockBias / 32; ++w) { a += sh[0][w]; b += sh[1][w]; c += sh[2][w]; }
    if (s.ncv == 2) {
        double gv, gg0, gg1;
        grid_value(s, x0, x1, gv, gg0, gg1);
        a += gv;
        b += gg0;
        c += gg1;
    }
    double *out = s.bias_out;
    out[0] = a;
    out[1] = b;
    out[2] = c;
    s.ticket[2] = 0u;
    if (s.deposit) {
        const double w = s.w0 * exp(-a / s.kbdt);
        s.hc[2 * (size_t)K] = x0;
        s.hc[2 * (size_t)K + 1] = x1;
        s.hw[K] = w;
        s.scal[kDepW] = w;
    }
}

__global__ void __launch_bounds__(kBlockBias) k_bias(Sys s) { bias(s, own_blk()); }

// Batched: every system evaluates at its own CVs (deposit 0) or deposits a
// hill there (deposit 1; only systems with s.deposit have blocks).
__global__ void __launch_bounds__(kBlockBias) kb_bias(BatchView v, int deposit)
{
    Blk k;
    Sys s = v.sys[batch_system(v, k)];
    s.bias_x = s.scal + kS0;
    s.bias_out = s.scal + (deposit ? kDepV : kV);
    s.deposit = deposit;
    bias(s, k);
}

// One thread per system: s1, s2, V and the error word, for one copy to the host.
__global__ void kb_collect(const Sys *sys, int nsys, double *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsys) return;
    const Sys &s = sys[k];
    out[4 * k + 0] = s.scal[kS0];
    out[4 * k + 1] = s.scal[kS1];
    out[4 * k + 2] = s.scal[kV];
    out[4 * k + 3] = (double)*s.err;
}

// One thread per grid node: exact sums over hills [0, K).
__global__ void k_grid_fold(Sys s, int K)
{
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= s.gn[0] * s.gn[1]) return;
    const int a = node / s.gn[1], b = node % s.gn[1];
    const double x = s.glo[0] + a * s.gh[0], y = s.glo[1] + b * s.gh[1];
    const double v0 = s.sigma[0] * s.sigma[0], v1 = s.sigma[1] * s.sigma[1];
    double f = 0.0, fx = 0.0, fy = 0.0, fxy = 0.0;
    for (int k = 0; k < K; ++k) {
        const double dx = x - s.hc[2 * (size_t)k], dy = y - s.hc[2 * (size_t)k + 1];
        const double g = s.hw[k] * exp(-(dx * dx / (2.0 * v0) + dy * dy / (2.0 * v1)));
        f += g;
        fx -= g * dx / v0;
        fy -= g * dy / v1;
        fxy += g * dx * dy / (v0 * v1);
    }
    double *nd = s.grid + (size_t)node * 4;
    nd[0] += f;
    nd[1] += fx;
    nd[2] += fy;
    nd[3] += fxy;
}

}  // namespace

int bias_blocks(int K)
{
    int b = (K + kBlockBias - 1) / kBlockBias;
    if (b < 1) b = 1;
    if (b > kMaxBiasBlocks) b = kMaxBiasBlocks;
    return b;
}

void launch_bias(const Sys &s, int K, const double *x_dev, double *out_dev, int deposit, cudaStream_t st)
{
    Sys t = s;
    t.K = K;
    t.bias_x = x_dev;
    t.bias_out = out_dev;
    t.deposit = deposit;
    k_bias<<<bias_blocks(K), kBlockBias, 0, st>>>(t);
}

void launch_batch_bias(const BatchView &v, int total, int deposit, cudaStream_t st)
{
    if (total > 0) kb_bias<<<total, kBlockBias, 0, st>>>(v, deposit);
}

void launch_batch_collect(const BatchView &v, double *out, cudaStream_t st)
{
    kb_collect<<<(v.nsys + 127) / 128, 128, 0, st>>>(v.sys, v.nsys, out);
}

void launch_grid_fold(const Sys &s, int K, cudaStream_t st)
{
    const int nodes = s.gn[0] * s.gn[1];
    k_grid_fold<<<(nodes + 127) / 128, 128, 0, st>>>(s, K);
}

}  // namespace metad
