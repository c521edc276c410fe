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
#include "hills.cuh"

namespace metad {

namespace {

// V and dV/ds at s.bias_x into s.bias_out; with s.deposit, also appends the
// well-tempered hill there as hill s.K.
__device__ __forceinline__ void bias(const Sys &s, Blk blk) { hill_sum(s, blk, s.bias_x, s.bias_out, s.deposit); }

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

// One thread per system: s1, s2 (0 with one per-atom CV), V and the error
// word, for one copy to the host.
__global__ void kb_collect(const Sys *sys, int nsys, double *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsys) return;
    const Sys &s = sys[k];
    out[4 * k + 0] = s.scal[kS0];
    out[4 * k + 1] = s.ncv == 2 ? s.scal[kS1] : 0.0;
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
        const double dx = x - s.hc[(size_t)s.hstride * k], dy = y - s.hc[(size_t)s.hstride * k + 1];
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

// About kHillsPerBlock hills per block (one per thread).  Fewer hills per
// block spread one system's FP64 work over more SMs (a lone 10,000-hill
// walker's step: 22.5 -> 18.4 us at 64 per block) but halve the throughput
// of batched walkers, whose blocks fill the GPU anyway; a system's grid must
// not depend on whether it is batched, or the two would round differently.
int bias_blocks(int K)
{
    int b = (K + kHillsPerBlock - 1) / kHillsPerBlock;
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


// The kernels of this file whose only argument is the system descriptor
// (a captured step's nodes of these can take new I/O buffers in place).
bool sys_kernel_bias(const void *func)
{
    static const void *const kernels[] = {
        (const void *)k_bias,
    };
    for (const void *k : kernels)
        if (k == func) return true;
    return false;
}

}  // namespace metad
