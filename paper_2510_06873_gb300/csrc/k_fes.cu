// Free-energy surface from a context's bias (an analysis pass, not per step).
//
// The methods section recovers the FES by reweighting the biased ensemble,
// P_unbias(s) = <delta(s - s(R)) exp(beta V)> / <exp(beta V)> and
// F = -(1/beta) log P (Eqs. 4-5); for a well-tempered bias the deposited
// bias itself estimates it, F = -(gamma / (gamma - 1)) V + const.  Both are
// computed here in FP64 with fixed summation orders.
#include "metad_impl.cuh"

namespace metad {

namespace {

constexpr int kFesThreads = 256;

__device__ __forceinline__ double fes_block_sum(double v, double *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    __syncthreads();
    return t;
}

struct FesGrid {
    double lo[2], hi[2];
    int n[2];
};

// V at grid point b, the centre of bin b (one block per point): thread t
// sums hills t, t + blockDim, ... in order, then a fixed tree, then the grid
// patch (as the hill kernel).
__global__ void __launch_bounds__(kFesThreads) k_fes_points(Sys s, int K, FesGrid g, int M, double *V)
{
    __shared__ double sh[kFesThreads / 32];
    const int b = blockIdx.x;
    if (b >= M) return;
    const int i0 = s.ncv == 2 ? b / g.n[1] : b, i1 = s.ncv == 2 ? b % g.n[1] : 0;
    const double x0 = g.lo[0] + (i0 + 0.5) * ((g.hi[0] - g.lo[0]) / g.n[0]);
    const double x1 = s.ncv == 2 ? g.lo[1] + (i1 + 0.5) * ((g.hi[1] - g.lo[1]) / g.n[1]) : 0.0;
    const double inv2v0 = 0.5 / (s.sigma[0] * s.sigma[0]), inv2v1 = 0.5 / (s.sigma[1] * s.sigma[1]);
    double acc = 0.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double d0 = hill_diff(s, 0, x0 - s.hc[(size_t)s.hstride * k]);
        double e = d0 * d0 * inv2v0;
        if (s.ncv == 2) {
            const double d1 = hill_diff(s, 1, x1 - s.hc[(size_t)s.hstride * k + 1]);
            e += d1 * d1 * inv2v1;
        }
        acc += s.hw[k] * exp(-e);
    }
    acc = fes_block_sum(acc, sh);
    if (threadIdx.x == 0) {
        if (s.ncv == 2) {
            double gv, g0, g1;
            grid_value(s, x0, x1, gv, g0, g1);
            acc += gv;
        }
        V[b] = acc;
    }
}

// F = -fac V, shifted so the minimum is 0 (one block; fixed order).
__global__ void __launch_bounds__(kFesThreads) k_fes_finish(const double *V, int M, double fac, double *F)
{
    __shared__ double sh[kFesThreads];
    double lo = INFINITY;
    for (int b = threadIdx.x; b < M; b += blockDim.x) lo = fmin(lo, -fac * V[b]);
    sh[threadIdx.x] = lo;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = INFINITY;
        for (int t = 0; t < (int)blockDim.x; ++t) m = fmin(m, sh[t]);
        sh[0] = m;
    }
    __syncthreads();
    const double m = sh[0];
    for (int b = threadIdx.x; b < M; b += blockDim.x) F[b] = -fac * V[b] - m;
}

// Bin of a CV point on the regular grid [lo, hi), the first CV slowest; -1
// when outside.
__device__ __forceinline__ int fes_bin(const double *x, int ncv, const double *lo, const double *hi, const int *n)
{
    int idx = 0;
    for (int d = 0; d < ncv; ++d) {
        const double h = (hi[d] - lo[d]) / n[d];
        if (!(x[d] >= lo[d] && x[d] < hi[d])) return -1;
        const int b = (int)floor((x[d] - lo[d]) / h);
        if (b >= n[d]) return -1;
        idx = idx * n[d] + b;
    }
    return idx;
}

// max_t V_t (one block).
__global__ void __launch_bounds__(kFesThreads) k_fes_vmax(const double *V, long long T, double *out)
{
    __shared__ double sh[kFesThreads];
    double m = -INFINITY;
    for (long long t = threadIdx.x; t < T; t += blockDim.x) m = fmax(m, V[t]);
    sh[threadIdx.x] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = -INFINITY;
        for (int i = 0; i < (int)blockDim.x; ++i) r = fmax(r, sh[i]);
        *out = r;
    }
}

// Weight sum per bin: one thread per bin walks the samples in order
// (exp(beta (V_t - max V)) for range), so every sum has a fixed order.
__global__ void k_fes_bins(const double *S, const double *V, long long T, int ncv, FesGrid g, double beta,
                           const double *vmax, int nbins, double *acc)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const double m = *vmax;
    double a = 0.0;
    for (long long t = 0; t < T; ++t) {
        double x[2] = {S[(size_t)ncv * t], ncv == 2 ? S[(size_t)ncv * t + 1] : 0.0};
        if (fes_bin(x, ncv, g.lo, g.hi, g.n) == b) a += exp(beta * (V[t] - m));
    }
    acc[b] = a;
}

// P_b = acc_b / sum acc, F_b = -(1/beta) log P_b shifted to minimum 0; empty
// bins +inf (one block; fixed order).
__global__ void __launch_bounds__(kFesThreads) k_fes_norm(const double *acc, int nbins, double beta, double *F)
{
    __shared__ double sh[kFesThreads];
    __shared__ double tot_s, min_s;
    double t = 0.0;
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) t += acc[b];
    sh[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) r += sh[i];
        tot_s = r;
    }
    __syncthreads();
    const double tot = tot_s;
    double m = INFINITY;
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        const double f = acc[b] > 0.0 ? -log(acc[b] / tot) / beta : INFINITY;
        F[b] = f;
        m = fmin(m, f);
    }
    sh[threadIdx.x] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = INFINITY;
        for (int i = 0; i < (int)blockDim.x; ++i) r = fmin(r, sh[i]);
        min_s = r;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (acc[b] > 0.0) F[b] -= min_s;
}

}  // namespace

void launch_fes_points(const Sys &s, int K, const double *lo, const double *hi, const int *n, double *V, double *F,
                       double fac, cudaStream_t st)
{
    FesGrid g{};
    int M = 1;
    for (int d = 0; d < s.ncv; ++d) {
        g.lo[d] = lo[d];
        g.hi[d] = hi[d];
        g.n[d] = n[d];
        M *= n[d];
    }
    k_fes_points<<<M, kFesThreads, 0, st>>>(s, K, g, M, V);
    k_fes_finish<<<1, kFesThreads, 0, st>>>(V, M, fac, F);
}

void launch_fes_reweight(const double *S, const double *V, long long T, int ncv, const double *lo, const double *hi,
                         const int *n, double beta, double *scratch, double *F, cudaStream_t st)
{
    FesGrid g{};
    int nbins = 1;
    for (int d = 0; d < ncv; ++d) {
        g.lo[d] = lo[d];
        g.hi[d] = hi[d];
        g.n[d] = n[d];
        nbins *= n[d];
    }
    double *vmax = scratch, *acc = scratch + 1;
    k_fes_vmax<<<1, kFesThreads, 0, st>>>(V, T, vmax);
    k_fes_bins<<<(nbins + 127) / 128, 128, 0, st>>>(S, V, T, ncv, g, beta, vmax, nbins, acc);
    k_fes_norm<<<1, kFesThreads, 0, st>>>(acc, nbins, beta, F);
}

}  // namespace metad
