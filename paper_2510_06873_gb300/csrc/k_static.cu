// Hill-bias evaluation that allocates nothing (metad_bias_eval_noalloc).
//
// Some callers cannot allocate device memory at the point where they need
// the bias: an MD engine whose step runs on its own stream while other work
// is in flight (cudaMalloc and cudaFree can synchronise the whole device and
// stall that pipeline), code that owns a fixed memory budget or pool and
// forbids allocations outside it, and code that must not create a context
// object of this library.  For them this entry point evaluates V(s) and
// dV/ds from hill arrays they already hold on the device, using only a
// scratch array that lives in this file for the whole life of the process.
//
// The scratch is a file-scope static __device__ array: it holds one FP64
// partial triple per thread block (at most kNoAllocBlocks blocks of
// kNoAllocThreads threads, one hill per thread, so at most 131,072 hills per
// call) and the completion ticket of the last-block reduction.  Every GPU
// that loads the library holds it (about 12 KB) until the process exits.
#include <cstdint>
#include <mutex>

#include "metad.h"
#include "metad_impl.cuh"

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocBlocks = 512;
constexpr int kNoAllocMaxHills = kNoAllocThreads * kNoAllocBlocks;
constexpr int kTicketSlot = 3 * kNoAllocBlocks;      // one double slot, used as an unsigned counter
constexpr int kScratchDoubles = 3 * kNoAllocBlocks + 32;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Same sum as the context's hill kernel: each thread takes at most one hill,
// block partials go to the scratch, and the last block to finish adds them in
// block order (fixed, so repeated calls give identical bits).
__global__ void __launch_bounds__(kNoAllocThreads)
    k_bias_noalloc(const double *s, int ncv, const double *c, const double *w, int K, double inv2v0, double inv2v1,
                   double *scratch, double *out)
{
    const double x0 = s[0];
    const double x1 = ncv == 2 ? s[1] : 0.0;
    double V = 0.0, g0 = 0.0, g1 = 0.0;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K) {
        const double d0 = x0 - c[(size_t)ncv * k];
        double e = d0 * d0 * inv2v0;
        double d1 = 0.0;
        if (ncv == 2) {
            d1 = x1 - c[(size_t)ncv * k + 1];
            e += d1 * d1 * inv2v1;
        }
        const double gk = w[k] * exp(-e);
        V = gk;
        g0 = -gk * d0 * (2.0 * inv2v0);
        g1 = -gk * d1 * (2.0 * inv2v1);
    }
    __shared__ double sh[3][kNoAllocThreads / 32];
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        V += __shfl_down_sync(0xffffffffu, V, o);
        g0 += __shfl_down_sync(0xffffffffu, g0, o);
        g1 += __shfl_down_sync(0xffffffffu, g1, o);
    }
    if (lane == 0) {
        sh[0][wid] = V;
        sh[1][wid] = g0;
        sh[2][wid] = g1;
    }
    __syncthreads();
    unsigned *ticket = reinterpret_cast<unsigned *>(scratch + kTicketSlot);
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, cc = 0.0;
        for (int q = 0; q < kNoAllocThreads / 32; ++q) {
            a += sh[0][q];
            b += sh[1][q];
            cc += sh[2][q];
        }
        scratch[3 * blockIdx.x + 0] = a;
        scratch[3 * blockIdx.x + 1] = b;
        scratch[3 * blockIdx.x + 2] = cc;
        __threadfence();
        am_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last || threadIdx.x != 0) return;
    __threadfence();
    double a = 0.0, b = 0.0, cc = 0.0;
    for (int q = 0; q < (int)gridDim.x; ++q) {
        a += __ldcg(scratch + 3 * q);
        b += __ldcg(scratch + 3 * q + 1);
        cc += __ldcg(scratch + 3 * q + 2);
    }
    out[0] = a;
    out[1] = b;
    out[2] = cc;
    *ticket = 0u;
}

std::mutex g_mu;
constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on `device` (the current device).  Looked
// up once per device: in host code the array's name is only a stand-in.
// The cached address belongs to the device's primary context; a caller that
// resets the device (cudaDeviceReset) must not call this entry point again
// in the same process.
cudaError_t scratch_address(int device, double **out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" metad_status metad_bias_eval_noalloc(const double *s_dev, int32_t n_cv, const double *centers_dev,
                                                const double *heights_dev, int32_t K, const double *sigma_host,
                                                double *out_dev, int32_t device, void *stream)
{
    if (!s_dev || !out_dev || !sigma_host || (n_cv != 1 && n_cv != 2) || K < 0) return METAD_ERR_INVALID;
    if (K > 0 && (!centers_dev || !heights_dev)) return METAD_ERR_INVALID;
    if (K > kNoAllocMaxHills) return METAD_ERR_CAPACITY;  // more hills than the static scratch has blocks for
    for (int d = 0; d < n_cv; ++d)
        if (!(sigma_host[d] > 0.0)) return METAD_ERR_INVALID;
    if (device < 0 || device >= kMaxDevices) return METAD_ERR_INVALID;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return METAD_ERR_CUDA;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return METAD_ERR_CUDA;
    metad_status st = METAD_OK;
    double *scratch = nullptr;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    if (scratch_address(device, &scratch) != cudaSuccess) {
        st = METAD_ERR_CUDA;
    } else if (cudaMemsetAsync(scratch + kTicketSlot, 0, sizeof(double), cs) != cudaSuccess) {
        st = METAD_ERR_CUDA;
    } else {
        const int blocks = K > 0 ? (K + kNoAllocThreads - 1) / kNoAllocThreads : 1;
        const double inv2v0 = 0.5 / (sigma_host[0] * sigma_host[0]);
        const double inv2v1 = n_cv == 2 ? 0.5 / (sigma_host[1] * sigma_host[1]) : 0.0;
        // the launch's own status (an error left by an unrelated earlier
        // call stays with its owner)
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)blocks);
        cfg.blockDim = dim3((unsigned)kNoAllocThreads);
        cfg.stream = cs;
        if (cudaLaunchKernelEx(&cfg, k_bias_noalloc, s_dev, (int)n_cv, centers_dev, heights_dev, (int)K, inv2v0,
                               inv2v1, scratch, out_dev) != cudaSuccess)
            st = METAD_ERR_CUDA;
    }
    if (prev != device) cudaSetDevice(prev);
    return st;
}
