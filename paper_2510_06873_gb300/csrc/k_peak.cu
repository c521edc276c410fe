// FP32 throughput probe: the denominator of the FP32 roofline fraction.
//
// Every thread runs kChains independent multiply-add chains, so each
// scheduler always has an independent FMA to issue; the grid fills every SM
// with 2048 threads.  Work = 2 flop x kChains x iters per thread.  The
// chains' inputs come from memory and their results are stored only under a
// condition the host never meets, so nothing is folded away.
#include <cuda_runtime.h>
#include <stdint.h>

#include "metad.h"
#include "metad_impl.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__global__ void __launch_bounds__(kThreads) k_fma_chains(const float *in, float *out, int iters, float guard)
{
    float a[kChains];
    const float x = in[0], y = in[1];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = in[2 + c] + (float)threadIdx.x * 1e-7f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], x, y);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == guard) out[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" metad_status metad_probe_fp32_peak(int32_t device, int32_t iters, int32_t repeats, double *tflops_host)
{
    if (!tflops_host || iters < 1 || repeats < 1) return METAD_ERR_INVALID;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return METAD_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return METAD_ERR_CUDA;
    metad_status st = METAD_OK;
    int sms = 0;
    float *buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = nullptr;
    const float init[2 + kChains] = {0.999999f, 1e-6f, 1.0f, 1.1f, 1.2f, 1.3f, 1.4f, 1.5f, 1.6f, 1.7f};
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = METAD_ERR_CUDA;
    } else {
        const int blocks = sms * kBlocksPerSm;
        if (cudaMalloc(&buf, sizeof(float) * ((size_t)blocks * kThreads + 16)) != cudaSuccess ||
            cudaMemcpyAsync(buf, init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess) {
            st = METAD_ERR_CUDA;
        } else {
            // one untimed launch, then `repeats` launches between two events
            k_fma_chains<<<blocks, kThreads, 0, s>>>(buf, buf + 16, iters, -1.0f);
            cudaEventRecord(e0, s);
            for (int r = 0; r < repeats; ++r) k_fma_chains<<<blocks, kThreads, 0, s>>>(buf, buf + 16, iters, -1.0f);
            cudaEventRecord(e1, s);
            float ms = 0.0f;
            if (cudaStreamSynchronize(s) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
                ms <= 0.0f) {
                st = METAD_ERR_CUDA;
            } else {
                const double flop = 2.0 * kChains * (double)iters * kThreads * blocks * repeats;
                *tflops_host = flop / (ms * 1e-3) / 1e12;
            }
        }
    }
    if (buf) cudaFree(buf);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaSetDevice(prev);
    return st;
}

// Accuracy probe of the kernels' FP32 reciprocal square root and reciprocal
// against CUDA's correctly rounded intrinsics, on the caller's inputs.
namespace {

__global__ void k_recip_probe(const float *v, float *out, int64_t n, int which)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = v[i];
    float y;
    switch (which) {
    case 0: y = metad::rsqrt_newton(x); break;
    case 1: y = __frsqrt_rn(x); break;
    case 2: y = metad::recip_newton(x); break;
    default: y = __frcp_rn(x); break;
    }
    out[i] = y;
}

}  // namespace

extern "C" metad_status metad_probe_recip(const float *v_dev, float *out_dev, int64_t n, int32_t which, void *stream)
{
    if (!v_dev || !out_dev || n < 0 || which < 0 || which > 3) return METAD_ERR_INVALID;
    if (n == 0) return METAD_OK;
    const int threads = 256;
    k_recip_probe<<<(unsigned)((n + threads - 1) / threads), threads, 0, (cudaStream_t)stream>>>(v_dev, out_dev, n, which);
    return cudaGetLastError() == cudaSuccess ? METAD_OK : METAD_ERR_CUDA;
}
