// Measurement probes.  The double kernels of the path (K1, the coarsest
// level, the DFT solve) are bound by the FP64 FMA rate, which the measured
// peaks of the device (a copy bandwidth and a bf16 GEMM rate) do not give,
// so the FMA rates are measured here: independent FMA chains on every SM,
// timed with CUDA events.  The reciprocal probe exposes the Newton
// reciprocal of the K1 kernels so that it can be tested against CUDA's own
// double division.
#include <algorithm>
#include <cmath>

#include "dev_math.cuh"
#include "kernels.h"

namespace ptp {
namespace {

constexpr int kProbeBlock = 256;

// kChains independent FMA chains per thread
template <typename T, int kChains>
__global__ void __launch_bounds__(kProbeBlock) k_fma_probe(int iters, T a, T b, T* out) {
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

__global__ void k_recip_probe(size_t n, const double* __restrict__ d, double* __restrict__ out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = recip_newton(d[i]);
}

struct ProbeError {
    int code;
};

#define PROBE_CUDA(call)                              \
    do {                                              \
        if ((call) != cudaSuccess) throw ProbeError{PTP_ECUDA}; \
    } while (0)

template <typename T, int kChains>
double fma_rate_chains(int device) {
    PROBE_CUDA(cudaSetDevice(device));
    int sms = 0, per_sm = 0;
    PROBE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    PROBE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<T, kChains>, kProbeBlock, 0));
    const int grid = sms * std::max(1, per_sm);
    const size_t threads = (size_t)grid * kProbeBlock;
    T* out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double best = 0.0;
    try {
        PROBE_CUDA(cudaMalloc(&out, threads * sizeof(T)));
        PROBE_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        PROBE_CUDA(cudaEventCreate(&e0));
        PROBE_CUDA(cudaEventCreate(&e1));
        const T a = T(0.999999), b = T(1e-6);   // x -> b / (1 - a) = 1: no overflow
        // size the loop from a short run so that one timed launch takes about 40 ms
        int iters = 256;
        k_fma_probe<T, kChains><<<grid, kProbeBlock, 0, s>>>(iters, a, b, out);
        PROBE_CUDA(cudaGetLastError());
        PROBE_CUDA(cudaEventRecord(e0, s));
        k_fma_probe<T, kChains><<<grid, kProbeBlock, 0, s>>>(iters, a, b, out);
        PROBE_CUDA(cudaEventRecord(e1, s));
        PROBE_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        PROBE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        const double scale = 40.0 / std::max(1e-3, (double)ms);
        iters = (int)std::min(1e7, std::max(256.0, iters * scale));
        for (int rep = 0; rep < 3; ++rep) {
            PROBE_CUDA(cudaEventRecord(e0, s));
            k_fma_probe<T, kChains><<<grid, kProbeBlock, 0, s>>>(iters, a, b, out);
            PROBE_CUDA(cudaEventRecord(e1, s));
            PROBE_CUDA(cudaEventSynchronize(e1));
            PROBE_CUDA(cudaGetLastError());
            PROBE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            const double flops = 2.0 * kChains * (double)iters * (double)threads;
            best = std::max(best, flops / (ms * 1e-3) / 1e12);
        }
    } catch (const ProbeError&) {
        best = -1.0;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    return best;
}

// the best rate over 8 and 16 chains per thread (latency hidden either way
// when the pipe is the limit; the better of the two is the measured peak)
template <typename T>
double fma_rate(int device) {
    return std::max(fma_rate_chains<T, 8>(device), fma_rate_chains<T, 16>(device));
}

}  // namespace
}  // namespace ptp

extern "C" {

int ptp_probe_fma(int device, int fp64, double* tflops) {
    if (!tflops || device < 0) return PTP_EINVAL;
    const double r = fp64 ? ptp::fma_rate<double>(device) : ptp::fma_rate<float>(device);
    if (!(r > 0.0)) return PTP_ECUDA;
    *tflops = r;
    return PTP_OK;
}

int ptp_probe_recip_dev(int device, const double* d, double* out, int64_t n, void* stream) {
    if (n < 0 || (n > 0 && (!d || !out)) || device < 0 || (const void*)d == (const void*)out) return PTP_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return PTP_ECUDA;
    if (n == 0) return PTP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    ptp::k_recip_probe<<<grid, 256, 0, s>>>((size_t)n, d, out);
    if (cudaGetLastError() != cudaSuccess) return PTP_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PTP_ECUDA;
    return PTP_OK;
}

}  // extern "C"
