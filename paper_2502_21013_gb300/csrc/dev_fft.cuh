// Radix-2 FFT helpers in shared memory, double complex, shared by the DFT
// in time (k_dft.cu) and the discrete sine transforms of the exact coarsest
// spatial solve (k_poisson.cu).
#pragma once

#include <cuda_runtime.h>

namespace ptp {
namespace {

__device__ __forceinline__ int bit_reverse(int t, int logN) {
    return logN == 0 ? 0 : (int)(__brev((unsigned)t) >> (32 - logN));
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place iterative radix-2 FFT (decimation in time) of nb rows of length N
// held in shared memory in bit-reversed order; W[j] = e^{-2 pi i j / N}, the
// inverse uses conj(W).
template <bool INV>
__device__ void fft_stages(double2* sh, int nb, int N, const double2* __restrict__ W) {
    const int half = N / 2;
    for (int len = 2; len <= N; len <<= 1) {
        const int h = len >> 1, stride = N / len;
        for (int b = threadIdx.x; b < nb * half; b += blockDim.x) {
            const int j = b / half, bb = b - j * half;
            const int grp = bb / h, pos = bb - grp * h;
            const int i0 = j * N + grp * len + pos, i1 = i0 + h;
            double2 w = __ldg(W + pos * stride);
            if (INV) w.y = -w.y;
            const double2 u = sh[i0];
            const double2 t = cmul(w, sh[i1]);
            sh[i0] = make_double2(u.x + t.x, u.y + t.y);
            sh[i1] = make_double2(u.x - t.x, u.y - t.y);
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace ptp
