// Kernel bodies shared by their own kernels and by the fused program of the
// coarse time levels (k_stencil.cu): the coarsest dense apply and the time
// prolongation (k_sparse.cu), the last PCG update (k_krylov.cu) and the sine
// transforms of the coarsest time level (k_poisson.cu).  Each body works on
// one virtual grid (VGrid) of blocks.
#pragma once

#include <algorithm>

#include "dev_async.cuh"
#include "dev_fft.cuh"
#include "dev_util.cuh"

namespace ptp {
namespace {

constexpr int kDstThreads = 256;

// Loads transforms t1 = 2p and t2 = 2p + 1 (of ntr) as the odd extension, in
// bit-reversed order, into sh (2m complex values).
template <typename TI>
__device__ __forceinline__ void dst_load(double2* sh, int p, int ntr, int n, int logM2, const TI* __restrict__ in,
                                         long in_tr, long in_el) {
    const int m = n + 1, M2 = 2 * m;
    const int t1 = 2 * p, t2 = 2 * p + 1;
    for (int idx = threadIdx.x; idx < M2; idx += blockDim.x) {
        double2 v = make_double2(0.0, 0.0);
        int j = 0;
        double sgn = 1.0;
        if (idx >= 1 && idx <= n) {
            j = idx - 1;
        } else if (idx > m) {
            j = M2 - idx - 1;
            sgn = -1.0;
        } else {
            j = -1;
        }
        if (j >= 0) {
            v.x = sgn * (double)in[(long)t1 * in_tr + (long)j * in_el];
            if (t2 < ntr) v.y = sgn * (double)in[(long)t2 * in_tr + (long)j * in_el];
        }
        sh[bit_reverse(idx, logM2)] = v;
    }
}

// out = S in along each transform (two per block pass); with TWICE the
// transform is scaled elementwise by scale[t][k] and transformed again
// (S (scale * S in)), in one pass over shared memory.
template <typename TI, typename TO, bool TWICE>
__device__ __forceinline__ void dst_body(const DstArgs& p, const VGrid& g) {
    pdl_enter();
    if (skip_now(p.sk)) return;
    const int ntr = p.ntr, n = p.n, logM2 = p.logM2;
    const TI* __restrict__ in = static_cast<const TI*>(p.in);
    TO* __restrict__ out = static_cast<TO*>(p.out);
    const double* __restrict__ scale = p.scale;
    const double2* __restrict__ Wt = p.Wt;
    extern __shared__ double2 dsm[];
    const int m = n + 1, M2 = 2 * m;
    double2* sh = dsm;
    double2* sh2 = dsm + M2;
    for (int q = g.bx; 2 * q < ntr; q += g.gx) {
        const int t1 = 2 * q, t2 = 2 * q + 1;
        dst_load<TI>(sh, q, ntr, n, logM2, in, p.in_tr, p.in_el);
        __syncthreads();
        fft_stages<false>(sh, 1, M2, Wt);
        if constexpr (TWICE) {
            // S z_k of both transforms, scaled, as the new odd extension
            for (int idx = threadIdx.x; idx < M2; idx += blockDim.x) {
                double2 v = make_double2(0.0, 0.0);
                int k = -1;
                double sgn = 1.0;
                if (idx >= 1 && idx <= n) {
                    k = idx;
                } else if (idx > m) {
                    k = M2 - idx;
                    sgn = -1.0;
                }
                if (k > 0) {
                    const double2 Y = sh[k];
                    v.x = sgn * (-0.5 * Y.y) * __ldg(scale + (long)t1 * n + (k - 1));
                    if (t2 < ntr) v.y = sgn * (0.5 * Y.x) * __ldg(scale + (long)t2 * n + (k - 1));
                }
                sh2[bit_reverse(idx, logM2)] = v;
            }
            __syncthreads();
            fft_stages<false>(sh2, 1, M2, Wt);
        }
        const double2* res = TWICE ? sh2 : sh;
        for (int k = 1 + threadIdx.x; k <= n; k += blockDim.x) {
            const double2 Y = res[k];
            out[(long)t1 * p.out_tr + (long)(k - 1) * p.out_el] = (TO)(-0.5 * Y.y);
            if (t2 < ntr) out[(long)t2 * p.out_tr + (long)(k - 1) * p.out_el] = (TO)(0.5 * Y.x);
        }
        __syncthreads();
    }
}


template <typename T, int VEC>
__device__ __forceinline__ void pcg_xupdate_body(const XUpdateArgs<T>& a, const VGrid& g) {
    pdl_enter();
    if (skip_now(a.sk)) return;
    const int N = a.N, NC = N / VEC, rpb = blockDim.x / NC;
    const T xscale = a.xscale;
    const T* p = a.p;
    const T* alpha = a.alpha;
    T* x = a.x;
    PTP_ROW_LOOP_G(a.rows, NC, rpb, g) {
        const size_t o = (size_t)row * N + col0;
        T pv[VEC], xv[VEC];
        ld_vec<T, VEC>(p + o, pv);   // a plain load: p may be written earlier in the same fused program
        if (a.assign) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) xv[v] = T(0);
        } else {
            ld_vec<T, VEC>(x + o, xv);
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) xv[v] += xscale * alpha[col0 + v] * pv[v];
        st_vec<T, VEC>(x + o, xv);
    }
}


// Y = Ainv B on the coarsest spatial level (dense, row-major Ainv, n <= 600).
// A block computes an 8 x 32 tile of Y (one row and column per thread) from
// the 8 rows of Ainv and the 32 columns of B it needs, copied to shared
// memory kc values of k at a time (kc = n when it fits, so one chunk in
// float).  Every copy of a chunk is in flight at once (cp.async, zero-filled
// outside the matrices).  The product is small and bound by latency: small
// tiles give many blocks, and two partial sums per thread halve the chain of
// dependent FMAs.
constexpr int kDT = 32;   // columns of a tile
constexpr int kDR = 8;    // rows of a tile
constexpr size_t kDenseSmem = 96 * 1024;
template <typename T>
int dense_chunk(int n) {   // k values per chunk
    const int fit = (int)((kDenseSmem / sizeof(T) - kDR) / (kDR + kDT));
    return std::max(1, std::min(n, fit));
}
template <typename T>
size_t dense_smem(int kc) { return (size_t)(kDR * (kc + 1) + kc * kDT) * sizeof(T); }

template <typename T>
__device__ __forceinline__ void dense_apply_body(const DenseArgs<T>& p, const VGrid& g) {
    pdl_enter();
    if (skip_now(p.sk)) return;
    const int n = p.n, N = p.N, kc = p.kc;
    const T* __restrict__ A = p.A;
    const T* __restrict__ B = p.B;
    T* __restrict__ Y = p.Y;
    extern __shared__ __align__(16) unsigned char dense_smem_raw[];
    T* As = reinterpret_cast<T*>(dense_smem_raw);   // [8][kc + 1]
    T* Bs = As + kDR * (kc + 1);                    // [kc][32]
    const int tx = threadIdx.x % kDT, ty = threadIdx.x / kDT;   // column, row of the tile
    const int c0 = g.bx * kDT, i0 = g.by * kDR;
    T acc0 = T(0), acc1 = T(0);
    for (int k0 = 0; k0 < n; k0 += kc) {
        const int kk = min(kc, n - k0);
        for (int e = threadIdx.x; e < kDR * kc; e += blockDim.x) {
            const int r = e / kc, q = e - r * kc;
            const bool ok = i0 + r < n && q < kk;
            cp_async<sizeof(T)>(As + r * (kc + 1) + q, ok ? A + (size_t)(i0 + r) * n + (k0 + q) : A, ok);
        }
        for (int e = threadIdx.x; e < kc * kDT; e += blockDim.x) {
            const int r = e / kDT, q = e - r * kDT;
            const bool ok = r < kk && c0 + q < N;
            cp_async<sizeof(T)>(Bs + r * kDT + q, ok ? B + (size_t)(k0 + r) * N + (c0 + q) : B, ok);
        }
        cp_commit();
        cp_wait<0>();
        __syncthreads();
        const T* ar = As + ty * (kc + 1);
        int k = 0;
#pragma unroll 4
        for (; k + 1 < kk; k += 2) {
            acc0 += ar[k] * Bs[k * kDT + tx];
            acc1 += ar[k + 1] * Bs[(k + 1) * kDT + tx];
        }
        if (k < kk) acc0 += ar[k] * Bs[k * kDT + tx];
        __syncthreads();
    }
    const int c = c0 + tx, i = i0 + ty;
    if (c < N && i < n) Y[(size_t)i * N + c] = acc0 + acc1;
}

template <typename T>
__device__ __forceinline__ void time_prolong_add_body(const ProlongArgs<T>& p, const VGrid& g) {
    pdl_enter();
    if (skip_now(p.sk)) return;
    const int Nc = p.Nc;
    const size_t total = (size_t)p.rows * Nc;
    for (size_t q = (size_t)g.bx * blockDim.x + threadIdx.x; q < total; q += (size_t)g.gx * blockDim.x) {
        const size_t i = q / Nc, m = q - i * Nc;
        const T v = p.xc[q];
        T* xr = p.x + i * (2 * (size_t)Nc) + 2 * m;
        xr[0] += v;
        xr[1] += v;
    }
}

}  // namespace
}  // namespace ptp
