// Device helpers shared by the sparse and spectral kernel translation units:
// vector loads/stores on the node-major, time-fastest layout X[row * N + n],
// the (row, column chunk) walk of the row kernels, and the deterministic
// per-column reductions with a last-block finish that carry the scalars of
// the batched Krylov solvers (one independent solve per column, or per pair
// of columns holding the real and imaginary parts of one complex unknown).
#pragma once

#include <cmath>

#include "kernels.h"

namespace ptp {

// Launch shape of the row kernels: N / vec threads per row, as many rows per
// block as the host thread's row-block size allows, one resident wave.
struct Launch {
    int grid, block;
};
Launch row_launch(int rows, int N, int vec, const void* kernel);

template <typename... KArgs, typename... Args>
void launch_rows(void (*kernel)(KArgs...), int rows, int N, int vec, cudaStream_t s, Args&&... args) {
    const Launch l = row_launch(rows, N, vec, (const void*)kernel);
    launch_k(kernel, dim3(l.grid), dim3(l.block), s, std::forward<Args>(args)...);
}

namespace {

constexpr int kMaxBlock = 512;

__device__ __forceinline__ bool skip_now(const Skip& s) {
    return (s.done && *(volatile const int*)s.done) || (s.pdone && *(volatile const int*)s.pdone);
}

template <typename T, int VEC>
__device__ __forceinline__ void ldg_vec(const T* p, T (&o)[VEC]) {
    if constexpr (sizeof(T) == 4 && VEC == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    } else if constexpr (sizeof(T) == 4 && VEC == 2) {
        const float2 a = __ldg(reinterpret_cast<const float2*>(p));
        o[0] = a.x; o[1] = a.y;
    } else if constexpr (sizeof(T) == 8 && VEC == 2) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p));
        o[0] = a.x; o[1] = a.y;
    } else {
#pragma unroll
        for (int v = 0; v < VEC; ++v) o[v] = __ldg(p + v);
    }
}

template <typename T, int VEC>
__device__ __forceinline__ void ld_vec(const T* p, T (&o)[VEC]) {  // coherent load
    if constexpr (sizeof(T) == 4 && VEC == 4) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    } else if constexpr (sizeof(T) == 4 && VEC == 2) {
        const float2 a = *reinterpret_cast<const float2*>(p);
        o[0] = a.x; o[1] = a.y;
    } else if constexpr (sizeof(T) == 8 && VEC == 2) {
        const double2 a = *reinterpret_cast<const double2*>(p);
        o[0] = a.x; o[1] = a.y;
    } else {
#pragma unroll
        for (int v = 0; v < VEC; ++v) o[v] = p[v];
    }
}

template <typename T, int VEC>
__device__ __forceinline__ void st_vec(T* p, const T (&o)[VEC]) {
    if constexpr (sizeof(T) == 4 && VEC == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else if constexpr (sizeof(T) == 4 && VEC == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
    } else if constexpr (sizeof(T) == 8 && VEC == 2) {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    } else {
#pragma unroll
        for (int v = 0; v < VEC; ++v) p[v] = o[v];
    }
}

// grid-stride walk over (row, chunk); NC = N / VEC, rpb = rows per block
#define PTP_ROW_LOOP(rows, NC, rpb)                                                    \
    const int chunk_ = threadIdx.x % (NC);                                             \
    const int rsub_ = threadIdx.x / (NC);                                              \
    const int col0 = chunk_ * VEC;                                                     \
    for (int rg_ = blockIdx.x; rg_ * (rpb) < (rows); rg_ += gridDim.x)                  \
        for (int row = rg_ * (rpb) + rsub_; row < (rows) && rsub_ < (rpb); row = (rows))

// the same walk over the blocks of a virtual grid g
#define PTP_ROW_LOOP_G(rows, NC, rpb, g)                                               \
    const int chunk_ = threadIdx.x % (NC);                                             \
    const int rsub_ = threadIdx.x / (NC);                                              \
    const int col0 = chunk_ * VEC;                                                     \
    for (int rg_ = (g).bx; rg_ * (rpb) < (rows); rg_ += (g).gx)                        \
        for (int row = rg_ * (rpb) + rsub_; row < (rows) && rsub_ < (rpb); row = (rows))

// ---------------------------------------------------------------------------
// per-column reductions with a last-block finish
// ---------------------------------------------------------------------------

// Real finishes act on every column; complex finishes (FIN_C_*) act on column
// pairs (2k, 2k+1) = (re, im) of complex unknown k, with bilinear (unconjugated)
// products for the conjugate-orthogonal CG recurrence and |.|^2 for norms.
enum Fin {
    FIN_ALPHA = 0, FIN_UPDATE_JACOBI = 1, FIN_UPDATE_RR = 2, FIN_RZ_FIRST = 3, FIN_RZ_NEXT = 4,
    FIN_C_ALPHA = 10,     // s = p^T A p (re, im):      alpha = rho / s
    FIN_C_UPDATE = 11,    // s = (|r_re|^2, |r_im|^2):   rr = sum, convergence test
    FIN_C_RZ_FIRST = 12,  // s = (r^T z, |r|^2 parts):   rho = r^T z, bb = rr = |r|^2
    FIN_C_RZ_NEXT = 13,   // s = r^T z:                  beta = s / rho, rho = s
};


// num / den for PCG scalars, evaluated in double; 0 when the column has
// no (or a non-finite) search direction, so a column whose right-hand side
// is zero or underflows stays untouched instead of propagating NaN.
template <typename T>
__device__ __forceinline__ T safe_ratio(T num, T den) {
    if (!(num > T(0) && den > T(0))) return T(0);
    const double r = (double)num / (double)den;
    return isfinite(r) && r < 1e30 ? (T)r : T(0);
}

// complex num / den; 0 when den vanishes or the quotient is not finite
__device__ __forceinline__ double2 safe_cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    if (!(d > 0.0) || !isfinite(d)) return make_double2(0.0, 0.0);
    const double re = (a.x * b.x + a.y * b.y) / d, im = (a.y * b.x - a.x * b.y) / d;
    if (!isfinite(re) || !isfinite(im)) return make_double2(0.0, 0.0);
    return make_double2(re, im);
}

// Blocks are grouped by kGroup; the last block of each group to finish sums
// its group's partials, and the last group finisher sums the group results
// and applies FIN to every column (or column pair).  Both sums run in a fixed
// order, so the result does not depend on block scheduling.  Counters: [0] for
// the groups, [1 + g] for group g; each is reset by the block that consumed it.
constexpr int kGroup = 32;

template <typename T, int VEC, int NQ, int FIN>
__device__ void col_reduce_finish(T (&acc)[NQ][VEC], int N, int NC, int rpb, const ColRed<T>& cr, const VGrid& vg) {
    __shared__ T sm[NQ * kMaxBlock * VEC];
    __shared__ int stage;
    __shared__ int all_conv;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int v = 0; v < VEC; ++v) sm[(q * blockDim.x + threadIdx.x) * VEC + v] = acc[q][v];
    __syncthreads();
    const int G = vg.gx;
    const int QN = NQ * N;
    for (int e = threadIdx.x; e < QN; e += blockDim.x) {
        const int q = e / N, col = e - q * N;
        const int chunk = col / VEC, v = col - chunk * VEC;
        T s = T(0);
        for (int r = 0; r < rpb; ++r) s += sm[(q * blockDim.x + r * NC + chunk) * VEC + v];
        cr.partials[(size_t)vg.bx * QN + e] = s;
    }
    __threadfence();
    __syncthreads();
    const int ng = (G + kGroup - 1) / kGroup;
    const int g = vg.bx / kGroup;
    const int b0 = g * kGroup;
    const int gsz = min(kGroup, G - b0);
    T* part2 = cr.partials + (size_t)G * QN;
    if (threadIdx.x == 0) {
        const unsigned ticket = atomicAdd(cr.counter + 1 + g, 1u);
        stage = ticket == (unsigned)(gsz - 1) ? 1 : 0;
        all_conv = 1;
    }
    __syncthreads();
    if (!stage) return;
    for (int e = threadIdx.x; e < QN; e += blockDim.x) {
        T a = T(0);
#pragma unroll 8
        for (int b = 0; b < gsz; ++b) a += __ldcg(cr.partials + (size_t)(b0 + b) * QN + e);
        part2[(size_t)g * QN + e] = a;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        cr.counter[1 + g] = 0u;
        const unsigned ticket = atomicAdd(cr.counter, 1u);
        stage = ticket == (unsigned)(ng - 1) ? 2 : 0;
    }
    __syncthreads();
    if (stage != 2) return;
    constexpr bool CPLX = FIN >= FIN_C_ALPHA;
    constexpr int CW = CPLX ? 2 : 1;
    for (int u = threadIdx.x; u < N / CW; u += blockDim.x) {
        const int col = u * CW;
        T s[NQ][CW];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int w = 0; w < CW; ++w) {
                T a = T(0);
                for (int b = 0; b < ng; ++b) a += __ldcg(part2 + (size_t)b * QN + q * N + col + w);
                s[q][w] = a;
            }
        T* c = cr.col;
        if constexpr (FIN == FIN_ALPHA) {
            c[S_ALPHA * N + col] = safe_ratio<T>(c[S_RHO * N + col], s[0][0]);
        } else if constexpr (FIN == FIN_UPDATE_JACOBI) {  // s = (rz, rr)
            c[S_BETA * N + col] = safe_ratio<T>(s[0][0], c[S_RHO * N + col]);
            c[S_RHO * N + col] = s[0][0];
            c[S_RR * N + col] = s[1][0];
            if (!(s[1][0] <= cr.tol2 * c[S_BB * N + col])) all_conv = 0;
        } else if constexpr (FIN == FIN_UPDATE_RR) {
            c[S_RR * N + col] = s[0][0];
            if (!(s[0][0] <= cr.tol2 * c[S_BB * N + col])) all_conv = 0;
        } else if constexpr (FIN == FIN_RZ_FIRST) {  // s = (rz, rr)
            c[S_RHO * N + col] = s[0][0];
            c[S_BB * N + col] = s[1][0];
            c[S_RR * N + col] = s[1][0];
        } else if constexpr (FIN == FIN_RZ_NEXT) {
            c[S_BETA * N + col] = safe_ratio<T>(s[0][0], c[S_RHO * N + col]);
            c[S_RHO * N + col] = s[0][0];
        } else if constexpr (CPLX) {
            static_assert(sizeof(T) == 8, "complex finishes are double");
            const double2 rho = make_double2(c[S_RHO * N + col], c[S_RHO * N + col + 1]);
            if constexpr (FIN == FIN_C_ALPHA) {
                const double2 a = safe_cdiv(rho, make_double2(s[0][0], s[0][1]));
                c[S_ALPHA * N + col] = a.x;
                c[S_ALPHA * N + col + 1] = a.y;
            } else if constexpr (FIN == FIN_C_UPDATE) {
                const T rr = s[0][0] + s[0][1];
                c[S_RR * N + col] = rr;
                if (!(rr <= cr.tol2 * c[S_BB * N + col])) all_conv = 0;
            } else if constexpr (FIN == FIN_C_RZ_FIRST) {
                const T rr = s[1][0] + s[1][1];
                c[S_RHO * N + col] = s[0][0];
                c[S_RHO * N + col + 1] = s[0][1];
                c[S_BB * N + col] = rr;
                c[S_RR * N + col] = rr;
            } else if constexpr (FIN == FIN_C_RZ_NEXT) {
                const double2 b = safe_cdiv(make_double2(s[0][0], s[0][1]), rho);
                c[S_BETA * N + col] = b.x;
                c[S_BETA * N + col + 1] = b.y;
                c[S_RHO * N + col] = s[0][0];
                c[S_RHO * N + col + 1] = s[0][1];
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if constexpr (FIN == FIN_UPDATE_JACOBI || FIN == FIN_UPDATE_RR || FIN == FIN_C_UPDATE)
            if (cr.pdone && all_conv) *cr.pdone = 1;
        cr.counter[0] = 0u;
    }
}

}  // namespace
}  // namespace ptp
