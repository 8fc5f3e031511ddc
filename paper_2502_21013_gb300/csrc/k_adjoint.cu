// Adjoint of the period-averaged eddy-current loss (double precision).
//
//   J = (1/N) sum_n sum_{e in iron} sigma_e (d_tau u^n)_e^T M1_e (d_tau u^n)_e
//
// At the solution U of Problem 1 the implicit-function theorem gives
// dJ/dp = dJ/dp|_U - lambda^T dG/dp with G = A(U) - F and the adjoint system
// (dA/dU)^T lambda = dJ/dU, i.e.
//   M (lambda^n - lambda^{n+1}) / tau + DK(u^n) lambda^n = g^n,  lambda^{N+1} = lambda^1,
// backward in time (proof of Theorem 2 for the operator A; its Jacobian has
// blocks M/tau + DK(u^n) and -M/tau).  Stored with the time columns reversed
// (column m holds step N - m), this is the forward periodic operator again,
// so the fixed point of eq. (iter1) with K_hat = L and multigrid in time
// solve it unchanged; only the element flux differs: DK's element block is
// |T| grad(phi)^T [nu I + 2 nu'(s^2) g g^T] grad(phi), with nu' = dnu/d(s^2).
#include <cmath>

#include "kernels.h"

namespace ptp {
namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums NQ per-thread values over the grid: block partials, then the last block
// adds them in a fixed order and writes out[0..NQ).
template <int NQ>
__device__ void grid_sum(double (&v)[NQ], double* partials, unsigned* counter, double* out) {
    __shared__ double sm[NQ][kBlock / 32];
    __shared__ bool last;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double s = warp_sum(v[q]);
        if ((threadIdx.x & 31) == 0) sm[q][threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[q][w];
            partials[(size_t)blockIdx.x * NQ + q] = s;
        }
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    if (threadIdx.x < NQ) {
        double s = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(partials + (size_t)b * NQ + threadIdx.x);
        out[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) *counter = 0u;
}

__device__ __forceinline__ void elem_grad(const int* e_nodes, const double* G, const double* X, int N, int e,
                                          int col, double& gx, double& gy) {
    const int a = __ldg(e_nodes + 3 * e), b = __ldg(e_nodes + 3 * e + 1), c = __ldg(e_nodes + 3 * e + 2);
    const double x0 = a >= 0 ? __ldg(X + (size_t)a * N + col) : 0.0;
    const double x1 = b >= 0 ? __ldg(X + (size_t)b * N + col) : 0.0;
    const double x2 = c >= 0 ? __ldg(X + (size_t)c * N + col) : 0.0;
    const double d1 = x1 - x0, d2 = x2 - x0;
    gx = fma(d1, __ldg(G + 0), d2 * __ldg(G + 2));
    gy = fma(d1, __ldg(G + 1), d2 * __ldg(G + 3));
}

// Jacobian coefficients of the iron elements at every step:
// A = |T| [nu I + 2 nu'(s^2) g g^T] as (a11, a12, a22), stored at the reversed
// column (adjoint) or at the step's own column (Newton's forward Jacobian).
__global__ void __launch_bounds__(kBlock)
k_adj_jacobian(AdjointArgs a, const double* __restrict__ U, int reversed) {
    pdl_enter();
    const int N = a.N;
    const size_t total = (size_t)a.n_iron * N;
    const double c = a.s2sat, dnu = a.nu_max - a.nu_min;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(g / N);
        const int n = (int)(g - (size_t)e * N);
        double gx, gy;
        elem_grad(a.e_nodes, a.e_geo + 6 * (size_t)e, U, N, e, n, gx, gy);
        const double s2 = fma(gx, gx, gy * gy);
        const double den = s2 + c;
        const double nu = a.nu_min + dnu * s2 / den;
        const double dnu_ds2 = dnu * c / (den * den);
        const double A = __ldg(a.e_area + e);
        const double w = 2.0 * dnu_ds2 * A;
        const size_t o = (size_t)e * N + (reversed ? N - 1 - n : n);
        a.Jc[o] = A * nu + w * gx * gx;
        a.Jc[total + o] = w * gx * gy;
        a.Jc[2 * total + o] = A * nu + w * gy * gy;
    }
}

// Right-hand side g = dJ/dU at reversed columns and J itself:
// g^n = (2/(N tau)) (M_J d^n - M_J d^{n+1}),  J = (1/N) sum_n d^n . M_J d^n.
__global__ void __launch_bounds__(kBlock)
k_adj_rhs(AdjointArgs a, const double* __restrict__ U, double* __restrict__ Gout) {
    pdl_enter();
    const int N = a.N;
    const size_t total = (size_t)a.n * N;
    const double itau = 1.0 / a.tau;
    double acc[1] = {0.0};
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(g / N);
        const int n = (int)(g - (size_t)i * N);
        const int nm = n == 0 ? N - 1 : n - 1, np = n == N - 1 ? 0 : n + 1;
        double md = 0.0, mdn = 0.0;
        for (int k = __ldg(a.mj_ptr + i), ke = __ldg(a.mj_ptr + i + 1); k < ke; ++k) {
            const double* uj = U + (size_t)__ldg(a.mj_idx + k) * N;
            const double v = __ldg(a.mj_val + k);
            const double un = __ldg(uj + n);
            md = fma(v, un - __ldg(uj + nm), md);
            mdn = fma(v, __ldg(uj + np) - un, mdn);
        }
        md *= itau;
        mdn *= itau;
        Gout[(size_t)i * N + (N - 1 - n)] = 2.0 / (N * a.tau) * (md - mdn);
        const double di = (__ldg(U + g) - __ldg(U + (size_t)i * N + nm)) * itau;
        acc[0] = fma(di, md, acc[0]);
    }
    grid_sum<1>(acc, a.partials, a.counter, a.scalars + 0);
}

// adjoint element flux q = A grad(lambda) at reversed column m
__global__ void __launch_bounds__(kBlock)
k_adj_elem_flux(AdjointArgs a, const double* __restrict__ Lam, double* __restrict__ Qx, double* __restrict__ Qy,
                const int* done) {
    pdl_enter();
    if (done && *(volatile const int*)done) return;
    const int N = a.N;
    const size_t total = (size_t)a.n_iron * N;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(g / N);
        const int m = (int)(g - (size_t)e * N);
        double hx, hy;
        elem_grad(a.e_nodes, a.e_geo + 6 * (size_t)e, Lam, N, e, m, hx, hy);
        const double a11 = __ldg(a.Jc + g), a12 = __ldg(a.Jc + total + g), a22 = __ldg(a.Jc + 2 * total + g);
        Qx[g] = fma(a11, hx, a12 * hy);
        Qy[g] = fma(a12, hx, a22 * hy);
    }
}

// dJ/d(amp_c) = sum_n sum_i lambda_i^n sin(2 pi t^n/T + phase_c) b_c,i  (up to kMaxCoils coils)
// and dJ/d(nu_min, nu_max, s_sat) = - sum_n sum_iron |T| dnu/dtheta (g . grad lambda)
__global__ void __launch_bounds__(kBlock)
k_adj_grad_coils(AdjointArgs a, const double* __restrict__ Lam) {
    pdl_enter();
    const int N = a.N;
    const size_t total = (size_t)a.n * N;
    double acc[kMaxCoils];
#pragma unroll
    for (int c = 0; c < kMaxCoils; ++c) acc[c] = 0.0;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(g / N);
        const int m = (int)(g - (size_t)i * N);
        const int n = N - 1 - m;
        const double l = __ldg(Lam + g);
#pragma unroll
        for (int c = 0; c < kMaxCoils; ++c)
            if (c < a.n_coils)
                acc[c] = fma(l * __ldg(a.coil_b + (size_t)c * a.n + i), __ldg(a.coil_sin + (size_t)c * N + n), acc[c]);
    }
    grid_sum<kMaxCoils>(acc, a.partials, a.counter, a.scalars + 1);
}

__global__ void __launch_bounds__(kBlock)
k_adj_grad_nu(AdjointArgs a, const double* __restrict__ U, const double* __restrict__ Lam) {
    pdl_enter();
    const int N = a.N;
    const size_t total = (size_t)a.n_iron * N;
    const double c = a.s2sat, dnu = a.nu_max - a.nu_min, ssat = sqrt(a.s2sat);
    double acc[3] = {0.0, 0.0, 0.0};
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(g / N);
        const int n = (int)(g - (size_t)e * N);
        const double* G = a.e_geo + 6 * (size_t)e;
        double gx, gy, hx, hy;
        elem_grad(a.e_nodes, G, U, N, e, n, gx, gy);
        elem_grad(a.e_nodes, G, Lam, N, e, N - 1 - n, hx, hy);
        const double s2 = fma(gx, gx, gy * gy);
        const double den = s2 + c;
        const double w = -__ldg(a.e_area + e) * fma(gx, hx, gy * hy);
        const double q = s2 / den;
        acc[0] = fma(w, 1.0 - q, acc[0]);
        acc[1] = fma(w, q, acc[1]);
        acc[2] = fma(w, -dnu * s2 * 2.0 * ssat / (den * den), acc[2]);
    }
    grid_sum<3>(acc, a.partials, a.counter, a.scalars + 1 + kMaxCoils);
}

// dJ/dsigma_e = [iron] (1/N) sum_n |T|/12 ((sum d)^2 + sum d^2)
//               - sum_n |T|/12 ((sum l)(sum d) + sum l d),  d = d_tau u at the vertices
// one warp per element, lanes over the steps
__global__ void __launch_bounds__(kBlock)
k_adj_grad_sigma(AdjointArgs a, const double* __restrict__ U, const double* __restrict__ Lam,
                 double* __restrict__ dsigma) {
    pdl_enter();
    const int N = a.N;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const double itau = 1.0 / a.tau;
    for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < a.n_tri; e += warps) {
        int v[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = __ldg(a.all_nodes + 3 * e + k);
        double quu = 0.0, qlu = 0.0;
        for (int n = lane; n < N; n += 32) {
            const int nm = n == 0 ? N - 1 : n - 1;
            double d[3], l[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (v[k] >= 0) {
                    const double* u = U + (size_t)v[k] * N;
                    d[k] = (__ldg(u + n) - __ldg(u + nm)) * itau;
                    l[k] = __ldg(Lam + (size_t)v[k] * N + (N - 1 - n));
                } else {
                    d[k] = 0.0;
                    l[k] = 0.0;
                }
            }
            const double sd = d[0] + d[1] + d[2], sl = l[0] + l[1] + l[2];
            quu += sd * sd + d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            qlu += sl * sd + l[0] * d[0] + l[1] * d[1] + l[2] * d[2];
        }
        quu = warp_sum(quu);
        qlu = warp_sum(qlu);
        if (lane == 0) {
            const double A = __ldg(a.all_area + e) / 12.0;
            const double own = __ldg(a.all_iron + e) ? A * quu / N : 0.0;
            dsigma[e] = own - A * qlu;
        }
    }
}

int flat_grid(size_t total) {
    size_t want = (total + kBlock - 1) / kBlock;
    size_t cap = (size_t)num_sms() * 8;
    return (int)std::max<size_t>(1, std::min(want, cap));
}

}  // namespace

int launch_adj_jacobian(const AdjointArgs& a, const double* U, cudaStream_t s, bool reversed) {
    if (a.n_iron == 0) return 0;
    launch_k(k_adj_jacobian, dim3(flat_grid((size_t)a.n_iron * a.N)), dim3(kBlock), s, a, U, reversed ? 1 : 0);
    return 1;
}

int launch_adj_rhs(const AdjointArgs& a, const double* U, double* Gout, cudaStream_t s) {
    launch_k(k_adj_rhs, dim3(flat_grid((size_t)a.n * a.N)), dim3(kBlock), s, a, U, Gout);
    return 1;
}

int launch_adj_elem_flux(const AdjointArgs& a, const double* Lam, double* Qx, double* Qy, const int* done,
                         cudaStream_t s) {
    if (a.n_iron == 0) return 0;
    launch_k(k_adj_elem_flux, dim3(flat_grid((size_t)a.n_iron * a.N)), dim3(kBlock), s, a, Lam, Qx, Qy, done);
    return 1;
}

int launch_adj_gradients(const AdjointArgs& a, const double* U, const double* Lam, double* dsigma, cudaStream_t s) {
    launch_k(k_adj_grad_coils, dim3(flat_grid((size_t)a.n * a.N)), dim3(kBlock), s, a, Lam);
    int k = 1;
    if (a.n_iron > 0) {
        launch_k(k_adj_grad_nu, dim3(flat_grid((size_t)a.n_iron * a.N)), dim3(kBlock), s, a, U, Lam);
        ++k;
    }
    launch_k(k_adj_grad_sigma, dim3(flat_grid((size_t)a.n_tri * 32)), dim3(kBlock), s, a, U, Lam, dsigma);
    return k + 1;
}

}  // namespace ptp
