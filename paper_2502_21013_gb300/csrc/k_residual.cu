// K1: the outer residual R = F - A(U) of Problem 1 in double precision.
//
//   R^n_i = f^n_i - sum_j (M_ij / tau) (u^n_j - u^{n-1}_j) - K(u^n)_i,   u^0 = u^N,
//   K(u)_i = sum_{T containing i} nu(|g_T|^2) |T| g_T . grad(phi_i),
//   g_T = sum_j u_j grad(phi_j) = (u_1 - u_0) grad(phi_1) + (u_2 - u_0) grad(phi_2),
//   nu(s^2) = nu_min + (nu_max - nu_min) s^2 / (s^2 + s_sat^2) on iron, nu_linear else,
//   f^n_i = sum_c b_c,i amp_c sin(2 pi t^n / T + phase_c).
//
// (Problem 1; the operator A of the proof of Theorem 2; the model and
// material law of Section 4.)  On elements with the constant nu_linear the
// contribution is the linear stencil nu_linear A_lin u, so K splits exactly
// into a CSR product and the iron part.  Two passes over the space-time block:
//   1. iron-element pass: flux q_T^n = nu |T| g_T^n for every (iron element, step),
//   2. node pass: gather sum_T q_T . grad(phi_i) over the incident iron
//      elements (CSR gather, no atomics, deterministic), add the linear
//      stencil, mass and source terms, write R (and the scaled right-hand
//      side of the correction equation) and reduce ||R||^2; the last block
//      applies the stopping rule.
// Threads are mapped with the time index fastest, so every load of a node's
// N values is a contiguous, coalesced run.
#include <cmath>
#include <cstdlib>

#include "dev_math.cuh"
#include "kernels.h"

namespace ptp {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ bool skip_now(const int* done) {
    return done != nullptr && *(volatile const int*)done != 0;
}

// Iron elements only: q = nu(|g|^2) |T| g with
// nu |T| = |T| nu_max - |T| (nu_max - nu_min) s_sat^2 / (|g|^2 + s_sat^2).
__global__ void __launch_bounds__(kBlock)
k_elem_flux(int n_iron, int N, const int* __restrict__ e_nodes, const double* __restrict__ e_geo,
            const double* __restrict__ U, double* __restrict__ Qx, double* __restrict__ Qy,
            double s2sat, const int* done) {
    pdl_enter();
    if (skip_now(done)) return;
    const size_t total = (size_t)n_iron * N;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(g / N);
        const int t = (int)(g - (size_t)e * N);
        const int a = __ldg(e_nodes + 3 * e), b = __ldg(e_nodes + 3 * e + 1),
                  c = __ldg(e_nodes + 3 * e + 2);
        const double u0 = a >= 0 ? __ldg(U + (size_t)a * N + t) : 0.0;
        const double u1 = b >= 0 ? __ldg(U + (size_t)b * N + t) : 0.0;
        const double u2 = c >= 0 ? __ldg(U + (size_t)c * N + t) : 0.0;
        const double* G = e_geo + 6 * (size_t)e;
        const double d1 = u1 - u0, d2 = u2 - u0;
        const double gx = fma(d1, __ldg(G + 0), d2 * __ldg(G + 2));
        const double gy = fma(d1, __ldg(G + 1), d2 * __ldg(G + 3));
        const double s2 = fma(gx, gx, gy * gy);
        const double w = fma(-__ldg(G + 5), recip_newton(s2 + s2sat), __ldg(G + 4));
        Qx[g] = w * gx;
        Qy[g] = w * gy;
    }
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kBlock)
k_node_residual(ResidualArgs a) {
    pdl_enter();
    if (skip_now(a.done)) return;
    const int N = a.N;
    const size_t total = (size_t)a.n * N;
    // The float right-hand side is tau R / s with s the previous residual
    // norm, so its entries stay O(tau / sqrt(n N)) however small R becomes.
    // (Every block reads s before the last block replaces it below.)
    const double fscale = a.b_f ? a.scale / a.status->bscale : 0.0;
    double local = 0.0;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(g / N);
        const int t = (int)(g - (size_t)i * N);
        const int tm = t == 0 ? N - 1 : t - 1;
        double kv = 0.0;   // iron elements: sum_T q_T . grad(phi_i)
        for (int k = __ldg(a.inc_ptr + i), ke = __ldg(a.inc_ptr + i + 1); k < ke; ++k) {
            const size_t q = (size_t)__ldg(a.inc_elem + k) * N + t;
            kv = fma(__ldg(a.Qx + q), __ldg(a.inc_grad + 2 * k), kv);
            kv = fma(__ldg(a.Qy + q), __ldg(a.inc_grad + 2 * k + 1), kv);
        }
        for (int k = __ldg(a.l_ptr + i), ke = __ldg(a.l_ptr + i + 1); k < ke; ++k)  // linear elements
            kv = fma(__ldg(a.l_val + k), __ldg(a.U + (size_t)__ldg(a.l_idx + k) * N + t), kv);
        double mv = 0.0;   // (M / tau)(u^n - u^{n-1})
        for (int k = __ldg(a.m_ptr + i), ke = __ldg(a.m_ptr + i + 1); k < ke; ++k) {
            const size_t j = (size_t)__ldg(a.m_idx + k) * N;
            mv = fma(__ldg(a.m_val + k), __ldg(a.U + j + t) - __ldg(a.U + j + tm), mv);
        }
        double f = 0.0;
        if (a.Fext) {
            f = __ldg(a.Fext + g);
        } else {
            for (int c = 0; c < a.n_coils; ++c) {
                const double cb = __ldg(a.coil_b + (size_t)c * a.n + i);
                if (cb != 0.0) f = fma(cb, __ldg(a.coil_s + (size_t)c * N + t), f);   // warp-uniform
            }
        }
        const double r = f - mv - kv;
        if (a.R) a.R[g] = r;
        if (a.b_d) a.b_d[g] = a.scale * r;
        if (a.b_f) a.b_f[g] = (float)(fscale * r);
        local += r * r;
    }
    // block reduction of ||R||^2, then the last block finishes the sum
    __shared__ double sm[kBlock / 32];
    __shared__ bool last;
    local = warp_sum(local);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < kBlock / 32 ? sm[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) {
            a.partials[blockIdx.x] = v;
            __threadfence();
            const unsigned ticket = atomicAdd(a.counter, 1u);
            last = ticket == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!last) return;
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(a.partials + b);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) tot += sm[w];
        const double nrm = sqrt(tot);
        if (a.norm_out) *a.norm_out = nrm;
        Status* st = a.status;
        if (!st) {
            *a.counter = 0u;
            return;
        }
        st->bscale_used = st->bscale;
        if (isfinite(nrm) && nrm > 0.0) st->bscale = nrm;
        if (a.check) {
            const int it = st->iteration;
            if (it == 0) st->res0 = nrm;
            st->res = nrm;
            st->iteration = it + 1;
            if (!isfinite(nrm)) {
                st->done = 2;
                if (a.done) *a.done = 1;
            } else if (nrm <= st->tol * st->res0) {
                st->done = 1;
                if (a.done) *a.done = 1;
            }
        } else {
            st->res = nrm;
        }
        *a.counter = 0u;
    }
}

__global__ void k_source(int n, int N, int n_coils, const double* __restrict__ coil_b,
                         const double* __restrict__ coil_s, double* __restrict__ F) {
    pdl_enter();
    const size_t total = (size_t)n * N;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(g / N);
        const int t = (int)(g - (size_t)i * N);
        double f = 0.0;
        for (int c = 0; c < n_coils; ++c) f += coil_b[(size_t)c * n + i] * coil_s[(size_t)c * N + t];
        F[g] = f;
    }
}

int grid_for(size_t total, int per_sm) {
    size_t want = (total + kBlock - 1) / kBlock;
    size_t cap = (size_t)num_sms() * per_sm;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (int)want;
}

}  // namespace

bool pdl_enabled() {
    static int on = -1;
    if (on < 0) on = getenv("PTP_NO_PDL") ? 0 : 1;
    return on == 1;
}

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

int residual_grid(size_t total) { return grid_for(total, 8); }

int launch_residual(const ResidualArgs& a, cudaStream_t s) {
    int launched = 0;
    if (a.n_iron > 0 && !a.skip_flux) {
        const size_t te = (size_t)a.n_iron * a.N;
        launch_k(k_elem_flux, dim3(grid_for(te, 8)), dim3(kBlock), s, a.n_iron, a.N, a.e_nodes, a.e_geo, a.U,
                 a.Qx, a.Qy, a.s2sat, (const int*)a.done);
        ++launched;
    }
    const size_t tn = (size_t)a.n * a.N;
    launch_k(k_node_residual, dim3(grid_for(tn, 8)), dim3(kBlock), s, a);
    return launched + 1;
}

void launch_source(int n, int N, int n_coils, const double* coil_b, const double* coil_s,
                   double* F, cudaStream_t s) {
    const size_t t = (size_t)n * N;
    launch_k(k_source, dim3(grid_for(t, 8)), dim3(kBlock), s, n, N, n_coils, coil_b, coil_s, F);
}

}  // namespace ptp
