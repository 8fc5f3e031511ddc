// Iron element fluxes of the reluctivity law of the paper's transformer
// (Section 4, "Test problem"), in double precision:
//
//   nu(s) = a min(exp(b s^2), c) + d,   q_T^n = nu(|g_T^n|^2) |T| g_T^n,
//
// with per-element constants (iron and steel differ).  The cap is applied in
// the exponent, exp(min(b s^2, ln c)) = min(exp(b s^2), c), and exp is CUDA's
// double-precision exp.  The node pass of K1 (k_residual.cu) then gathers
// these fluxes like those of the saturating law, so only this element pass
// depends on the law.
#include "kernels.h"

namespace ptp {

namespace {

constexpr int kBlock = 256;

// e_law per iron element: |T| a, b, ln c, |T| d
__global__ void __launch_bounds__(kBlock)
k_elem_flux_exp(int n_iron, int N, const int* __restrict__ e_nodes, const double* __restrict__ e_geo,
                const double* __restrict__ e_law, const double* __restrict__ U, double* __restrict__ Qx,
                double* __restrict__ Qy, const int* done) {
    pdl_enter();
    if (done != nullptr && *(volatile const int*)done != 0) return;
    const size_t total = (size_t)n_iron * N;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(g / N);
        const int t = (int)(g - (size_t)e * N);
        const int i0 = __ldg(e_nodes + 3 * e), i1 = __ldg(e_nodes + 3 * e + 1), i2 = __ldg(e_nodes + 3 * e + 2);
        const double u0 = i0 >= 0 ? __ldg(U + (size_t)i0 * N + t) : 0.0;
        const double u1 = i1 >= 0 ? __ldg(U + (size_t)i1 * N + t) : 0.0;
        const double u2 = i2 >= 0 ? __ldg(U + (size_t)i2 * N + t) : 0.0;
        const double* G = e_geo + 6 * (size_t)e;
        const double* Lw = e_law + 4 * (size_t)e;
        const double d1 = u1 - u0, d2 = u2 - u0;
        const double gx = fma(d1, __ldg(G + 0), d2 * __ldg(G + 2));
        const double gy = fma(d1, __ldg(G + 1), d2 * __ldg(G + 3));
        const double s2 = fma(gx, gx, gy * gy);
        const double w = fma(__ldg(Lw + 0), exp(fmin(__ldg(Lw + 1) * s2, __ldg(Lw + 2))), __ldg(Lw + 3));
        Qx[g] = w * gx;
        Qy[g] = w * gy;
    }
}

}  // namespace

int launch_residual_law(const ResidualArgs& a, const double* e_law, cudaStream_t s) {
    if (e_law == nullptr || a.n_iron == 0 || a.skip_flux) return launch_residual(a, s);
    const size_t total = (size_t)a.n_iron * a.N;
    const size_t want = (total + kBlock - 1) / kBlock;
    const int grid = (int)std::max<size_t>(1, std::min(want, (size_t)num_sms() * 8));
    launch_k(k_elem_flux_exp, dim3(grid), dim3(kBlock), s, a.n_iron, a.N, a.e_nodes, a.e_geo, e_law, a.U, a.Qx,
             a.Qy, (const int*)a.done);
    ResidualArgs b = a;
    b.skip_flux = 1;
    return 1 + launch_residual(b, s);
}

}  // namespace ptp
