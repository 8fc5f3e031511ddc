// Exact solve of the coarsest time level on a uniform structured grid by the
// discrete sine transform, in double precision.
//
// With one step on the coarsest time level (N_c = 1) its periodic system is
// tau_c L x = b (the mass terms cancel).  On the uniform grid whose cells
// are split along one diagonal, L = nu_max A and the P1 stiffness A of the
// free nodes is the five-point operator
//   (A x)_{a,b} = 2 (hy/hx + hx/hy) x_{a,b} - hy/hx (x_{a+1,b} + x_{a-1,b})
//                 - hx/hy (x_{a,b+1} + x_{a,b-1})
// (right triangles couple no hypotenuse ends), with zero Dirichlet values
// outside.  The sine vectors sin(pi k (a+1) / m_x) sin(pi l (b+1) / m_y),
// m_x = W + 1, m_y = H + 1, diagonalise it with eigenvalues
//   lambda_kl = hy/hx (2 - 2 cos(pi k / m_x)) + hx/hy (2 - 2 cos(pi l / m_y)),
// so x = (2/m_x)(2/m_y) S_x S_y [ b^ / (tau_c nu_max lambda) ] with the
// unnormalised DST-I  (S z)_k = sum_j z_j sin(pi j k / m)  applied along the
// rows and the columns.  This is the solve, not an approximation of it: the
// result is exact up to the rounding of the transforms.
//
// Each DST-I of length n = m - 1 (m a power of two) is a complex radix-2 FFT
// of length 2m of the odd extension y = [0, z, 0, -reverse(z)]:
// FFT(y)_k = -2i (S z)_k.  Two real transforms share one FFT: with
// z = z1 + i z2, (S z1)_k = -Im FFT(y)_k / 2 and (S z2)_k = Re FFT(y)_k / 2.
#include <algorithm>
#include <map>
#include <mutex>

#include "dev_bodies.cuh"

namespace ptp {

namespace {

template <typename TI, typename TO, bool TWICE>
__global__ void __launch_bounds__(kDstThreads) k_dst(DstArgs p) {
    dst_body<TI, TO, TWICE>(p, native_grid());
}
template <typename TI, typename TO, bool TWICE>
__global__ void __launch_bounds__(kDstThreads) k_dst_b(const DstArgs* __restrict__ ps, BatchMap m) {
    pdl_enter();
    int i;
    VGrid g;
    if (batch_block(m, i, g)) {
        const auto a_ = ps[i];   // a local copy: no store of the body aliases it
        dst_body<TI, TO, TWICE>(a_, g);
    }
}

template <typename... KArgs, typename... Args>
void dst_launch(void (*kernel)(KArgs...), int blocks, size_t smem, cudaStream_t s, Args&&... args) {
    ensure_dynamic_smem((const void*)kernel, smem);
    launch_k_smem(kernel, dim3(std::max(1, blocks)), dim3(kDstThreads), smem, s, std::forward<Args>(args)...);
}

template <typename TI, typename TO, bool TWICE>
int dst_batch(const void* args, BatchMap m, int blocks, const KShape& sh, cudaStream_t s) {
    dst_launch(k_dst_b<TI, TO, TWICE>, blocks, sh.smem, s, static_cast<const DstArgs*>(args), m);
    return 1;
}

// one transform pass: recorded for a batched step, else launched
template <typename TI, typename TO, bool TWICE>
void dst_pass(const DstArgs& a, cudaStream_t s) {
    KShape sh;
    sh.gx = std::max(1, (a.ntr + 1) / 2);
    sh.gy = 1;
    sh.block = kDstThreads;
    sh.smem = (size_t)(TWICE ? 4 : 2) * (a.n + 1) * sizeof(double2);
    int body = 0;
    if constexpr (sizeof(TI) == 4 && sizeof(TO) == 8 && !TWICE) body = body_id(BF_DST_FD, 0, 0);
    if constexpr (sizeof(TI) == 8 && sizeof(TO) == 8 && TWICE) body = body_id(BF_DST_DD2, 0, 0);
    if constexpr (sizeof(TI) == 8 && sizeof(TO) == 4 && !TWICE) body = body_id(BF_DST_DF, 0, 0);
    if (record_launch(dst_batch<TI, TO, TWICE>, a, sh, body)) return;
    dst_launch(k_dst<TI, TO, TWICE>, sh.gx, sh.smem, s, a);
}

}  // namespace

template <typename T>
int launch_dst_solve(const DstSolve& d, const T* b, T* x, Skip sk, cudaStream_t s) {
    const int W = d.W, H = d.H;
    // rows: along a for every b, written transposed to tmp[k][b]
    dst_pass<T, double, false>(DstArgs{H, W, d.logx, b, (long)W, 1L, d.tmp, 1L, (long)H, nullptr, d.wx, sk}, s);
    // columns: along b for every k, scaled by 1 / eigenvalue, and back
    dst_pass<double, double, true>(DstArgs{W, H, d.logy, d.tmp, (long)H, 1L, d.tmp2, (long)H, 1L, d.scale, d.wy, sk},
                                   s);
    // rows again: along k for every b, written back in node order
    dst_pass<double, T, false>(DstArgs{H, W, d.logx, d.tmp2, 1L, (long)H, x, (long)W, 1L, nullptr, d.wx, sk}, s);
    return 3;
}

template int launch_dst_solve<float>(const DstSolve&, const float*, float*, Skip, cudaStream_t);
template int launch_dst_solve<double>(const DstSolve&, const double*, double*, Skip, cudaStream_t);

}  // namespace ptp
