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
    static std::mutex mu;
    static std::map<const void*, size_t> granted;   // dynamic shared memory granted per kernel
    if (smem > 48 * 1024) {
        std::lock_guard<std::mutex> lock(mu);
        size_t& g = granted[(const void*)kernel];
        if (smem > g) {
            PTP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            g = smem;
        }
    }
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
    if (record_launch(dst_batch<TI, TO, TWICE>, a, sh)) return;
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
