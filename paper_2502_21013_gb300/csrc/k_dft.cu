// Exact periodic solve of one time level by a discrete Fourier transform in
// time (Remark on parallel solvers, Section 3), in double precision.
//
// The periodic, time-invariant system of the level,
//   (M + tau L) x^n - M x^{n-1} = b^n,  n = 0..N-1,  x^{-1} = x^{N-1},
// becomes block diagonal under the DFT  x_k = sum_n x^n e^{-2 pi i k n / N}:
//   ((1 - e^{-2 pi i k / N}) M + tau L) x_k = b_k,   k = 0..N-1.
// (The discrete shift gives the factor 1 - e^{-2 pi i k/N}; the remark writes
// the continuous-time symbol.)  b is real, so x_{N-k} = conj(x_k) and only
// k = 0..N/2 are solved.  Each block is complex symmetric; the K = N/2 + 1
// solves run batched, one complex column per mode, stored as interleaved
// (re, im) double pairs [row][2K], by the conjugate-orthogonal CG method:
// the CG recurrence with the bilinear form x^T y in place of x^H y.  The
// preconditioner of every mode is the real SPD operator tau L (one spatial
// multigrid V-cycle applied to the 2K real columns), so the preconditioned
// spectrum is 1 + c_k [0, lambda_max((tau L)^{-1} M)], a segment in the right
// half-plane.
//
// Transforms: radix-2 FFT in shared memory per node (N a power of two, one
// block holds 512 / N nodes), otherwise a direct sum over the N steps.
// N <= 1022, so the K <= 512 complex columns of a row fit one block.
#include "dev_fft.cuh"
#include "dev_util.cuh"

namespace ptp {

namespace {

constexpr int kFftThreads = 256;

// forward: H[i][k] = sum_t x[i][t] e^{-2 pi i k t / N}, k < K (N a power of two)
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
k_fft_fwd(int n, int N, int logN, int K, const T* __restrict__ x, const double2* __restrict__ W,
          double* __restrict__ H, Skip sk) {
    pdl_enter();
    if (skip_now(sk)) return;
    extern __shared__ double2 sh[];
    const int nb = max(1, (int)blockDim.x / max(1, N / 2));
    for (int base = blockIdx.x * nb; base < n; base += gridDim.x * nb) {
        for (int e = threadIdx.x; e < nb * N; e += blockDim.x) {
            const int j = e / N, t = e - j * N, node = base + j;
            const double v = node < n ? (double)x[(size_t)node * N + t] : 0.0;
            sh[j * N + bit_reverse(t, logN)] = make_double2(v, 0.0);
        }
        __syncthreads();
        fft_stages<false>(sh, nb, N, W);
        for (int e = threadIdx.x; e < nb * K; e += blockDim.x) {
            const int j = e / K, k = e - j * K, node = base + j;
            if (node < n) reinterpret_cast<double2*>(H)[(size_t)node * K + k] = sh[j * N + k];
        }
        __syncthreads();
    }
}

// inverse: x[i][t] = scale * Re sum_{k<N} H_k e^{+2 pi i k t / N} with
// H_{N-k} = conj(H_k) (N a power of two)
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
k_fft_inv(int n, int N, int logN, int K, const double* __restrict__ H, const double2* __restrict__ W,
          T* __restrict__ x, double scale, Skip sk) {
    pdl_enter();
    if (skip_now(sk)) return;
    extern __shared__ double2 sh[];
    const int nb = max(1, (int)blockDim.x / max(1, N / 2));
    const double2* Hc = reinterpret_cast<const double2*>(H);
    for (int base = blockIdx.x * nb; base < n; base += gridDim.x * nb) {
        for (int e = threadIdx.x; e < nb * N; e += blockDim.x) {
            const int j = e / N, t = e - j * N, node = base + j;
            double2 v = make_double2(0.0, 0.0);
            if (node < n) {
                if (t < K) {
                    v = Hc[(size_t)node * K + t];
                } else {
                    v = Hc[(size_t)node * K + (N - t)];
                    v.y = -v.y;
                }
            }
            sh[j * N + bit_reverse(t, logN)] = v;
        }
        __syncthreads();
        fft_stages<true>(sh, nb, N, W);
        for (int e = threadIdx.x; e < nb * N; e += blockDim.x) {
            const int j = e / N, t = e - j * N, node = base + j;
            if (node < n) x[(size_t)node * N + t] = (T)(sh[e].x * scale);
        }
        __syncthreads();
    }
}

// direct transforms for N that is not a power of two (O(N) per output)
template <typename T>
__global__ void k_dft_direct_fwd(int n, int N, int K, const T* __restrict__ x, const double2* __restrict__ W,
                                 double* __restrict__ H, Skip sk) {
    pdl_enter();
    if (skip_now(sk)) return;
    const size_t total = (size_t)n * K;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(g / K), k = (int)(g - (size_t)i * K);
        const T* xr = x + (size_t)i * N;
        double re = 0.0, im = 0.0;
        int idx = 0;   // k t mod N
        for (int t = 0; t < N; ++t) {
            const double v = (double)xr[t];
            const double2 w = __ldg(W + idx);
            re = fma(v, w.x, re);
            im = fma(v, w.y, im);
            idx += k;
            if (idx >= N) idx -= N;
        }
        reinterpret_cast<double2*>(H)[g] = make_double2(re, im);
    }
}

template <typename T>
__global__ void k_dft_direct_inv(int n, int N, int K, const double* __restrict__ H, const double2* __restrict__ W,
                                 T* __restrict__ x, double scale, Skip sk) {
    pdl_enter();
    if (skip_now(sk)) return;
    const size_t total = (size_t)n * N;
    const double2* Hc = reinterpret_cast<const double2*>(H);
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(g / N), t = (int)(g - (size_t)i * N);
        const double2* hr = Hc + (size_t)i * K;
        double s = hr[0].x;
        int idx = t;   // k t mod N
        for (int k = 1; k < K; ++k) {
            const double2 h = hr[k];
            if (2 * k == N) {
                s += (t & 1) ? -h.x : h.x;   // the real Nyquist mode, counted once
            } else {
                // 2 Re(h e^{+i theta}) with W[idx] = e^{-i theta}
                const double2 w = __ldg(W + idx);
                s += 2.0 * (h.x * w.x + h.y * w.y);
            }
            idx += t;
            if (idx >= N) idx -= N;
        }
        x[g] = (T)(s * scale);
    }
}

// ---------------------------------------------------------------------------
// Conjugate-orthogonal CG over K complex columns (D = 2K doubles per row).
// Thread = (row, mode k); VEC = 2 real columns = one complex value.
// ---------------------------------------------------------------------------

// mode-k operator of one row: c_k (M x)_row + tau (L x)_row, complex x
__device__ __forceinline__ double2 row_capply(const Op<double>& op, int D, int row, int col0, const double* X,
                                              double2 ck, double tau) {
    double mr = 0.0, mi = 0.0, lr = 0.0, li = 0.0;
    if (op.ell_w > 0) {
        const size_t base = (size_t)row * op.ell_w;
        for (int e = 0; e < op.ell_w; ++e) {
            const int j = __ldg(op.eidx + base + e);
            const double m = __ldg(op.ev1 + base + e), l = __ldg(op.ev2 + base + e);
            const double2 x = __ldg(reinterpret_cast<const double2*>(X + (size_t)j * D + col0));
            mr = fma(m, x.x, mr);
            mi = fma(m, x.y, mi);
            lr = fma(l, x.x, lr);
            li = fma(l, x.y, li);
        }
    } else {
        for (int e = __ldg(op.ptr + row), ee = __ldg(op.ptr + row + 1); e < ee; ++e) {
            const int j = __ldg(op.idx + e);
            const double m = __ldg(op.v1 + e), l = __ldg(op.v2 + e);
            const double2 x = __ldg(reinterpret_cast<const double2*>(X + (size_t)j * D + col0));
            mr = fma(m, x.x, mr);
            mi = fma(m, x.y, mi);
            lr = fma(l, x.x, lr);
            li = fma(l, x.y, li);
        }
    }
    return make_double2(ck.x * mr - ck.y * mi + tau * lr, ck.x * mi + ck.y * mr + tau * li);
}

__device__ __forceinline__ double2 ld2(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ void st2(double* p, double2 v) { *reinterpret_cast<double2*>(p) = v; }

// q = A_k p ; alpha_k = rho_k / (p^T q)
__global__ void __launch_bounds__(kMaxBlock)
k_capply_alpha(Op<double> op, int D, const double2* __restrict__ ck, double tau, const double* __restrict__ p,
               double* __restrict__ q, ColRed<double> cr, Skip sk) {
    pdl_enter();
    if (skip_now(sk)) return;
    constexpr int VEC = 2;
    const int NC = D / VEC, rpb = blockDim.x / NC;
    double acc[1][VEC] = {{0.0, 0.0}};
    PTP_ROW_LOOP(op.rows, NC, rpb) {
        const double2 y = row_capply(op, D, row, col0, p, __ldg(ck + chunk_), tau);
        const double2 pv = ld2(p + (size_t)row * D + col0);
        st2(q + (size_t)row * D + col0, y);
        acc[0][0] += pv.x * y.x - pv.y * y.y;
        acc[0][1] += pv.x * y.y + pv.y * y.x;
    }
    col_reduce_finish<double, VEC, 1, FIN_C_ALPHA>(acc, D, NC, rpb, cr, native_grid());
}

// x += alpha p (x = alpha p when assign) ; r -= alpha q ; rr = |r|^2 and the convergence test
__global__ void __launch_bounds__(kMaxBlock)
k_cupdate(int rows, int D, int assign, double* x, const double* __restrict__ p, double* r,
          const double* __restrict__ q, ColRed<double> cr, Skip sk) {
    pdl_enter();
    if (skip_now(sk)) return;
    constexpr int VEC = 2;
    const int NC = D / VEC, rpb = blockDim.x / NC;
    double acc[1][VEC] = {{0.0, 0.0}};
    const double* alpha = cr.col + S_ALPHA * D;
    PTP_ROW_LOOP(rows, NC, rpb) {
        const size_t o = (size_t)row * D + col0;
        const double2 a = make_double2(alpha[col0], alpha[col0 + 1]);
        const double2 ap = cmul(a, ld2(p + o));
        const double2 aq = cmul(a, ld2(q + o));
        double2 xv = assign ? make_double2(0.0, 0.0) : ld2(x + o);
        double2 rv = ld2(r + o);
        xv.x += ap.x; xv.y += ap.y;
        rv.x -= aq.x; rv.y -= aq.y;
        st2(x + o, xv);
        st2(r + o, rv);
        acc[0][0] += rv.x * rv.x;
        acc[0][1] += rv.y * rv.y;
    }
    col_reduce_finish<double, VEC, 1, FIN_C_UPDATE>(acc, D, NC, rpb, cr, native_grid());
}

// first: rho = r^T z, bb = rr = |r|^2 ; else beta = (r^T z) / rho, rho = r^T z
template <bool FIRST>
__global__ void __launch_bounds__(kMaxBlock)
k_cdot_rz(int rows, int D, const double* __restrict__ r, const double* __restrict__ z, ColRed<double> cr, Skip sk) {
    pdl_enter();
    if (skip_now(sk)) return;
    constexpr int VEC = 2;
    constexpr int NQ = FIRST ? 2 : 1;
    const int NC = D / VEC, rpb = blockDim.x / NC;
    double acc[NQ][VEC];
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) acc[qq][0] = acc[qq][1] = 0.0;
    PTP_ROW_LOOP(rows, NC, rpb) {
        const size_t o = (size_t)row * D + col0;
        const double2 rv = ld2(r + o), zv = ld2(z + o);
        acc[0][0] += rv.x * zv.x - rv.y * zv.y;
        acc[0][1] += rv.x * zv.y + rv.y * zv.x;
        if constexpr (FIRST) {
            acc[1][0] += rv.x * rv.x;
            acc[1][1] += rv.y * rv.y;
        }
    }
    col_reduce_finish<double, VEC, NQ, FIRST ? FIN_C_RZ_FIRST : FIN_C_RZ_NEXT>(acc, D, NC, rpb, cr, native_grid());
}

// p = z + beta p
__global__ void __launch_bounds__(kMaxBlock)
k_cdirection(int rows, int D, const double* __restrict__ z, double* p, ColRed<double> cr, Skip sk) {
    pdl_enter();
    if (skip_now(sk)) return;
    constexpr int VEC = 2;
    const int NC = D / VEC, rpb = blockDim.x / NC;
    const double* beta = cr.col + S_BETA * D;
    PTP_ROW_LOOP(rows, NC, rpb) {
        const size_t o = (size_t)row * D + col0;
        const double2 bp = cmul(make_double2(beta[col0], beta[col0 + 1]), ld2(p + o));
        const double2 zv = ld2(z + o);
        st2(p + o, make_double2(zv.x + bp.x, zv.y + bp.y));
    }
}

int log2_exact(int N) {
    int l = 0;
    while ((1 << l) < N) ++l;
    return (1 << l) == N ? l : -1;
}

int fft_grid(int n, int nb) {
    const int want = (n + nb - 1) / nb;
    return std::max(1, std::min(want, num_sms() * 8));
}

int flat_blocks(size_t total) {
    const size_t want = (total + 255) / 256;
    return (int)std::max<size_t>(1, std::min(want, (size_t)num_sms() * 8));
}

void check_dft_size(int N) {
    if (N < 1 || N > kMaxDftSteps) throw Error(PTP_EINVAL, "DFT in time: the level must have 1..1022 steps");
}

}  // namespace

template <typename T>
int launch_dft_fwd(int n, int N, const T* x, const double* W, double* H, Skip sk, cudaStream_t s) {
    check_dft_size(N);
    const int K = N / 2 + 1;
    const int logN = log2_exact(N);
    const double2* W2 = reinterpret_cast<const double2*>(W);
    if (logN >= 0) {
        const int nb = std::max(1, kFftThreads / std::max(1, N / 2));
        const size_t smem = (size_t)nb * N * sizeof(double2);
        launch_k_smem(k_fft_fwd<T>, dim3(fft_grid(n, nb)), dim3(kFftThreads), smem, s, n, N, logN, K, x, W2, H, sk);
    } else {
        launch_k(k_dft_direct_fwd<T>, dim3(flat_blocks((size_t)n * K)), dim3(256), s, n, N, K, x, W2, H, sk);
    }
    return 1;
}

template <typename T>
int launch_dft_inv(int n, int N, const double* H, const double* W, T* x, Skip sk, cudaStream_t s) {
    check_dft_size(N);
    const int K = N / 2 + 1;
    const int logN = log2_exact(N);
    const double2* W2 = reinterpret_cast<const double2*>(W);
    const double scale = 1.0 / N;
    if (logN >= 0) {
        const int nb = std::max(1, kFftThreads / std::max(1, N / 2));
        const size_t smem = (size_t)nb * N * sizeof(double2);
        launch_k_smem(k_fft_inv<T>, dim3(fft_grid(n, nb)), dim3(kFftThreads), smem, s, n, N, logN, K, H, W2, x, scale,
                      sk);
    } else {
        launch_k(k_dft_direct_inv<T>, dim3(flat_blocks((size_t)n * N)), dim3(256), s, n, N, K, H, W2, x, scale, sk);
    }
    return 1;
}

int launch_capply_alpha(const Op<double>& op, int D, const double* ck, double tau, const double* p, double* q,
                        ColRed<double> cr, Skip sk, cudaStream_t s) {
    launch_rows(k_capply_alpha, op.rows, D, 2, s, op, D, reinterpret_cast<const double2*>(ck), tau, p, q, cr, sk);
    return 1;
}

int launch_cupdate(int rows, int D, int assign, double* x, const double* p, double* r, const double* q,
                   ColRed<double> cr, Skip sk, cudaStream_t s) {
    launch_rows(k_cupdate, rows, D, 2, s, rows, D, assign, x, p, r, q, cr, sk);
    return 1;
}

int launch_cdot_rz(int rows, int D, const double* r, const double* z, ColRed<double> cr, int first, Skip sk,
                   cudaStream_t s) {
    if (first)
        launch_rows(k_cdot_rz<true>, rows, D, 2, s, rows, D, r, z, cr, sk);
    else
        launch_rows(k_cdot_rz<false>, rows, D, 2, s, rows, D, r, z, cr, sk);
    return 1;
}

int launch_cdirection(int rows, int D, const double* z, double* p, ColRed<double> cr, Skip sk, cudaStream_t s) {
    launch_rows(k_cdirection, rows, D, 2, s, rows, D, z, p, cr, sk);
    return 1;
}

template int launch_dft_fwd<float>(int, int, const float*, const double*, double*, Skip, cudaStream_t);
template int launch_dft_fwd<double>(int, int, const double*, const double*, double*, Skip, cudaStream_t);
template int launch_dft_inv<float>(int, int, const double*, const double*, float*, Skip, cudaStream_t);
template int launch_dft_inv<double>(int, int, const double*, const double*, double*, Skip, cudaStream_t);

}  // namespace ptp
