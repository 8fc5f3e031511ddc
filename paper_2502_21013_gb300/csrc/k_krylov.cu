// Vector kernels of the flexible GMRES used by Newton's method (method (M2)
// of Section 4), in double over whole space-time blocks of `count` values:
// several dot products against one vector at once, a combination of several
// basis vectors, and a division by a device scalar.  The dot products are
// deterministic: per-block partials, then the last block to finish (atomic
// ticket, no waiting) sums them in block order.
#include "dev_bodies.cuh"

namespace ptp {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// out[i] = sum_g V[i * stride + g] w[g], i < k <= KB (KB a power of two, so
// a launch issues at most twice the FMAs its k dot products need)
template <int KB>
__global__ void __launch_bounds__(kThreads)
k_mdot(size_t count, int k, const double* __restrict__ V, size_t stride, const double* __restrict__ w,
       double* __restrict__ partials, unsigned* counter, double* __restrict__ out) {
    pdl_enter();
    double acc[KB];
#pragma unroll
    for (int i = 0; i < KB; ++i) acc[i] = 0.0;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < count; g += (size_t)gridDim.x * blockDim.x) {
        const double wg = __ldg(w + g);
#pragma unroll
        for (int i = 0; i < KB; ++i)
            if (i < k) acc[i] = fma(__ldg(V + (size_t)i * stride + g), wg, acc[i]);
    }
    __shared__ double sm[KB][kThreads / 32];
    __shared__ bool last;
#pragma unroll
    for (int i = 0; i < KB; ++i) {
        if (i >= k) break;
        const double s = warp_sum(acc[i]);
        if ((threadIdx.x & 31) == 0) sm[i][threadIdx.x >> 5] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        double s = 0.0;
        for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) s += sm[i][wi];
        partials[(size_t)blockIdx.x * k + i] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    // the whole last block sums the partials of each dot product: a strided
    // share per thread, then the warp and block trees (a fixed order)
    __shared__ double red[kThreads / 32];
    for (int i = 0; i < k; ++i) {
        double t = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(partials + (size_t)b * k + i);
        t = warp_sum(t);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            double u = 0.0;
            for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) u += red[wi];
            out[i] = u;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// w += sign * sum_{i<k} coef[i] V[i * stride + g]
__global__ void __launch_bounds__(kThreads)
k_maxpy(size_t count, int k, const double* __restrict__ V, size_t stride, const double* __restrict__ coef,
        double sign, double* __restrict__ w) {
    pdl_enter();
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < count; g += (size_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s = fma(__ldg(coef + i), __ldg(V + (size_t)i * stride + g), s);
        w[g] = fma(sign, s, w[g]);
    }
}

// y = x / *h
__global__ void __launch_bounds__(kThreads)
k_div_scalar(size_t count, const double* __restrict__ x, const double* __restrict__ h, double* __restrict__ y) {
    pdl_enter();
    const double inv = 1.0 / *h;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < count; g += (size_t)gridDim.x * blockDim.x)
        y[g] = x[g] * inv;
}

// *x = sqrt(*x) when positive and finite, else 1 (a norm used as a divisor)
__global__ void k_sqrt_or_one(double* x) {
    pdl_enter();
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const double v = *x;
        *x = (v > 0.0 && isfinite(v)) ? sqrt(v) : 1.0;
    }
}

// The last update of a batched PCG whose residual and residual norm are not
// used again: x = xscale alpha p (assign) or x += xscale alpha p, with the
// per-column alpha of the ColRed scalars (the same arithmetic as the full update).
template <typename T, int VEC>
__global__ void __launch_bounds__(kMaxBlock) k_pcg_xupdate(XUpdateArgs<T> a) {
    pcg_xupdate_body<T, VEC>(a, native_grid());
}
template <typename T, int VEC>
__global__ void __launch_bounds__(kMaxBlock) k_pcg_xupdate_b(const XUpdateArgs<T>* __restrict__ ps, BatchMap m) {
    pdl_enter();
    int i;
    VGrid g;
    if (batch_block(m, i, g)) {
        const auto a_ = ps[i];   // a local copy: no store of the body aliases it
        pcg_xupdate_body<T, VEC>(a_, g);
    }
}

int grid_of(size_t count) {
    const size_t want = (count + kThreads - 1) / kThreads;
    return (int)std::max<size_t>(1, std::min(want, (size_t)num_sms() * 8));
}

}  // namespace

int launch_mdot(size_t count, int k, const double* V, size_t stride, const double* w, double* partials,
                unsigned* counter, double* out, cudaStream_t s) {
    if (k < 1 || k > kMaxKrylovDots) throw Error(PTP_EINVAL, "launch_mdot: 1..32 dot products per launch");
    const dim3 gr(grid_of(count)), bl(kThreads);
    if (k == 1) launch_k(k_mdot<1>, gr, bl, s, count, k, V, stride, w, partials, counter, out);
    else if (k <= 2) launch_k(k_mdot<2>, gr, bl, s, count, k, V, stride, w, partials, counter, out);
    else if (k <= 4) launch_k(k_mdot<4>, gr, bl, s, count, k, V, stride, w, partials, counter, out);
    else if (k <= 8) launch_k(k_mdot<8>, gr, bl, s, count, k, V, stride, w, partials, counter, out);
    else if (k <= 16) launch_k(k_mdot<16>, gr, bl, s, count, k, V, stride, w, partials, counter, out);
    else launch_k(k_mdot<32>, gr, bl, s, count, k, V, stride, w, partials, counter, out);
    return 1;
}

int launch_maxpy(size_t count, int k, const double* V, size_t stride, const double* coef, double sign, double* w,
                 cudaStream_t s) {
    if (k < 1) return 0;
    launch_k(k_maxpy, dim3(grid_of(count)), dim3(kThreads), s, count, k, V, stride, coef, sign, w);
    return 1;
}

int launch_div_scalar(size_t count, const double* x, const double* h, double* y, cudaStream_t s) {
    launch_k(k_div_scalar, dim3(grid_of(count)), dim3(kThreads), s, count, x, h, y);
    return 1;
}

template <typename T>
int launch_pcg_xupdate_batch(const void* args, BatchMap m, int blocks, const KShape& sh, cudaStream_t s) {
    const XUpdateArgs<T>* a = static_cast<const XUpdateArgs<T>*>(args);
    if (sh.vec == 4) {
        if constexpr (sizeof(T) == 4) launch_k(k_pcg_xupdate_b<T, 4>, dim3(blocks), dim3(sh.block), s, a, m);
    } else if (sh.vec == 2) {
        launch_k(k_pcg_xupdate_b<T, 2>, dim3(blocks), dim3(sh.block), s, a, m);
    } else {
        launch_k(k_pcg_xupdate_b<T, 1>, dim3(blocks), dim3(sh.block), s, a, m);
    }
    return 1;
}

template <typename T>
int launch_pcg_xupdate(int rows, int N, T xscale, int assign, T* x, const T* p, ColRed<T> cr, Skip sk,
                       cudaStream_t s) {
    const XUpdateArgs<T> a{rows, N, xscale, assign, x, p, cr.col + S_ALPHA * N, sk};
    auto al = [](const void* q, size_t b) { return ((uintptr_t)q % b) == 0; };
    int vec = 1;
    const void* kern = (const void*)k_pcg_xupdate<T, 1>;
    if (sizeof(T) == 4 && N % 4 == 0 && al(x, 16) && al(p, 16)) {
        vec = 4;
        if constexpr (sizeof(T) == 4) kern = (const void*)k_pcg_xupdate<T, 4>;
    } else if (N % 2 == 0 && al(x, 2 * sizeof(T)) && al(p, 2 * sizeof(T))) {
        vec = 2;
        kern = (const void*)k_pcg_xupdate<T, 2>;
    }
    const Launch l = row_launch(rows, N, vec, kern);
    KShape sh;
    sh.gx = l.grid;
    sh.gy = 1;
    sh.block = l.block;
    sh.vec = vec;
    if (record_launch(launch_pcg_xupdate_batch<T>, a, sh, sizeof(T) == 4 ? body_id(BF_XUPDATE_F, vec, 0) : 0))
        return 1;
    if (vec == 4) {
        if constexpr (sizeof(T) == 4) launch_k(k_pcg_xupdate<T, 4>, dim3(l.grid), dim3(l.block), s, a);
    } else if (vec == 2) {
        launch_k(k_pcg_xupdate<T, 2>, dim3(l.grid), dim3(l.block), s, a);
    } else {
        launch_k(k_pcg_xupdate<T, 1>, dim3(l.grid), dim3(l.block), s, a);
    }
    return 1;
}
template int launch_pcg_xupdate<float>(int, int, float, int, float*, const float*, ColRed<float>, Skip, cudaStream_t);
template int launch_pcg_xupdate<double>(int, int, double, int, double*, const double*, ColRed<double>, Skip,
                                        cudaStream_t);

int launch_sqrt_or_one(double* x, cudaStream_t s) {
    launch_k(k_sqrt_or_one, dim3(1), dim3(32), s, x);
    return 1;
}

}  // namespace ptp
