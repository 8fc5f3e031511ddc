// Sparse kernels on node-major, time-fastest column blocks X[row * N + n].
//
// Every kernel maps a thread to (row, chunk of VEC consecutive columns) so a
// row's N values are read as 16/8-byte vectors and a warp covers a contiguous
// run; the CSR row structure is shared by all threads of the row (L1
// broadcast).  A block holds rpb = 256 / (N / VEC) rows and walks the row
// range with a grid stride, so each thread keeps the same columns and can
// accumulate per-column dot products in registers.  Per-column reductions
// are deterministic: block partials, then the last block to finish (atomic
// ticket, no waiting) sums them in a fixed order and applies the PCG scalar
// update for every column.
//
// Operators are cm * v1 + cl * v2 on a CSR pattern: at time level l the
// spatial block of the periodic system is M + tau_l L (Remark on parallel
// solvers, Section 3), with v1 = M and v2 = L = nu_max * stiffness.
#include <cmath>
#include <map>
#include <mutex>

#include "dev_bodies.cuh"

namespace ptp {

namespace {

// threads per block of the row kernels for launches issued by this host thread
// (each context sets its autotuned value before launching)
thread_local int g_row_block = 256;

// Padded-ELL row with W entries, fully unrolled: every index and value load
// is issued, then every X load, so a row costs two memory round trips
// instead of one per entry.  PERIODIC adds -M X^{n-1} (time shift by one
// column, X^0 = X^N).
template <typename T, int VEC, int W, bool PERIODIC>
__device__ __forceinline__ void row_ell(const Op<T>& op, int N, int row, int col0, const T* X,
                                        T (&acc)[VEC]) {
    int j[W];
    T a[W], m[W];
    const size_t base = (size_t)row * W;
    if constexpr (sizeof(T) == 4) {
        // one 16-byte load per entry: {column, v1, v2, 0}
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const int4 e = __ldg(op.pk + base + k);
            j[k] = e.x;
            m[k] = __int_as_float(e.y);
            a[k] = op.cm * m[k] + op.cl * __int_as_float(e.z);
        }
    } else if (op.ecomb) {
        // double: the combined values are precomputed; M is only needed for the time shift
#pragma unroll
        for (int k = 0; k < W; ++k) {
            j[k] = __ldg(op.eidx + base + k);
            a[k] = __ldg(op.ecomb + base + k);
            if constexpr (PERIODIC) m[k] = __ldg(op.ev1 + base + k);
        }
    } else {
#pragma unroll
        for (int k = 0; k < W; ++k) {
            j[k] = __ldg(op.eidx + base + k);
            m[k] = __ldg(op.ev1 + base + k);
            a[k] = op.cm * m[k];
        }
        if (op.ev2) {
#pragma unroll
            for (int k = 0; k < W; ++k) a[k] += op.cl * __ldg(op.ev2 + base + k);
        }
    }
    T x[W][VEC];
    T xp[W];
    const int cprev = col0 == 0 ? N - 1 : col0 - 1;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const T* xr = X + (size_t)j[k] * N;
        ldg_vec<T, VEC>(xr + col0, x[k]);
        if constexpr (PERIODIC) xp[k] = __ldg(xr + cprev);
    }
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = T(0);
#pragma unroll
    for (int k = 0; k < W; ++k) {
        if constexpr (PERIODIC) {
            T prev = xp[k];
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                acc[v] += a[k] * x[k][v] - m[k] * prev;
                prev = x[k][v];
            }
        } else {
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[v] += a[k] * x[k][v];
        }
    }
}

// CSR row (any width): the fallback for rows wider than 8 entries
template <typename T, int VEC, bool PERIODIC>
__device__ __forceinline__ void row_csr(const Op<T>& op, int N, int row, int col0, const T* X,
                                        T (&acc)[VEC]) {
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = T(0);
    const int k0 = __ldg(op.ptr + row), k1 = __ldg(op.ptr + row + 1);
    const int cprev = col0 == 0 ? N - 1 : col0 - 1;
    for (int k = k0; k < k1; ++k) {
        const int j = __ldg(op.idx + k);
        const T m = __ldg(op.v1 + k);
        T a = op.cm * m;
        if (op.v2) a += op.cl * __ldg(op.v2 + k);
        T x[VEC];
        const T* xr = X + (size_t)j * N;
        ldg_vec<T, VEC>(xr + col0, x);
        if constexpr (PERIODIC) {
            T xp = __ldg(xr + cprev);
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                acc[v] += a * x[v] - m * xp;
                xp = x[v];
            }
        } else {
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[v] += a * x[v];
        }
    }
}

template <typename T, int VEC, bool PERIODIC>
__device__ __forceinline__ void row_dispatch(const Op<T>& op, int N, int row, int col0, const T* X,
                                             T (&acc)[VEC]) {
    switch (op.ell_w) {
        case 2: row_ell<T, VEC, 2, PERIODIC>(op, N, row, col0, X, acc); return;
        case 4: row_ell<T, VEC, 4, PERIODIC>(op, N, row, col0, X, acc); return;
        case 8: row_ell<T, VEC, 8, PERIODIC>(op, N, row, col0, X, acc); return;
        default: row_csr<T, VEC, PERIODIC>(op, N, row, col0, X, acc); return;
    }
}

// acc = (cm v1 + cl v2)[row, :] X[:, col0 .. col0+VEC)
template <typename T, int VEC>
__device__ __forceinline__ void row_apply(const Op<T>& op, int N, int row, int col0, const T* X,
                                          T (&acc)[VEC]) {
    row_dispatch<T, VEC, false>(op, N, row, col0, X, acc);
}

// periodic operator of one row: (cm M + cl L) X^n - M X^{n-1}, X^0 = X^N
template <typename T, int VEC>
__device__ __forceinline__ void row_papply(const Op<T>& op, int N, int row, int col0, const T* X,
                                           T (&acc)[VEC]) {
    row_dispatch<T, VEC, true>(op, N, row, col0, X, acc);
}

// periodic residual of one row: B^n - [(cm M + cl L) X^n - M X^{n-1}]
template <typename T, int VEC>
__device__ __forceinline__ void row_presid(const Op<T>& op, int N, int row, int col0, const T* X,
                                           const T* B, T (&r)[VEC]) {
    T acc[VEC];
    row_papply<T, VEC>(op, N, row, col0, X, acc);
    T b[VEC];
    ldg_vec<T, VEC>(B + (size_t)row * N + col0, b);
#pragma unroll
    for (int v = 0; v < VEC; ++v) r[v] = b[v] - acc[v];
}

template <typename T>
__device__ __forceinline__ T diag_of(const Op<T>& op, int row) {
    if (op.dcomb) return __ldg(op.dcomb + row);
    T d = op.cm * __ldg(op.d1 + row);
    if (op.d2) d += op.cl * __ldg(op.d2 + row);
    return d;
}

template <typename T, int VEC>
__device__ __forceinline__ void fused_sweep(const Aux<T>& aux, int N, int row, int col0, const T (&y)[VEC]) {
    if (!aux.Y2) return;
    T d = aux.cm * __ldg(aux.d1 + row);
    if (aux.d2) d += aux.cl * __ldg(aux.d2 + row);
    const T w = aux.omega / d;
    T o[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) o[v] = w * y[v];
    st_vec<T, VEC>(aux.Y2 + (size_t)row * N + col0, o);
}


// argument structs of the row kernels (one per launch; arrays of them in a batched launch)
template <typename T>
struct SpmmArgs {
    Op<T> op;
    int N;
    const T* X;
    const T* B;
    T* Y;
    T omega;
    Skip sk;
    Aux<T> aux;
};
template <typename T>
struct AlphaArgs {
    Op<T> op;
    int N;
    const T* p;
    T* q;
    ColRed<T> cr;
    Skip sk;
};
template <typename T>
struct UpdateArgs {
    Op<T> op;
    int N;
    T xscale;
    int assign;
    T* x;
    const T* p;
    T* r;
    const T* q;
    T* z;
    ColRed<T> cr;
    Skip sk;
    Aux<T> aux;
};
template <typename T>
struct InitJacArgs {
    Op<T> op;
    int N;
    const T* r;
    T* z;
    T* p;
    ColRed<T> cr;
    Skip sk;
};
template <typename T>
struct DotRzArgs {
    int rows, N;
    const T* r;
    const T* z;
    ColRed<T> cr;
    int first;
    Skip sk;
};
template <typename T>
struct DirArgs {
    int rows, N;
    const T* z;
    T* p;
    ColRed<T> cr;
    Skip sk;
};

template <typename T, int VEC, int MODE>
__device__ __forceinline__ void spmm_body(const SpmmArgs<T>& a_, const VGrid& g_) {
    const Op<T>& op = a_.op;
    const int N = a_.N;
    const T* __restrict__ X = a_.X;
    const T* __restrict__ B = a_.B;
    T* Y = a_.Y;
    const T omega = a_.omega;
    const Skip& sk = a_.sk;
    const Aux<T>& aux = a_.aux;
    pdl_enter();
    if (skip_now(sk)) return;
    const int NC = N / VEC;
    const int rpb = blockDim.x / NC;
    PTP_ROW_LOOP_G(op.rows, NC, rpb, g_) {
        if constexpr (MODE == SP_APPLY || MODE == SP_RESTRICT) {
            T acc[VEC];
            row_apply<T, VEC>(op, N, row, col0, X, acc);
            st_vec<T, VEC>(Y + (size_t)row * N + col0, acc);
            if constexpr (MODE == SP_RESTRICT) fused_sweep<T, VEC>(aux, N, row, col0, acc);
        } else if constexpr (MODE == SP_COPY) {
            T b[VEC];
            ldg_vec<T, VEC>(B + (size_t)row * N + col0, b);
            st_vec<T, VEC>(Y + (size_t)row * N + col0, b);
            fused_sweep<T, VEC>(aux, N, row, col0, b);
        } else if constexpr (MODE == SP_RESID) {
            T acc[VEC], b[VEC];
            row_apply<T, VEC>(op, N, row, col0, X, acc);
            ldg_vec<T, VEC>(B + (size_t)row * N + col0, b);
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[v] = b[v] - acc[v];
            st_vec<T, VEC>(Y + (size_t)row * N + col0, acc);
        } else if constexpr (MODE == SP_JACOBI) {
            T b[VEC], out[VEC];
            ldg_vec<T, VEC>(B + (size_t)row * N + col0, b);
            const T w = omega / diag_of(op, row);
            if (X) {
                T acc[VEC], x[VEC];
                row_apply<T, VEC>(op, N, row, col0, X, acc);
                ldg_vec<T, VEC>(X + (size_t)row * N + col0, x);
#pragma unroll
                for (int v = 0; v < VEC; ++v) out[v] = x[v] + w * (b[v] - acc[v]);
            } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) out[v] = w * b[v];
            }
            st_vec<T, VEC>(Y + (size_t)row * N + col0, out);
        } else if constexpr (MODE == SP_PAPPLY) {
            T acc[VEC];
            row_papply<T, VEC>(op, N, row, col0, X, acc);
            st_vec<T, VEC>(Y + (size_t)row * N + col0, acc);
        } else if constexpr (MODE == SP_PRESID) {
            T r[VEC];
            row_presid<T, VEC>(op, N, row, col0, X, B, r);
            st_vec<T, VEC>(Y + (size_t)row * N + col0, r);
            fused_sweep<T, VEC>(aux, N, row, col0, r);
        } else if constexpr (MODE == SP_PRESID_RESTRICT) {
            T r[VEC];
            row_presid<T, VEC>(op, N, row, col0, X, B, r);
            constexpr int H = VEC / 2;
            T o[H];
#pragma unroll
            for (int v = 0; v < H; ++v) o[v] = r[2 * v] + r[2 * v + 1];
            st_vec<T, H>(Y + (size_t)row * (N / 2) + col0 / 2, o);
        } else if constexpr (MODE == SP_INTERP_ADD) {
            T acc[VEC], y[VEC];
            row_apply<T, VEC>(op, N, row, col0, X, acc);
            T* yp = Y + (size_t)row * N + col0;
            ld_vec<T, VEC>(yp, y);
#pragma unroll
            for (int v = 0; v < VEC; ++v) y[v] += acc[v];
            st_vec<T, VEC>(yp, y);
        }
    }
}

// q = A p ; alpha = rho / (p . q)
template <typename T, int VEC>
__device__ __forceinline__ void apply_alpha_body(const AlphaArgs<T>& a_, const VGrid& g_) {
    const Op<T>& op = a_.op;
    const int N = a_.N;
    const T* __restrict__ p = a_.p;
    T* __restrict__ q = a_.q;
    const ColRed<T>& cr = a_.cr;
    const Skip& sk = a_.sk;
    pdl_enter();
    if (skip_now(sk)) return;
    const int NC = N / VEC, rpb = blockDim.x / NC;
    T acc[1][VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[0][v] = T(0);
    PTP_ROW_LOOP_G(op.rows, NC, rpb, g_) {
        T y[VEC], x[VEC];
        row_apply<T, VEC>(op, N, row, col0, p, y);
        ldg_vec<T, VEC>(p + (size_t)row * N + col0, x);
        st_vec<T, VEC>(q + (size_t)row * N + col0, y);
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[0][v] += x[v] * y[v];
    }
    col_reduce_finish<T, VEC, 1, FIN_ALPHA>(acc, N, NC, rpb, cr, g_);
}

// x += xscale alpha p ; r -= alpha q ; (jacobi) z = r / D ; dots (rz, rr) or (rr)
template <typename T, int VEC, bool JAC>
__device__ __forceinline__ void pcg_update_body(const UpdateArgs<T>& a_, const VGrid& g_) {
    const Op<T>& op = a_.op;
    const int N = a_.N;
    const T xscale = a_.xscale;
    const int assign = a_.assign;
    T* x = a_.x;
    const T* __restrict__ p = a_.p;
    T* r = a_.r;
    const T* __restrict__ q = a_.q;
    T* z = a_.z;
    const ColRed<T>& cr = a_.cr;
    const Skip& sk = a_.sk;
    const Aux<T>& aux = a_.aux;
    pdl_enter();
    if (skip_now(sk)) return;
    const int NC = N / VEC, rpb = blockDim.x / NC;
    constexpr int NQ = JAC ? 2 : 1;
    T acc[NQ][VEC];
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[qq][v] = T(0);
    const T* alpha = cr.col + S_ALPHA * N;
    PTP_ROW_LOOP_G(op.rows, NC, rpb, g_) {
        const size_t o = (size_t)row * N + col0;
        T pv[VEC], qv[VEC], xv[VEC], rv[VEC], al[VEC];
        ldg_vec<T, VEC>(p + o, pv);
        ldg_vec<T, VEC>(q + o, qv);
        if (assign) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) xv[v] = T(0);
        } else {
            ld_vec<T, VEC>(x + o, xv);
        }
        ld_vec<T, VEC>(r + o, rv);
#pragma unroll
        for (int v = 0; v < VEC; ++v) al[v] = alpha[col0 + v];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            xv[v] += xscale * al[v] * pv[v];
            rv[v] -= al[v] * qv[v];
        }
        st_vec<T, VEC>(x + o, xv);
        st_vec<T, VEC>(r + o, rv);
        if constexpr (JAC) {
            const T dinv = T(1) / diag_of(op, row);
            T zv[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                zv[v] = rv[v] * dinv;
                acc[0][v] += rv[v] * zv[v];
                acc[1][v] += rv[v] * rv[v];
            }
            st_vec<T, VEC>(z + o, zv);
        } else {
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[0][v] += rv[v] * rv[v];
            fused_sweep<T, VEC>(aux, N, row, col0, rv);
        }
    }
    col_reduce_finish<T, VEC, NQ, JAC ? FIN_UPDATE_JACOBI : FIN_UPDATE_RR>(acc, N, NC, rpb, cr, g_);
}

// z = r / D ; p = z ; rho = r.z ; bb = rr = r.r
template <typename T, int VEC>
__device__ __forceinline__ void init_jacobi_body(const InitJacArgs<T>& a_, const VGrid& g_) {
    const Op<T>& op = a_.op;
    const int N = a_.N;
    const T* __restrict__ r = a_.r;
    T* __restrict__ z = a_.z;
    T* __restrict__ p = a_.p;
    const ColRed<T>& cr = a_.cr;
    const Skip& sk = a_.sk;
    pdl_enter();
    if (skip_now(sk)) return;
    const int NC = N / VEC, rpb = blockDim.x / NC;
    T acc[2][VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[0][v] = acc[1][v] = T(0);
    PTP_ROW_LOOP_G(op.rows, NC, rpb, g_) {
        const size_t o = (size_t)row * N + col0;
        T rv[VEC], zv[VEC];
        ldg_vec<T, VEC>(r + o, rv);
        const T dinv = T(1) / diag_of(op, row);
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            zv[v] = rv[v] * dinv;
            acc[0][v] += rv[v] * zv[v];
            acc[1][v] += rv[v] * rv[v];
        }
        st_vec<T, VEC>(z + o, zv);
        st_vec<T, VEC>(p + o, zv);
    }
    col_reduce_finish<T, VEC, 2, FIN_RZ_FIRST>(acc, N, NC, rpb, cr, g_);
}

template <typename T, int VEC>
__device__ __forceinline__ void dot_rz_body(const DotRzArgs<T>& a_, const VGrid& g_) {
    const int rows = a_.rows;
    const int N = a_.N;
    const T* __restrict__ r = a_.r;
    const T* __restrict__ z = a_.z;
    const ColRed<T>& cr = a_.cr;
    const int first = a_.first;
    const Skip& sk = a_.sk;
    pdl_enter();
    if (skip_now(sk)) return;
    const int NC = N / VEC, rpb = blockDim.x / NC;
    T acc[2][VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[0][v] = acc[1][v] = T(0);
    PTP_ROW_LOOP_G(rows, NC, rpb, g_) {
        const size_t o = (size_t)row * N + col0;
        T rv[VEC], zv[VEC];
        ldg_vec<T, VEC>(r + o, rv);
        ldg_vec<T, VEC>(z + o, zv);
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            acc[0][v] += rv[v] * zv[v];
            acc[1][v] += rv[v] * rv[v];
        }
    }
    if (first)
        col_reduce_finish<T, VEC, 2, FIN_RZ_FIRST>(acc, N, NC, rpb, cr, g_);
    else
        col_reduce_finish<T, VEC, 2, FIN_RZ_NEXT>(acc, N, NC, rpb, cr, g_);
}

// p = z + beta p
template <typename T, int VEC>
__device__ __forceinline__ void direction_body(const DirArgs<T>& a_, const VGrid& g_) {
    const int rows = a_.rows;
    const int N = a_.N;
    const T* __restrict__ z = a_.z;
    T* p = a_.p;
    const ColRed<T>& cr = a_.cr;
    const Skip& sk = a_.sk;
    pdl_enter();
    if (skip_now(sk)) return;
    const int NC = N / VEC, rpb = blockDim.x / NC;
    const T* beta = cr.col + S_BETA * N;
    PTP_ROW_LOOP_G(rows, NC, rpb, g_) {
        const size_t o = (size_t)row * N + col0;
        T zv[VEC], pv[VEC];
        ldg_vec<T, VEC>(z + o, zv);
        ld_vec<T, VEC>(p + o, pv);
#pragma unroll
        for (int v = 0; v < VEC; ++v) pv[v] = zv[v] + beta[col0 + v] * pv[v];
        st_vec<T, VEC>(p + o, pv);
    }
}


// ---- kernels: one single-instance and one batched entry per body ----
#define PTP_ROW_KERNELS(NAME, BODY, ARGS, TPARAMS, TARGS)                                            \
    template <TPARAMS>                                                                              \
    __global__ void __launch_bounds__(kMaxBlock) NAME(ARGS a) { BODY<TARGS>(a, native_grid()); }    \
    template <TPARAMS>                                                                              \
    __global__ void __launch_bounds__(kMaxBlock) NAME##_b(const ARGS* __restrict__ ps, BatchMap m) { \
        pdl_enter();                                                                                \
        int i;                                                                                      \
        VGrid g;                                                                                    \
        if (batch_block(m, i, g)) {                                                    \
            const auto a_ = ps[i];                                                  \
            BODY<TARGS>(a_, g);                                                     \
        }                                            \
    }
#define PTP_COMMA ,
PTP_ROW_KERNELS(k_spmm, spmm_body, SpmmArgs<T>, typename T PTP_COMMA int VEC PTP_COMMA int MODE, T PTP_COMMA VEC PTP_COMMA MODE)
PTP_ROW_KERNELS(k_pcg_apply_alpha, apply_alpha_body, AlphaArgs<T>, typename T PTP_COMMA int VEC, T PTP_COMMA VEC)
PTP_ROW_KERNELS(k_pcg_update, pcg_update_body, UpdateArgs<T>, typename T PTP_COMMA int VEC PTP_COMMA bool JAC,
                T PTP_COMMA VEC PTP_COMMA JAC)
PTP_ROW_KERNELS(k_pcg_init_jacobi, init_jacobi_body, InitJacArgs<T>, typename T PTP_COMMA int VEC, T PTP_COMMA VEC)
PTP_ROW_KERNELS(k_pcg_dot_rz, dot_rz_body, DotRzArgs<T>, typename T PTP_COMMA int VEC, T PTP_COMMA VEC)
PTP_ROW_KERNELS(k_pcg_direction, direction_body, DirArgs<T>, typename T PTP_COMMA int VEC, T PTP_COMMA VEC)
#undef PTP_ROW_KERNELS
#undef PTP_COMMA

template <typename T>
__global__ void __launch_bounds__(256) k_dense_apply(DenseArgs<T> p) { dense_apply_body<T>(p, native_grid()); }
template <typename T>
__global__ void __launch_bounds__(256) k_dense_apply_b(const DenseArgs<T>* __restrict__ ps, BatchMap m) {
    pdl_enter();
    int i;
    VGrid g;
    if (batch_block(m, i, g)) {
        const auto a_ = ps[i];   // a local copy: no store of the body aliases it
        dense_apply_body<T>(a_, g);
    }
}

template <typename T>
__global__ void k_time_prolong_add(ProlongArgs<T> p) { time_prolong_add_body<T>(p, native_grid()); }
template <typename T>
__global__ void k_time_prolong_add_b(const ProlongArgs<T>* __restrict__ ps, BatchMap m) {
    pdl_enter();
    int i;
    VGrid g;
    if (batch_block(m, i, g)) {
        const auto a_ = ps[i];   // a local copy: no store of the body aliases it
        time_prolong_add_body<T>(a_, g);
    }
}

// VEC consecutive columns n0.. of one node per thread.  The sum runs from
// the coarsest level to the finest, the order of the level-by-level
// prolongations, so U receives the same float value.
template <typename T, int VEC>
__device__ __forceinline__ void prolong_chain_add_body(const ChainAddArgs<T>& p, const VGrid& g) {
    pdl_enter();
    if (skip_now(p.sk)) return;
    const double sc = p.scale ? *p.scale : 1.0;
    const int N = p.N, NC = N / VEC, D = p.D;
    const size_t total = (size_t)p.rows * NC;
    for (size_t q = (size_t)g.bx * blockDim.x + threadIdx.x; q < total; q += (size_t)g.gx * blockDim.x) {
        const size_t i = q / NC;
        const int n0 = (int)(q - i * NC) * VEC;
        T s[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) s[k] = T(0);
#pragma unroll
        for (int l = kMaxChain - 1; l >= 0; --l) {
            if (l > D) continue;
            const T* xl = p.x[l] + i * (size_t)(N >> l);
            T v[VEC];
            if (l == 0) {
                ld_vec<T, VEC>(xl + n0, v);
            } else {
#pragma unroll
                for (int k = 0; k < VEC; ++k) v[k] = xl[(n0 + k) >> l];
            }
#pragma unroll
            for (int k = 0; k < VEC; ++k) s[k] = l == D ? v[k] : v[k] + s[k];
        }
        double* u = p.U + i * (size_t)N + n0;
#pragma unroll
        for (int k = 0; k < VEC; ++k) u[k] += sc * (double)s[k];
    }
}
template <typename T, int VEC>
__global__ void k_prolong_chain_add(ChainAddArgs<T> p) { prolong_chain_add_body<T, VEC>(p, native_grid()); }
template <typename T, int VEC>
__global__ void k_prolong_chain_add_b(const ChainAddArgs<T>* __restrict__ ps, BatchMap m) {
    pdl_enter();
    int i;
    VGrid g;
    if (batch_block(m, i, g)) {
        const auto a_ = ps[i];   // a local copy: no store of the body aliases it
        prolong_chain_add_body<T, VEC>(a_, g);
    }
}

template <typename T>
__device__ __forceinline__ void add_to_double_body(const AddArgs<T>& p, const VGrid& g) {
    pdl_enter();
    if (skip_now(p.sk)) return;
    const double s = p.scale ? *p.scale : 1.0;
    for (size_t q = (size_t)g.bx * blockDim.x + threadIdx.x; q < p.count; q += (size_t)g.gx * blockDim.x)
        p.U[q] += s * (double)p.d[q];
}
template <typename T>
__global__ void k_add_to_double(AddArgs<T> p) { add_to_double_body<T>(p, native_grid()); }
template <typename T>
__global__ void k_add_to_double_b(const AddArgs<T>* __restrict__ ps, BatchMap m) {
    pdl_enter();
    int i;
    VGrid g;
    if (batch_block(m, i, g)) {
        const auto a_ = ps[i];   // a local copy: no store of the body aliases it
        add_to_double_body<T>(a_, g);
    }
}

template <typename T>
__global__ void k_axpy(size_t count, T a, const T* __restrict__ x, T* __restrict__ y, Skip sk) {
    pdl_enter();
    if (skip_now(sk)) return;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < count; g += (size_t)gridDim.x * blockDim.x)
        y[g] += a * x[g];
}

template <typename T>
__global__ void k_fill(size_t count, T v, T* __restrict__ y, Skip sk) {
    pdl_enter();
    if (skip_now(sk)) return;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < count; g += (size_t)gridDim.x * blockDim.x)
        y[g] = v;
}

template <typename TI, typename TO>
__global__ void k_cast(size_t count, const TI* __restrict__ x, TO* __restrict__ y, Skip sk) {
    pdl_enter();
    if (skip_now(sk)) return;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < count; g += (size_t)gridDim.x * blockDim.x)
        y[g] = (TO)x[g];
}

template <typename TI, typename TO>
__global__ void k_cast_scaled(size_t count, const TI* __restrict__ x, TO* __restrict__ y,
                              const double* __restrict__ mul, const double* __restrict__ div) {
    pdl_enter();
    const double s = (mul ? *mul : 1.0) / (div ? *div : 1.0);
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < count; g += (size_t)gridDim.x * blockDim.x)
        y[g] = (TO)(s * (double)x[g]);
}

template <typename T>
__global__ void k_split2(int rows, const T* __restrict__ b, double* __restrict__ bs, double* __restrict__ bd, Skip sk) {
    pdl_enter();
    if (skip_now(sk)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
        const double b0 = (double)b[2 * (size_t)i], b1 = (double)b[2 * (size_t)i + 1];
        bs[i] = b0 + b1;
        bd[i] = b0 - b1;
    }
}

template <typename T>
__global__ void k_combine2(int rows, const double* __restrict__ xs, const double* __restrict__ xd, T* __restrict__ x,
                           Skip sk) {
    pdl_enter();
    if (skip_now(sk)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
        x[2 * (size_t)i] = (T)(0.5 * (xs[i] + xd[i]));
        x[2 * (size_t)i + 1] = (T)(0.5 * (xs[i] - xd[i]));
    }
}

__global__ void k_flag(int* flag, int v, Skip sk) {
    pdl_enter();
    if (skip_now(sk)) return;
    if (threadIdx.x == 0 && blockIdx.x == 0) *flag = v;
}

template <typename T>
__global__ void k_norm2(size_t count, const T* __restrict__ x, double* partials, unsigned* counter, double* out) {
    pdl_enter();
    double s = 0.0;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < count; g += (size_t)gridDim.x * blockDim.x) {
        const double v = (double)x[g];
        s += v * v;
    }
    __shared__ double sm[kMaxBlock];
    __shared__ bool last;
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = sm[0];
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(partials + b);
        *out = t;
        *counter = 0u;
    }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------

inline bool aligned(const void* p, size_t a) { return p == nullptr || ((uintptr_t)p % a) == 0; }

template <typename T>
int pick_vec(int N, std::initializer_list<const void*> ptrs, bool need_even = false) {
    int vmax = sizeof(T) == 4 ? 4 : 2;
    for (int v = vmax; v >= 1; v /= 2) {
        if (N % v) continue;
        if (need_even && v < 2) continue;
        bool ok = true;
        for (const void* p : ptrs) ok = ok && aligned(p, v * sizeof(T));
        if (need_even && v == 4 && N % 4) ok = false;
        if (ok) return v;
    }
    if (need_even) throw Error(PTP_EINVAL, "time restriction needs an even number of steps and aligned buffers");
    return 1;
}


// resident blocks per SM of `kernel` at `block` threads (cached per kernel)
int blocks_per_sm(const void* kernel, int block) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair(kernel, block);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, block, 0) != cudaSuccess || nb < 1) nb = 1;
    cache[key] = nb;
    return nb;
}


int flat_grid(size_t total) {
    size_t want = (total + 255) / 256;
    size_t cap = (size_t)num_sms() * 8;
    return (int)std::max<size_t>(1, std::min(want, cap));
}

}  // namespace

Launch row_launch(int rows, int N, int vec, const void* kernel) {
    const int NC = N / vec;
    if (NC > kMaxBlock) throw Error(PTP_EINVAL, "too many time steps per level for one block (N/VEC > 512)");
    const int target = std::max(g_row_block, NC);
    const int rpb = std::max(1, target / NC);
    const int block = NC * rpb;
    long groups = ((long)rows + rpb - 1) / rpb;
    // one full wave: grid-stride loops cover the rest (no partial second wave)
    long cap = (long)num_sms() * std::min(8, blocks_per_sm(kernel, block));
    Launch l;
    l.grid = (int)std::max(1L, std::min(groups, cap));
    l.block = block;
    return l;
}

__global__ void k_lincomb(size_t n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                          double* __restrict__ out) {
    pdl_enter();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

void launch_lincomb(size_t n, double a, const double* x, double b, const double* y, double* out, cudaStream_t s) {
    if (n == 0) return;
    launch_k(k_lincomb, dim3(flat_grid(n)), dim3(256), s, n, a, x, b, y, out);
}

void set_row_block(int threads) {
    g_row_block = std::min(kMaxBlock, std::max(64, threads));
}

// max partial-buffer entries a reduction launch can need for N columns
size_t reduction_partials(int Nmax) { return (size_t)num_sms() * 9 * 2 * (size_t)Nmax; }

#define PTP_VEC_DISPATCH(vec, ...)                               \
    switch (vec) {                                               \
        case 4: { constexpr int VEC = 4; __VA_ARGS__; } break;   \
        case 2: { constexpr int VEC = 2; __VA_ARGS__; } break;   \
        default: { constexpr int VEC = 1; __VA_ARGS__; } break;  \
    }

// launch shape of a row kernel as a KShape (variant: the template's mode)
template <typename... KArgs>
KShape row_shape(void (*kernel)(KArgs...), int rows, int N, int vec, int variant) {
    const Launch l = row_launch(rows, N, vec, (const void*)kernel);
    KShape sh;
    sh.gx = l.grid;
    sh.gy = 1;
    sh.block = l.block;
    sh.vec = vec;
    sh.variant = variant;
    return sh;
}

// recorded for a batched step, else launched
template <typename A, typename... KArgs>
void row_go(void (*kernel)(KArgs...), BatchLaunch bfn, int rows, int N, int vec, int variant, cudaStream_t s,
            const A& a) {
    const KShape sh = row_shape(kernel, rows, N, vec, variant);
    if (record_launch(bfn, a, sh)) return;
    launch_k(kernel, dim3(sh.gx), dim3(sh.block), s, a);
}

// batched launch of a row-kernel family: VEC from the shape (4 only in float;
// the time restriction needs VEC >= 2)
#define PTP_ROW_BATCH(FN, KB, ARGS, TPARAMS, ...)                                                   \
    template <TPARAMS>                                                                              \
    int FN(const void* args, BatchMap m, int blocks, const KShape& sh, cudaStream_t s) {             \
        const ARGS* a = static_cast<const ARGS*>(args);                                             \
        const dim3 g(blocks), b(sh.block);                                                          \
        if (sh.vec == 4) {                                                                          \
            if constexpr (sizeof(T) == 4) launch_k(KB<T, 4, ##__VA_ARGS__>, g, b, s, a, m);         \
        } else if (sh.vec == 2) {                                                                   \
            launch_k(KB<T, 2, ##__VA_ARGS__>, g, b, s, a, m);                                       \
        } else {                                                                                    \
            one_vec<T>(KB<T, 1, ##__VA_ARGS__>, g, b, s, a, m);                                     \
        }                                                                                           \
        return 1;                                                                                   \
    }

template <typename T, typename... KArgs, typename... Args>
void one_vec(void (*kernel)(KArgs...), dim3 g, dim3 b, cudaStream_t s, Args&&... args) {
    launch_k(kernel, g, b, s, std::forward<Args>(args)...);
}

#define PTP_COMMA ,
PTP_ROW_BATCH(alpha_batch, k_pcg_apply_alpha_b, AlphaArgs<T>, typename T)
PTP_ROW_BATCH(init_jacobi_batch, k_pcg_init_jacobi_b, InitJacArgs<T>, typename T)
PTP_ROW_BATCH(dot_rz_batch, k_pcg_dot_rz_b, DotRzArgs<T>, typename T)
PTP_ROW_BATCH(direction_batch, k_pcg_direction_b, DirArgs<T>, typename T)
PTP_ROW_BATCH(update_batch, k_pcg_update_b, UpdateArgs<T>, typename T PTP_COMMA bool JAC, JAC)
#undef PTP_COMMA
#undef PTP_ROW_BATCH

template <typename T, int MODE>
int spmm_batch(const void* args, BatchMap m, int blocks, const KShape& sh, cudaStream_t s) {
    const SpmmArgs<T>* a = static_cast<const SpmmArgs<T>*>(args);
    const dim3 g(blocks), b(sh.block);
    if (sh.vec == 4) {
        if constexpr (sizeof(T) == 4) launch_k(k_spmm_b<T, 4, MODE>, g, b, s, a, m);
    } else if (sh.vec == 2) {
        launch_k(k_spmm_b<T, 2, MODE>, g, b, s, a, m);
    } else {
        if constexpr (MODE != SP_PRESID_RESTRICT) launch_k(k_spmm_b<T, 1, MODE>, g, b, s, a, m);
    }
    return 1;
}

template <typename T, int MODE>
void spmm_go(const SpmmArgs<T>& a, int vec, cudaStream_t s) {
    const int rows = a.op.rows, N = a.N;
    if (vec == 4) {
        if constexpr (sizeof(T) == 4) row_go(k_spmm<T, 4, MODE>, spmm_batch<T, MODE>, rows, N, 4, MODE, s, a);
    } else if (vec == 2) {
        row_go(k_spmm<T, 2, MODE>, spmm_batch<T, MODE>, rows, N, 2, MODE, s, a);
    } else {
        if constexpr (MODE != SP_PRESID_RESTRICT) row_go(k_spmm<T, 1, MODE>, spmm_batch<T, MODE>, rows, N, 1, MODE, s, a);
    }
}

template <typename T>
int launch_spmm(SpMode mode, const Op<T>& op, int N, const T* X, const T* B, T* Y, T omega, Skip sk,
                cudaStream_t s, Aux<T> aux) {
    const bool restrict_time = mode == SP_PRESID_RESTRICT;
    int vec = pick_vec<T>(N, {X, B, Y, aux.Y2}, restrict_time);
    if (sizeof(T) == 8 && vec == 4) vec = 2;
    if (restrict_time && sizeof(T) == 4 && vec == 4 && !aligned(Y, 8)) vec = 2;
    const SpmmArgs<T> a{op, N, X, B, Y, omega, sk, aux};
    switch (mode) {
        case SP_APPLY: spmm_go<T, SP_APPLY>(a, vec, s); break;
        case SP_RESID: spmm_go<T, SP_RESID>(a, vec, s); break;
        case SP_JACOBI: spmm_go<T, SP_JACOBI>(a, vec, s); break;
        case SP_PRESID: spmm_go<T, SP_PRESID>(a, vec, s); break;
        case SP_PRESID_RESTRICT: spmm_go<T, SP_PRESID_RESTRICT>(a, vec, s); break;
        case SP_INTERP_ADD: spmm_go<T, SP_INTERP_ADD>(a, vec, s); break;
        case SP_RESTRICT: spmm_go<T, SP_RESTRICT>(a, vec, s); break;
        case SP_PAPPLY: spmm_go<T, SP_PAPPLY>(a, vec, s); break;
        case SP_COPY: spmm_go<T, SP_COPY>(a, vec, s); break;
    }
    return 1;
}

// the PCG row kernels: vec 4 (float) / 2 / 1 as for the SpMM
#define PTP_ROW_GO(K, BATCH, ROWS, VARIANT, ...)                                                   \
    if (vec == 4) {                                                                                 \
        if constexpr (sizeof(T) == 4) row_go(K<T, 4, ##__VA_ARGS__>, BATCH, ROWS, N, 4, VARIANT, s, a); \
    } else if (vec == 2) {                                                                          \
        row_go(K<T, 2, ##__VA_ARGS__>, BATCH, ROWS, N, 2, VARIANT, s, a);                           \
    } else {                                                                                        \
        row_go(K<T, 1, ##__VA_ARGS__>, BATCH, ROWS, N, 1, VARIANT, s, a);                           \
    }

template <typename T>
int launch_pcg_init_jacobi(const Op<T>& op, int N, T* r, T* z, T* p, ColRed<T> cr, Skip sk, cudaStream_t s) {
    int vec = pick_vec<T>(N, {r, z, p});
    if (sizeof(T) == 8 && vec == 4) vec = 2;
    const InitJacArgs<T> a{op, N, r, z, p, cr, sk};
    PTP_ROW_GO(k_pcg_init_jacobi, init_jacobi_batch<T>, op.rows, 0)
    return 1;
}

template <typename T>
int launch_pcg_dot_rz(int rows, int N, const T* r, const T* z, ColRed<T> cr, int first, Skip sk, cudaStream_t s) {
    int vec = pick_vec<T>(N, {r, z});
    if (sizeof(T) == 8 && vec == 4) vec = 2;
    const DotRzArgs<T> a{rows, N, r, z, cr, first, sk};
    PTP_ROW_GO(k_pcg_dot_rz, dot_rz_batch<T>, rows, 0)
    return 1;
}

template <typename T>
int launch_pcg_apply_alpha(const Op<T>& op, int N, const T* p, T* q, ColRed<T> cr, Skip sk, cudaStream_t s) {
    int vec = pick_vec<T>(N, {p, q});
    if (sizeof(T) == 8 && vec == 4) vec = 2;
    const AlphaArgs<T> a{op, N, p, q, cr, sk};
    PTP_ROW_GO(k_pcg_apply_alpha, alpha_batch<T>, op.rows, 0)
    return 1;
}

template <typename T>
int launch_pcg_update(const Op<T>& op, int N, T xscale, int assign, T* x, const T* p, T* r, const T* q, T* z,
                      int jacobi, ColRed<T> cr, Skip sk, cudaStream_t s, Aux<T> aux) {
    int vec = pick_vec<T>(N, {x, p, r, q, z, aux.Y2});
    if (sizeof(T) == 8 && vec == 4) vec = 2;
    const UpdateArgs<T> a{op, N, xscale, assign, x, p, r, q, z, cr, sk, aux};
    if (jacobi) {
        PTP_ROW_GO(k_pcg_update, (update_batch<T, true>), op.rows, 1, true)
    } else {
        PTP_ROW_GO(k_pcg_update, (update_batch<T, false>), op.rows, 0, false)
    }
    return 1;
}

template <typename T>
int launch_pcg_direction(int rows, int N, const T* z, T* p, ColRed<T> cr, Skip sk, cudaStream_t s) {
    int vec = pick_vec<T>(N, {z, p});
    if (sizeof(T) == 8 && vec == 4) vec = 2;
    const DirArgs<T> a{rows, N, z, p, cr, sk};
    PTP_ROW_GO(k_pcg_direction, direction_batch<T>, rows, 0)
    return 1;
}
#undef PTP_ROW_GO

// raises a kernel's dynamic shared memory limit to smem once per size
template <typename... KArgs>
void grant_smem(void (*kernel)(KArgs...), size_t smem) {
    ensure_dynamic_smem((const void*)kernel, smem);
}

template <typename T>
int launch_dense_apply_batch(const void* args, BatchMap m, int blocks, const KShape& sh, cudaStream_t s) {
    grant_smem(k_dense_apply_b<T>, sh.smem);
    launch_k_smem(k_dense_apply_b<T>, dim3(blocks), dim3(256), sh.smem, s, static_cast<const DenseArgs<T>*>(args),
                  m);
    return 1;
}

template <typename T>
int launch_dense_apply(int n, int N, const T* Ainv, const T* B, T* Y, Skip sk, cudaStream_t s) {
    const int kc = dense_chunk<T>(n);
    const DenseArgs<T> a{n, N, kc, Ainv, B, Y, sk};
    KShape sh;
    sh.gx = (N + kDT - 1) / kDT;
    sh.gy = (n + kDR - 1) / kDR;
    sh.block = 256;
    sh.smem = dense_smem<T>(kc);
    if (record_launch(launch_dense_apply_batch<T>, a, sh, sizeof(T) == 4 ? body_id(BF_DENSE_F, 0, 0) : 0)) return 1;
    grant_smem(k_dense_apply<T>, sh.smem);
    launch_k_smem(k_dense_apply<T>, dim3(sh.gx, sh.gy), dim3(256), sh.smem, s, a);
    return 1;
}

template <typename T>
int launch_time_prolong_add_batch(const void* args, BatchMap m, int blocks, const KShape&, cudaStream_t s) {
    launch_k(k_time_prolong_add_b<T>, dim3(blocks), dim3(256), s, static_cast<const ProlongArgs<T>*>(args), m);
    return 1;
}

template <typename T>
int launch_time_prolong_add(int rows, int Nc, const T* xc, T* x, Skip sk, cudaStream_t s) {
    const ProlongArgs<T> a{rows, Nc, xc, x, sk};
    KShape sh;
    sh.gx = flat_grid((size_t)rows * Nc);
    sh.gy = 1;
    sh.block = 256;
    if (record_launch(launch_time_prolong_add_batch<T>, a, sh, sizeof(T) == 4 ? body_id(BF_PROLONG_F, 0, 0) : 0))
        return 1;
    launch_k(k_time_prolong_add<T>, dim3(sh.gx), 256, s, a);
    return 1;
}

template <typename T>
int launch_axpy(size_t count, T a, const T* x, T* y, Skip sk, cudaStream_t s) {
    launch_k(k_axpy<T>, flat_grid(count), 256, s, count, a, x, y, sk);
    return 1;
}

template <typename T>
int launch_fill(size_t count, T v, T* y, Skip sk, cudaStream_t s) {
    launch_k(k_fill<T>, flat_grid(count), 256, s, count, v, y, sk);
    return 1;
}

template <typename TI, typename TO>
int launch_cast(size_t count, const TI* x, TO* y, Skip sk, cudaStream_t s) {
    launch_k(k_cast<TI, TO>, flat_grid(count), 256, s, count, x, y, sk);
    return 1;
}

template <typename T>
int launch_add_to_double_batch(const void* args, BatchMap m, int blocks, const KShape&, cudaStream_t s) {
    launch_k(k_add_to_double_b<T>, dim3(blocks), dim3(256), s, static_cast<const AddArgs<T>*>(args), m);
    return 1;
}

template <typename T>
int launch_add_to_double(size_t count, const T* d, double* U, const double* scale, Skip sk, cudaStream_t s) {
    const AddArgs<T> a{count, d, U, scale, sk};
    KShape sh;
    sh.gx = flat_grid(count);
    sh.gy = 1;
    sh.block = 256;
    if (record_launch(launch_add_to_double_batch<T>, a, sh)) return 1;
    launch_k(k_add_to_double<T>, dim3(sh.gx), 256, s, a);
    return 1;
}

template <typename T>
int launch_prolong_chain_add_batch(const void* args, BatchMap m, int blocks, const KShape& sh, cudaStream_t s) {
    const auto* a = static_cast<const ChainAddArgs<T>*>(args);
    if (sh.vec == 4) launch_k(k_prolong_chain_add_b<T, 4>, dim3(blocks), dim3(256), s, a, m);
    else launch_k(k_prolong_chain_add_b<T, 1>, dim3(blocks), dim3(256), s, a, m);
    return 1;
}

template <typename T>
int launch_prolong_chain_add(int rows, int N, int D, const T* const* x, double* U, const double* scale, Skip sk,
                             cudaStream_t s) {
    PTP_REQUIRE(D >= 0 && D < kMaxChain && (N >> D) << D == N, "prolongation chain: bad level count");
    ChainAddArgs<T> a{};
    a.rows = rows;
    a.N = N;
    a.D = D;
    for (int l = 0; l <= D; ++l) a.x[l] = x[l];
    a.U = U;
    a.scale = scale;
    a.sk = sk;
    const bool v4 = N % 4 == 0 && ((uintptr_t)x[0] % (4 * sizeof(T))) == 0;
    KShape sh;
    sh.gx = flat_grid((size_t)rows * (N / (v4 ? 4 : 1)));
    sh.gy = 1;
    sh.block = 256;
    sh.vec = v4 ? 4 : 1;
    if (record_launch(launch_prolong_chain_add_batch<T>, a, sh)) return 1;
    if (v4) launch_k(k_prolong_chain_add<T, 4>, dim3(sh.gx), 256, s, a);
    else launch_k(k_prolong_chain_add<T, 1>, dim3(sh.gx), 256, s, a);
    return 1;
}

template <typename TI, typename TO>
int launch_cast_scaled(size_t count, const TI* x, TO* y, const double* mul, const double* div, cudaStream_t s) {
    launch_k(k_cast_scaled<TI, TO>, flat_grid(count), 256, s, count, x, y, mul, div);
    return 1;
}

template <typename T>
int launch_split2(int rows, const T* b, double* bs, double* bd, Skip sk, cudaStream_t s) {
    launch_k(k_split2<T>, flat_grid(rows), 256, s, rows, b, bs, bd, sk);
    return 1;
}

template <typename T>
int launch_combine2(int rows, const double* xs, const double* xd, T* x, Skip sk, cudaStream_t s) {
    launch_k(k_combine2<T>, flat_grid(rows), 256, s, rows, xs, xd, x, sk);
    return 1;
}

int launch_flag(int* flag, int v, Skip sk, cudaStream_t s) {
    launch_k(k_flag, 1, 32, s, flag, v, sk);
    return 1;
}

template <typename T>
int launch_norm2(size_t count, const T* x, double* partials, unsigned* counter, double* out, cudaStream_t s) {
    launch_k(k_norm2<T>, flat_grid(count), 256, s, count, x, partials, counter, out);
    return 1;
}

#define PTP_INST(T)                                                                                        \
    template int launch_spmm<T>(SpMode, const Op<T>&, int, const T*, const T*, T*, T, Skip, cudaStream_t, Aux<T>); \
    template int launch_pcg_init_jacobi<T>(const Op<T>&, int, T*, T*, T*, ColRed<T>, Skip, cudaStream_t);  \
    template int launch_pcg_dot_rz<T>(int, int, const T*, const T*, ColRed<T>, int, Skip, cudaStream_t);   \
    template int launch_pcg_apply_alpha<T>(const Op<T>&, int, const T*, T*, ColRed<T>, Skip, cudaStream_t); \
    template int launch_pcg_update<T>(const Op<T>&, int, T, int, T*, const T*, T*, const T*, T*, int, ColRed<T>, \
                                      Skip, cudaStream_t, Aux<T>);                                         \
    template int launch_pcg_direction<T>(int, int, const T*, T*, ColRed<T>, Skip, cudaStream_t);          \
    template int launch_dense_apply<T>(int, int, const T*, const T*, T*, Skip, cudaStream_t);              \
    template int launch_time_prolong_add<T>(int, int, const T*, T*, Skip, cudaStream_t);                   \
    template int launch_axpy<T>(size_t, T, const T*, T*, Skip, cudaStream_t);                              \
    template int launch_fill<T>(size_t, T, T*, Skip, cudaStream_t);                                        \
    template int launch_add_to_double<T>(size_t, const T*, double*, const double*, Skip, cudaStream_t);    \
    template int launch_prolong_chain_add<T>(int, int, int, const T* const*, double*, const double*, Skip,    \
                                             cudaStream_t);                                                   \
    template int launch_split2<T>(int, const T*, double*, double*, Skip, cudaStream_t);                    \
    template int launch_combine2<T>(int, const double*, const double*, T*, Skip, cudaStream_t);            \
    template int launch_norm2<T>(size_t, const T*, double*, unsigned*, double*, cudaStream_t);

PTP_INST(float)
PTP_INST(double)
template int launch_cast<double, float>(size_t, const double*, float*, Skip, cudaStream_t);
template int launch_cast<float, double>(size_t, const float*, double*, Skip, cudaStream_t);
template int launch_cast_scaled<double, float>(size_t, const double*, float*, const double*, const double*,
                                               cudaStream_t);
template int launch_cast_scaled<float, double>(size_t, const float*, double*, const double*, const double*,
                                               cudaStream_t);

}  // namespace ptp
