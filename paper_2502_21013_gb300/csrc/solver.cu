// Host orchestration of the hot path (all work runs in the kernels of
// k_residual.cu and k_sparse.cu):
//
//   outer step k (fixed point of eq. iter1-iter2 in correction form)
//     R = F - A(U^k), ||R||, stopping rule          (K1, double)
//     b = tau R
//     x = V-cycle(s) of multigrid in time on  (M + tau L) x^n - M x^{n-1} = b^n,  x^0 = x^N
//     U^{k+1} = U^k + x                             (double)
//
//   multigrid in time, level l (N_l steps, tau_l = T/N_l):
//     damped block-Jacobi sweeps  x += w_t (M + tau_l L)^{-1} (b + M x^{n-1} - (M + tau_l L) x^n),
//       each spatial solve = batched PCG over the N_l columns (Jacobi or GMG preconditioned)
//     residual restricted to N_l/2 steps by summing pairs (2m, 2m+1)
//     coarse correction prolongated by injection to both steps of the pair
//     coarsest level N_c = 1: tau_c L x = b;  N_c = 2: sum / difference split into
//       tau_c L s = b^0 + b^1 and (2M + tau_c L) d = b^0 - b^1, both SPD, PCG in double.
//
// With piecewise-constant prolongation P and restriction P^T the Galerkin
// coarse operator of the level-l periodic operator is exactly the level-(l+1)
// operator with tau_{l+1} = 2 tau_l, so coarse levels are rediscretisations.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "kernels.h"

namespace ptp {

size_t reduction_partials(int Nmax);
int residual_grid(size_t total);

Ctx::~Ctx() {
    for (auto& g : graph_exec)
        if (g) cudaGraphExecDestroy(g);
    if (newton_exec) cudaGraphExecDestroy(newton_exec);
    if (h_status) cudaFreeHost(h_status);
    if (own_stream) cudaStreamDestroy(own_stream);
}

namespace {

// per-iron-element constants of the exponential law, or null for the saturating law
const double* law_data(const Ctx& c) { return c.law_exp ? c.e_law.p : nullptr; }

// device-to-device copy inside a step (foreign work while a batched step is recorded)
static void copy_async(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    if (record_foreign()) return;
    PTP_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st));
}

template <typename T> T* wbuf(Ctx& c, int k);
template <> double* wbuf<double>(Ctx& c, int k) { return c.w_d[k].p; }
template <> float* wbuf<float>(Ctx& c, int k) { return c.w_f[k].p; }

template <typename T> T* gx(Ctx& c, int s);
template <typename T> T* gb(Ctx& c, int s);
template <typename T> T* gr(Ctx& c, int s);
template <> double* gx<double>(Ctx& c, int s) { return c.g_xd[s].p; }
template <> double* gb<double>(Ctx& c, int s) { return c.g_bd[s].p; }
template <> double* gr<double>(Ctx& c, int s) { return c.g_rd[s].p; }
template <> float* gx<float>(Ctx& c, int s) { return c.g_xf[s].p; }
template <> float* gb<float>(Ctx& c, int s) { return c.g_bf[s].p; }
template <> float* gr<float>(Ctx& c, int s) { return c.g_rf[s].p; }

template <typename T> T* mgx(Ctx& c, int l);
template <typename T> T* mgb(Ctx& c, int l);
template <> double* mgx<double>(Ctx& c, int l) { return c.mg_xd[l].p; }
template <> double* mgb<double>(Ctx& c, int l) { return c.mg_bd[l].p; }
template <> float* mgx<float>(Ctx& c, int l) { return c.mg_xf[l].p; }
template <> float* mgb<float>(Ctx& c, int l) { return c.mg_bf[l].p; }

template <typename T>
Op<T> make_op(const DevCSR& d, double cm, double cl) {
    Op<T> o;
    o.rows = d.rows;
    o.cols = d.cols;
    o.ptr = d.ptr.p;
    o.idx = d.idx.p;
    if constexpr (sizeof(T) == 8) {
        o.v1 = d.v1d.p; o.v2 = d.v2d.p; o.d1 = d.d1d.p; o.d2 = d.d2d.p;
        o.ev1 = d.e1d.p; o.ev2 = d.e2d.p;
    } else {
        o.v1 = d.v1f.p; o.v2 = d.v2f.p; o.d1 = d.d1f.p; o.d2 = d.d2f.p;
        o.ev1 = d.e1f.p; o.ev2 = d.e2f.p;
    }
    o.ell_w = d.ell_w;
    o.eidx = d.eidx.p;
    o.pk = sizeof(T) == 4 ? d.pk.p : nullptr;
    o.cm = (T)cm;
    o.cl = (T)cl;
    return o;
}

// operator cm M + cl L of op pair opi on spatial level s (double: precombined values)
template <typename T>
Op<T> level_op(Ctx& c, int s, int opi) {
    const OpPair& p = c.ops[opi];
    Op<T> o = make_op<T>(c.sl[s].op, p.cm, p.cl);
    if constexpr (sizeof(T) == 8) {
        if (s < (int)p.comb.size()) {
            o.ecomb = p.comb[s].p;
            o.dcomb = p.dcomb[s].p;
        }
    }
    return o;
}

template <typename T>
ColRed<T> make_cr(Ctx& c) {
    ColRed<T> r;
    if constexpr (sizeof(T) == 8) {
        r.partials = c.part_d.p;
        r.capacity = c.part_d.n;
        r.col = c.col_d.p;
    } else {
        r.partials = c.part_f.p;
        r.capacity = c.part_f.n;
        r.col = c.col_f.p;
    }
    r.counter = c.counter.p;
    return r;
}

bool use_gmg(const Ctx& c) {
    return c.opts.spatial_prec == PTP_PREC_GMG &&
           (c.sl.size() > 1 || c.ops[0].inv_d.p != nullptr);
}

// The float inner solve runs the structured-grid stencil kernels
// (k_stencil.cu): every spatial level has its 7-point stencil, GMG with one
// sweep per level, and the option is on.
template <typename T>
bool use_stencil(const Ctx& c) {
    if constexpr (sizeof(T) != 4) {
        return false;
    } else {
        return c.stencil_ok && c.opts.stencil != 0 && use_gmg(c) && std::max(1, c.opts.gmg_smooth) == 1;
    }
}

// operator cm M + cl L of op pair opi on spatial level s as a stencil
StencilOp<float> st_op(const Ctx& c, int s, int opi) {
    StencilOp<float> o;
    o.W = c.sl[s].nx - 2;
    o.H = c.sl[s].ny - 2;
    o.coef = c.sl[s].st_coef.p;
    o.acoef = c.ops[opi].st_a[s].p;
    o.cm = (float)c.ops[opi].cm;
    o.cl = (float)c.ops[opi].cl;
    return o;
}

// Aux for a fused first damped-Jacobi sweep of spatial level s under op pair opi
template <typename T>
Aux<T> sweep_aux(Ctx& c, int s, int opi, T* Y2) {
    Aux<T> a;
    const DevCSR& d = c.sl[s].op;
    if constexpr (sizeof(T) == 8) {
        a.d1 = d.d1d.p;
        a.d2 = d.d2d.p;
    } else {
        a.d1 = d.d1f.p;
        a.d2 = d.d2f.p;
    }
    a.cm = (T)c.ops[opi].cm;
    a.cl = (T)c.ops[opi].cl;
    a.omega = (T)c.opts.gmg_omega;
    a.Y2 = Y2;
    return a;
}

// Spatial geometric-multigrid V-cycle for (cm M + cl L) on N columns:
// z = V(b).  Damped-Jacobi pre/post sweeps (symmetric), Galerkin coarse
// operators, dense inverse on the coarsest level.  The first pre-smoothing
// sweep of a level starts from zero, x = w D^-1 b, which is pointwise: it is
// fused into the kernel that produces b (the restriction for coarser levels;
// for level 0 the caller's producer of b0 when first_done).  Returns the
// buffer that holds z (xa or xb).
template <typename T>
T* gmg_vcycle(Ctx& c, int opi, int N, const T* b0, T* xa, T* xb, Skip sk, bool first_done, int dots = 0);

// The same V-cycle with the stencil kernels: the residual and its
// restriction in one pass per level (with the coarse level's first sweep),
// the interpolation and the post-smoothing sweep in one pass per level, and
// on the finest level the PCG dot products of b0 and z (dots 1: rho, bb, rr;
// dots 2: beta, rho) in that same pass.
float* gmg_vcycle_stencil(Ctx& c, int opi, int N, const float* b0, float* xa, float* xb, Skip sk, bool first_done,
                          int dots) {
    const int S = (int)c.sl.size();
    const float w = (float)c.opts.gmg_omega;
    cudaStream_t st = c.stream;
    std::vector<const float*> b(S);
    std::vector<float*> cur(S), oth(S);
    b[0] = b0;
    cur[0] = xa;
    oth[0] = xb;
    for (int s = 1; s < S; ++s) {
        b[s] = gb<float>(c, s);
        cur[s] = gx<float>(c, s);
        oth[s] = gr<float>(c, s);
    }
    if (!first_done) {
        Op<float> A = level_op<float>(c, 0, opi);
        c.launches += launch_spmm<float>(SP_JACOBI, A, N, nullptr, b[0], cur[0], w, sk, st);
    }
    for (int s = 0; s < S - 1; ++s) {
        // the next level's first sweep rides on the restriction unless it is the dense level
        float* x_next = (s + 1 < S - 1) ? cur[s + 1] : nullptr;
        c.launches += launch_st_resid_restrict(st_op(c, s, opi), st_op(c, s + 1, opi), N, cur[s], b[s],
                                               const_cast<float*>(b[s + 1]), x_next, w, sk, st);
    }
    {
        const int s = S - 1;
        const float* inv = c.ops[opi].inv_f.p;
        if (inv) {
            c.launches += launch_dense_apply<float>(c.sl[s].n, N, inv, b[s], cur[s], sk, st);
        } else {
            Op<float> A = level_op<float>(c, s, opi);
            c.launches += launch_spmm<float>(SP_JACOBI, A, N, nullptr, b[s], cur[s], w, sk, st);
            for (int k = 1; k < 4; ++k) {
                c.launches += launch_spmm<float>(SP_JACOBI, A, N, cur[s], b[s], oth[s], w, sk, st);
                std::swap(cur[s], oth[s]);
            }
        }
    }
    ColRed<float> cr = make_cr<float>(c);
    for (int s = S - 2; s >= 0; --s) {
        const int d = s == 0 ? dots : 0;
        c.launches += launch_st_interp_sweep(st_op(c, s, opi), c.sl[s + 1].nx - 2, c.sl[s + 1].ny - 2, N, cur[s + 1],
                                             cur[s], b[s], oth[s], w, cr, d, sk, st);
        std::swap(cur[s], oth[s]);
    }
    return cur[0];
}

template <typename T>
T* gmg_vcycle(Ctx& c, int opi, int N, const T* b0, T* xa, T* xb, Skip sk, bool first_done, int dots) {
    if constexpr (sizeof(T) == 4) {
        if (use_stencil<T>(c)) return gmg_vcycle_stencil(c, opi, N, b0, xa, xb, sk, first_done, dots);
    }
    if (dots) throw Error(PTP_EINVAL, "fused dot products need the stencil V-cycle");
    const int S = (int)c.sl.size();
    const double cm = c.ops[opi].cm, cl = c.ops[opi].cl;
    const int nu = std::max(1, c.opts.gmg_smooth);
    const T w = (T)c.opts.gmg_omega;
    cudaStream_t st = c.stream;
    std::vector<const T*> b(S);
    std::vector<T*> cur(S), oth(S);
    b[0] = b0;
    cur[0] = xa;
    oth[0] = xb;
    for (int s = 1; s < S; ++s) {
        b[s] = gb<T>(c, s);
        cur[s] = gx<T>(c, s);
        oth[s] = gr<T>(c, s);
    }
    for (int s = 0; s < S - 1; ++s) {
        Op<T> A = level_op<T>(c, s, opi);
        const bool have_first = (s == 0) ? first_done : true;
        if (!have_first) c.launches += launch_spmm<T>(SP_JACOBI, A, N, nullptr, b[s], cur[s], w, sk, st);
        for (int k = 1; k < nu; ++k) {
            c.launches += launch_spmm<T>(SP_JACOBI, A, N, cur[s], b[s], oth[s], w, sk, st);
            std::swap(cur[s], oth[s]);
        }
        c.launches += launch_spmm<T>(SP_RESID, A, N, cur[s], b[s], oth[s], T(0), sk, st);
        Op<T> R = make_op<T>(c.sl[s].R, 1.0, 0.0);
        // the next level's first sweep rides on the restriction unless it is the dense level
        Aux<T> aux = (s + 1 < S - 1) ? sweep_aux<T>(c, s + 1, opi, cur[s + 1]) : Aux<T>();
        c.launches += launch_spmm<T>(SP_RESTRICT, R, N, oth[s], nullptr, const_cast<T*>(b[s + 1]), T(0), sk, st, aux);
    }
    {
        const int s = S - 1;
        const OpPair& p = c.ops[opi];
        const T* inv = nullptr;
        if constexpr (sizeof(T) == 8) inv = p.inv_d.p; else inv = p.inv_f.p;
        if (inv) {
            c.launches += launch_dense_apply<T>(c.sl[s].n, N, inv, b[s], cur[s], sk, st);
        } else {
            Op<T> A = level_op<T>(c, s, opi);
            if (!(s == 0 && first_done))
                c.launches += launch_spmm<T>(SP_JACOBI, A, N, nullptr, b[s], cur[s], w, sk, st);
            for (int k = 1; k < 4 * nu; ++k) {
                c.launches += launch_spmm<T>(SP_JACOBI, A, N, cur[s], b[s], oth[s], w, sk, st);
                std::swap(cur[s], oth[s]);
            }
        }
    }
    for (int s = S - 2; s >= 0; --s) {
        Op<T> P = make_op<T>(c.sl[s].P, 1.0, 0.0);
        c.launches += launch_spmm<T>(SP_INTERP_ADD, P, N, cur[s + 1], nullptr, cur[s], T(0), sk, st);
        Op<T> A = level_op<T>(c, s, opi);
        for (int k = 0; k < nu; ++k) {
            c.launches += launch_spmm<T>(SP_JACOBI, A, N, cur[s], b[s], oth[s], w, sk, st);
            std::swap(cur[s], oth[s]);
        }
    }
    return cur[0];
}

// Batched PCG on (cm M + cl L) X = B over N columns, X accumulated as
// X += xscale * (solution from zero).  `r` holds B on entry and is
// destroyed.  Work buffers: w[1..5] of the precision.  With tol > 0 the
// iteration stops early on the device once every column has
// ||r|| <= tol ||b|| (later kernels of the solve see the flag and return).
template <typename T>
struct PCG {
    Ctx& c;
    int opi, N;
    T* r;
    T* x;
    T xscale;
    bool gmg;
    Skip sk, sk2;
    ColRed<T> cr;
    T *p = nullptr, *q = nullptr, *z = nullptr, *pa = nullptr, *pb = nullptr;
    Op<T> A;

    bool assign_first;   // x is not initialised: the first update assigns
    int iter = 0;

    PCG(Ctx& c_, int opi_, int N_, T* r_, T* x_, T xscale_, double tol, Skip sk_, bool x_uninit)
        : c(c_), opi(opi_), N(N_), r(r_), x(x_), xscale(xscale_), sk(sk_), assign_first(x_uninit) {
        gmg = use_gmg(c);
        cr = make_cr<T>(c);
        sk2 = sk;
        if (tol > 0) {
            cr.pdone = c.flag.p + 1;
            cr.tol2 = (T)(tol * tol);
            sk2.pdone = c.flag.p + 1;
        }
        A = level_op<T>(c, 0, opi);
        q = wbuf<T>(c, 3);
    }

    // Buffer into which the producer of r may write the fused first
    // V-cycle sweep (GMG only).
    T* first_sweep_buffer() const { return wbuf<T>(c, 1); }

    // j0_done: the producer of r already wrote w D^-1 r into first_sweep_buffer()
    void init(bool j0_done = false) {
        cudaStream_t st = c.stream;
        if (cr.pdone) c.launches += launch_flag(c.flag.p + 1, 0, sk, st);
        if (!gmg) {
            z = wbuf<T>(c, 1);
            p = wbuf<T>(c, 2);
            c.launches += launch_pcg_init_jacobi<T>(A, N, r, z, p, cr, sk2, st);
        } else {
            // the stencil V-cycle forms rho = r.z and bb = rr = r.r in its last pass
            const bool fused = use_stencil<T>(c);
            T* zr = gmg_vcycle<T>(c, opi, N, r, wbuf<T>(c, 1), wbuf<T>(c, 4), sk2, j0_done, fused ? 1 : 0);
            if (!fused) c.launches += launch_pcg_dot_rz<T>(A.rows, N, r, zr, cr, 1, sk2, st);
            p = zr;
            pa = zr == wbuf<T>(c, 1) ? wbuf<T>(c, 4) : wbuf<T>(c, 1);
            pb = wbuf<T>(c, 5);
        }
    }

    // Whether the last iteration from a zero start can leave x = xscale
    // alpha p to its consumer (the time restriction forms it on the fly).
    bool can_defer_update(int iters) const {
        if constexpr (sizeof(T) == 4) return iters == 1 && assign_first && !cr.pdone && use_stencil<T>(c);
        return false;
    }

    // defer: skip the final x update (only where can_defer_update holds);
    // p and alpha() then define x
    void iterate(bool last, bool defer = false) {
        cudaStream_t st = c.stream;
        const int assign = (assign_first && iter == 0) ? 1 : 0;
        if (last && !cr.pdone) {   // no tolerance: the final r and its norm are never read
            ++iter;
            if constexpr (sizeof(T) == 4) {
                if (use_stencil<T>(c)) {   // q = A p is not needed: only p.(A p) for alpha
                    c.launches += launch_st_apply_dot(st_op(c, 0, opi), N, p, cr, sk2, st);
                    if (!(defer && assign))
                        c.launches += launch_pcg_xupdate<T>(A.rows, N, xscale, assign, x, p, cr, sk2, st);
                    return;
                }
            }
            c.launches += launch_pcg_apply_alpha<T>(A, N, p, q, cr, sk2, st);
            c.launches += launch_pcg_xupdate<T>(A.rows, N, xscale, assign, x, p, cr, sk2, st);
            return;
        }
        c.launches += launch_pcg_apply_alpha<T>(A, N, p, q, cr, sk2, st);
        ++iter;
        // the next V-cycle's first sweep rides on the residual update
        Aux<T> aux = (gmg && !last) ? sweep_aux<T>(c, 0, opi, pa) : Aux<T>();
        c.launches += launch_pcg_update<T>(A, N, xscale, assign, x, p, r, q, gmg ? nullptr : z, gmg ? 0 : 1, cr,
                                           sk2, st, aux);
        if (last) return;
        if (gmg) {
            const bool fused = use_stencil<T>(c);
            z = gmg_vcycle<T>(c, opi, N, r, pa, pb, sk2, true, fused ? 2 : 0);
            if (!fused) c.launches += launch_pcg_dot_rz<T>(A.rows, N, r, z, cr, 0, sk2, st);
        }
        c.launches += launch_pcg_direction<T>(A.rows, N, z, p, cr, sk2, st);
    }

    const T* alpha() const { return cr.col + S_ALPHA * N; }
};

// x = xscale alpha[n] p left for the time restriction to form (bj_sweep)
struct DeferredUpdate {
    bool on = false;
    const float* p = nullptr;
    const float* alpha = nullptr;
    float xscale = 0.f;
};

// One damped block-Jacobi sweep at time level l on x (in place).  With
// `defer` set, a sweep from zero whose single PCG iteration would end with
// x = omega_t alpha p leaves that update out and describes it in *defer
// (on = false where it cannot).
template <typename T>
void bj_sweep(Ctx& c, int l, T* x, const T* b, bool x_zero, Skip sk, DeferredUpdate* defer = nullptr) {
    const TimeLevel& t = c.tl[l];
    T* r = wbuf<T>(c, 0);
    const size_t cnt = (size_t)c.n * t.N;
    // a zero start means x holds stale data: the first PCG update assigns it
    PCG<T> pcg(c, t.op, t.N, r, x, (T)c.opts.omega_t, 0.0, sk, x_zero);
    Op<T> A = level_op<T>(c, 0, t.op);
    Aux<T> aux = pcg.gmg ? sweep_aux<T>(c, 0, t.op, pcg.first_sweep_buffer()) : Aux<T>();
    if (x_zero) {
        bool done = false;
        if constexpr (sizeof(T) == 4) {
            if (pcg.gmg && use_stencil<T>(c)) {
                c.launches += launch_st_copy_sweep(st_op(c, 0, t.op), t.N, b, r, aux.Y2, aux.omega, sk, c.stream);
                done = true;
            }
        }
        if (done) {
        } else if (pcg.gmg) {
            c.launches += launch_spmm<T>(SP_COPY, A, t.N, nullptr, b, r, T(0), sk, c.stream, aux);
        } else {
            copy_async(r, b, cnt * sizeof(T), c.stream);
        }
    } else if (use_stencil<T>(c)) {
        if constexpr (sizeof(T) == 4)
            c.launches += launch_st_presid(st_op(c, 0, t.op), t.N, x, b, r, aux.Y2, aux.omega, false, sk, c.stream);
    } else {
        c.launches += launch_spmm<T>(SP_PRESID, A, t.N, x, b, r, T(0), sk, c.stream, aux);
    }
    pcg.init(pcg.gmg);
    const int it = std::max(1, c.opts.pcg_iters);
    const bool dfr = defer && pcg.can_defer_update(it);
    for (int k = 0; k < it; ++k) pcg.iterate(k == it - 1, dfr);
    if (defer) {
        defer->on = false;
        if constexpr (sizeof(T) == 4) {
            if (dfr) {
                defer->on = true;
                defer->p = pcg.p;
                defer->alpha = pcg.alpha();
                defer->xscale = pcg.xscale;
            }
        }
    }
}

DstSolve dst_of(Ctx& c) {
    DstSolve d;
    d.W = c.gnx - 2;
    d.H = c.gny - 2;
    d.logx = c.dst_logx;
    d.logy = c.dst_logy;
    d.wx = c.dst_wx.p;
    d.wy = c.dst_wy.p;
    d.scale = c.dst_scale.p;
    d.tmp = c.dst_tmp.p;
    d.tmp2 = c.dst_tmp2.p;
    return d;
}

// exact solve on the coarsest time level, in double: direct by sine
// transforms where the grid allows, else PCG to coarse_tol
template <typename T>
void coarse_solve(Ctx& c, Skip sk) {
    const int L = (int)c.tl.size();
    const int Nc = c.tl[L - 1].N;
    const int n = c.n;
    cudaStream_t st = c.stream;
    T* xc = mgx<T>(c, L - 1);
    const T* bc = mgb<T>(c, L - 1);
    double* cb = c.w_d[0].p;   // rhs (destroyed by PCG)
    double* cx = c.Ud.p;       // solution columns
    const double tol = c.opts.coarse_tol;
    const int maxit = std::max(1, c.opts.coarse_max_it);
    auto run = [&](int opi, double* rhs, double* sol) {
        // the fill is kept: with early exit the assigning update may be skipped
        c.launches += launch_fill<double>((size_t)n, 0.0, sol, sk, st);
        PCG<double> pcg(c, opi, 1, rhs, sol, 1.0, tol, sk, false);
        pcg.init();
        for (int k = 0; k < maxit; ++k) pcg.iterate(k == maxit - 1);
    };
    if (Nc == 1 && c.dst_ok) {   // direct: tau_c L x = b by sine transforms, in double
        c.launches += launch_dst_solve<T>(dst_of(c), bc, xc, sk, st);
        return;
    }
    if (Nc == 1) {
        if constexpr (sizeof(T) == 8)
            copy_async(cb, bc, (size_t)n * sizeof(double), st);
        else
            c.launches += launch_cast<float, double>((size_t)n, bc, cb, sk, st);
        run(c.coarse_ops[0], cb, cx);
        if constexpr (sizeof(T) == 8)
            copy_async(xc, cx, (size_t)n * sizeof(double), st);
        else
            c.launches += launch_cast<double, float>((size_t)n, cx, xc, sk, st);
    } else {
        double* bs = cb;
        double* bd = cb + n;
        double* xs = cx;
        double* xd = cx + n;
        c.launches += launch_split2<T>(n, bc, bs, bd, sk, st);
        if (c.dst_ok) c.launches += launch_dst_solve<double>(dst_of(c), bs, xs, sk, st);
        else run(c.coarse_ops[0], bs, xs);
        run(c.coarse_ops[1], bd, xd);
        c.launches += launch_combine2<T>(n, xs, xd, xc, sk, st);
    }
}

// Exact periodic solve of time level l by the DFT in time, in double
// (k_dft.cu): b_l -> spectrum, one conjugate-orthogonal CG solve per mode
// k = 0..N_l/2 on ((1 - e^{-2 pi i k/N_l}) M + tau_l L) x_k = b_k with the
// tau_l L V-cycle (or its diagonal) as preconditioner, spectrum -> x_l.  The
// iteration stops on the device once every mode has |r_k| <= coarse_tol |b_k|.
template <typename T>
void dft_solve(Ctx& c, int l, Skip sk) {
    const int N = c.tl[l].N;
    const int K = N / 2 + 1, D = 2 * K;
    const int n = c.n;
    const double tau = c.tl[l].tau;
    cudaStream_t st = c.stream;
    double* r = c.dft_w[0].p;   // spectrum of b, then the residual
    double* x = c.dft_w[1].p;
    double* q = c.dft_w[2].p;
    double* za = c.dft_w[3].p;
    double* zb = c.dft_w[4].p;
    double* zc = c.dft_w[5].p;
    c.launches += launch_dft_fwd<T>(n, N, mgb<T>(c, l), c.dft_W.p, r, sk, st);
    ColRed<double> cr = make_cr<double>(c);
    cr.pdone = c.flag.p + 1;
    cr.tol2 = c.opts.coarse_tol * c.opts.coarse_tol;
    Skip sk2 = sk;
    sk2.pdone = c.flag.p + 1;
    c.launches += launch_flag(c.flag.p + 1, 0, sk, st);
    const bool gmg = use_gmg(c);
    Op<double> P = level_op<double>(c, 0, c.dft_op);
    auto precond = [&](double* xa, double* xb) -> double* {
        if (gmg) return gmg_vcycle<double>(c, c.dft_op, D, r, xa, xb, sk2, false);
        c.launches += launch_spmm<double>(SP_JACOBI, P, D, nullptr, r, xa, 1.0, sk2, st);
        return xa;
    };
    double* p = precond(za, zb);
    double* pa = p == za ? zb : za;
    c.launches += launch_cdot_rz(n, D, r, p, cr, 1, sk2, st);
    Op<double> A = make_op<double>(c.sl[0].op, 1.0, 0.0);   // v1 = M, v2 = L
    const int maxit = std::max(1, c.opts.dft_max_it);
    for (int it = 0; it < maxit; ++it) {
        c.launches += launch_capply_alpha(A, D, c.dft_ck.p, tau, p, q, cr, sk2, st);
        c.launches += launch_cupdate(n, D, it == 0 ? 1 : 0, x, p, r, q, cr, sk2, st);
        if (it == maxit - 1) break;
        double* z = precond(pa, zc);
        c.launches += launch_cdot_rz(n, D, r, z, cr, 0, sk2, st);
        c.launches += launch_cdirection(n, D, z, p, cr, sk2, st);
    }
    c.launches += launch_dft_inv<T>(n, N, x, c.dft_W.p, mgx<T>(c, l), sk, st);
}

// multigrid-in-time V-cycle at level l: improves x_l for P_l x_l = b_l.
// The V-cycle uses levels 0..active_levels-1.  Its last level is solved
// exactly: by the DFT in time when that solver is chosen, directly when it
// is the 1- or 2-step bottom of the hierarchy, otherwise by coarse_cycles
// V-cycles over the levels below it (full = true).
template <typename T>
void mgt_vcycle(Ctx& c, int l, bool x_zero, Skip sk, bool full = false) {
    const int L = (int)c.tl.size();
    T* x = mgx<T>(c, l);
    const T* b = mgb<T>(c, l);
    const TimeLevel& t = c.tl[l];
    cudaStream_t st = c.stream;
    if (l == c.dft_level) {
        dft_solve<T>(c, l, sk);  // x_zero is implied: exact solve
        return;
    }
    if (l == L - 1) {
        coarse_solve<T>(c, sk);  // x_zero is implied: exact solve
        return;
    }
    if constexpr (sizeof(T) == 4) {
        if (c.fz_on && l == c.fz_level && x_zero && !full) {   // the recorded program of levels l..L-1
            c.launches += launch_fused_program(reinterpret_cast<const FusedPhase*>(c.fz_blob.p), c.fz_nph, c.fz_grid,
                                               c.fz_smem, st);
            return;
        }
    }
    if (!full && l == c.active_levels - 1) {
        const int cyc = std::max(1, c.opts.coarse_cycles);
        for (int k = 0; k < cyc; ++k) mgt_vcycle<T>(c, l, x_zero && k == 0, sk, true);
        return;
    }
    const int pre = c.opts.pre_smooth, post = c.opts.post_smooth;
    bool zero = x_zero;
    if (pre == 0 && zero) {
        c.launches += launch_fill<T>((size_t)c.n * t.N, T(0), x, sk, st);
        zero = false;
    }
    const bool st_restrict = use_stencil<T>(c) && sizeof(T) == 4 && t.N % 2 == 0;
    DeferredUpdate du;
    for (int k = 0; k < pre; ++k) {
        // the last pre-sweep from zero hands x = omega_t alpha p to the restriction
        const bool hand_over = st_restrict && c.opts.fuse_update && k == pre - 1;
        bj_sweep<T>(c, l, x, b, zero, sk, hand_over ? &du : nullptr);
        zero = false;
    }
    bool restricted = false;
    if constexpr (sizeof(T) == 4) {
        if (st_restrict && du.on) {
            c.launches += launch_st_presid_restrict_update(st_op(c, 0, t.op), t.N, du.p, du.alpha, du.xscale, x, b,
                                                           mgb<T>(c, l + 1), sk, st);
            restricted = true;
        } else if (st_restrict) {
            c.launches += launch_st_presid(st_op(c, 0, t.op), t.N, x, b, mgb<T>(c, l + 1), nullptr, 0.f, true, sk, st);
            restricted = true;
        }
    }
    if (!restricted) {
        Op<T> A = level_op<T>(c, 0, t.op);
        c.launches += launch_spmm<T>(SP_PRESID_RESTRICT, A, t.N, x, b, mgb<T>(c, l + 1), T(0), sk, st);
    }
    mgt_vcycle<T>(c, l + 1, true, sk, full);
    if (l >= c.chain_depth)   // else x stays the smoothed iterate; the chain pass adds the prolongations
        c.launches += launch_time_prolong_add<T>(c.n, c.tl[l + 1].N, mgx<T>(c, l + 1), x, sk, st);
    for (int k = 0; k < post; ++k) bj_sweep<T>(c, l, x, b, false, sk);
}

// Levels of one V(pre, 0) cycle from zero whose final iterate is only read
// by the prolongation to the level above: 0 .. D - 1, where level D is the
// first whose cycle is not the plain recursion (the exact last level, the
// DFT level, the fused coarse program, the coarse cycles) and x_D is final
// when its cycle returns.  0 where post-smoothing or a second cycle reads
// the finer iterates.
static int prolong_chain_depth(const Ctx& c) {
    if (c.opts.post_smooth != 0 || std::max(1, c.opts.vcycles) != 1) return 0;
    int D = (int)c.tl.size() - 1;
    if (c.dft_level >= 0) D = std::min(D, c.dft_level);
    if (c.fz_on) D = std::min(D, c.fz_level);
    if (c.active_levels < (int)c.tl.size()) D = std::min(D, c.active_levels - 1);
    if (D < 1 || D >= kMaxChain) return 0;
    for (int l = 0; l <= D; ++l)
        if (c.tl[l].N != c.N >> l) return 0;
    return D;
}

// One outer step of the fixed point (correction form of eq. iter1) on the
// iterate X:
//   STEP_FORWARD  X = U, residual F - A(U), periodic inner solve;
//   STEP_ADJOINT  X = lambda in reversed time, residual g - (dA/dU)^T lambda;
//   STEP_STATIC   X = U with sigma = 0 (the initialisation of Section 4): the
//                 mass term drops, the steps decouple, and the inner solve is
//                 tau_c L x = tau_c (F - K(U)) for every column (batched PCG
//                 with the spatial multigrid preconditioner), i.e. eq. (iter1)
//                 with M = 0.
template <typename T>
void outer_step(Ctx& c, Skip sk, int kind) {
    const bool adjoint = kind == STEP_ADJOINT;
    double* X = adjoint ? c.Lam.p : c.U.p;
    ResidualArgs a = residual_args(c, X, nullptr);
    a.scale = kind == STEP_STATIC ? c.tl.back().tau : c.T / c.N;
    if constexpr (sizeof(T) == 8) a.b_d = mgb<double>(c, 0); else a.b_f = mgb<float>(c, 0);
    a.done = c.flag.p;
    a.check = 1;
    if (adjoint) {
        c.launches += launch_adj_elem_flux(adjoint_args(c), X, c.Qx.p, c.Qy.p, c.flag.p, c.stream);
        a.Fext = c.Gadj.p;
        a.skip_flux = 1;
    }
    if (kind == STEP_STATIC) {   // every mass row empty
        a.m_ptr = c.zero_ptr.p;
        a.st_no_mass = 1;
    }
    c.launches += launch_residual_law(a, law_data(c), c.stream);
    int D = 0;   // levels whose prolongation the chain pass below adds
    if (kind == STEP_STATIC) {
        PCG<T> pcg(c, c.coarse_ops[0], c.N, mgb<T>(c, 0), mgx<T>(c, 0), T(1), 0.0, sk, true);
        pcg.init();
        const int it = std::max(1, c.opts.pcg_iters);
        for (int k = 0; k < it; ++k) pcg.iterate(k == it - 1);
    } else {
        // set for this cycle only: other callers of the V-cycle (also after an
        // exception here) see 0 and prolongate level by level
        struct Reset {
            int& v;
            ~Reset() { v = 0; }
        } reset{c.chain_depth};
        c.chain_depth = c.opts.fuse_update ? prolong_chain_depth(c) : 0;
        D = c.chain_depth;
        const int cyc = std::max(1, c.opts.vcycles);
        for (int v = 0; v < cyc; ++v) mgt_vcycle<T>(c, 0, v == 0, sk);
    }
    const double* sc = sizeof(T) == 4 ? &c.status.p->bscale_used : nullptr;
    if (D > 0) {
        const T* xs[kMaxChain];
        for (int l = 0; l <= D; ++l) xs[l] = mgx<T>(c, l);
        c.launches += launch_prolong_chain_add<T>(c.n, c.N, D, xs, X, sc, sk, c.stream);
    } else {
        c.launches += launch_add_to_double<T>((size_t)c.n * c.N, mgx<T>(c, 0), X, sc, sk, c.stream);
    }
}

void final_residual(Ctx& c, int kind) {
    const bool adjoint = kind == STEP_ADJOINT;
    double* X = adjoint ? c.Lam.p : c.U.p;
    ResidualArgs a = residual_args(c, X, nullptr);
    a.done = c.flag.p;
    a.check = 1;
    if (adjoint) {
        c.launches += launch_adj_elem_flux(adjoint_args(c), X, c.Qx.p, c.Qy.p, c.flag.p, c.stream);
        a.Fext = c.Gadj.p;
        a.skip_flux = 1;
    }
    if (kind == STEP_STATIC) {
        a.m_ptr = c.zero_ptr.p;
        a.st_no_mass = 1;
    }
    c.launches += launch_residual_law(a, law_data(c), c.stream);
}

template <typename T>
void alloc_levels(Ctx& c, std::vector<DBuf<T>>& x, std::vector<DBuf<T>>& b) {
    x.clear();
    b.clear();
    x.resize(c.tl.size());
    b.resize(c.tl.size());
    for (size_t l = 0; l < c.tl.size(); ++l) {
        x[l].alloc((size_t)c.n * c.tl[l].N);
        b[l].alloc((size_t)c.n * c.tl[l].N);
    }
}

}  // namespace

ResidualArgs residual_args(Ctx& c, const double* U, double* R) {
    ResidualArgs a{};
    a.n = c.n;
    a.N = c.N;
    a.n_iron = c.n_iron;
    a.n_coils = c.n_coils;
    a.e_nodes = c.e_nodes.p;
    a.e_geo = c.e_geo.p;
    a.inc_ptr = c.inc_ptr.p;
    a.inc_elem = c.inc_elem.p;
    a.inc_grad = c.inc_grad.p;
    a.m_ptr = c.m_ptr.p;
    a.m_idx = c.m_idx.p;
    a.m_val = c.m_val.p;
    a.l_ptr = c.l_ptr.p;
    a.l_idx = c.l_idx.p;
    a.l_val = c.l_val.p;
    a.coil_b = c.coil_b.p;
    a.coil_s = c.coil_s.p;
    a.s2sat = c.s_sat * c.s_sat;
    a.U = U;
    a.Qx = c.Qx.p;
    a.Qy = c.Qy.p;
    a.R = R;
    a.partials = c.part_d.p;
    a.partials_cap = c.part_d.n;
    a.counter = c.counter.p;
    a.status = c.status.p;
    if (c.k1_struct && c.opts.k1_fused) {
        a.st_W = c.gnx - 2;
        a.st_H = c.gny - 2;
        a.st_cell = c.k1_cell.p;
        a.st_flag = c.k1_flag.p;
        a.st_mass = c.k1_mass.p;
        a.st_lin = c.k1_lin.p;
        a.st_ihx2 = c.k1_ihx2;
        a.st_ihy2 = c.k1_ihy2;
        a.st_At = c.k1_At;
        a.st_Bt = c.k1_Bt;
    }
    return a;
}

// Allocates what a solve in the set-up precision needs.  In mixed mode the
// double work vectors only serve the one- or two-column coarsest time level;
// double entry points called on a mixed context grow them on demand
// (ensure_double_work).
void alloc_work(Ctx& c) {
    const size_t big = (size_t)c.n * c.N;
    const bool mixed = c.opts.precision == PTP_MIXED;
    const size_t dcols = mixed ? 2 : (size_t)std::max(c.N, 2);
    for (int k = 0; k < 6; ++k) {
        c.w_d[k].alloc((size_t)c.n * dcols);
        if (mixed) c.w_f[k].alloc(big); else c.w_f[k].release();
    }
    c.U.alloc(big);
    c.R.release();
    c.Ud.alloc((size_t)c.n * 2);
    c.Qx.alloc((size_t)std::max(c.n_iron, 1) * c.N);
    c.Qy.alloc((size_t)std::max(c.n_iron, 1) * c.N);
    if (mixed) {
        alloc_levels<float>(c, c.mg_xf, c.mg_bf);
        c.mg_xd.clear();
        c.mg_bd.clear();
    } else {
        alloc_levels<double>(c, c.mg_xd, c.mg_bd);
        c.mg_xf.clear();
        c.mg_bf.clear();
    }
    // the DFT solve works on 2 (N_l/2 + 1) double columns of its own
    const size_t dft_cols = c.dft_level >= 0 ? 2 * (size_t)(c.tl[c.dft_level].N / 2 + 1) : 0;
    for (int k = 0; k < 6; ++k) {
        if (dft_cols) c.dft_w[k].alloc((size_t)c.n * dft_cols); else c.dft_w[k].release();
    }
    const size_t gcols = std::max(dcols, dft_cols);
    const size_t S = c.sl.size();
    c.g_xd.clear(); c.g_bd.clear(); c.g_rd.clear();
    c.g_xf.clear(); c.g_bf.clear(); c.g_rf.clear();
    c.g_xd.resize(S); c.g_bd.resize(S); c.g_rd.resize(S);
    c.g_xf.resize(S); c.g_bf.resize(S); c.g_rf.resize(S);
    for (size_t s = 1; s < S; ++s) {
        const size_t m = (size_t)c.sl[s].n * c.N;
        const size_t md = (size_t)c.sl[s].n * gcols;
        c.g_xd[s].alloc(md); c.g_bd[s].alloc(md); c.g_rd[s].alloc(md);
        if (mixed) { c.g_xf[s].alloc(m); c.g_bf[s].alloc(m); c.g_rf[s].alloc(m); }
    }
    const int colmax = std::max({c.N, 2, (int)dft_cols});
    c.col_d.alloc(8 * (size_t)colmax);
    c.scal.alloc(8);
    c.col_f.alloc(8 * (size_t)std::max(c.N, 2));
    const size_t parts = std::max(reduction_partials(colmax), (size_t)num_sms() * 64);
    c.part_d.alloc(parts);
    c.part_f.alloc(mixed ? parts : 0);
    c.counter.alloc(256);
    PTP_CUDA(cudaMemsetAsync(c.counter.p, 0, 256 * sizeof(unsigned), c.stream));
    c.status.alloc(1);
    c.flag.alloc(4);
    PTP_CUDA(cudaMemsetAsync(c.flag.p, 0, 4 * sizeof(int), c.stream));
    if (!c.h_status) PTP_CUDA(cudaHostAlloc((void**)&c.h_status, 2 * sizeof(Status), cudaHostAllocDefault));
}

template <typename T>
static bool grow(DBuf<T>& b, size_t n) {
    if (b.n >= n) return false;
    b.alloc(n);
    return true;
}

// full-size work vectors of precision T (entry points that run in the other
// precision than the set-up one, and host staging of [n][N] blocks)
// A reallocated buffer may be baked into a captured graph (of this context or
// of a batch holding it): bumping buf_gen changes the step key, so those
// graphs are captured again before their next launch.
void ensure_work(Ctx& c, bool doubles) {
    const size_t big = (size_t)c.n * c.N;
    bool changed = false;
    for (int k = 0; k < 6; ++k) {
        if (doubles) changed |= grow(c.w_d[k], big); else changed |= grow(c.w_f[k], big);
    }
    for (size_t s = 1; s < c.sl.size(); ++s) {
        const size_t m = (size_t)c.sl[s].n * c.N;
        if (doubles) { changed |= grow(c.g_xd[s], m); changed |= grow(c.g_bd[s], m); changed |= grow(c.g_rd[s], m); }
        else { changed |= grow(c.g_xf[s], m); changed |= grow(c.g_bf[s], m); changed |= grow(c.g_rf[s], m); }
    }
    if (!doubles) changed |= grow(c.part_f, c.part_d.n);
    if (changed) ++c.buf_gen;
}

void ensure_staging(Ctx& c) {
    const size_t big = (size_t)c.n * c.N;
    bool changed = grow(c.R, big);
    changed |= grow(c.Ud, std::max(big, (size_t)c.n * 2));
    if (changed) ++c.buf_gen;
}

void residual_dev(Ctx& c, const double* U, double* R, double* b_out_d, float* b_out_f, double scale,
                  bool outer_check) {
    ResidualArgs a = residual_args(c, U, R);
    a.b_d = b_out_d;
    a.b_f = b_out_f;
    a.scale = scale;
    a.check = outer_check ? 1 : 0;
    c.launches += launch_residual_law(a, law_data(c), c.stream);
}

double norm_dev(Ctx& c, const double* x, size_t count) {
    double* out = c.scal.p + 1;
    c.launches += launch_norm2<double>(count, x, c.part_d.p, c.counter.p, out, c.stream);
    double h = 0.0;
    PTP_CUDA(cudaMemcpyAsync(&h, out, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    PTP_CUDA(cudaStreamSynchronize(c.stream));
    return std::sqrt(h);
}

void source_dev(Ctx& c, double* F) {
    launch_source(c.n, c.N, c.n_coils, c.coil_b.p, c.coil_s.p, F, c.stream);
    c.launches += 1;
}

template <typename T>
void apply_op(Ctx& c, int s, int op, int N, const T* X, T* Y) {
    Op<T> A = level_op<T>(c, s, op);
    c.launches += launch_spmm<T>(SP_APPLY, A, N, X, nullptr, Y, T(0), Skip{}, c.stream);
}

template <typename T>
void periodic_apply(Ctx& c, int level, const T* X, T* Y) {
    const TimeLevel& t = c.tl[level];
    Op<T> A = level_op<T>(c, 0, t.op);
    c.launches += launch_spmm<T>(SP_PAPPLY, A, t.N, X, nullptr, Y, T(0), Skip{}, c.stream);
}

void periodic_residual_f32(Ctx& c, int level, const float* X, const float* B, float* R) {
    const TimeLevel& t = c.tl[level];
    if (use_stencil<float>(c)) {
        c.launches += launch_st_presid(st_op(c, 0, t.op), t.N, X, B, R, nullptr, 0.f, false, Skip{}, c.stream);
    } else {
        Op<float> A = level_op<float>(c, 0, t.op);
        c.launches += launch_spmm<float>(SP_PRESID, A, t.N, X, B, R, 0.f, Skip{}, c.stream);
    }
}

template <typename T>
int spatial_pcg(Ctx& c, int op, int N, const T* B, T* X, double tol, int max_it, bool host_check) {
    ensure_work(c, sizeof(T) == 8);
    cudaStream_t st = c.stream;
    const size_t cnt = (size_t)c.n * N;
    T* r = wbuf<T>(c, 0);
    PTP_CUDA(cudaMemcpyAsync(r, B, cnt * sizeof(T), cudaMemcpyDeviceToDevice, st));
    c.launches += launch_fill<T>(cnt, T(0), X, Skip{}, st);
    PCG<T> pcg(c, op, N, r, X, T(1), tol, Skip{}, false);
    pcg.init();
    int it = 0;
    for (; it < max_it; ++it) {
        pcg.iterate(it == max_it - 1);
        if (host_check && tol > 0) {
            int done = 0;
            PTP_CUDA(cudaMemcpyAsync(&done, c.flag.p + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
            PTP_CUDA(cudaStreamSynchronize(st));
            if (done) { ++it; break; }
        }
    }
    PTP_CUDA(cudaStreamSynchronize(st));
    return it;
}

void require_coarse(const Ctx& c) {
    PTP_REQUIRE(c.coarse_ok || c.dft_level >= 0 || c.active_levels < (int)c.tl.size(),
                "multigrid in time needs a coarsest level with 1 or 2 steps (N must be a power of "
                "two times 1 or 2, and time_levels large enough to reach it), or the DFT coarse solver");
}

void periodic_mg_solve(Ctx& c, const double* B, double* X, int cycles, double* relres) {
    require_coarse(c);
    ensure_staging(c);
    cudaStream_t st = c.stream;
    const size_t cnt = (size_t)c.n * c.N;
    const bool mixed = c.opts.precision == PTP_MIXED;
    double* nb = c.scal.p;  // ||B||^2, then ||B|| (device scalar)
    if (mixed) {
        // the float V-cycle runs on B / ||B|| and its result is scaled back
        c.launches += launch_norm2<double>(cnt, B, c.part_d.p, c.counter.p, nb, st);
        double h = 0.0;
        PTP_CUDA(cudaMemcpyAsync(&h, nb, sizeof(double), cudaMemcpyDeviceToHost, st));
        PTP_CUDA(cudaStreamSynchronize(st));
        h = h > 0 ? std::sqrt(h) : 1.0;
        PTP_CUDA(cudaMemcpyAsync(nb, &h, sizeof(double), cudaMemcpyHostToDevice, st));
        c.launches += launch_cast_scaled<double, float>(cnt, B, mgb<float>(c, 0), nullptr, nb, st);
    } else {
        PTP_CUDA(cudaMemcpyAsync(mgb<double>(c, 0), B, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    for (int v = 0; v < std::max(1, cycles); ++v) {
        if (mixed) mgt_vcycle<float>(c, 0, v == 0, Skip{});
        else mgt_vcycle<double>(c, 0, v == 0, Skip{});
    }
    if (mixed) c.launches += launch_cast_scaled<float, double>(cnt, mgx<float>(c, 0), X, nb, nullptr, st);
    else PTP_CUDA(cudaMemcpyAsync(X, mgx<double>(c, 0), cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (relres) {
        // ||B - P X|| / ||B|| in double
        double* r = c.Ud.p;
        Op<double> A = level_op<double>(c, 0, c.tl[0].op);
        c.launches += launch_spmm<double>(SP_PRESID, A, c.N, X, B, r, 0.0, Skip{}, st);
        double* out = c.scal.p + 2;  // two scratch scalars
        c.launches += launch_norm2<double>(cnt, r, c.part_d.p, c.counter.p, out, st);
        c.launches += launch_norm2<double>(cnt, B, c.part_d.p, c.counter.p, out + 1, st);
        double h[2];
        PTP_CUDA(cudaMemcpyAsync(h, out, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        PTP_CUDA(cudaStreamSynchronize(st));
        *relres = h[1] > 0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
    }
    PTP_CUDA(cudaStreamSynchronize(st));
}

// z = one application of the inner periodic solve (opts.vcycles V-cycles of
// multigrid in time from zero) to v, in the set-up precision; the float
// cycle runs on v / ||v|| and is scaled back.  Used as the preconditioner of
// Newton's linear solves.
void mg_precondition(Ctx& c, const double* v, double* z) {
    cudaStream_t st = c.stream;
    const size_t cnt = (size_t)c.n * c.N;
    const int cyc = std::max(1, c.opts.vcycles);
    if (c.opts.precision == PTP_MIXED) {
        double* nb = c.scal.p + 4;
        c.launches += launch_mdot(cnt, 1, v, cnt, v, c.part_d.p, c.counter.p, nb, st);
        c.launches += launch_sqrt_or_one(nb, st);
        c.launches += launch_cast_scaled<double, float>(cnt, v, mgb<float>(c, 0), nullptr, nb, st);
        for (int k = 0; k < cyc; ++k) mgt_vcycle<float>(c, 0, k == 0, Skip{});
        c.launches += launch_cast_scaled<float, double>(cnt, mgx<float>(c, 0), z, nb, nullptr, st);
    } else {
        PTP_CUDA(cudaMemcpyAsync(mgb<double>(c, 0), v, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
        for (int k = 0; k < cyc; ++k) mgt_vcycle<double>(c, 0, k == 0, Skip{});
        PTP_CUDA(cudaMemcpyAsync(z, mgx<double>(c, 0), cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
}

// ---- pieces of a fixed-point solve (shared with the batched solve) ----

// identifies the captured outer step: everything that changes its launches
int64_t step_key(const Ctx& c, const ptp_opts& o) {
    // FNV-1a over every option whose value is baked into the captured step
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    };
    const int ints[18] = {o.precision, o.pcg_iters, o.vcycles, o.pre_smooth, o.post_smooth, o.gmg_smooth,
                          o.coarse_max_it, c.row_block, o.coarse_cycles, o.coarse_solver, o.dft_max_it,
                          o.stencil, o.k1_fused, o.coarse_direct, c.st_tt, c.st_waves, c.fz_on ? c.fz_level : -1,
                          o.fuse_update};
    const double dbls[3] = {o.omega_t, o.gmg_omega, o.coarse_tol};
    mix(ints, sizeof(ints));
    mix(dbls, sizeof(dbls));
    mix(&c.buf_gen, sizeof(c.buf_gen));   // buffers the captured step uses were reallocated
    return (int64_t)(h >> 1);
}

int autotune(Ctx& c, double* best_us) {
    const int cands[3] = {128, 256, 512};
    const bool mixed = c.opts.precision == PTP_MIXED;
    cudaStream_t st = c.stream;
    const size_t cnt = (size_t)c.n * c.N;
    if (mixed) PTP_CUDA(cudaMemsetAsync(c.w_f[0].p, 0, cnt * sizeof(float), st));
    else PTP_CUDA(cudaMemsetAsync(c.w_d[0].p, 0, cnt * sizeof(double), st));
    cudaEvent_t a, b;
    PTP_CUDA(cudaEventCreate(&a));
    PTP_CUDA(cudaEventCreate(&b));
    double best = 1e300;
    int bestb = c.row_block;
    for (int cb : cands) {
        set_row_block(cb);
        auto run = [&]() {
            if (mixed) apply_op<float>(c, 0, c.tl[0].op, c.N, c.w_f[0].p, c.w_f[1].p);
            else apply_op<double>(c, 0, c.tl[0].op, c.N, c.w_d[0].p, c.w_d[1].p);
        };
        for (int r = 0; r < 3; ++r) run();
        PTP_CUDA(cudaEventRecord(a, st));
        for (int r = 0; r < 10; ++r) run();
        PTP_CUDA(cudaEventRecord(b, st));
        PTP_CUDA(cudaEventSynchronize(b));
        float ms = 0;
        PTP_CUDA(cudaEventElapsedTime(&ms, a, b));
        const double us = ms * 100.0;  // per launch
        if (us < best) {
            best = us;
            bestb = cb;
        }
    }
    c.row_block = bestb;
    set_row_block(bestb);
    if (best_us) *best_us = best;
    // stencil schedule: whole outer steps (every level of both hierarchies
    // runs with the schedule) for every (largest time tile, blocks per SM),
    // from a zero start with the stopping rule off; a candidate whose launch
    // plan does not fit the reduction buffers is skipped
    const bool hierarchy = c.coarse_ok || c.dft_level >= 0 || c.active_levels < (int)c.tl.size();
    if (mixed && use_stencil<float>(c) && !c.tl.empty() && hierarchy) {
        ptp_opts o = c.opts;
        o.tol = 0.0;
        const int64_t launches0 = c.launches;
        solve_begin(c, o, nullptr, STEP_FORWARD);
        // each candidate: one warm-up step, then the better of two runs of three
        // steps; the default schedule stays unless another is 2% faster
        auto time_steps = [&]() -> double {
            enqueue_step(c, STEP_FORWARD);
            double t = 1e300;
            for (int rep = 0; rep < 2; ++rep) {
                PTP_CUDA(cudaEventRecord(a, st));
                for (int r = 0; r < 3; ++r) enqueue_step(c, STEP_FORWARD);
                PTP_CUDA(cudaEventRecord(b, st));
                PTP_CUDA(cudaEventSynchronize(b));
                float ms = 0;
                PTP_CUDA(cudaEventElapsedTime(&ms, a, b));
                t = std::min(t, (double)ms);
            }
            return t;
        };
        const int dt = c.st_tt, dw = c.st_waves;
        set_stencil_schedule(dt, dw);
        const double t_default = time_steps();
        double best_st = 1e300;
        int bt = dt, bw = dw;
        for (int tt : {8, 16, 32, 64}) {
            for (int wv : {2, 3, 4, 6}) {
                if (tt == dt && wv == dw) continue;
                set_stencil_schedule(tt, wv);
                double ms = 1e300;
                try {
                    ms = time_steps();
                } catch (const Error& e) {
                    if (e.code != PTP_EINVAL) throw;
                    PTP_CUDA(cudaStreamSynchronize(st));
                    continue;
                }
                if (ms < best_st) {
                    best_st = ms;
                    bt = tt;
                    bw = wv;
                }
            }
        }
        if (!(best_st < 0.98 * t_default)) {
            bt = dt;
            bw = dw;
        }
        c.st_tt = bt;
        c.st_waves = bw;
        apply_schedule(c);
        c.launches = launches0;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return bestb;
}

void apply_schedule(const Ctx& c) {
    set_row_block(c.row_block);
    set_stencil_schedule(c.st_tt, c.st_waves);
}

// Smallest eigenvalue of the pencil L x = lambda M x (M the sigma-weighted
// mass, singular on non-conducting nodes) by inverse iteration
// x <- (tau_c L)^{-1} M x with the double spatial PCG of the coarsest time
// level; the Rayleigh quotient x.Lx / x.Mx decreases to lambda_min.
double estimate_lambda_min(Ctx& c) {
    const int n = c.n;
    cudaStream_t st = c.stream;
    const int oL = c.coarse_ops[0];
    PTP_REQUIRE(oL >= 0, "no tau_c L operator");
    const double tc = c.ops[oL].cl;
    Op<double> Mop = make_op<double>(c.sl[0].op, 1.0, 0.0);
    Op<double> Lop = level_op<double>(c, 0, oL);
    DBuf<double> x, Mx, Lx;
    x.alloc(n);
    Mx.alloc(n);
    Lx.alloc(n);
    std::vector<double> hx(n), hm(n), hl(n);
    c.launches += launch_fill<double>((size_t)n, 1.0, x.p, Skip{}, st);
    double lam = -1.0;
    const int max_pcg = 200;
    for (int k = 0; k < 30; ++k) {
        double* r = c.w_d[0].p;   // M x, destroyed by the PCG
        c.launches += launch_spmm<double>(SP_APPLY, Mop, 1, x.p, nullptr, r, 0.0, Skip{}, st);
        c.launches += launch_fill<double>((size_t)n, 0.0, x.p, Skip{}, st);
        PCG<double> pcg(c, oL, 1, r, x.p, 1.0, 1e-10, Skip{}, false);
        pcg.init();
        for (int it = 0; it < max_pcg; ++it) {
            pcg.iterate(it == max_pcg - 1);
            if (it % 8 == 7) {
                int done = 0;
                PTP_CUDA(cudaMemcpyAsync(&done, c.flag.p + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
                PTP_CUDA(cudaStreamSynchronize(st));
                if (done) break;
            }
        }
        c.launches += launch_spmm<double>(SP_APPLY, Mop, 1, x.p, nullptr, Mx.p, 0.0, Skip{}, st);
        c.launches += launch_spmm<double>(SP_APPLY, Lop, 1, x.p, nullptr, Lx.p, 0.0, Skip{}, st);
        PTP_CUDA(cudaMemcpyAsync(hx.data(), x.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
        PTP_CUDA(cudaMemcpyAsync(hm.data(), Mx.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
        PTP_CUDA(cudaMemcpyAsync(hl.data(), Lx.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
        PTP_CUDA(cudaStreamSynchronize(st));
        double xm = 0.0, xl = 0.0;
        for (int i = 0; i < n; ++i) {
            xm += hx[i] * hm[i];
            xl += hx[i] * hl[i];
        }
        if (!(xm > 0.0)) return 1e300;   // M = 0: no time coupling, kappa is infinite
        if (!std::isfinite(xl)) return 0.0;
        const double now = xl / tc / xm;
        const bool settled = lam > 0 && std::fabs(lam - now) <= 1e-4 * now;
        lam = now;
        if (settled) break;
        const double sc = 1.0 / std::sqrt(xm);
        for (int i = 0; i < n; ++i) hx[i] *= sc;
        PTP_CUDA(cudaMemcpyAsync(x.p, hx.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    PTP_CUDA(cudaStreamSynchronize(st));
    return lam;
}

// Resolves omega_t <= 0 and post_smooth < 0 (automatic) from the smallest
// kappa = tau lambda_min of the problem (tsmooth.cpp).
void resolve_time_smoother(Ctx& c) {
    ptp_opts& o = c.opts;
    if ((o.omega_t > 0 && o.post_smooth >= 0) || c.tl.empty()) return;
    if (c.lambda_min < 0) c.lambda_min = estimate_lambda_min(c);
    c.kappa_min = std::min(1e6, c.tl[0].tau * c.lambda_min);
    // the model's hierarchy: the levels down to the one solved exactly
    int last = (int)c.tl.size() - 1;
    if (c.dft_level >= 0) last = std::min(last, c.dft_level);
    last = std::min(last, std::max(0, c.active_levels - 1));
    std::vector<int> Nl;
    for (int l = 0; l <= last; ++l) Nl.push_back(c.tl[l].N);
    // a 10% margin below the estimate (a Rayleigh quotient, which approaches
    // lambda_min from above; smaller kappa is the harder case)
    const TimeSmoother t = choose_time_smoother(Nl, 0.9 * c.kappa_min, std::max(0, o.pre_smooth), o.post_smooth,
                                                o.omega_t);
    o.post_smooth = t.post;
    o.omega_t = t.omega;
    c.rho_time = t.rho;
}

void solve_begin(Ctx& c, const ptp_opts& o, const double* X0, int kind) {
    const bool adjoint = kind == STEP_ADJOINT;
    if (kind != STEP_STATIC) require_coarse(c);   // the static step has no time hierarchy
    PTP_REQUIRE(o.precision == c.opts.precision && o.spatial_prec == c.opts.spatial_prec &&
                    o.time_levels == c.opts.time_levels && o.coarse_steps == c.opts.coarse_steps &&
                    o.coarse_solver == c.opts.coarse_solver,
                "precision / preconditioner / hierarchy options differ from ptp_setup");
    c.opts = o;
    c.fz_on = false;
    if (kind != STEP_STATIC) resolve_time_smoother(c);
    cudaStream_t st = c.stream;
    double* X = adjoint ? c.Lam.p : c.U.p;
    const size_t cnt = (size_t)c.n * c.N;
    if (X0 && X0 != X) PTP_CUDA(cudaMemcpyAsync(X, X0, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
    else if (!X0) PTP_CUDA(cudaMemsetAsync(X, 0, cnt * sizeof(double), st));
    Status s0{};
    s0.tol = kind == STEP_STATIC && o.init_tol > 0 ? o.init_tol : o.tol;
    // the residual norm of the zero start: ||F|| (forward) or ||g|| (adjoint)
    const double r0 = adjoint ? c.g_norm : c.f_norm;
    s0.bscale = r0 > 0 ? r0 : 1.0;
    s0.bscale_used = s0.bscale;
    c.h_status[0] = s0;
    PTP_CUDA(cudaMemcpyAsync(c.status.p, &c.h_status[0], sizeof(Status), cudaMemcpyHostToDevice, st));
    PTP_CUDA(cudaMemsetAsync(c.flag.p, 0, 4 * sizeof(int), st));
    PTP_CUDA(cudaStreamSynchronize(st));  // h_status[0] is reused below
}

// Enqueues one outer step on c.stream (also while a capture is active);
// returns the kernels it launched.
int64_t enqueue_step(Ctx& c, int kind) {
    Skip sk;
    sk.done = c.flag.p;
    const int64_t b = c.launches;
    if (c.opts.precision == PTP_MIXED) outer_step<float>(c, sk, kind);
    else outer_step<double>(c, sk, kind);
    const int64_t k = c.launches - b;
    c.launches = b;
    return k;
}

// Final residual of the returned iterate, status read-back and statistics.
int solve_end(Ctx& c, ptp_stats* stats, int kind, int64_t step_launches, double solve_ms, float dev_ms) {
    cudaStream_t st = c.stream;
    final_residual(c, kind);
    step_launches += 2;
    PTP_CUDA(cudaMemcpyAsync(&c.h_status[0], c.status.p, sizeof(Status), cudaMemcpyDeviceToHost, st));
    PTP_CUDA(cudaStreamSynchronize(st));
    PTP_CUDA(cudaGetLastError());
    const Status fs = c.h_status[0];
    c.launches += step_launches;
    const bool conv = fs.done == 1;
    if (stats) {
        stats->outer_iterations = fs.iteration > 0 ? fs.iteration - 1 : 0;
        stats->converged = conv ? 1 : 0;
        stats->res0 = fs.res0;
        stats->res_final = fs.res;
        stats->setup_ms = c.setup_ms;
        stats->solve_ms = solve_ms;
        stats->residual_ms = dev_ms;
        stats->kernel_launches = step_launches;
        stats->time_levels = c.active_levels;
        stats->spatial_levels = (int)c.sl.size();
        stats->omega_t = c.opts.omega_t;
        stats->post_smooth = c.opts.post_smooth;
        stats->kappa_min = c.kappa_min;
    }
    if (fs.done == 2) return PTP_ENAN;
    return conv ? PTP_OK : PTP_ENOTCONV;
}

// The fused program of the coarse time levels (k_stencil.cu): the launches
// of the V-cycle from the first time level with at most kFuseSteps steps
// down to the coarsest level and back, recorded once (from zero, as every
// level below the finest starts) and replayed as one cooperative kernel.
// Only on the float stencil path with the full hierarchy and an exact
// coarsest level; anything without a fused body keeps the separate launches.
constexpr int kFuseSteps = 16;
static void prepare_fused(Ctx& c, int kind) {
    c.fz_on = false;
    const int L = (int)c.tl.size();
    if (!c.opts.fuse_coarse || c.opts.precision != PTP_MIXED || kind != STEP_FORWARD || !use_stencil<float>(c) ||
        c.dft_level >= 0 ||
        c.active_levels != L || L < 3 || c.opts.vcycles < 1)
        return;
    int l0 = -1;
    for (int l = 1; l < L - 1; ++l)
        if (c.tl[l].N <= kFuseSteps) { l0 = l; break; }
    if (l0 < 0) return;
    const int64_t key = step_key(c, c.opts) ^ ((int64_t)l0 << 40);
    if (c.fz_level == l0 && c.fz_key == key && c.fz_blob.p) {
        c.fz_on = true;
        return;
    }
    c.fz_level = -1;
    const int64_t launches0 = c.launches;
    Recorder rec;
    active_recorder() = &rec;
    try {
        Skip sk;
        sk.done = c.flag.p;
        mgt_vcycle<float>(c, l0, true, sk, false);
    } catch (...) {
        active_recorder() = nullptr;
        throw;
    }
    active_recorder() = nullptr;
    c.launches = launches0;
    if (rec.foreign || rec.ops.empty()) return;
    size_t smem = 0;
    for (const RecordedLaunch& r : rec.ops) {
        if (!fused_body_supported(r.body) || r.shape.block != 256) return;
        smem = std::max(smem, r.shape.smem);
    }
    const int grid = fused_program_grid(smem);
    if (grid < 1) return;
    const size_t nph = rec.ops.size();
    size_t bytes = nph * sizeof(FusedPhase);
    std::vector<size_t> off(nph);
    for (size_t k = 0; k < nph; ++k) {
        bytes = (bytes + 15) / 16 * 16;
        off[k] = bytes;
        bytes += rec.ops[k].args.size();
    }
    c.fz_blob.alloc(bytes);
    std::vector<unsigned char> host(bytes, 0);
    FusedPhase* ph = reinterpret_cast<FusedPhase*>(host.data());
    for (size_t k = 0; k < nph; ++k) {
        const RecordedLaunch& r = rec.ops[k];
        ph[k] = FusedPhase{r.body, r.shape.gx, std::max(1, r.shape.gy), 0, c.fz_blob.p + off[k]};
        std::memcpy(host.data() + off[k], r.args.data(), r.args.size());
    }
    PTP_CUDA(cudaMemcpy(c.fz_blob.p, host.data(), bytes, cudaMemcpyHostToDevice));
    c.fz_nph = (int)nph;
    c.fz_grid = grid;
    c.fz_smem = smem;
    c.fz_level = l0;
    c.fz_key = key;
    c.fz_on = true;
}

// Fixed-point iteration of one kind from X0 (null: zero start) until its
// stopping rule or max_outer; the graph of one step is re-captured when the
// options change.
static int run_fixed_point(Ctx& c, const ptp_opts& o, const double* X0, double* U, ptp_stats* stats, int kind) {
    const auto t0 = std::chrono::steady_clock::now();
    solve_begin(c, o, X0, kind);
    prepare_fused(c, kind);
    double* X = kind == STEP_ADJOINT ? c.Lam.p : c.U.p;
    const int gi = kind;
    cudaStream_t st = c.stream;
    const size_t cnt = (size_t)c.n * c.N;
    // graph of one outer step, re-captured when the options change
    const int64_t key = step_key(c, c.opts);
    if (o.use_graph && (c.graph_exec[gi] == nullptr || c.graph_key[gi] != key)) {
        if (c.graph_exec[gi]) { cudaGraphExecDestroy(c.graph_exec[gi]); c.graph_exec[gi] = nullptr; }
        cudaGraph_t g;
        PTP_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        try {
            c.launches_per_step[gi] = enqueue_step(c, kind);
        } catch (...) {
            cudaStreamEndCapture(st, &g);
            throw;
        }
        PTP_CUDA(cudaStreamEndCapture(st, &g));
        PTP_CUDA(cudaGraphInstantiate(&c.graph_exec[gi], g, 0));
        cudaGraphDestroy(g);
        c.graph_key[gi] = key;
    }
    cudaEvent_t e0, e1;
    PTP_CUDA(cudaEventCreate(&e0));
    PTP_CUDA(cudaEventCreate(&e1));
    cudaEvent_t chk[2];
    PTP_CUDA(cudaEventCreateWithFlags(&chk[0], cudaEventDisableTiming));
    PTP_CUDA(cudaEventCreateWithFlags(&chk[1], cudaEventDisableTiming));
    PTP_CUDA(cudaEventRecord(e0, st));
    const int every = std::max(1, o.check_every);
    int launched = 0, slot = 0, pending = -1;
    bool stop = false;
    int64_t step_launches = 0;
    while (launched < o.max_outer && !stop) {
        const int chunk = std::min(every, o.max_outer - launched);
        for (int k = 0; k < chunk; ++k) {
            if (o.use_graph) {
                PTP_CUDA(cudaGraphLaunch(c.graph_exec[gi], st));
                step_launches += c.launches_per_step[gi];
            } else {
                step_launches += enqueue_step(c, kind);
            }
        }
        launched += chunk;
        PTP_CUDA(cudaMemcpyAsync(&c.h_status[slot], c.status.p, sizeof(Status), cudaMemcpyDeviceToHost, st));
        PTP_CUDA(cudaEventRecord(chk[slot], st));
        if (pending >= 0) {
            PTP_CUDA(cudaEventSynchronize(chk[pending]));
            if (c.h_status[pending].done) stop = true;
        }
        pending = slot;
        slot ^= 1;
    }
    PTP_CUDA(cudaEventRecord(e1, st));
    PTP_CUDA(cudaStreamSynchronize(st));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0); cudaEventDestroy(e1);
    cudaEventDestroy(chk[0]); cudaEventDestroy(chk[1]);
    const double wall = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    c.fz_on = false;
    const int rc = solve_end(c, stats, kind, step_launches, wall, ms);
    if (U) {
        PTP_CUDA(cudaMemcpyAsync(U, X, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
        PTP_CUDA(cudaStreamSynchronize(st));
    }
    return rc;
}

int solve(Ctx& c, const ptp_opts& o, const double* U0, double* U, ptp_stats* stats, int kind) {
    if (kind != STEP_FORWARD || !o.init_static || U0) return run_fixed_point(c, o, U0, U, stats, kind);
    // initialisation of Section 4: start from the static solutions (sigma = 0)
    ptp_stats si;
    std::memset(&si, 0, sizeof(si));
    const int rs = run_fixed_point(c, o, nullptr, nullptr, &si, STEP_STATIC);
    if (rs == PTP_ENAN) {
        if (stats) *stats = si;
        return rs;
    }
    const int rc = run_fixed_point(c, o, c.U.p, U, stats, STEP_FORWARD);
    if (stats) {
        stats->init_ms = si.solve_ms;
        stats->init_iterations = si.outer_iterations;
        stats->kernel_launches += si.kernel_launches;
    }
    return rc;
}

AdjointArgs adjoint_args(Ctx& c) {
    AdjointArgs a{};
    a.n = c.n;
    a.N = c.N;
    a.n_iron = c.n_iron;
    a.n_tri = c.n_tri;
    a.n_coils = c.n_coils;
    a.tau = c.T / c.N;
    a.nu_min = c.nu_min;
    a.nu_max = c.nu_max;
    a.s2sat = c.s_sat * c.s_sat;
    a.e_nodes = c.e_nodes.p;
    a.e_geo = c.e_geo.p;
    a.e_area = c.e_area.p;
    a.mj_ptr = c.mj_ptr.p;
    a.mj_idx = c.mj_idx.p;
    a.mj_val = c.mj_val.p;
    a.coil_b = c.coil_b.p;
    a.coil_sin = c.coil_sin.p;
    a.all_nodes = c.all_nodes.p;
    a.all_area = c.all_area.p;
    a.all_iron = c.all_iron.p;
    a.Jc = c.Jc.p;
    a.partials = c.part_d.p;
    a.counter = c.counter.p;
    a.scalars = c.adj_scal.p;
    return a;
}

void alloc_adjoint(Ctx& c) {
    const size_t cnt = (size_t)c.n * c.N;
    const size_t jc = 3 * (size_t)std::max(c.n_iron, 1) * c.N;
    if (c.Lam.n == cnt && c.Gadj.n == cnt && c.Ustar.n == cnt && c.Jc.n == jc && c.adj_scal.n >= 16) return;
    if (c.Lam.n != cnt) c.Lam.alloc(cnt);
    if (c.Gadj.n != cnt) c.Gadj.alloc(cnt);
    if (c.Ustar.n != cnt) c.Ustar.alloc(cnt);
    if (c.Jc.n != jc) c.Jc.alloc(jc);
    if (c.adj_scal.n < 16) c.adj_scal.alloc(16);
    ++c.buf_gen;
}

double loss_dev(Ctx& c, const double* U) {
    alloc_adjoint(c);
    AdjointArgs a = adjoint_args(c);
    c.launches += launch_adj_rhs(a, U, c.Gadj.p, c.stream);
    double h = 0.0;
    PTP_CUDA(cudaMemcpyAsync(&h, c.adj_scal.p, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    PTP_CUDA(cudaStreamSynchronize(c.stream));
    return h / c.N;
}

int adjoint_gradient(Ctx& c, const ptp_opts& o, const double* U, double* J, double* dJ_damp, double* dJ_dnu,
                     double* dJ_dsigma, ptp_stats* st) {
    PTP_REQUIRE(c.n_coils <= kMaxCoils, "the adjoint supports at most 8 coils");
    PTP_REQUIRE(!c.law_exp, "the adjoint supports the saturating reluctivity law only");
    cudaStream_t s = c.stream;
    const size_t cnt = (size_t)c.n * c.N;
    alloc_adjoint(c);
    PTP_CUDA(cudaMemcpyAsync(c.Ustar.p, U, cnt * sizeof(double), cudaMemcpyDeviceToDevice, s));
    AdjointArgs a = adjoint_args(c);
    c.launches += launch_adj_jacobian(a, c.Ustar.p, s);
    c.launches += launch_adj_rhs(a, c.Ustar.p, c.Gadj.p, s);
    double nJ = 0.0;
    PTP_CUDA(cudaMemcpyAsync(&nJ, c.adj_scal.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    c.g_norm = norm_dev(c, c.Gadj.p, cnt);   // synchronises
    const int rc = solve(c, o, nullptr, nullptr, st, STEP_ADJOINT);
    if (rc == PTP_ENAN) return rc;
    c.launches += launch_adj_gradients(a, c.Ustar.p, c.Lam.p, dJ_dsigma, s);
    double h[1 + kMaxCoils + 3];
    PTP_CUDA(cudaMemcpyAsync(h, c.adj_scal.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    PTP_CUDA(cudaStreamSynchronize(s));
    PTP_CUDA(cudaGetLastError());
    if (J) *J = nJ / c.N;
    if (dJ_damp)
        for (int k = 0; k < c.n_coils; ++k) dJ_damp[k] = h[1 + k];
    if (dJ_dnu)
        for (int k = 0; k < 3; ++k) dJ_dnu[k] = h[1 + kMaxCoils + k];
    return rc;
}

template void apply_op<double>(Ctx&, int, int, int, const double*, double*);
template void apply_op<float>(Ctx&, int, int, int, const float*, float*);
template void periodic_apply<double>(Ctx&, int, const double*, double*);
template int spatial_pcg<double>(Ctx&, int, int, const double*, double*, double, int, bool);
template int spatial_pcg<float>(Ctx&, int, int, const float*, float*, double, int, bool);

}  // namespace ptp
