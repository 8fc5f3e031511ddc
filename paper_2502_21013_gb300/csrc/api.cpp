// C ABI of the library (declared in include/ptp.h).  Every entry point
// catches exceptions and turns them into status codes and a message.
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>

#include "kernels.h"

using ptp::Ctx;
using ptp::Error;

struct ptp_ctx {
    Ctx c;
};

namespace ptp {
Ctx* ctx_of(ptp_ctx* h) { return h ? &h->c : nullptr; }
}  // namespace ptp

namespace {

// Runs f, mapping exceptions to status codes.  Entry points that only
// record host-side problem data pass device = false and never touch CUDA.
template <typename F>
int guarded(ptp_ctx* h, F&& f, bool device = true) {
    if (!h) return PTP_EINVAL;
    try {
        h->c.err.clear();
        if (device) {
            PTP_CUDA(cudaSetDevice(h->c.device));
            ptp::apply_schedule(h->c);
            if (!h->c.own_stream) {
                PTP_CUDA(cudaStreamCreateWithFlags(&h->c.own_stream, cudaStreamNonBlocking));
                if (!h->c.stream) h->c.stream = h->c.own_stream;
            }
        }
        return f(h->c);
    } catch (const Error& e) {
        h->c.err = e.what();
        return e.code;
    } catch (const std::exception& e) {
        h->c.err = e.what();
        return PTP_EINVAL;
    } catch (...) {
        h->c.err = "unknown error";
        return PTP_EINVAL;
    }
}

void need_ready(const Ctx& c) {
    if (!c.ready) throw Error(PTP_ESTATE, "call ptp_setup first");
}

}  // namespace

// The same error handling and per-call set-up (device, row-block size, own
// stream) for entry points defined in other translation units.
namespace ptp {
int run_entry(ptp_ctx* h, const std::function<int(Ctx&)>& f) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        return f(c);
    });
}
}  // namespace ptp

namespace {

void invalidate(Ctx& c) {
    c.ready = false;
    for (int k = 0; k < 3; ++k) {
        if (c.graph_exec[k]) {
            cudaGraphExecDestroy(c.graph_exec[k]);
            c.graph_exec[k] = nullptr;
        }
        c.graph_key[k] = -1;
    }
    if (c.newton_exec) {
        cudaGraphExecDestroy(c.newton_exec);
        c.newton_exec = nullptr;
    }
    c.newton_key = -1;
    c.lambda_min = -1.0;
}

// device copies for the host-pointer entry points
struct Staging {
    double* p = nullptr;
    ~Staging() { if (p) cudaFree(p); }
    double* get(size_t n) {
        if (n == 0) return nullptr;
        cudaError_t e = cudaMalloc(&p, n * sizeof(double));
        if (e != cudaSuccess) { p = nullptr; throw Error(PTP_ENOMEM, "staging allocation failed"); }
        return p;
    }
};

int check_level(const Ctx& c, int level) {
    if (level < 0 || level >= (int)c.tl.size()) throw Error(PTP_EINVAL, "time level out of range");
    return c.tl[level].N;
}

}  // namespace

extern "C" {

void ptp_default_opts(ptp_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-8;
    o->max_outer = 5000;
    o->precision = PTP_MIXED;
    o->time_levels = 0;
    o->coarse_steps = 1;
    o->vcycles = 1;
    o->pre_smooth = 1;
    o->post_smooth = -1;   // chosen per problem (with omega_t)
    o->omega_t = 0.0;
    o->pcg_iters = 1;
    o->spatial_prec = PTP_PREC_GMG;
    o->gmg_smooth = 1;
    o->gmg_omega = 0.7;
    o->coarse_tol = 1e-6;
    o->coarse_max_it = 4;
    o->use_graph = 1;
    o->check_every = 16;
    o->coarse_cycles = 8;
    o->coarse_solver = PTP_COARSE_VCYCLES;
    o->dft_max_it = 30;
    o->init_tol = 0.0;
    o->init_static = 0;
    o->newton_eta = 1e-2;
    o->krylov_dim = 20;
    o->stencil = 1;
    o->k1_fused = 0;
    o->coarse_direct = 1;
    o->fuse_coarse = 0;
    o->fuse_update = 1;
}

const char* ptp_version(void) { return "ptp 0.1 (sm_103a)"; }

int ptp_create(ptp_ctx** out, int device) {
    if (!out) return PTP_EINVAL;
    *out = nullptr;
    ptp_ctx* h = nullptr;
    try {
        h = new ptp_ctx();
    } catch (...) {
        return PTP_ENOMEM;
    }
    if (device < 0) {
        delete h;
        return PTP_EINVAL;
    }
    h->c.device = device;  // CUDA is first touched by ptp_setup / ptp_set_stream
    *out = h;
    return PTP_OK;
}

void ptp_abi_sizes(size_t* opts_bytes, size_t* stats_bytes) {
    if (opts_bytes) *opts_bytes = sizeof(ptp_opts);
    if (stats_bytes) *stats_bytes = sizeof(ptp_stats);
}

void ptp_destroy(ptp_ctx* h) {
    if (!h) return;
    if (h->c.own_stream || h->c.stream) {
        cudaSetDevice(h->c.device);
        cudaStreamSynchronize(h->c.stream);
    }
    delete h;
}

const char* ptp_last_error(const ptp_ctx* h) { return h ? h->c.err.c_str() : "null context"; }

int ptp_set_stream(ptp_ctx* h, void* stream) {
    return guarded(h, [&](Ctx& c) {
        PTP_CUDA(cudaStreamSynchronize(c.stream));
        c.stream = stream ? (cudaStream_t)stream : c.own_stream;
        invalidate(c);
        return PTP_OK;
    });
}

int ptp_set_mesh(ptp_ctx* h, int n_nodes, const double* xy, int n_tri, const int32_t* tri,
                 const uint8_t* dirichlet) {
    return guarded(h, [&](Ctx& c) {
        PTP_REQUIRE(n_nodes > 0 && n_tri > 0 && xy && tri && dirichlet, "ptp_set_mesh: bad arguments");
        for (int64_t k = 0; k < 3 * (int64_t)n_tri; ++k)
            PTP_REQUIRE(tri[k] >= 0 && tri[k] < n_nodes, "ptp_set_mesh: vertex id out of range");
        for (int64_t k = 0; k < 2 * (int64_t)n_nodes; ++k)
            PTP_REQUIRE(std::isfinite(xy[k]), "ptp_set_mesh: non-finite coordinate");
        c.n_nodes = n_nodes;
        c.n_tri = n_tri;
        c.xy.assign(xy, xy + 2 * (size_t)n_nodes);
        c.tri.assign(tri, tri + 3 * (size_t)n_tri);
        c.dirichlet.assign(dirichlet, dirichlet + n_nodes);
        c.structured = false;
        invalidate(c);
        return PTP_OK;
    }, false);
}

int ptp_set_structured(ptp_ctx* h, int nx, int ny, double x0, double y0, double x1, double y1) {
    return guarded(h, [&](Ctx& c) {
        ptp::make_structured_mesh(c, nx, ny, x0, y0, x1, y1);
        invalidate(c);
        return PTP_OK;
    }, false);
}

int ptp_set_materials(ptp_ctx* h, const double* sigma_e, const uint8_t* nonlinear_e, double nu_min,
                      double nu_max, double s_sat, double nu_linear) {
    return guarded(h, [&](Ctx& c) {
        PTP_REQUIRE(c.n_tri > 0, "ptp_set_materials: set the mesh first");
        PTP_REQUIRE(sigma_e && nonlinear_e, "ptp_set_materials: null array");
        PTP_REQUIRE(nu_min > 0 && nu_max >= nu_min && nu_linear > 0 && s_sat >= 1e-15 && s_sat <= 1e15 &&
                        std::isfinite(nu_max) && std::isfinite(nu_linear),
                    "ptp_set_materials: need 0 < nu_min <= nu_max, nu_linear > 0 (finite), 1e-15 <= s_sat <= 1e15");
        for (int e = 0; e < c.n_tri; ++e)
            PTP_REQUIRE(sigma_e[e] >= 0.0 && std::isfinite(sigma_e[e]),
                        "ptp_set_materials: negative or non-finite conductivity");
        c.sigma.assign(sigma_e, sigma_e + c.n_tri);
        c.nonlinear.assign(nonlinear_e, nonlinear_e + c.n_tri);
        c.nu_min = nu_min;
        c.nu_max = nu_max;
        c.s_sat = s_sat;
        c.nu_linear = nu_linear;
        c.have_materials = true;
        invalidate(c);
        return PTP_OK;
    }, false);
}

int ptp_set_law_exp(ptp_ctx* h, const double* abcd) {
    return guarded(h, [&](Ctx& c) {
        PTP_REQUIRE(c.have_materials, "ptp_set_law_exp: set the materials first");
        PTP_REQUIRE((int)c.nonlinear.size() == c.n_tri, "ptp_set_law_exp: the materials do not match the mesh");
        if (!abcd) {
            c.law_exp = false;
            c.law_abcd.clear();
        } else {
            for (int e = 0; e < c.n_tri; ++e) {
                if (!c.nonlinear[e]) continue;
                const double* L = abcd + 4 * (size_t)e;
                PTP_REQUIRE(L[0] >= 0.0 && L[1] > 0.0 && L[2] >= 1.0 && L[3] > 0.0 && std::isfinite(L[0]) &&
                                std::isfinite(L[1]) && std::isfinite(L[2]) && std::isfinite(L[3]),
                            "ptp_set_law_exp: need a >= 0, b > 0, c >= 1, d > 0 on every nonlinear element");
            }
            c.law_abcd.assign(abcd, abcd + 4 * (size_t)c.n_tri);
            c.law_exp = true;
        }
        invalidate(c);
        return PTP_OK;
    }, false);
}

int ptp_set_khat(ptp_ctx* h, const double* khat_e) {
    return guarded(h, [&](Ctx& c) {
        PTP_REQUIRE(c.n_tri > 0, "ptp_set_khat: set the mesh first");
        if (!khat_e) {
            c.khat.clear();
        } else {
            for (int e = 0; e < c.n_tri; ++e)
                PTP_REQUIRE(khat_e[e] > 0.0 && std::isfinite(khat_e[e]), "ptp_set_khat: weights must be positive");
            c.khat.assign(khat_e, khat_e + c.n_tri);
        }
        invalidate(c);
        return PTP_OK;
    }, false);
}

int ptp_set_sources(ptp_ctx* h, int n_coils, const int32_t* coil_of_elem, const double* amp,
                    const double* phase) {
    return guarded(h, [&](Ctx& c) {
        PTP_REQUIRE(c.n_tri > 0, "ptp_set_sources: set the mesh first");
        PTP_REQUIRE(n_coils >= 0, "ptp_set_sources: negative coil count");
        PTP_REQUIRE(n_coils == 0 || (coil_of_elem && amp && phase), "ptp_set_sources: null array");
        // everything is checked before the context changes, so a rejected
        // call leaves the previous sources in place
        if (n_coils > 0) {
            for (int e = 0; e < c.n_tri; ++e)
                PTP_REQUIRE(coil_of_elem[e] >= -1 && coil_of_elem[e] < n_coils,
                            "ptp_set_sources: coil id out of range");
            for (int k = 0; k < n_coils; ++k)
                PTP_REQUIRE(std::isfinite(amp[k]) && std::isfinite(phase[k]),
                            "ptp_set_sources: non-finite amplitude or phase");
        }
        c.n_coils = n_coils;
        if (n_coils > 0) {
            c.coil_of_elem.assign(coil_of_elem, coil_of_elem + c.n_tri);
            c.amp.assign(amp, amp + n_coils);
            c.phase.assign(phase, phase + n_coils);
        } else {
            c.coil_of_elem.assign(c.n_tri, -1);
            c.amp.clear();
            c.phase.clear();
        }
        invalidate(c);
        return PTP_OK;
    }, false);
}

int ptp_set_time(ptp_ctx* h, double T, int N) {
    return guarded(h, [&](Ctx& c) {
        PTP_REQUIRE(T > 0 && std::isfinite(T) && N >= 1, "ptp_set_time: need a finite T > 0 and N >= 1");
        c.T = T;
        c.N = N;
        invalidate(c);
        return PTP_OK;
    }, false);
}

int ptp_setup(ptp_ctx* h, const ptp_opts* opts) {
    return guarded(h, [&](Ctx& c) {
        const auto t0 = std::chrono::steady_clock::now();
        invalidate(c);
        ptp_opts o;
        if (opts) o = *opts; else ptp_default_opts(&o);
        PTP_REQUIRE(o.precision == PTP_FP64 || o.precision == PTP_MIXED, "ptp_setup: bad precision");
        PTP_REQUIRE(o.spatial_prec == PTP_PREC_JACOBI || o.spatial_prec == PTP_PREC_GMG,
                    "ptp_setup: bad spatial preconditioner");
        PTP_REQUIRE(o.coarse_steps == 1 || o.coarse_steps == 2, "ptp_setup: coarse_steps must be 1 or 2");
        PTP_REQUIRE(o.coarse_solver == PTP_COARSE_VCYCLES || o.coarse_solver == PTP_COARSE_DFT,
                    "ptp_setup: bad coarse_solver");
        c.opts = o;
        ptp::build_problem(c);
        ptp::build_hierarchy(c);
        ptp::alloc_work(c);
        {   // ||F|| scales the float right-hand side of the first outer step
            const size_t cnt = (size_t)c.n * c.N;
            double* F = nullptr;
            PTP_CUDA(cudaMallocAsync((void**)&F, cnt * sizeof(double), c.stream));
            ptp::source_dev(c, F);
            c.f_norm = ptp::norm_dev(c, F, cnt);
            PTP_CUDA(cudaFreeAsync(F, c.stream));
        }
        // the smallest kappa that selects an automatic time smoother
        if ((o.omega_t <= 0 || o.post_smooth < 0) && c.coarse_ops[0] >= 0) {
            c.lambda_min = ptp::estimate_lambda_min(c);
            ptp::resolve_time_smoother(c);   // c.opts as the entry points without options use it
        }
        PTP_CUDA(cudaStreamSynchronize(c.stream));
        c.ready = true;
        c.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return PTP_OK;
    });
}

int ptp_sizes(const ptp_ctx* h, int* n_free, int* N, int* n_tri, int* time_levels) {
    if (!h) return PTP_EINVAL;
    const Ctx& c = h->c;
    if (!c.ready) return PTP_ESTATE;
    if (n_free) *n_free = c.n;
    if (N) *N = c.N;
    if (n_tri) *n_tri = c.n_tri;
    if (time_levels) *time_levels = (int)c.tl.size();
    return PTP_OK;
}

int ptp_autotune(ptp_ctx* h, int* block_threads, double* best_us) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        const int b = ptp::autotune(c, best_us);
        if (block_threads) *block_threads = b;
        return PTP_OK;
    });
}

int ptp_info(const ptp_ctx* h, int64_t* counts, int n) {
    if (!h || !counts || n < 0) return PTP_EINVAL;
    const Ctx& c = h->c;
    if (!c.ready) return PTP_ESTATE;
    const int64_t v[PTP_INFO_COUNT] = {c.n, c.N, c.n_tri, c.n_iron, (int64_t)c.inc_elem.n, (int64_t)c.l_idx.n,
                                       (int64_t)c.m_idx.n, c.sl[0].op.nnz, (int64_t)c.sl.size(),
                                       (int64_t)c.tl.size(), c.n_coils, c.row_block, c.st_tt, c.st_waves};
    const int m = n < PTP_INFO_COUNT ? n : PTP_INFO_COUNT;
    for (int k = 0; k < m; ++k) counts[k] = v[k];
    return m;
}

int ptp_source_dev(ptp_ctx* h, double* F) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        PTP_REQUIRE(F, "ptp_source: null output");
        ptp::source_dev(c, F);
        PTP_CUDA(cudaGetLastError());
        return PTP_OK;
    });
}

int ptp_source(ptp_ctx* h, double* F) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        PTP_REQUIRE(F, "ptp_source: null output");
        const size_t cnt = (size_t)c.n * c.N;
        ptp::ensure_staging(c);
        ptp::source_dev(c, c.R.p);
        PTP_CUDA(cudaMemcpyAsync(F, c.R.p, cnt * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        PTP_CUDA(cudaStreamSynchronize(c.stream));
        return PTP_OK;
    });
}

static int residual_impl(Ctx& c, const double* U, double* R, double* norm) {
    ptp::residual_dev(c, U, R, nullptr, nullptr, 0.0, false);
    PTP_CUDA(cudaGetLastError());
    if (norm) {
        ptp::Status s;
        PTP_CUDA(cudaMemcpyAsync(&s, c.status.p, sizeof(s), cudaMemcpyDeviceToHost, c.stream));
        PTP_CUDA(cudaStreamSynchronize(c.stream));
        *norm = s.res;
    }
    return PTP_OK;
}

int ptp_residual_dev(ptp_ctx* h, const double* U, double* R, double* norm) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        PTP_REQUIRE(U && U != R, "ptp_residual: null input, or R is U");
        return residual_impl(c, U, R, norm);
    });
}

int ptp_residual(ptp_ctx* h, const double* U, double* R, double* norm) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        PTP_REQUIRE(U, "ptp_residual: null input");
        const size_t cnt = (size_t)c.n * c.N;
        ptp::ensure_staging(c);
        PTP_CUDA(cudaMemcpyAsync(c.Ud.p, U, cnt * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        residual_impl(c, c.Ud.p, R ? c.R.p : nullptr, norm);
        if (R) PTP_CUDA(cudaMemcpyAsync(R, c.R.p, cnt * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        PTP_CUDA(cudaStreamSynchronize(c.stream));
        return PTP_OK;
    });
}

int ptp_apply_shifted_dev(ptp_ctx* h, int level, const double* X, double* Y) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        const int N = check_level(c, level);
        PTP_REQUIRE(X && Y && (const void*)X != (const void*)Y, "ptp_apply_shifted: null or aliased pointers");
        ptp::apply_op<double>(c, 0, c.tl[level].op, N, X, Y);
        PTP_CUDA(cudaGetLastError());
        return PTP_OK;
    });
}

int ptp_apply_shifted_f32_dev(ptp_ctx* h, int level, const float* X, float* Y) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        const int N = check_level(c, level);
        PTP_REQUIRE(X && Y && (const void*)X != (const void*)Y, "ptp_apply_shifted_f32: null or aliased pointers");
        ptp::apply_op<float>(c, 0, c.tl[level].op, N, X, Y);
        PTP_CUDA(cudaGetLastError());
        return PTP_OK;
    });
}

int ptp_periodic_apply_dev(ptp_ctx* h, int level, const double* X, double* Y) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        check_level(c, level);
        PTP_REQUIRE(X && Y && X != Y, "ptp_periodic_apply: null or aliased pointers");
        ptp::periodic_apply<double>(c, level, X, Y);
        PTP_CUDA(cudaGetLastError());
        return PTP_OK;
    });
}

int ptp_periodic_residual_f32_dev(ptp_ctx* h, int level, const float* X, const float* B, float* R) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        check_level(c, level);
        PTP_REQUIRE(c.opts.precision == PTP_MIXED, "ptp_periodic_residual_f32: needs a PTP_MIXED context");
        PTP_REQUIRE(X && B && R && (const void*)R != (const void*)X && (const void*)R != (const void*)B,
                    "ptp_periodic_residual_f32: null or aliased pointers");
        ptp::periodic_residual_f32(c, level, X, B, R);
        PTP_CUDA(cudaGetLastError());
        return PTP_OK;
    });
}

int ptp_spatial_solve_dev(ptp_ctx* h, int level, const double* B, double* X, double tol, int max_it,
                          int* iters) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        const int N = check_level(c, level);
        PTP_REQUIRE(B && X && (const void*)B != (const void*)X && max_it >= 1, "ptp_spatial_solve: bad arguments");
        int it = ptp::spatial_pcg<double>(c, c.tl[level].op, N, B, X, tol, max_it, true);
        PTP_CUDA(cudaGetLastError());
        if (iters) *iters = it;
        return PTP_OK;
    });
}

int ptp_spatial_solve_f32_dev(ptp_ctx* h, int level, const float* B, float* X, double tol, int max_it,
                              int* iters) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        const int N = check_level(c, level);
        PTP_REQUIRE(B && X && (const void*)B != (const void*)X && max_it >= 1, "ptp_spatial_solve_f32: bad arguments");
        int it = ptp::spatial_pcg<float>(c, c.tl[level].op, N, B, X, tol, max_it, true);
        PTP_CUDA(cudaGetLastError());
        if (iters) *iters = it;
        return PTP_OK;
    });
}

int ptp_periodic_solve_dev(ptp_ctx* h, const ptp_opts* opts, const double* B, double* X, int cycles,
                           double* relres) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        PTP_REQUIRE(B && X && (const void*)B != (const void*)X && cycles >= 1, "ptp_periodic_solve: bad arguments");
        if (opts) {
            PTP_REQUIRE(opts->precision == c.opts.precision && opts->spatial_prec == c.opts.spatial_prec &&
                            opts->time_levels == c.opts.time_levels && opts->coarse_steps == c.opts.coarse_steps &&
                            opts->coarse_solver == c.opts.coarse_solver,
                        "ptp_periodic_solve: hierarchy options differ from ptp_setup");
            c.opts = *opts;
        }
        ptp::resolve_time_smoother(c);
        ptp::periodic_mg_solve(c, B, X, cycles, relres);
        PTP_CUDA(cudaGetLastError());
        return PTP_OK;
    });
}

int ptp_solve_dev(ptp_ctx* h, const ptp_opts* opts, const double* U0, double* U, ptp_stats* stats) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        ptp_opts o = opts ? *opts : c.opts;
        PTP_REQUIRE(o.max_outer >= 1 && o.tol >= 0, "ptp_solve: bad options");
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return ptp::solve(c, o, U0, U, stats);
    });
}

int ptp_static_solve_dev(ptp_ctx* h, const ptp_opts* opts, double* U, ptp_stats* stats) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        ptp_opts o = opts ? *opts : c.opts;
        PTP_REQUIRE(o.max_outer >= 1 && o.tol >= 0 && o.init_tol >= 0, "ptp_static_solve: bad options");
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return ptp::solve(c, o, nullptr, U, stats, ptp::STEP_STATIC);
    });
}

int ptp_static_solve(ptp_ctx* h, const ptp_opts* opts, double* U, ptp_stats* stats) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        ptp_opts o = opts ? *opts : c.opts;
        PTP_REQUIRE(o.max_outer >= 1 && o.tol >= 0 && o.init_tol >= 0, "ptp_static_solve: bad options");
        if (stats) std::memset(stats, 0, sizeof(*stats));
        int rc = ptp::solve(c, o, nullptr, nullptr, stats, ptp::STEP_STATIC);
        if (U) {
            const size_t cnt = (size_t)c.n * c.N;
            PTP_CUDA(cudaMemcpyAsync(U, c.U.p, cnt * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
            PTP_CUDA(cudaStreamSynchronize(c.stream));
        }
        return rc;
    });
}

int ptp_newton_solve_dev(ptp_ctx* h, const ptp_opts* opts, const double* U0, double* U, ptp_stats* stats) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        ptp_opts o = opts ? *opts : c.opts;
        PTP_REQUIRE(o.max_outer >= 1 && o.tol >= 0, "ptp_newton_solve: bad options");
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return ptp::newton_solve(c, o, U0, U, stats);
    });
}

int ptp_newton_solve(ptp_ctx* h, const ptp_opts* opts, const double* U0, double* U, ptp_stats* stats) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        ptp_opts o = opts ? *opts : c.opts;
        PTP_REQUIRE(o.max_outer >= 1 && o.tol >= 0, "ptp_newton_solve: bad options");
        if (stats) std::memset(stats, 0, sizeof(*stats));
        const size_t cnt = (size_t)c.n * c.N;
        Staging s0;
        double* d0 = nullptr;
        if (U0) {
            d0 = s0.get(cnt);
            PTP_CUDA(cudaMemcpyAsync(d0, U0, cnt * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        }
        int rc = ptp::newton_solve(c, o, d0, nullptr, stats);
        if (U) {
            PTP_CUDA(cudaMemcpyAsync(U, c.U.p, cnt * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
            PTP_CUDA(cudaStreamSynchronize(c.stream));
        }
        return rc;
    });
}

int ptp_jacobian_apply_dev(ptp_ctx* h, const double* U, const double* V, double* Y) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        PTP_REQUIRE(U && V && Y && Y != U && Y != V, "ptp_jacobian_apply_dev: null pointer, or Y is U or V");
        PTP_REQUIRE(!c.law_exp, "ptp_jacobian_apply_dev: saturating reluctivity law only");
        ptp::alloc_adjoint(c);
        c.launches += ptp::launch_adj_jacobian(ptp::adjoint_args(c), U, c.stream, false);
        ptp::jacobian_apply(c, V, Y);
        PTP_CUDA(cudaStreamSynchronize(c.stream));
        PTP_CUDA(cudaGetLastError());
        return PTP_OK;
    });
}

int ptp_solve(ptp_ctx* h, const ptp_opts* opts, const double* U0, double* U, ptp_stats* stats) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        ptp_opts o = opts ? *opts : c.opts;
        PTP_REQUIRE(o.max_outer >= 1 && o.tol >= 0, "ptp_solve: bad options");
        if (stats) std::memset(stats, 0, sizeof(*stats));
        const size_t cnt = (size_t)c.n * c.N;
        Staging s0;
        double* d0 = nullptr;
        if (U0) {
            d0 = s0.get(cnt);
            PTP_CUDA(cudaMemcpyAsync(d0, U0, cnt * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        }
        int rc = ptp::solve(c, o, d0, nullptr, stats);
        if (U) {
            PTP_CUDA(cudaMemcpyAsync(U, c.U.p, cnt * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
            PTP_CUDA(cudaStreamSynchronize(c.stream));
        }
        return rc;
    });
}

int ptp_loss_dev(ptp_ctx* h, const double* U, double* J) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        PTP_REQUIRE(U && J, "ptp_loss_dev: null pointer");
        *J = ptp::loss_dev(c, U);
        return PTP_OK;
    });
}

int ptp_adjoint_gradient_dev(ptp_ctx* h, const ptp_opts* opts, const double* U, double* J, double* dJ_damp,
                             double* dJ_dnu, double* dJ_dsigma, ptp_stats* stats) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        PTP_REQUIRE(U && dJ_dsigma, "ptp_adjoint_gradient_dev: null U or dJ_dsigma");
        ptp_opts o = opts ? *opts : c.opts;
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return ptp::adjoint_gradient(c, o, U, J, dJ_damp, dJ_dnu, dJ_dsigma, stats);
    });
}

int ptp_adjoint_gradient(ptp_ctx* h, const ptp_opts* opts, const double* U, double* J, double* dJ_damp,
                         double* dJ_dnu, double* dJ_dsigma, ptp_stats* stats) {
    return guarded(h, [&](Ctx& c) {
        need_ready(c);
        PTP_REQUIRE(U && dJ_dsigma, "ptp_adjoint_gradient: null U or dJ_dsigma");
        ptp_opts o = opts ? *opts : c.opts;
        if (stats) std::memset(stats, 0, sizeof(*stats));
        const size_t cnt = (size_t)c.n * c.N;
        Staging su, sg;
        double* du = su.get(cnt);
        double* dg = sg.get((size_t)c.n_tri);
        PTP_CUDA(cudaMemcpyAsync(du, U, cnt * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        int rc = ptp::adjoint_gradient(c, o, du, J, dJ_damp, dJ_dnu, dg, stats);
        PTP_CUDA(cudaMemcpyAsync(dJ_dsigma, dg, (size_t)c.n_tri * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        PTP_CUDA(cudaStreamSynchronize(c.stream));
        return rc;
    });
}

}  // extern "C"
