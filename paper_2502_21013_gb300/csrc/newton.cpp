// Newton's method for Problem 1 (method (M2) of Section 4), with Armijo
// back-tracking on the residual norm:
//
//   R_k = F - A(U_k),  J(U_k) d = R_k,  U_{k+1} = U_k + t d,
//   t = 1, 1/2, ... until ||R(U_k + t d)|| <= (1 - 1e-4 t) ||R_k||,
//
// stopped by the rule of Section 4, ||R_k|| <= tol ||R_0||.  J = dA/dU has
// the periodic block structure M/tau + DK(u^n) on the diagonal and -M/tau on
// the cyclic sub-diagonal, with the iron element blocks
// |T| [nu I + 2 nu'(s^2) g g^T] of the adjoint (k_adjoint.cu) in forward time
// order.  Each linear system is solved by right-preconditioned flexible GMRES
// whose preconditioner is the inner solve of the fixed point: V-cycles of
// multigrid in time for the time-invariant operator M d_tau + K_hat.  All
// vectors stay on the device; the Hessenberg least-squares problem (at most
// krylov_dim columns) is solved on the host.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "kernels.h"

namespace ptp {

namespace {

// ||F - A(X)||, written to R when R is set (synchronises)
double residual_norm(Ctx& c, const double* X, double* R) {
    ResidualArgs a = residual_args(c, X, R);
    a.status = nullptr;
    a.check = 0;
    a.done = nullptr;
    a.norm_out = c.kr_s.p;
    c.launches += launch_residual_law(a, c.law_exp ? c.e_law.p : nullptr, c.stream);
    double h = 0.0;
    PTP_CUDA(cudaMemcpyAsync(&h, c.kr_s.p, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    PTP_CUDA(cudaStreamSynchronize(c.stream));
    return h;
}

// The preconditioner and Jacobian of one Krylov step, zout = P^{-1} vin and
// w = J zout, on fixed buffers: captured once as a CUDA graph (re-captured
// when the step key of the context changes) or enqueued directly.
void krylov_step(Ctx& c, const ptp_opts& o) {
    auto enqueue = [&]() {
        mg_precondition(c, c.kr_vin.p, c.kr_zout.p);
        jacobian_apply(c, c.kr_zout.p, c.kr_w.p);
    };
    if (!o.use_graph) {
        enqueue();
        return;
    }
    const int64_t key = step_key(c, o);
    if (!c.newton_exec || c.newton_key != key) {
        if (c.newton_exec) {
            cudaGraphExecDestroy(c.newton_exec);
            c.newton_exec = nullptr;
        }
        cudaGraph_t g;
        PTP_CUDA(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
        const int64_t l0 = c.launches;
        try {
            enqueue();
        } catch (...) {
            cudaStreamEndCapture(c.stream, &g);
            throw;
        }
        c.launches = l0;
        PTP_CUDA(cudaStreamEndCapture(c.stream, &g));
        PTP_CUDA(cudaGraphInstantiate(&c.newton_exec, g, 0));
        cudaGraphDestroy(g);
        c.newton_key = key;
    }
    PTP_CUDA(cudaGraphLaunch(c.newton_exec, c.stream));
}

// Flexible GMRES (right preconditioning, classical Gram-Schmidt with a
// second pass only when the first removed most of the vector: ||w|| after
// < 0.7 ||w|| before, the "twice is enough" rule) for J x = b from x = 0;
// stops when the least-squares residual is below eta ||b|| or after m
// iterations.  Returns the iterations taken.
int fgmres(Ctx& c, const ptp_opts& o, const double* b, double* x, double eta, int m, double* relres) {
    cudaStream_t st = c.stream;
    const size_t cnt = (size_t)c.n * c.N;
    double* V = c.kr_v.p;   // m + 1 basis vectors
    double* Z = c.kr_z.p;   // m preconditioned vectors
    double* w = c.kr_w.p;
    double* ds = c.kr_s.p;  // device scalars: [1 .. 1+32) dots, [33 .. 65) second pass, [65] ||w||^2
    double* d1 = ds + 1;
    double* d2 = ds + 1 + kMaxKrylovDots;
    double* dn = ds + 1 + 2 * kMaxKrylovDots;   // ||w||^2 after the first pass, then ||w||
    double* dy = ds + 2 + 2 * kMaxKrylovDots;   // solution coefficients
    double* d0 = ds + 2 + 3 * kMaxKrylovDots;   // ||w||^2 before orthogonalisation
    c.launches += launch_mdot(cnt, 1, b, cnt, b, c.part_d.p, c.counter.p, dn, st);
    double beta2 = 0.0;
    PTP_CUDA(cudaMemcpyAsync(&beta2, dn, sizeof(double), cudaMemcpyDeviceToHost, st));
    PTP_CUDA(cudaStreamSynchronize(st));
    PTP_CUDA(cudaMemsetAsync(x, 0, cnt * sizeof(double), st));
    const double beta = std::sqrt(beta2);
    if (!(beta > 0.0) || !std::isfinite(beta)) {
        *relres = 0.0;
        return 0;
    }
    PTP_CUDA(cudaMemcpyAsync(dn, &beta, sizeof(double), cudaMemcpyHostToDevice, st));
    c.launches += launch_div_scalar(cnt, b, dn, V, st);
    PTP_CUDA(cudaMemcpyAsync(c.kr_vin.p, V, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
    std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m, 0.0), sn(m, 0.0), g(m + 1, 0.0);
    auto Hat = [&](int i, int j) -> double& { return H[(size_t)j * (m + 1) + i]; };
    g[0] = beta;
    std::vector<double> hd(2 * kMaxKrylovDots + 1);   // both passes and ||w||^2, one copy
    int k = 0;
    double res = beta;
    for (int j = 0; j < m; ++j) {
        double* zj = Z + (size_t)j * cnt;
        krylov_step(c, o);   // vin holds v_j
        ++c.launches;
        PTP_CUDA(cudaMemcpyAsync(zj, c.kr_zout.p, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
        c.launches += launch_mdot(cnt, 1, w, cnt, w, c.part_d.p, c.counter.p, d0, st);
        c.launches += launch_mdot(cnt, j + 1, V, cnt, w, c.part_d.p, c.counter.p, d1, st);
        c.launches += launch_maxpy(cnt, j + 1, V, cnt, d1, -1.0, w, st);
        c.launches += launch_mdot(cnt, 1, w, cnt, w, c.part_d.p, c.counter.p, dn, st);
        double w0 = 0.0;
        PTP_CUDA(cudaMemcpyAsync(hd.data(), d1, hd.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        PTP_CUDA(cudaMemcpyAsync(&w0, d0, sizeof(double), cudaMemcpyDeviceToHost, st));
        PTP_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i <= j; ++i) Hat(i, j) = hd[i];
        if (hd[2 * kMaxKrylovDots] < 0.49 * w0) {   // second pass
            c.launches += launch_mdot(cnt, j + 1, V, cnt, w, c.part_d.p, c.counter.p, d2, st);
            c.launches += launch_maxpy(cnt, j + 1, V, cnt, d2, -1.0, w, st);
            c.launches += launch_mdot(cnt, 1, w, cnt, w, c.part_d.p, c.counter.p, dn, st);
            PTP_CUDA(cudaMemcpyAsync(hd.data(), d1, hd.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
            PTP_CUDA(cudaStreamSynchronize(st));
            for (int i = 0; i <= j; ++i) Hat(i, j) += hd[kMaxKrylovDots + i];
        }
        const double hn = std::sqrt(std::max(hd[2 * kMaxKrylovDots], 0.0));
        Hat(j + 1, j) = hn;
        if (!std::isfinite(hn)) throw Error(PTP_ENAN, "newton: non-finite Krylov vector");
        if (hn > 0.0 && j + 1 < m) {
            PTP_CUDA(cudaMemcpyAsync(dn, &hn, sizeof(double), cudaMemcpyHostToDevice, st));
            c.launches += launch_div_scalar(cnt, w, dn, V + (size_t)(j + 1) * cnt, st);
            PTP_CUDA(cudaMemcpyAsync(c.kr_vin.p, V + (size_t)(j + 1) * cnt, cnt * sizeof(double),
                                     cudaMemcpyDeviceToDevice, st));
        }
        // Givens rotations on column j
        for (int i = 0; i < j; ++i) {
            const double a = Hat(i, j), bb = Hat(i + 1, j);
            Hat(i, j) = cs[i] * a + sn[i] * bb;
            Hat(i + 1, j) = -sn[i] * a + cs[i] * bb;
        }
        const double a = Hat(j, j), bb = Hat(j + 1, j);
        const double r = std::hypot(a, bb);
        cs[j] = r > 0.0 ? a / r : 1.0;
        sn[j] = r > 0.0 ? bb / r : 0.0;
        Hat(j, j) = r;
        Hat(j + 1, j) = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        k = j + 1;
        res = std::fabs(g[j + 1]);
        if (res <= eta * beta || hn == 0.0) break;
    }
    // back substitution H(0:k, 0:k) y = g(0:k), then x = Z y
    std::vector<double> y(k, 0.0);
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int l = i + 1; l < k; ++l) s -= Hat(i, l) * y[l];
        y[i] = Hat(i, i) != 0.0 ? s / Hat(i, i) : 0.0;
    }
    PTP_CUDA(cudaMemcpyAsync(dy, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, st));
    c.launches += launch_maxpy(cnt, k, Z, cnt, dy, 1.0, x, st);
    PTP_CUDA(cudaStreamSynchronize(st));   // y (host) is released on return
    *relres = res / beta;
    return k;
}

void grow(DBuf<double>& b, size_t n) {
    if (b.n < n) b.alloc(n);
}

}  // namespace

void jacobian_apply(Ctx& c, const double* V, double* Y) {
    // fluxes of the iron elements: A_T grad v with the stored coefficients
    c.launches += launch_adj_elem_flux(adjoint_args(c), V, c.Qx.p, c.Qy.p, nullptr, c.stream);
    // node pass with no source: r = -(M d_tau v + K_lin v + gathered fluxes), written as -r
    ResidualArgs a = residual_args(c, V, nullptr);
    a.n_coils = 0;
    a.Fext = nullptr;
    a.skip_flux = 1;
    a.b_d = Y;
    a.scale = -1.0;
    a.status = nullptr;
    a.check = 0;
    a.done = nullptr;
    c.launches += launch_residual(a, c.stream);
}

int newton_solve(Ctx& c, const ptp_opts& o, const double* U0, double* Uout, ptp_stats* stats) {
    const auto t0 = std::chrono::steady_clock::now();
    PTP_REQUIRE(!c.law_exp, "Newton's method supports the saturating reluctivity law only");
    PTP_REQUIRE(o.krylov_dim >= 1 && o.krylov_dim <= kMaxKrylovDots - 1, "newton: krylov_dim must be 1..31");
    PTP_REQUIRE(o.newton_eta > 0.0 && o.newton_eta < 1.0, "newton: newton_eta must lie in (0, 1)");
    require_coarse(c);
    PTP_REQUIRE(o.precision == c.opts.precision && o.spatial_prec == c.opts.spatial_prec &&
                    o.time_levels == c.opts.time_levels && o.coarse_steps == c.opts.coarse_steps &&
                    o.coarse_solver == c.opts.coarse_solver,
                "precision / preconditioner / hierarchy options differ from ptp_setup");
    cudaStream_t st = c.stream;
    const size_t cnt = (size_t)c.n * c.N;
    const int m = o.krylov_dim;
    // initial iterate: U0, the static solutions (init_static), or zero
    ptp_stats si;
    std::memset(&si, 0, sizeof(si));
    if (!U0 && o.init_static) {
        const int rs = solve(c, o, nullptr, nullptr, &si, STEP_STATIC);
        if (rs == PTP_ENAN) throw Error(PTP_ENAN, "newton: the static initialisation diverged");
    } else if (U0) {
        PTP_CUDA(cudaMemcpyAsync(c.U.p, U0, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
        PTP_CUDA(cudaMemsetAsync(c.U.p, 0, cnt * sizeof(double), st));
    }
    c.opts = o;
    resolve_time_smoother(c);
    alloc_adjoint(c);
    ensure_staging(c);
    grow(c.kr_v, (size_t)(m + 1) * cnt);
    grow(c.kr_z, (size_t)m * cnt);
    grow(c.kr_w, cnt);
    grow(c.kr_t, cnt);
    grow(c.kr_r, cnt);
    grow(c.kr_d, cnt);
    grow(c.kr_vin, cnt);
    grow(c.kr_zout, cnt);
    grow(c.kr_s, 8 + 4 * (size_t)kMaxKrylovDots);
    const int64_t launches0 = c.launches;
    double* U = c.U.p;
    double* R = c.R.p;
    double* Ut = c.kr_t.p;
    double* Rt = c.kr_r.p;
    double* d = c.kr_d.p;   // Newton direction
    const double r0 = residual_norm(c, U, R);
    double r = r0;
    int it = 0, inner = 0;
    bool conv = r0 == 0.0;
    while (!conv && it < o.max_outer) {
        if (!std::isfinite(r)) break;
        c.launches += launch_adj_jacobian(adjoint_args(c), U, st, false);
        double rel = 0.0;
        inner += fgmres(c, o, R, d, o.newton_eta, m, &rel);
        double t = 1.0, rt = 0.0;
        for (;;) {
            launch_lincomb(cnt, 1.0, U, t, d, Ut, st);
            ++c.launches;
            rt = residual_norm(c, Ut, Rt);
            if ((std::isfinite(rt) && rt <= (1.0 - 1e-4 * t) * r) || t < 1.0 / 1024.0) break;
            t *= 0.5;
        }
        // accept the trial iterate (copied: captured graphs of this context
        // hold the address of U) and its residual (local buffers, swapped)
        PTP_CUDA(cudaMemcpyAsync(U, Ut, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
        std::swap(R, Rt);
        r = rt;
        ++it;
        conv = r <= o.tol * r0;
    }
    const double wall = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (stats) {
        stats->outer_iterations = it;
        stats->converged = conv ? 1 : 0;
        stats->res0 = r0;
        stats->res_final = r;
        stats->setup_ms = c.setup_ms;
        stats->solve_ms = wall - si.solve_ms;
        stats->time_levels = c.active_levels;
        stats->spatial_levels = (int)c.sl.size();
        stats->init_ms = si.solve_ms;
        stats->init_iterations = si.outer_iterations;
        stats->inner_iterations = inner;
        stats->kernel_launches = c.launches - launches0 + si.kernel_launches;
    }
    if (Uout) {
        PTP_CUDA(cudaMemcpyAsync(Uout, U, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
        PTP_CUDA(cudaStreamSynchronize(st));
    }
    if (!std::isfinite(r)) return PTP_ENAN;
    return conv ? PTP_OK : PTP_ENOTCONV;
}

}  // namespace ptp
