// Internal declarations of the time-periodic solver library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <functional>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/ptp.h"

namespace ptp {

// Thrown inside the library, turned into a status code at the ABI boundary.
struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define PTP_CUDA(call)                                                         \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess)                                                 \
            throw ::ptp::Error(PTP_ECUDA, std::string(#call) + ": " +          \
                                              cudaGetErrorString(e_));         \
    } while (0)

#define PTP_REQUIRE(cond, msg)                                                 \
    do {                                                                       \
        if (!(cond)) throw ::ptp::Error(PTP_EINVAL, msg);                      \
    } while (0)

// Owning device allocation (cudaMalloc / cudaFree).
template <typename T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count) {
        release();
        if (count == 0) return;
        cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            throw Error(PTP_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) +
                                        " bytes failed: " + cudaGetErrorString(e));
        }
        n = count;
    }
    void upload(const std::vector<T>& h, cudaStream_t s) {
        alloc(h.size());
        if (!h.empty())
            PTP_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T),
                                     cudaMemcpyHostToDevice, s));
    }
};

// Host CSR matrix (sorted column indices per row).
struct HostCSR {
    int rows = 0, cols = 0;
    std::vector<int> ptr, idx;
    std::vector<double> val;
    int nnz() const { return (int)idx.size(); }
};

// Device CSR whose values are a combination  cm * v1 + cl * v2  (v2 optional),
// stored in double and in float.
struct DevCSR {
    int rows = 0, cols = 0, nnz = 0;
    DBuf<int> ptr, idx;
    DBuf<double> v1d, v2d;
    DBuf<float> v1f, v2f;
    // the same matrix as padded ELL (row-major, width ell_w; padding points
    // at the row itself with value 0) so a row's loads can all be in flight
    int ell_w = 0;
    DBuf<int> eidx;
    DBuf<int4> pk;          // float path: one 16-byte load per entry {idx, v1, v2, 0}
    DBuf<double> e1d, e2d;
    DBuf<float> e1f, e2f;
    DBuf<double> d1d, d2d;  // diagonals of v1 / v2 (rows == cols only)
    DBuf<float> d1f, d2f;
};

// One level of the spatial (geometric) hierarchy.
struct SpatialLevel {
    int n = 0;          // free nodes on this level
    int nx = 0, ny = 0; // grid nodes (structured)
    DevCSR op;          // pattern with v1 = mass, v2 = stiffness L (Galerkin)
    DevCSR P;           // interpolation from the next coarser level (n x n_c)
    DevCSR R;           // restriction = P^T (n_c x n)
    HostCSR hM, hL, hP;
    // the same operators as a 7-point stencil on the structured grid (free
    // nodes (a, b), W = nx - 2 per row, H = ny - 2 rows, row-major), float,
    // 4 float4 per node: M {C, E, W, N}, M {S, NE, SW, 0}, L {...}, L {...}
    bool st_ok = false;
    DBuf<float4> st_coef;
};

// A spatial operator  cm * M + cl * L  used somewhere in the hierarchy.
struct OpPair {
    double cm = 1.0, cl = 0.0;
    DBuf<double> inv_d;  // dense inverse on the coarsest spatial level (row-major)
    DBuf<float> inv_f;
    // per spatial level, double: padded-ELL values cm M + cl L and its diagonal,
    // formed once so the double row kernels spend no FMA on the combination
    std::vector<DBuf<double>> comb, dcomb;
    // per spatial level, float stencil of cm M + cl L (structured hierarchies)
    std::vector<DBuf<float4>> st_a;
};

struct TimeLevel {
    int N = 0;        // time steps on this level
    double tau = 0.0; // T / N
    int op = 0;       // index into Ctx::ops of (1, tau)
};

// Device-side status of a solve (one allocation, copied to pinned host).
struct Status {
    double res;      // ||R|| of the latest residual evaluation
    double res0;     // ||R|| at the first evaluation
    double tol;      // relative tolerance
    double bscale;   // divisor of the float right-hand side of the next step
    double bscale_used;  // divisor used by the current step (its correction is multiplied back)
    int iteration;   // residual evaluations so far
    int done;        // stopping rule met (1) or non-finite (2)
};

struct Ctx {
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    std::string err;

    // ---- problem definition (host copies) ----
    int n_nodes = 0, n_tri = 0;
    std::vector<double> xy;
    std::vector<int> tri;
    std::vector<uint8_t> dirichlet;
    bool structured = false;
    int gnx = 0, gny = 0;
    double gx0 = 0, gy0 = 0, gx1 = 1, gy1 = 1;
    std::vector<double> sigma;
    std::vector<uint8_t> nonlinear;
    double nu_min = 1, nu_max = 100, s_sat = 1, nu_linear = 100;
    bool have_materials = false;
    bool law_exp = false;             // iron follows a min(exp(b s^2), c) + d (Section 4)
    std::vector<double> law_abcd;     // 4 per element: a, b, c, d
    std::vector<double> khat;         // per-element weights of K_hat (empty: nu_max everywhere)
    int n_coils = 0;
    std::vector<int> coil_of_elem;
    std::vector<double> amp, phase;
    double T = 0;
    int N = 0;

    // ---- derived, after setup ----
    bool ready = false;
    ptp_opts opts{};
    int n = 0;                  // free nodes
    std::vector<int> free_id;   // node -> free index or -1
    double setup_ms = 0;
    double f_norm = 0;          // ||F||, computed at setup
    double g_norm = 0;          // ||g|| of the current adjoint right-hand side

    // residual (K1) data
    int n_iron = 0;             // iron (nonlinear) elements
    DBuf<int> e_nodes;          // 3 per iron element, free index or -1
    DBuf<double> e_geo;         // 6 per iron element: g1x g1y g2x g2y |T| nu_max, |T| dnu s_sat^2
    DBuf<double> e_law;         // exponential law: 4 per iron element |T| a, b, ln c, |T| d
    DBuf<int> inc_ptr, inc_elem;// node -> incident iron elements
    DBuf<double> inc_grad;      // 2 per incidence: grad phi_i on that element
    DBuf<int> m_ptr, m_idx;     // mass rows (only nonzero entries), scaled 1/tau
    DBuf<int> zero_ptr;         // n + 1 zeros: a mass pattern with every row empty (sigma = 0)
    DBuf<double> m_val;
    DBuf<int> l_ptr, l_idx;     // stiffness of the linear elements (nu_linear)
    DBuf<double> l_val;
    DBuf<double> coil_b;        // n_coils x n
    DBuf<double> coil_s;        // n_coils x N: amp sin(2 pi t^n/T + phase)
    std::vector<int> coil_rows; // nodes with a nonzero coil load (host)
    DBuf<double> Qx, Qy;        // iron element flux scratch, n_iron x N each
    // structured grid, saturating law: the residual in one fused pass
    bool k1_struct = false;
    double k1_ihx2 = 0, k1_ihy2 = 0, k1_At = 0, k1_Bt = 0;
    DBuf<uint8_t> k1_cell, k1_flag;
    DBuf<double> k1_mass, k1_lin;
    // adjoint data
    DBuf<double> e_area;        // |T| per iron element
    DBuf<int> mj_ptr, mj_idx;   // loss mass sum_iron sigma_e M1_e
    DBuf<double> mj_val;
    DBuf<double> coil_sin;      // n_coils x N: sin(2 pi t^n / T + phase_c)
    DBuf<int> all_nodes;        // 3 per element, free index or -1
    DBuf<double> all_area;
    DBuf<uint8_t> all_iron;
    DBuf<double> Jc, Lam, Gadj, Ustar;  // adjoint work (allocated on first use)
    DBuf<double> adj_scal;
    // Newton (method M2): Krylov bases, trial iterate and residual, device scalars
    DBuf<double> kr_v, kr_z, kr_w, kr_t, kr_r, kr_d, kr_s;
    DBuf<double> kr_vin, kr_zout;      // fixed input / output of the captured Krylov step
    cudaGraphExec_t newton_exec = nullptr;   // graph: precondition vin -> zout, w = J zout
    int64_t newton_key = -1;

    // spatial hierarchy (level 0 = the mesh itself)
    std::vector<SpatialLevel> sl;
    std::vector<OpPair> ops;
    std::vector<TimeLevel> tl;
    int coarse_ops[2] = {-1, -1};  // ops of the coarsest time level (N_c = 1 or 2)
    // exact tau_c L solve by sine transforms (uniform structured grid, K_hat = nu_max A)
    bool dst_ok = false;
    int dst_logx = 0, dst_logy = 0;
    DBuf<double2> dst_wx, dst_wy;
    DBuf<double> dst_scale, dst_tmp, dst_tmp2;
    bool coarse_ok = false;        // the coarsest time level has 1 or 2 steps
    int active_levels = 0;         // levels of the V-cycle (opts.time_levels)
    // exact periodic solve of one time level by a DFT in time (opts.coarse_solver)
    int dft_level = -1;            // level solved this way, -1 = none
    int dft_op = -1;               // op pair tau_l L: the preconditioner of every mode
    DBuf<double> dft_W;            // e^{-2 pi i j / N_l}, j < N_l (re, im pairs)
    DBuf<double> dft_ck;           // mode shifts c_k = 1 - e^{-2 pi i k / N_l}, k <= N_l / 2
    DBuf<double> dft_w[6];         // complex work vectors, n x 2 (N_l / 2 + 1) doubles

    // work vectors (sized n * N on the finest level)
    DBuf<double> U, R, F, Ud;              // double state / residual / scratch
    // multigrid in time, per level: correction x, right-hand side b (T = float or double)
    std::vector<DBuf<double>> mg_xd, mg_bd;
    std::vector<DBuf<float>> mg_xf, mg_bf;
    // PCG and GMG work (largest level size), double and float
    DBuf<double> w_d[6];
    DBuf<float> w_f[6];
    std::vector<DBuf<double>> g_xd, g_bd, g_rd;  // per spatial level
    std::vector<DBuf<float>> g_xf, g_bf, g_rf;
    DBuf<double> scal;    // device scalars of the host-driven entry points (norms, scales)
    DBuf<double> col_d;   // per-column PCG scalars: 8 x N
    DBuf<float> col_f;
    DBuf<double> part_d;  // block partials for column reductions
    DBuf<float> part_f;
    DBuf<unsigned> counter;  // last-block counters
    DBuf<Status> status;
    Status* h_status = nullptr;  // pinned
    DBuf<int> flag;              // device early-exit flags
    int red_blocks = 0;          // blocks of reduction kernels

    // CUDA graphs of one outer step, per step kind (STEP_FORWARD, STEP_ADJOINT, STEP_STATIC)
    cudaGraphExec_t graph_exec[3] = {nullptr, nullptr, nullptr};
    int64_t graph_key[3] = {-1, -1, -1};
    int64_t launches = 0;        // kernels issued (counting while capturing)
    int64_t launches_per_step[3] = {0, 0, 0};
    int row_block = 256;         // threads per block of the row kernels (autotuned)
    int st_tt = 32, st_waves = 3;  // stencil schedule: largest time tile, blocks per SM (autotuned)
    bool stencil_ok = false;     // every spatial level has a 7-point stencil (structured GMG hierarchy)
    int64_t buf_gen = 0;         // bumped when a buffer a captured graph may use is reallocated
    // smallest eigenvalue of L x = lambda M x (inverse iteration, on first need;
    // < 0: not yet estimated) and the time smoother it selected
    double lambda_min = -1.0;
    double kappa_min = 0.0;      // tau lambda_min on the finest time level
    double rho_time = 0.0;       // model spectral radius of the chosen cycle
    // fused program of the coarse time levels (one cooperative kernel)
    int fz_level = -1;           // time level the program starts at (-1: none)
    bool fz_on = false;          // used by the step being enqueued
    int fz_nph = 0, fz_grid = 0;
    size_t fz_smem = 0;
    int64_t fz_key = -1;
    // time levels 0 .. chain_depth - 1 of the V-cycle being enqueued leave
    // their prolongation to one pass that also updates U (0: none)
    int chain_depth = 0;
    DBuf<unsigned char> fz_blob; // phases, then the argument structs

    ~Ctx();
};

// ---- setup.cpp ----
void build_problem(Ctx& c);       // free numbering, K1 data, mass, coils
void build_hierarchy(Ctx& c);     // spatial levels, time levels, op pairs
void make_structured_mesh(Ctx& c, int nx, int ny, double x0, double y0, double x1, double y1);
void upload_csr(DevCSR& d, const HostCSR& a, const HostCSR* b, bool diag, cudaStream_t s);

// kinds of fixed-point step (solver.cu)
enum StepKind { STEP_FORWARD = 0, STEP_ADJOINT = 1, STEP_STATIC = 2 };

// ---- solver.cu ----
void alloc_work(Ctx& c);
void ensure_work(Ctx& c, bool doubles);   // full-size work vectors of one precision
void ensure_staging(Ctx& c);              // R and Ud at [n][N]
void residual_dev(Ctx& c, const double* U, double* R, double* b_out_d, float* b_out_f,
                  double scale, bool outer_check);
void source_dev(Ctx& c, double* F);
double norm_dev(Ctx& c, const double* x, size_t count);   // ||x||_2, synchronises
template <typename T>
void apply_op(Ctx& c, int s, int op, int N, const T* X, T* Y);
template <typename T>
void periodic_apply(Ctx& c, int level, const T* X, T* Y);
void periodic_residual_f32(Ctx& c, int level, const float* X, const float* B, float* R);
template <typename T>
int spatial_pcg(Ctx& c, int op, int N, const T* B, T* X, double tol, int max_it, bool host_check);
void periodic_mg_solve(Ctx& c, const double* B, double* X, int cycles, double* relres);
int solve(Ctx& c, const ptp_opts& o, const double* U0, double* U, ptp_stats* st, int kind = STEP_FORWARD);
int adjoint_gradient(Ctx& c, const ptp_opts& o, const double* U, double* J, double* dJ_damp, double* dJ_dnu,
                     double* dJ_dsigma, ptp_stats* st);
double loss_dev(Ctx& c, const double* U);
void solve_begin(Ctx& c, const ptp_opts& o, const double* X0, int kind);
int64_t step_key(const Ctx& c, const ptp_opts& o);
int64_t enqueue_step(Ctx& c, int kind);
int solve_end(Ctx& c, ptp_stats* stats, int kind, int64_t step_launches, double solve_ms, float dev_ms);
int autotune(Ctx& c, double* best_us);     // picks c.row_block (and the stencil schedule) by timing
void apply_schedule(const Ctx& c);         // the context's launch schedule for this host thread
void require_coarse(const Ctx& c);         // the time hierarchy has an exact last-level solve
void alloc_adjoint(Ctx& c);                // Jacobian coefficients and adjoint work
void mg_precondition(Ctx& c, const double* v, double* z);   // z = inner periodic solve of v
double estimate_lambda_min(Ctx& c);        // smallest eigenvalue of L x = lambda M x
// replaces an automatic omega_t (<= 0) / post_smooth (< 0) in c.opts by the
// choice for the problem's smallest kappa (estimating lambda_min on first need)
void resolve_time_smoother(Ctx& c);

// ---- tsmooth.cpp ----
struct TimeSmoother {
    int post;       // post-smoothing sweeps
    double omega;   // block-Jacobi damping
    double rho;     // worst model spectral radius over kappa >= kappa_min
};
// spectral radius of the V(pre, post) cycle on the scalar periodic model
// (1 + kappa_l) x^n - x^{n-1}, levels Nl (halving, last one exact), kappa_0 = kappa0
double tmg_cycle_rho(const std::vector<int>& Nl, double kappa0, int pre, int post, double omega);
// post < 0 / omega <= 0: free choices; the cheapest candidate with rho <= 0.6
TimeSmoother choose_time_smoother(const std::vector<int>& Nl, double kappa_min, int pre, int post, double omega);

// ---- api.cpp ----
// Runs f on the context of h (which must be set up) with the error handling
// and per-call set-up of every entry point: exceptions become status codes
// and the message of ptp_last_error.
int run_entry(ptp_ctx* h, const std::function<int(Ctx&)>& f);

// ---- newton.cpp ----
int newton_solve(Ctx& c, const ptp_opts& o, const double* U0, double* U, ptp_stats* st);
void jacobian_apply(Ctx& c, const double* V, double* Y);    // Y = J(U) V, coefficients of U in c.Jc
void set_row_block(int threads);           // row-kernel block size for launches from this thread

}  // namespace ptp
