// Kernel launchers (host functions) shared by the solver translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstring>
#include <utility>
#include <vector>

#include "common.h"

namespace ptp {

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  Every kernel of the library is launched
// with programmatic stream serialisation, so the next kernel in the stream is
// scheduled while the current one drains.  Each kernel therefore starts with
// pdl_wait() (griddepcontrol.wait: block until the preceding grid has
// completed and its memory is visible) as its FIRST statement, before any
// early return, so that completion stays transitive along the stream; then
// pdl_trigger() lets the following grid launch.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
    pdl_wait();
    pdl_trigger();
}

bool pdl_enabled();   // false if the environment sets PTP_NO_PDL

// ---------------------------------------------------------------------------
// Virtual grids.  Kernel bodies index blocks through a VGrid so that one
// launch can serve many instances (the batched step): a single launch passes
// the native grid; a batched launch gives instance i a contiguous range of
// the blocks of a 1-D grid and maps them onto its own gx x gy.
// ---------------------------------------------------------------------------
struct VGrid {
    int bx, by, gx, gy;
};
struct BatchMap {
    const int* inst_of;   // instance of every block of the launch
    const int4* geo;      // per instance: first block, gx, gy
    int n;
};
#ifdef __CUDACC__
__device__ __forceinline__ VGrid native_grid() {
    return VGrid{(int)blockIdx.x, (int)blockIdx.y, (int)gridDim.x, (int)gridDim.y};
}
// instance and virtual block of this block in a batched launch (two
// dependent loads: the block's instance, then that instance's geometry)
__device__ __forceinline__ bool batch_block(const BatchMap& m, int& inst, VGrid& g) {
    const int b = (int)blockIdx.x;
    inst = __ldg(m.inst_of + b);
    const int4 q = __ldg(m.geo + inst);
    const int local = b - q.x;
    if (local < 0 || local >= q.y * q.z) return false;
    g = VGrid{local % q.y, local / q.y, q.y, q.z};
    return true;
}
#endif

// Launch shape of one kernel call: virtual grid gx x gy of `block` threads,
// dynamic shared memory, vector width and kernel variant.
struct KShape {
    int gx = 0, gy = 0, block = 0;
    size_t smem = 0;
    int vec = 0, variant = 0;
};

// ---------------------------------------------------------------------------
// Recording (the batched step).  While a recorder is active on the host
// thread, the launcher of every kernel that has a batched form appends its
// kind, shape and argument struct instead of launching; any other launch or
// stream operation counts as foreign (and the instance is then not merged
// with others).
// ---------------------------------------------------------------------------
// one phase of the fused program of the coarse time levels (k_stencil.cu)
struct FusedPhase {
    int body, gx, gy, pad;
    const void* args;   // device copy of the argument struct
};
bool fused_body_supported(int body);
int fused_program_grid(size_t smem);   // blocks that can be co-resident (cooperative launch)
int launch_fused_program(const FusedPhase* phases, int nphases, int grid, size_t smem, cudaStream_t s);

// batched form of a kernel kind: one launch over the instances of `args`
// (device array of argument structs) with their virtual grids in m
using BatchLaunch = int (*)(const void* args, BatchMap m, int blocks, const KShape& sh, cudaStream_t s);
struct RecordedLaunch {
    BatchLaunch fn = nullptr;
    KShape shape;
    std::vector<unsigned char> args;
    int body = 0;   // body id for the fused program of the coarse time levels (0: none)
};
// body ids: family * 100 + VEC * 10 + variant
enum BodyFamily {
    BF_ST_COPY = 1, BF_ST_PRESID = 2, BF_ST_RESTRICT = 3, BF_ST_INTERP = 4, BF_ST_APPLYDOT = 5,
    BF_DENSE_F = 6, BF_XUPDATE_F = 7, BF_PROLONG_F = 8, BF_DST_FD = 9, BF_DST_DD2 = 10, BF_DST_DF = 11,
};
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int body_id(int family, int vec, int variant) { return family * 100 + vec * 10 + variant; }
struct Recorder {
    std::vector<RecordedLaunch> ops;
    int foreign = 0;
};
Recorder*& active_recorder();   // this host thread's recorder (null: launch)

template <typename A>
inline bool record_launch(BatchLaunch fn, const A& a, const KShape& sh, int body = 0) {
    Recorder* r = active_recorder();
    if (!r) return false;
    RecordedLaunch l;
    l.fn = fn;
    l.shape = sh;
    l.body = body;
    l.args.resize(sizeof(A));
    std::memcpy(l.args.data(), &a, sizeof(A));
    r->ops.push_back(std::move(l));
    return true;
}
// a launch or copy without batched form: true (and counted) while recording
inline bool record_foreign() {
    Recorder* r = active_recorder();
    if (!r) return false;
    ++r->foreign;
    return true;
}


// A launch the runtime refused: the error names the kernel and its shape
// (and clears the runtime's last-error state, so later calls do not see it).
[[noreturn]] void launch_failed(cudaError_t e, const void* kernel, const cudaLaunchConfig_t& cfg);

// Raise `kernel`'s dynamic shared-memory limit on the current device to at
// least `smem` bytes.  One record per (device, kernel) for the whole
// process, so the limit only grows: launches of one kernel from different
// call sites cannot lower it under one another.
void ensure_dynamic_smem(const void* kernel, size_t smem);

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args&&... args) {
    if (record_foreign()) return;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
    if (e != cudaSuccess) launch_failed(e, (const void*)kernel, cfg);
}

// the same with dynamic shared memory
template <typename... KArgs, typename... Args>
inline void launch_k_smem(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          Args&&... args) {
    if (record_foreign()) return;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
    if (e != cudaSuccess) launch_failed(e, (const void*)kernel, cfg);
}

// ---------------------------------------------------------------------------
// K1: outer residual R = F - A(U), double (fused source, mass, K(u), norm)
// ---------------------------------------------------------------------------
struct ResidualArgs {
    int n, N, n_iron, n_coils;
    const int* e_nodes;
    const double* e_geo;
    const int* inc_ptr;
    const int* inc_elem;
    const double* inc_grad;
    const int* m_ptr;
    const int* m_idx;
    const double* m_val;      // mass / tau
    const int* l_ptr;         // linear-element stiffness (nu_linear)
    const int* l_idx;
    const double* l_val;
    const double* coil_b;
    const double* coil_s;
    const double* Fext;       // if set, the source term is Fext[i*N + n] instead of the coils
    int skip_flux;            // the iron fluxes Qx, Qy were written by another kernel
    double s2sat;             // s_sat^2
    const double* U;
    double* Qx;
    double* Qy;
    double* R;                // may be null
    double* b_d;              // scale * R in double (may be null)
    float* b_f;               // scale * R in float (may be null)
    double scale;
    double* partials;         // >= grid doubles
    unsigned* counter;
    Status* status;           // norm written to status->res (and check); may be null
    double* norm_out;         // if set, the last block also writes ||R|| here
    int* done;                // outer early-exit flag (may be null)
    int check;                // apply the stopping rule in the last block
    size_t partials_cap;      // entries of `partials`
    // structured grid with the saturating law (set: one fused pass, see
    // launch_residual): W x H free nodes, cells (nx-1) x (ny-1)
    int st_W, st_H;
    const uint8_t* st_cell;   // per grid cell: bit 0 lower-right triangle iron, bit 1 upper-left
    const uint8_t* st_flag;   // per free node: bit 0 mass row nonzero, bit 1 linear stiffness row nonzero
    const double* st_mass;    // per free node 8: M / tau at C, E, W, N, S, NE, SW, 0
    const double* st_lin;     // per free node 8: nu_linear stiffness at C, E, W, N, S, 0, 0, 0
    double st_ihx2, st_ihy2;  // 1 / hx^2, 1 / hy^2
    double st_At, st_Bt;      // |T| nu_max, |T| (nu_max - nu_min) s_sat^2
    int st_no_mass;           // sigma = 0 (static problems)
};
int launch_residual(const ResidualArgs& a, cudaStream_t s);  // returns kernels launched
struct ElemFluxArgs {         // iron element fluxes of the two-pass residual
    int n_iron, N;
    const int* e_nodes;
    const double* e_geo;
    const double* U;
    double* Qx;
    double* Qy;
    double s2sat;
    const int* done;
};
// the two-pass residual's element pass (returned: whether it runs) and node pass
bool plan_residual(const ResidualArgs& a, ElemFluxArgs& ef, KShape& kef, KShape& knr);
int launch_elem_flux_batch(const void* args, BatchMap m, int blocks, const KShape& sh, cudaStream_t s);
int launch_node_residual_batch(const void* args, BatchMap m, int blocks, const KShape& sh, cudaStream_t s);
// the same, with the iron fluxes of the exponential law of Section 4 when e_law
// (4 per iron element: |T| a, b, ln c, |T| d) is set (k_law.cu)
int launch_residual_law(const ResidualArgs& a, const double* e_law, cudaStream_t s);
// residual arguments of a set-up context (scratch pointers point into the context)
ResidualArgs residual_args(Ctx& c, const double* U, double* R);

// ---------------------------------------------------------------------------
// Adjoint of the period-averaged eddy-current loss (k_adjoint.cu), double
// ---------------------------------------------------------------------------
constexpr int kMaxCoils = 8;
struct AdjointArgs {
    int n, N, n_iron, n_tri, n_coils;
    double tau, nu_min, nu_max, s2sat;
    const int* e_nodes;       // iron elements (as for the residual)
    const double* e_geo;
    const double* e_area;     // |T| of the iron elements
    const int* mj_ptr;        // loss mass: sum over iron of sigma_e M1_e
    const int* mj_idx;
    const double* mj_val;
    const double* coil_b;
    const double* coil_sin;   // n_coils x N: sin(2 pi t^n / T + phase_c)
    const int* all_nodes;     // 3 per element, free index or -1
    const double* all_area;
    const uint8_t* all_iron;
    double* Jc;               // 3 x n_iron x N Jacobian coefficients (reversed columns)
    double* partials;
    unsigned* counter;
    double* scalars;          // [0] N*J, [1..kMaxCoils] dJ/damp, [1+kMaxCoils..+3) dJ/dnu
};
AdjointArgs adjoint_args(Ctx& c);
// reversed: store at the reversed column (adjoint); else at the step's column (Newton)
int launch_adj_jacobian(const AdjointArgs& a, const double* U, cudaStream_t s, bool reversed = true);
int launch_adj_rhs(const AdjointArgs& a, const double* U, double* Gout, cudaStream_t s);
int launch_adj_elem_flux(const AdjointArgs& a, const double* Lam, double* Qx, double* Qy, const int* done,
                         cudaStream_t s);
int launch_adj_gradients(const AdjointArgs& a, const double* U, const double* Lam, double* dsigma, cudaStream_t s);
void launch_source(int n, int N, int n_coils, const double* coil_b, const double* coil_s,
                   double* F, cudaStream_t s);

// ---------------------------------------------------------------------------
// Sparse kernels on [rows][N] column blocks (node-major, time fastest)
// ---------------------------------------------------------------------------
template <typename T>
struct Op {             // cm * v1 + cl * v2 on a CSR pattern
    int rows = 0, cols = 0;
    const int* ptr = nullptr;
    const int* idx = nullptr;
    const T* v1 = nullptr;
    const T* v2 = nullptr;   // may be null
    const T* d1 = nullptr;   // diagonal of v1
    const T* d2 = nullptr;   // diagonal of v2
    T cm = 1, cl = 0;
    int ell_w = 0;           // > 0: use the padded ELL arrays below
    const int* eidx = nullptr;
    const int4* pk = nullptr; // float: packed {idx, v1, v2, 0} per entry
    const T* ecomb = nullptr; // precombined ELL values cm v1 + cl v2 (double path)
    const T* dcomb = nullptr; // precombined diagonal
    const T* ev1 = nullptr;
    const T* ev2 = nullptr;
};

// column scalar slots in ColRed::col (each N long; complex scalars of
// unknown k at columns 2k (re) and 2k+1 (im))
enum Slot { S_RHO = 0, S_ALPHA = 1, S_BETA = 2, S_RR = 3, S_BB = 4 };

template <typename T>
struct ColRed {         // per-column reduction workspace
    T* partials = nullptr;   // grid * N * 2
    size_t capacity = 0;     // entries of `partials`
    unsigned* counter = nullptr;
    T* col = nullptr;        // per-column scalars, 8 x N: rho alpha beta rr bb . . .
    int* pdone = nullptr;    // PCG early-exit flag
    T tol2 = 0;              // squared relative tolerance for pdone
};

struct Skip {           // early-exit flags checked by every kernel of a step
    const int* done = nullptr;
    const int* pdone = nullptr;
};

// Diagonal scaling fused into a producer: Y2 = omega Y / (cm d1 + cl d2) is the
// first damped-Jacobi sweep (from zero) of the level whose right-hand side Y is.
template <typename T>
struct Aux {
    const T* d1 = nullptr;
    const T* d2 = nullptr;
    T cm = 0, cl = 0, omega = 0;
    T* Y2 = nullptr;          // null: no fused sweep
};

enum SpMode {
    SP_APPLY = 0,       // Y = A X
    SP_RESID = 1,       // Y = B - A X
    SP_JACOBI = 2,      // Y = X + w D^-1 (B - A X)   (X null: Y = w D^-1 B)
    SP_PRESID = 3,      // Y^n = B^n - A X^n + M X^{n-1}  (periodic, M = v1)
    SP_PRESID_RESTRICT = 4,  // Y^m = sum over the pair (2m, 2m+1) of the periodic residual
    SP_INTERP_ADD = 5,  // Y += Op X   (interpolation, v1 only)
    SP_RESTRICT = 6,    // Y = Op X    (restriction, v1 only)
    SP_PAPPLY = 7,      // Y^n = A X^n - M X^{n-1}  (periodic operator)
    SP_COPY = 8,        // Y = B (used with a fused sweep)
};

template <typename T>
int launch_spmm(SpMode mode, const Op<T>& op, int N, const T* X, const T* B, T* Y, T omega,
                Skip sk, cudaStream_t s, Aux<T> aux = Aux<T>());

// PCG pieces (batched over N independent columns)
template <typename T>
int launch_pcg_init_jacobi(const Op<T>& op, int N, T* r, T* z, T* p, ColRed<T> cr, Skip sk,
                           cudaStream_t s);  // z = r/d, p = z, rho = r.z, bb = r.r
template <typename T>
int launch_pcg_dot_rz(int rows, int N, const T* r, const T* z, ColRed<T> cr, int first, Skip sk,
                      cudaStream_t s);       // first: rho = r.z, bb = r.r ; else beta = rz/rho, rho = rz
template <typename T>
int launch_pcg_apply_alpha(const Op<T>& op, int N, const T* p, T* q, ColRed<T> cr, Skip sk,
                           cudaStream_t s);  // q = A p, alpha = rho / p.q
template <typename T>
int launch_pcg_update(const Op<T>& op, int N, T xscale, int assign, T* x, const T* p, T* r,
                      const T* q, T* z, int jacobi, ColRed<T> cr, Skip sk, cudaStream_t s,
                      Aux<T> aux = Aux<T>());
// (assign = 1: x = xscale alpha p instead of x += ..., for a zero start)
template <typename T>
int launch_pcg_direction(int rows, int N, const T* z, T* p, ColRed<T> cr, Skip sk, cudaStream_t s);
// x (+)= xscale alpha p only: the last update when r and its norm are not needed (k_krylov.cu)
template <typename T>
struct XUpdateArgs {   // x = (assign ? 0 : x) + xscale alpha p, alpha per column
    int rows, N;
    T xscale;
    int assign;
    T* x;
    const T* p;
    const T* alpha;
    Skip sk;
};
template <typename T>
int launch_pcg_xupdate(int rows, int N, T xscale, int assign, T* x, const T* p, ColRed<T> cr, Skip sk,
                       cudaStream_t s);

// ---------------------------------------------------------------------------
// Structured-grid stencil kernels of the float inner solve (k_stencil.cu).
// Level grid: W free nodes per row, H rows, free node (a, b) at b W + a;
// coef: 4 float4 per node (M {C,E,W,N}, M {S,NE,SW,0}, L {..}, L {..}).
// ---------------------------------------------------------------------------
template <typename T>
struct StencilOp {      // cm M + cl L as a 7-point stencil
    int W = 0, H = 0;
    const float4* coef = nullptr;    // the level's M and L (4 float4 per node)
    const float4* acoef = nullptr;   // cm M + cl L precombined: {C, E, W, N}, {S, NE, SW, 1 / C}
    T cm = 1, cl = 0;
};
// schedule of the stencil launches from this host thread: the largest time
// tile (columns per block) and the blocks per SM the row strips aim at
void set_stencil_schedule(int tt, int waves);
// out (2 float4 per node) = cm M + cl L of coef, with 1 / diagonal in the last slot
void launch_st_combine(int n, const float4* coef, float cm, float cl, float4* out, cudaStream_t s);
struct StPresidArgs {
    StencilOp<float> A;
    int N, TT, sy, nseg;
    const float* X;
    const float* B;
    float* R;
    float* Z0;
    float omega;
    Skip sk;
    // time restriction only: if alpha is set, X holds the PCG direction p and
    // the iterate is x = (xscale alpha[n]) p (the last PCG update from zero),
    // formed on the fly and written to Xw
    const float* alpha = nullptr;
    float xscale = 0.f;
    float* Xw = nullptr;
};
struct StRestrictArgs {
    StencilOp<float> Af, Ac;
    int N, TT, cy, nseg;
    const float* Xf;
    const float* Bf;
    float* Bc;
    float* Xc;
    float omega;
    Skip sk;
};
struct StInterpArgs {
    StencilOp<float> A;
    int Wc, Hc, N, TT, sy, nseg;
    const float* Xc;
    const float* X;
    const float* B;
    float* Out;
    float omega;
    ColRed<float> cr;
    Skip sk;
};
struct StApplyDotArgs {
    StencilOp<float> A;
    int N, TT, sy, nseg;
    const float* P;
    ColRed<float> cr;
    Skip sk;
};
// R = B - (A X^n - M X^{n-1}) and Z0 = omega D^-1 R (Z0 may be null); with
// time_restrict R instead receives the pair sums over (2m, 2m+1) (N/2 columns)
StPresidArgs plan_st_presid(const StencilOp<float>& A, int N, const float* X, const float* B, float* R, float* Z0,
                            float omega, bool time_restrict, Skip sk, KShape& sh);
int launch_st_presid(const StencilOp<float>& A, int N, const float* X, const float* B, float* R, float* Z0,
                     float omega, bool time_restrict, Skip sk, cudaStream_t s);
// the time restriction of B - P x with x = (xscale alpha[n]) p, x written to Xw
int launch_st_presid_restrict_update(const StencilOp<float>& A, int N, const float* p, const float* alpha,
                                     float xscale, float* Xw, const float* B, float* Bc, Skip sk, cudaStream_t s);
// Bc = P^T (Bf - Af Xf); Xc = omega Dc^-1 Bc if Xc is set
StRestrictArgs plan_st_resid_restrict(const StencilOp<float>& Af, const StencilOp<float>& Ac, int N, const float* Xf,
                                      const float* Bf, float* Bc, float* Xc, float omega, Skip sk, KShape& sh);
int launch_st_resid_restrict(const StencilOp<float>& Af, const StencilOp<float>& Ac, int N, const float* Xf,
                             const float* Bf, float* Bc, float* Xc, float omega, Skip sk, cudaStream_t s);
// Out = x' + omega D^-1 (B - A x'), x' = X + P Xc; dots 1: rho = B.Out, bb = rr = B.B;
// dots 2: beta = B.Out / rho, rho = B.Out (per column, cr)
StInterpArgs plan_st_interp_sweep(const StencilOp<float>& A, int Wc, int Hc, int N, const float* Xc, const float* X,
                                  const float* B, float* Out, float omega, ColRed<float> cr, int dots, Skip sk,
                                  KShape& sh);
int launch_st_interp_sweep(const StencilOp<float>& A, int Wc, int Hc, int N, const float* Xc, const float* X,
                           const float* B, float* Out, float omega, ColRed<float> cr, int dots, Skip sk,
                           cudaStream_t s);
// alpha = rho / (P . A P) per column
StApplyDotArgs plan_st_apply_dot(const StencilOp<float>& A, int N, const float* P, ColRed<float> cr, Skip sk,
                                 KShape& sh);
int launch_st_apply_dot(const StencilOp<float>& A, int N, const float* P, ColRed<float> cr, Skip sk, cudaStream_t s);
// R = B and Z0 = omega D^-1 B (Z0 may be null): a block-Jacobi sweep from zero
struct StCopyArgs {
    const float4* acoef;
    int n, N;
    const float* B;
    float* R;
    float* Z0;
    float omega;
    Skip sk;
};
int launch_st_copy_sweep(const StencilOp<float>& A, int N, const float* B, float* R, float* Z0, float omega, Skip sk,
                         cudaStream_t s);
// One launch of a kernel kind for many instances: `args` (device array, one
// per instance), the batch map (device arrays) and the common shape (vec,
// variant, block and the largest smem); `blocks` = the sum of gx * gy.
int launch_st_presid_batch(const void* args, BatchMap m, int blocks, const KShape& sh, cudaStream_t s);
int launch_st_resid_restrict_batch(const void* args, BatchMap m, int blocks, const KShape& sh,
                                   cudaStream_t s);
int launch_st_interp_sweep_batch(const void* args, BatchMap m, int blocks, const KShape& sh, cudaStream_t s);
int launch_st_apply_dot_batch(const void* args, BatchMap m, int blocks, const KShape& sh, cudaStream_t s);

// ---------------------------------------------------------------------------
// Exact solve of tau_c L x = b on a uniform structured grid by discrete sine
// transforms along rows and columns (k_poisson.cu), double arithmetic.
// ---------------------------------------------------------------------------
struct DstSolve {
    int W = 0, H = 0;              // free nodes per row, rows; W + 1 and H + 1 powers of two
    int logx = 0, logy = 0;        // log2 of the FFT lengths 2 (W + 1), 2 (H + 1)
    const double2* wx = nullptr;   // e^{-2 pi i j / (2 (W + 1))}, j < W + 1
    const double2* wy = nullptr;
    const double* scale = nullptr; // [k][l]: (2 / m_x)(2 / m_y) / (tau_c nu_max lambda_kl)
    double* tmp = nullptr;         // W x H work arrays
    double* tmp2 = nullptr;
};
struct DstArgs {   // one DST-I pass over ntr transforms of length n (element types fixed by the kernel)
    int ntr, n, logM2;
    const void* in;
    long in_tr, in_el;
    void* out;
    long out_tr, out_el;
    const double* scale;
    const double2* Wt;
    Skip sk;
};
template <typename T>   // x = (tau_c L)^{-1} b, both [W x H] node order (one column)
int launch_dst_solve(const DstSolve& d, const T* b, T* x, Skip sk, cudaStream_t s);

// dense coarse-level apply Y = Ainv B  (n x n, row-major)
template <typename T>
struct DenseArgs {
    int n, N, kc;   // kc: k values staged in shared memory per chunk
    const T* A;
    const T* B;
    T* Y;
    Skip sk;
};
template <typename T>
int launch_dense_apply(int n, int N, const T* Ainv, const T* B, T* Y, Skip sk, cudaStream_t s);
template <typename T>
struct ProlongArgs {   // x^{2m}, x^{2m+1} += xc^m
    int rows, Nc;
    const T* xc;
    T* x;
    Skip sk;
};
// U += (*scale) (x_0 + P (x_1 + P (x_2 + ... + P x_D))), P the injection
// in time (x_l has N >> l columns): the prolongations of a V(pre, 0) cycle
// from level D down to 0 and the update of U in one pass
constexpr int kMaxChain = 16;
template <typename T>
struct ChainAddArgs {
    int rows, N, D;
    const T* x[kMaxChain];
    double* U;
    const double* scale;
    Skip sk;
};
template <typename T>
struct AddArgs {       // U += (*scale) d
    size_t count;
    const T* d;
    double* U;
    const double* scale;
    Skip sk;
};

// time transfers and vector helpers
template <typename T>
int launch_time_prolong_add(int rows, int Nc, const T* xc, T* x, Skip sk, cudaStream_t s);
template <typename T>
int launch_axpy(size_t count, T a, const T* x, T* y, Skip sk, cudaStream_t s);   // y += a x
template <typename T>
int launch_fill(size_t count, T v, T* y, Skip sk, cudaStream_t s);
template <typename TI, typename TO>
int launch_cast(size_t count, const TI* x, TO* y, Skip sk, cudaStream_t s);
template <typename T>   // U += s d with s = *scale (scale may be null: s = 1)
int launch_add_to_double(size_t count, const T* d, double* U, const double* scale, Skip sk, cudaStream_t s);
template <typename T>   // ChainAddArgs: x[0..D] the time levels' iterates, D < kMaxChain
int launch_prolong_chain_add(int rows, int N, int D, const T* const* x, double* U, const double* scale, Skip sk,
                             cudaStream_t s);
template <typename TI, typename TO>   // y = x * (*mul) / (*div)   (null pointers read as 1)
int launch_cast_scaled(size_t count, const TI* x, TO* y, const double* mul, const double* div, cudaStream_t s);
// coarsest level with two steps: split b into sum / difference columns, and combine
template <typename T>
int launch_split2(int rows, const T* b, double* bs, double* bd, Skip sk, cudaStream_t s);
template <typename T>
int launch_combine2(int rows, const double* xs, const double* xd, T* x, Skip sk, cudaStream_t s);
int launch_flag(int* flag, int v, Skip sk, cudaStream_t s);   // *flag = v
// squared norm of a column block into status-like scalar (double)
template <typename T>
int launch_norm2(size_t count, const T* x, double* partials, unsigned* counter, double* out,
                 cudaStream_t s);

// ---------------------------------------------------------------------------
// Exact periodic solve of a time level by a DFT in time (k_dft.cu), double.
// Spectra are [n][K] complex as interleaved (re, im) doubles, K = N/2 + 1;
// W holds e^{-2 pi i j / N}, j < N, as (re, im) pairs.
// ---------------------------------------------------------------------------
constexpr int kMaxDftSteps = 1022;   // K = N/2 + 1 <= 512 complex columns per row
template <typename T>   // H_k = sum_t x_t e^{-2 pi i k t / N}
int launch_dft_fwd(int n, int N, const T* x, const double* W, double* H, Skip sk, cudaStream_t s);
template <typename T>   // x_t = (1/N) sum_k H_k e^{2 pi i k t / N}, H_{N-k} = conj(H_k)
int launch_dft_inv(int n, int N, const double* H, const double* W, T* x, Skip sk, cudaStream_t s);
// conjugate-orthogonal CG pieces over D = 2K doubles per row (complex scalars in ColRed)
int launch_capply_alpha(const Op<double>& op, int D, const double* ck, double tau, const double* p, double* q,
                        ColRed<double> cr, Skip sk, cudaStream_t s);   // q = (c_k M + tau L) p, alpha
int launch_cupdate(int rows, int D, int assign, double* x, const double* p, double* r, const double* q,
                   ColRed<double> cr, Skip sk, cudaStream_t s);      // x += alpha p, r -= alpha q, test
int launch_cdot_rz(int rows, int D, const double* r, const double* z, ColRed<double> cr, int first, Skip sk,
                   cudaStream_t s);                                  // rho (and bb) or beta
int launch_cdirection(int rows, int D, const double* z, double* p, ColRed<double> cr, Skip sk,
                      cudaStream_t s);                               // p = z + beta p

// ---------------------------------------------------------------------------
// Flexible GMRES vectors for Newton's method (k_krylov.cu), double
// ---------------------------------------------------------------------------
constexpr int kMaxKrylovDots = 32;   // dot products per k_mdot launch
int launch_mdot(size_t count, int k, const double* V, size_t stride, const double* w, double* partials,
                unsigned* counter, double* out, cudaStream_t s);    // out[i] = V_i . w
int launch_maxpy(size_t count, int k, const double* V, size_t stride, const double* coef, double sign, double* w,
                 cudaStream_t s);                                    // w += sign sum_i coef_i V_i
int launch_div_scalar(size_t count, const double* x, const double* h, double* y, cudaStream_t s);   // y = x / *h
int launch_sqrt_or_one(double* x, cudaStream_t s);   // *x = sqrt(*x), or 1 if not positive

int num_sms();
// out = a x + b y (elementwise, double), for set-up
void launch_lincomb(size_t n, double a, const double* x, double b, const double* y, double* out, cudaStream_t s);

}  // namespace ptp
