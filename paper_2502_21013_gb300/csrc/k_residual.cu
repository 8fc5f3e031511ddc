// K1: the outer residual R = F - A(U) of Problem 1 in double precision.
//
//   R^n_i = f^n_i - sum_j (M_ij / tau) (u^n_j - u^{n-1}_j) - K(u^n)_i,   u^0 = u^N,
//   K(u)_i = sum_{T containing i} nu(|g_T|^2) |T| g_T . grad(phi_i),
//   g_T = sum_j u_j grad(phi_j) = (u_1 - u_0) grad(phi_1) + (u_2 - u_0) grad(phi_2),
//   nu(s^2) = nu_min + (nu_max - nu_min) s^2 / (s^2 + s_sat^2) on iron, nu_linear else,
//   f^n_i = sum_c b_c,i amp_c sin(2 pi t^n / T + phase_c).
//
// (Problem 1; the operator A of the proof of Theorem 2; the model and
// material law of Section 4.)  On elements with the constant nu_linear the
// contribution is the linear stencil nu_linear A_lin u, so K splits exactly
// into a CSR product and the iron part.  Two passes over the space-time block:
//   1. iron-element pass: flux q_T^n = nu |T| g_T^n for every (iron element, step),
//   2. node pass: gather sum_T q_T . grad(phi_i) over the incident iron
//      elements (CSR gather, no atomics, deterministic), add the linear
//      stencil, mass and source terms, write R (and the scaled right-hand
//      side of the correction equation) and reduce ||R||^2; the last block
//      applies the stopping rule.
// Threads are mapped with the time index fastest, so every load of a node's
// N values is a contiguous, coalesced run.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>

#include "dev_math.cuh"
#include "kernels.h"

namespace ptp {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ bool skip_now(const int* done) {
    return done != nullptr && *(volatile const int*)done != 0;
}

// Iron elements only: q = nu(|g|^2) |T| g with
// nu |T| = |T| nu_max - |T| (nu_max - nu_min) s_sat^2 / (|g|^2 + s_sat^2).
__device__ __forceinline__ void elem_flux_body(const ElemFluxArgs& p, const VGrid& vg) {
    pdl_enter();
    if (skip_now(p.done)) return;
    const int n_iron = p.n_iron, N = p.N;
    const int* __restrict__ e_nodes = p.e_nodes;
    const double* __restrict__ e_geo = p.e_geo;
    const double* __restrict__ U = p.U;
    double* __restrict__ Qx = p.Qx;
    double* __restrict__ Qy = p.Qy;
    const double s2sat = p.s2sat;
    const size_t total = (size_t)n_iron * N;
    for (size_t g = (size_t)vg.bx * blockDim.x + threadIdx.x; g < total;
         g += (size_t)vg.gx * blockDim.x) {
        const int e = (int)(g / N);
        const int t = (int)(g - (size_t)e * N);
        const int a = __ldg(e_nodes + 3 * e), b = __ldg(e_nodes + 3 * e + 1),
                  c = __ldg(e_nodes + 3 * e + 2);
        const double u0 = a >= 0 ? __ldg(U + (size_t)a * N + t) : 0.0;
        const double u1 = b >= 0 ? __ldg(U + (size_t)b * N + t) : 0.0;
        const double u2 = c >= 0 ? __ldg(U + (size_t)c * N + t) : 0.0;
        const double* G = e_geo + 6 * (size_t)e;
        const double d1 = u1 - u0, d2 = u2 - u0;
        const double gx = fma(d1, __ldg(G + 0), d2 * __ldg(G + 2));
        const double gy = fma(d1, __ldg(G + 1), d2 * __ldg(G + 3));
        const double s2 = fma(gx, gx, gy * gy);
        const double w = fma(-__ldg(G + 5), recip_newton(s2 + s2sat), __ldg(G + 4));
        Qx[g] = w * gx;
        Qy[g] = w * gy;
    }
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block reduction of ||R||^2 (every thread passes its partial sum), then
// the last block to finish (atomic ticket, no waiting) sums the block
// partials in a fixed order, writes ||R|| and applies the stopping rule of
// Section 4 to the solve status.  Called by every thread of every block.
__device__ void residual_norm_finish(double local, const ResidualArgs& a, const VGrid& vg) {
    __shared__ double sm[32];
    __shared__ bool last;
    const int nw = (blockDim.x + 31) / 32;
    local = warp_sum(local);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = (int)threadIdx.x < nw ? sm[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) {
            const unsigned nblk = (unsigned)(vg.gx * vg.gy);
            const unsigned bid = (unsigned)(vg.by * vg.gx + vg.bx);
            a.partials[bid] = v;
            __threadfence();
            const unsigned ticket = atomicAdd(a.counter, 1u);
            last = ticket == nblk - 1;
        }
    }
    __syncthreads();
    if (!last) return;
    const int nblk = vg.gx * vg.gy;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += __ldcg(a.partials + b);
    s = warp_sum(s);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < nw; ++w) tot += sm[w];
        const double nrm = sqrt(tot);
        if (a.norm_out) *a.norm_out = nrm;
        Status* st = a.status;
        if (!st) {
            *a.counter = 0u;
            return;
        }
        st->bscale_used = st->bscale;
        if (isfinite(nrm) && nrm > 0.0) st->bscale = nrm;
        if (a.check) {
            const int it = st->iteration;
            if (it == 0) st->res0 = nrm;
            st->res = nrm;
            st->iteration = it + 1;
            if (!isfinite(nrm)) {
                st->done = 2;
                if (a.done) *a.done = 1;
            } else if (nrm <= st->tol * st->res0) {
                st->done = 1;
                if (a.done) *a.done = 1;
            }
        } else {
            st->res = nrm;
        }
        *a.counter = 0u;
    }
}

__device__ __forceinline__ void node_residual_body(const ResidualArgs& a, const VGrid& vg) {
    pdl_enter();
    if (skip_now(a.done)) return;
    const int N = a.N;
    const size_t total = (size_t)a.n * N;
    // The float right-hand side is tau R / s with s the previous residual
    // norm, so its entries stay O(tau / sqrt(n N)) however small R becomes.
    // (Every block reads s before the last block replaces it below.)
    const double fscale = a.b_f ? a.scale / a.status->bscale : 0.0;
    double local = 0.0;
    for (size_t g = (size_t)vg.bx * blockDim.x + threadIdx.x; g < total;
         g += (size_t)vg.gx * blockDim.x) {
        const int i = (int)(g / N);
        const int t = (int)(g - (size_t)i * N);
        const int tm = t == 0 ? N - 1 : t - 1;
        double kv = 0.0;   // iron elements: sum_T q_T . grad(phi_i)
        for (int k = __ldg(a.inc_ptr + i), ke = __ldg(a.inc_ptr + i + 1); k < ke; ++k) {
            const size_t q = (size_t)__ldg(a.inc_elem + k) * N + t;
            kv = fma(__ldg(a.Qx + q), __ldg(a.inc_grad + 2 * k), kv);
            kv = fma(__ldg(a.Qy + q), __ldg(a.inc_grad + 2 * k + 1), kv);
        }
        for (int k = __ldg(a.l_ptr + i), ke = __ldg(a.l_ptr + i + 1); k < ke; ++k)  // linear elements
            kv = fma(__ldg(a.l_val + k), __ldg(a.U + (size_t)__ldg(a.l_idx + k) * N + t), kv);
        double mv = 0.0;   // (M / tau)(u^n - u^{n-1})
        for (int k = __ldg(a.m_ptr + i), ke = __ldg(a.m_ptr + i + 1); k < ke; ++k) {
            const size_t j = (size_t)__ldg(a.m_idx + k) * N;
            mv = fma(__ldg(a.m_val + k), __ldg(a.U + j + t) - __ldg(a.U + j + tm), mv);
        }
        double f = 0.0;
        if (a.Fext) {
            f = __ldg(a.Fext + g);
        } else {
            for (int c = 0; c < a.n_coils; ++c) {
                const double cb = __ldg(a.coil_b + (size_t)c * a.n + i);
                if (cb != 0.0) f = fma(cb, __ldg(a.coil_s + (size_t)c * N + t), f);   // warp-uniform
            }
        }
        const double r = f - mv - kv;
        if (a.R) a.R[g] = r;
        if (a.b_d) a.b_d[g] = a.scale * r;
        if (a.b_f) a.b_f[g] = (float)(fscale * r);
        local += r * r;
    }
    residual_norm_finish(local, a, vg);
}

__global__ void __launch_bounds__(kBlock) k_elem_flux(ElemFluxArgs p) { elem_flux_body(p, native_grid()); }
__global__ void __launch_bounds__(kBlock) k_elem_flux_b(const ElemFluxArgs* __restrict__ ps, BatchMap m) {
    pdl_enter();
    int i;
    VGrid g;
    if (batch_block(m, i, g)) {
        const auto a_ = ps[i];   // a local copy: no store of the body aliases it
        elem_flux_body(a_, g);
    }
}
__global__ void __launch_bounds__(kBlock) k_node_residual(ResidualArgs a) { node_residual_body(a, native_grid()); }
__global__ void __launch_bounds__(kBlock) k_node_residual_b(const ResidualArgs* __restrict__ ps, BatchMap m) {
    pdl_enter();
    int i;
    VGrid g;
    if (batch_block(m, i, g)) {
        const auto a_ = ps[i];   // a local copy: no store of the body aliases it
        node_residual_body(a_, g);
    }
}

// ---------------------------------------------------------------------------
// K1 on a structured grid with the saturating law: one fused pass.
//
// The grid's cells are split along (i, j)-(i+1, j+1) into the triangles
// T_a = {(i,j), (i+1,j), (i+1,j+1)} and T_b = {(i,j), (i+1,j+1), (i,j+1)}, all
// with area |T| = hx hy / 2 and axis-parallel legs, so on an iron triangle
//   T_a: dx = u(i+1,j) - u(i,j),     dy = u(i+1,j+1) - u(i+1,j)
//   T_b: dx = u(i+1,j+1) - u(i,j+1), dy = u(i,j+1) - u(i,j)
//   s^2 = dx^2 / hx^2 + dy^2 / hy^2,  nu |T| = |T| nu_max - |T| dnu s_sat^2 / (s^2 + s_sat^2)
//   Qx = nu |T| dx / hx^2, Qy = nu |T| dy / hy^2
// and the element's contributions nu |T| g . grad(phi_k) to its vertices are
//   T_a: (i,j) -Qx, (i+1,j) Qx - Qy, (i+1,j+1) Qy
//   T_b: (i,j) -Qy, (i+1,j+1) Qx,     (i,j+1) Qy - Qx.
// A block owns a time tile of TT columns, a segment of a grid row and a strip
// of rows, and marches up the strip with shared-memory rings of U and of
// u^n - u^{n-1} (four rows each) and of the iron fluxes (two cell rows):
// each iron flux is computed once per block, and U is read once (plus the
// halo).  The mass (M / tau) and the linear-element stiffness act as
// per-node stencils; the source, the outputs and ||R|| are as in the
// two-pass kernels.
constexpr int kK1TT = 16;                  // time columns per block (double2 per thread)
constexpr int kK1TPN = kK1TT / 2;          // threads per node
constexpr int kK1SX = kBlock / kK1TPN;     // node slots per block row (32)
constexpr size_t kK1Smem = (size_t)(8 + 8) * kK1SX * kK1TT * sizeof(double);   // 64 KB

__device__ __forceinline__ double* k1_u(double* base, int slot, int node) {
    return base + ((size_t)slot * kK1SX + node) * kK1TT;
}

__global__ void __launch_bounds__(kBlock)
k_k1_structured(ResidualArgs a, int sy, int nseg) {
    pdl_enter();
    if (skip_now(a.done)) return;
    extern __shared__ double2 k1_smem[];
    double* su = reinterpret_cast<double*>(k1_smem);           // U rows
    double* sd = su + 4 * kK1SX * kK1TT;                       // u^n - u^{n-1} rows
    double* sq = sd + 4 * kK1SX * kK1TT;                       // cell fluxes Qx_a, Qy_a, Qx_b, Qy_b
    const int N = a.N, W = a.st_W, H = a.st_H, nxc = W + 1;    // cells per grid row
    const int lc = threadIdx.x % kK1TPN, ln = threadIdx.x / kK1TPN;
    const int col = blockIdx.y * kK1TT + 2 * lc;
    const int colm = col == 0 ? N - 1 : col - 1;
    const int seg = blockIdx.x % nseg, strip = blockIdx.x / nseg;
    const int a0 = seg * (kK1SX - 2) - 1;
    const int y0 = strip * sy, y1 = min(H, y0 + sy);
    const int an = a0 + ln;                                     // this thread's free column
    const bool in_x = an >= 0 && an < W;
    const double fscale = a.b_f ? a.scale / a.status->bscale : 0.0;
    auto fetch = [&](int b, double2& v, double& pv) {
        if (in_x && b >= 0 && b < H) {
            const double* p = a.U + ((size_t)b * W + an) * N;
            v = __ldg(reinterpret_cast<const double2*>(p + col));
            pv = __ldg(p + colm);
        } else {
            v = make_double2(0.0, 0.0);
            pv = 0.0;
        }
    };
    auto stash = [&](int slot, double2 v, double pv) {
        *reinterpret_cast<double2*>(k1_u(su, slot, ln) + 2 * lc) = v;
        *reinterpret_cast<double2*>(k1_u(sd, slot, ln) + 2 * lc) = make_double2(v.x - pv, v.y - v.x);
    };
    // fluxes of grid cell row cj (free rows cj - 1 = slot sS, cj = slot sN) into flux slot q
    auto cell_row = [&](int cj, int sS, int sN, int q) {
        // cell slot cs = ln covers grid cell ci = a0 + 1 + cs, free columns ci - 1, ci = slots ln, ln + 1
        if (ln > kK1SX - 2) return;
        const int ci = a0 + 1 + ln;
        double* out = sq + ((size_t)q * kK1SX + ln) * 4 * kK1TT + 2 * lc;
        uint8_t f = 0;
        if (ci >= 0 && ci < nxc && cj >= 0 && cj <= H) f = __ldg(a.st_cell + (size_t)cj * nxc + ci);
        double2 r0 = make_double2(0.0, 0.0), r1 = r0, r2 = r0, r3 = r0;
        if (f) {
            const double2 u00 = *reinterpret_cast<const double2*>(k1_u(su, sS, ln) + 2 * lc);      // (i, j)
            const double2 u10 = *reinterpret_cast<const double2*>(k1_u(su, sS, ln + 1) + 2 * lc);  // (i+1, j)
            const double2 u01 = *reinterpret_cast<const double2*>(k1_u(su, sN, ln) + 2 * lc);      // (i, j+1)
            const double2 u11 = *reinterpret_cast<const double2*>(k1_u(su, sN, ln + 1) + 2 * lc);  // (i+1, j+1)
            auto flux = [&](double dx, double dy, double& qx, double& qy) {
                const double d = fma(dx * dx, a.st_ihx2, fma(dy * dy, a.st_ihy2, a.s2sat));
                const double nuT = fma(-a.st_Bt, recip_newton(d), a.st_At);
                qx = nuT * a.st_ihx2 * dx;
                qy = nuT * a.st_ihy2 * dy;
            };
            if (f & 1) {
                flux(u10.x - u00.x, u11.x - u10.x, r0.x, r1.x);
                flux(u10.y - u00.y, u11.y - u10.y, r0.y, r1.y);
            }
            if (f & 2) {
                flux(u11.x - u01.x, u01.x - u00.x, r2.x, r3.x);
                flux(u11.y - u01.y, u01.y - u00.y, r2.y, r3.y);
            }
        }
        *reinterpret_cast<double2*>(out) = r0;
        *reinterpret_cast<double2*>(out + kK1TT) = r1;
        *reinterpret_cast<double2*>(out + 2 * kK1TT) = r2;
        *reinterpret_cast<double2*>(out + 3 * kK1TT) = r3;
    };
    {
        double2 v;
        double pv;
        for (int r = 0; r < 3; ++r) {
            fetch(y0 - 1 + r, v, pv);
            stash(r, v, pv);
        }
    }
    __syncthreads();
    cell_row(y0, 0, 1, y0 & 1);
    double local = 0.0;
    const bool out_lane = ln >= 1 && ln <= kK1SX - 2 && in_x;
    for (int b = y0; b < y1; ++b) {
        const int k = b - y0;
        const int sS = k & 3, sC = (k + 1) & 3, sN = (k + 2) & 3;
        const bool pre = b + 1 < y1;
        double2 nv;
        double npv;
        if (pre) fetch(b + 2, nv, npv);
        cell_row(b + 1, sC, sN, (b + 1) & 1);
        __syncthreads();
        if (out_lane) {
            const size_t node = (size_t)b * W + an;
            // iron: cells (a, b) [this node is vertex (i+1, j+1) of both], (a+1, b) [(i, j+1) of T_b],
            // (a, b+1) [(i+1, j) of T_a], (a+1, b+1) [(i, j) of both], grid cell coordinates
            const double* qS = sq + ((size_t)(b & 1) * kK1SX) * 4 * kK1TT + 2 * lc;
            const double* qN = sq + ((size_t)((b + 1) & 1) * kK1SX) * 4 * kK1TT + 2 * lc;
            auto Q = [&](const double* base, int cs, int comp) {
                return *reinterpret_cast<const double2*>(base + ((size_t)cs * 4 + comp) * kK1TT);
            };
            const double2 sw_ya = Q(qS, ln - 1, 1), sw_xb = Q(qS, ln - 1, 2);
            const double2 se_xb = Q(qS, ln, 2), se_yb = Q(qS, ln, 3);
            const double2 nw_xa = Q(qN, ln - 1, 0), nw_ya = Q(qN, ln - 1, 1);
            const double2 ne_xa = Q(qN, ln, 0), ne_yb = Q(qN, ln, 3);
            double kv0 = (sw_ya.x + sw_xb.x) + (se_yb.x - se_xb.x) + (nw_xa.x - nw_ya.x) - (ne_xa.x + ne_yb.x);
            double kv1 = (sw_ya.y + sw_xb.y) + (se_yb.y - se_xb.y) + (nw_xa.y - nw_ya.y) - (ne_xa.y + ne_yb.y);
            const uint8_t fl = __ldg(a.st_flag + node);
            if (fl & 2) {   // linear elements: nu_linear stiffness, five-point
                const double* L = a.st_lin + 8 * node;
                const double2 c0 = __ldg(reinterpret_cast<const double2*>(L));      // C, E
                const double2 c1 = __ldg(reinterpret_cast<const double2*>(L + 2));  // W, N
                const double cS = __ldg(L + 4);
                const double2 uc = *reinterpret_cast<const double2*>(k1_u(su, sC, ln) + 2 * lc);
                const double2 ue = *reinterpret_cast<const double2*>(k1_u(su, sC, ln + 1) + 2 * lc);
                const double2 uw = *reinterpret_cast<const double2*>(k1_u(su, sC, ln - 1) + 2 * lc);
                const double2 un = *reinterpret_cast<const double2*>(k1_u(su, sN, ln) + 2 * lc);
                const double2 us = *reinterpret_cast<const double2*>(k1_u(su, sS, ln) + 2 * lc);
                kv0 = fma(c0.x, uc.x, fma(c0.y, ue.x, fma(c1.x, uw.x, fma(c1.y, un.x, fma(cS, us.x, kv0)))));
                kv1 = fma(c0.x, uc.y, fma(c0.y, ue.y, fma(c1.x, uw.y, fma(c1.y, un.y, fma(cS, us.y, kv1)))));
            }
            double mv0 = 0.0, mv1 = 0.0;
            if ((fl & 1) && !a.st_no_mass) {   // (M / tau)(u^n - u^{n-1}), seven-point
                const double* Mr = a.st_mass + 8 * node;
                const double2 m0 = __ldg(reinterpret_cast<const double2*>(Mr));      // C, E
                const double2 m1 = __ldg(reinterpret_cast<const double2*>(Mr + 2));  // W, N
                const double2 m2 = __ldg(reinterpret_cast<const double2*>(Mr + 4));  // S, NE
                const double mSW = __ldg(Mr + 6);
                const double2 dc = *reinterpret_cast<const double2*>(k1_u(sd, sC, ln) + 2 * lc);
                const double2 de = *reinterpret_cast<const double2*>(k1_u(sd, sC, ln + 1) + 2 * lc);
                const double2 dw = *reinterpret_cast<const double2*>(k1_u(sd, sC, ln - 1) + 2 * lc);
                const double2 dn = *reinterpret_cast<const double2*>(k1_u(sd, sN, ln) + 2 * lc);
                const double2 ds = *reinterpret_cast<const double2*>(k1_u(sd, sS, ln) + 2 * lc);
                const double2 dne = *reinterpret_cast<const double2*>(k1_u(sd, sN, ln + 1) + 2 * lc);
                const double2 dsw = *reinterpret_cast<const double2*>(k1_u(sd, sS, ln - 1) + 2 * lc);
                mv0 = fma(m0.x, dc.x, fma(m0.y, de.x, fma(m1.x, dw.x, fma(m1.y, dn.x, fma(m2.x, ds.x,
                          fma(m2.y, dne.x, mSW * dsw.x))))));
                mv1 = fma(m0.x, dc.y, fma(m0.y, de.y, fma(m1.x, dw.y, fma(m1.y, dn.y, fma(m2.x, ds.y,
                          fma(m2.y, dne.y, mSW * dsw.y))))));
            }
            double f0 = 0.0, f1 = 0.0;
            for (int cc = 0; cc < a.n_coils; ++cc) {
                const double cb = __ldg(a.coil_b + (size_t)cc * a.n + node);
                if (cb != 0.0) {
                    f0 = fma(cb, __ldg(a.coil_s + (size_t)cc * N + col), f0);
                    f1 = fma(cb, __ldg(a.coil_s + (size_t)cc * N + col + 1), f1);
                }
            }
            const double r0 = f0 - mv0 - kv0, r1 = f1 - mv1 - kv1;
            const size_t g = node * N + col;
            if (a.R) *reinterpret_cast<double2*>(a.R + g) = make_double2(r0, r1);
            if (a.b_d) *reinterpret_cast<double2*>(a.b_d + g) = make_double2(a.scale * r0, a.scale * r1);
            if (a.b_f) *reinterpret_cast<float2*>(a.b_f + g) = make_float2((float)(fscale * r0), (float)(fscale * r1));
            local = fma(r0, r0, fma(r1, r1, local));
        }
        if (pre) stash((k + 3) & 3, nv, npv);
        __syncthreads();
    }
    residual_norm_finish(local, a, native_grid());
}

__global__ void k_source(int n, int N, int n_coils, const double* __restrict__ coil_b,
                         const double* __restrict__ coil_s, double* __restrict__ F) {
    pdl_enter();
    const size_t total = (size_t)n * N;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(g / N);
        const int t = (int)(g - (size_t)i * N);
        double f = 0.0;
        for (int c = 0; c < n_coils; ++c) f += coil_b[(size_t)c * n + i] * coil_s[(size_t)c * N + t];
        F[g] = f;
    }
}

int grid_for(size_t total, int per_sm) {
    size_t want = (total + kBlock - 1) / kBlock;
    size_t cap = (size_t)num_sms() * per_sm;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (int)want;
}

}  // namespace

bool pdl_enabled() {
    static int on = -1;
    if (on < 0) on = getenv("PTP_NO_PDL") ? 0 : 1;
    return on == 1;
}

void ensure_dynamic_smem(const void* kernel, size_t smem) {
    if (smem <= 48 * 1024) return;
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> granted;
    int dev = 0;
    PTP_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    size_t& g = granted[std::make_pair(dev, kernel)];
    if (smem > g) {
        PTP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        g = smem;
    }
}

void launch_failed(cudaError_t e, const void* kernel, const cudaLaunchConfig_t& cfg) {
    (void)cudaGetLastError();   // the refused launch also set the last-error state
    const char* name = nullptr;
    if (cudaFuncGetName(&name, kernel) != cudaSuccess || !name) name = "?";
    throw Error(PTP_ECUDA, std::string("launch of ") + name + " (grid " + std::to_string(cfg.gridDim.x) + " x " +
                               std::to_string(cfg.gridDim.y) + " x " + std::to_string(cfg.gridDim.z) + ", block " +
                               std::to_string(cfg.blockDim.x) + ", dynamic shared memory " +
                               std::to_string(cfg.dynamicSmemBytes) + " B): " + cudaGetErrorString(e));
}

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

int residual_grid(size_t total) { return grid_for(total, 8); }

int launch_residual(const ResidualArgs& a, cudaStream_t s) {
    // structured grid, saturating law, the outer residual with its own source
    // and iron fluxes: one fused pass when its blocks fit the partial sums
    if (a.st_cell && !a.Fext && !a.skip_flux && a.N % kK1TT == 0 &&
        ((uintptr_t)a.U % 16) == 0 && ((uintptr_t)a.R % 16) == 0 && ((uintptr_t)a.b_d % 16) == 0 &&
        ((uintptr_t)a.b_f % 8) == 0) {
        const int nseg = (a.st_W + kK1SX - 3) / (kK1SX - 2);
        const int nch = a.N / kK1TT;
        const long want = 3L * num_sms();
        int sy = (int)std::max(2L, std::min(32L, ((long)a.st_H * nseg * nch) / std::max(1L, want)));
        long blocks = (long)nseg * ((a.st_H + sy - 1) / sy) * nch;
        while (blocks > (long)a.partials_cap && sy < a.st_H) {
            sy *= 2;
            blocks = (long)nseg * ((a.st_H + sy - 1) / sy) * nch;
        }
        if (blocks <= (long)a.partials_cap) {
            const int nstrip = (a.st_H + sy - 1) / sy;
            ensure_dynamic_smem((const void*)k_k1_structured, kK1Smem);
            launch_k_smem(k_k1_structured, dim3(nseg * nstrip, nch), dim3(kBlock), kK1Smem, s, a, sy, nseg);
            return 1;
        }
    }
    ElemFluxArgs ef;
    KShape kef, knr;
    const bool flux = plan_residual(a, ef, kef, knr);
    if (flux && !record_launch(launch_elem_flux_batch, ef, kef))
        launch_k(k_elem_flux, dim3(kef.gx), dim3(kBlock), s, ef);
    if (!record_launch(launch_node_residual_batch, a, knr))
        launch_k(k_node_residual, dim3(knr.gx), dim3(kBlock), s, a);
    return flux ? 2 : 1;
}

// the element and node passes of the two-pass residual: arguments and shapes
bool plan_residual(const ResidualArgs& a, ElemFluxArgs& ef, KShape& kef, KShape& knr) {
    const bool flux = a.n_iron > 0 && !a.skip_flux;
    ef = ElemFluxArgs{a.n_iron, a.N, a.e_nodes, a.e_geo, a.U, a.Qx, a.Qy, a.s2sat, (const int*)a.done};
    kef = KShape{};
    if (flux) kef = KShape{grid_for((size_t)a.n_iron * a.N, 8), 1, kBlock, 0, 1, 0};
    knr = KShape{grid_for((size_t)a.n * a.N, 8), 1, kBlock, 0, 1, 0};
    return flux;
}

int launch_elem_flux_batch(const void* args, BatchMap m, int blocks, const KShape&, cudaStream_t s) {
    launch_k(k_elem_flux_b, dim3(blocks), dim3(kBlock), s, static_cast<const ElemFluxArgs*>(args), m);
    return 1;
}

int launch_node_residual_batch(const void* args, BatchMap m, int blocks, const KShape&, cudaStream_t s) {
    launch_k(k_node_residual_b, dim3(blocks), dim3(kBlock), s, static_cast<const ResidualArgs*>(args), m);
    return 1;
}

void launch_source(int n, int N, int n_coils, const double* coil_b, const double* coil_s,
                   double* F, cudaStream_t s) {
    const size_t t = (size_t)n * N;
    launch_k(k_source, dim3(grid_for(t, 8)), dim3(kBlock), s, n, N, n_coils, coil_b, coil_s, F);
}

}  // namespace ptp
