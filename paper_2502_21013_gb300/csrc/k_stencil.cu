// Structured-grid stencil kernels of the float inner solve (multigrid in time
// whose block-Jacobi spatial solves are PCG with a geometric-multigrid
// preconditioner).
//
// On the nested structured grids every spatial operator cm M + cl L is a
// 7-point stencil (neighbours C, E, W, N, S, NE, SW of the P1 pattern whose
// cells are split along (i, j)-(i+1, j+1)); its coefficients are stored per
// free node.  A block owns a time tile of TT consecutive columns (one 128-byte
// line per node at TT = 32 floats), a segment of a grid row and a strip of
// rows.  It marches up the strip keeping the rows it needs in a shared-memory
// ring (the next row is fetched into registers while the current one is
// computed), so each value is read from global memory about once per pass,
// plus the halo, and from shared memory once per stencil entry.  Dirichlet
// neighbours outside the grid read as zero.
//
// Fused passes (each replaces two or three row-kernel passes):
//   st_presid          r = b - (A x^n - M x^{n-1})  and  z0 = w D^-1 r
//                      (the periodic residual of block Jacobi, Section 3's
//                      time-periodic system, with the first GMG sweep)
//   st_presid_restrict the same residual summed over the pairs (2m, 2m+1):
//                      restriction to the next time level
//   st_resid_restrict  t = b - A x on the fine level, restricted by P^T to
//                      the coarse level, and the coarse level's first sweep
//   st_interp_sweep    x' = x + P x_c, then one damped-Jacobi sweep
//                      x' + w D^-1 (b - A x'), with the PCG dot products
//                      r.z and r.r on the finest level
//   st_apply_dot       p.(A p) per column: the PCG step length, without
//                      writing A p
// Per-column sums are deterministic: block partials in global memory, summed
// in a fixed order by the last block of each time tile (atomic ticket, no
// waiting).
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include <cooperative_groups.h>

#include "dev_bodies.cuh"

namespace ptp {

namespace {

constexpr int kStBlock = 256;

struct A7 {
    float c, e, w, n, s, ne, sw;
};

// cm M + cl L of node `node` from the precombined array (2 float4 per node:
// {C, E, W, N}, {S, NE, SW, 1 / C}); idiag receives 1 / C
__device__ __forceinline__ void load_a(const float4* __restrict__ ac, size_t node, A7& a, float& idiag) {
    const float4 a0 = __ldg(ac + 2 * node), a1 = __ldg(ac + 2 * node + 1);
    a = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z};
    idiag = a1.w;
}

// M alone (the first two float4 of the level's 4 per node)
__device__ __forceinline__ void load_m(const float4* __restrict__ coef, size_t node, A7& m) {
    const float4 m0 = __ldg(coef + 4 * node), m1 = __ldg(coef + 4 * node + 1);
    m = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z};
}

__global__ void k_st_combine(int n, const float4* __restrict__ coef, float cm, float cl, float4* __restrict__ out) {
    pdl_enter();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 m0 = coef[4 * (size_t)i], m1 = coef[4 * (size_t)i + 1];
        const float4 l0 = coef[4 * (size_t)i + 2], l1 = coef[4 * (size_t)i + 3];
        const float c = cm * m0.x + cl * l0.x;
        out[2 * (size_t)i] = make_float4(c, cm * m0.y + cl * l0.y, cm * m0.z + cl * l0.z, cm * m0.w + cl * l0.w);
        out[2 * (size_t)i + 1] = make_float4(cm * m1.x + cl * l1.x, cm * m1.y + cl * l1.y, cm * m1.z + cl * l1.z,
                                             c != 0.f ? 1.0f / c : 0.f);
    }
}

// thread geometry of a block: TPN = TT / VEC threads per node (a time tile),
// SX = blockDim / TPN node slots
struct Lanes {
    int tpn, lc, ln, sx, col;   // col: first column of this thread
};

template <int VEC>
__device__ __forceinline__ Lanes lanes(int TT, int by) {
    Lanes L;
    L.tpn = TT / VEC;
    L.lc = threadIdx.x % L.tpn;
    L.ln = threadIdx.x / L.tpn;
    L.sx = blockDim.x / L.tpn;
    L.col = by * TT + L.lc * VEC;
    return L;
}

template <int VEC>
__device__ __forceinline__ void zero_vec(float (&v)[VEC]) {
#pragma unroll
    for (int k = 0; k < VEC; ++k) v[k] = 0.f;
}

// shared-memory row of SX nodes x TT floats: the VEC values of (slot, node, lane)
template <int VEC>
__device__ __forceinline__ float* srow(float* ring, int slot, int node, int sx, int TT, int lc) {
    return ring + ((size_t)slot * sx + node) * TT + lc * VEC;
}

template <int VEC>
__device__ __forceinline__ void lds(const float* p, float (&v)[VEC]) {
    if constexpr (VEC == 4) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else if constexpr (VEC == 2) {
        const float2 a = *reinterpret_cast<const float2*>(p);
        v[0] = a.x; v[1] = a.y;
    } else {
        v[0] = p[0];
    }
}

template <int VEC>
__device__ __forceinline__ void sts(float* p, const float (&v)[VEC]) {
    if constexpr (VEC == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (VEC == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    } else {
        p[0] = v[0];
    }
}

// Per-column sums of NQ quantities over the block, then over the blocks of
// the same time tile by the last of them (fixed order), then FIN on every
// column of the tile.  `scratch` holds at least NQ * SX * TT floats and is
// free (the caller synchronised after its last use).
template <int VEC, int NQ, int FIN>
__device__ void tile_reduce_finish(float (&acc)[NQ][VEC], const Lanes& L, int TT, int N, float* scratch,
                                   const ColRed<float>& cr, const VGrid& g) {
    __shared__ int last;
#pragma unroll
    for (int q = 0; q < NQ; ++q) sts<VEC>(scratch + ((size_t)q * L.sx + L.ln) * TT + L.lc * VEC, acc[q]);
    __syncthreads();
    const int tiles = g.gx;
    const int chunk = g.by;
    float* part = cr.partials + ((size_t)chunk * tiles) * NQ * TT;
    for (int e = threadIdx.x; e < NQ * TT; e += blockDim.x) {
        const int q = e / TT, j = e - q * TT;
        float s = 0.f;
        for (int r = 0; r < L.sx; ++r) s += scratch[((size_t)q * L.sx + r) * TT + j];
        part[(size_t)g.bx * NQ * TT + e] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(cr.counter + 1 + chunk, 1u);
        last = t == (unsigned)(tiles - 1);
    }
    __syncthreads();
    if (!last) return;
    // all threads of the last block: P = blockDim / (NQ TT) threads per sum,
    // each over a strided subset of the tiles, then P-way partials in order
    const int E = NQ * TT;
    const int P = max(1, (int)blockDim.x / E);
    float* red = scratch + E;   // P x E partial sums
    if ((int)threadIdx.x < P * E) {
        const int e = threadIdx.x % E, p = threadIdx.x / E;
        float s = 0.f;
        for (int b = p; b < tiles; b += P) s += __ldcg(part + (size_t)b * E + e);
        red[p * E + e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        float s = 0.f;
        for (int p = 0; p < P; ++p) s += red[p * E + e];
        scratch[e] = s;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < TT; j += blockDim.x) {
        const int col = chunk * TT + j;
        float* c = cr.col;
        if constexpr (FIN == FIN_ALPHA) {
            c[S_ALPHA * N + col] = safe_ratio<float>(c[S_RHO * N + col], scratch[j]);
        } else if constexpr (FIN == FIN_RZ_FIRST) {   // (rz, rr)
            c[S_RHO * N + col] = scratch[j];
            c[S_BB * N + col] = scratch[TT + j];
            c[S_RR * N + col] = scratch[TT + j];
        } else if constexpr (FIN == FIN_RZ_NEXT) {
            c[S_BETA * N + col] = safe_ratio<float>(scratch[j], c[S_RHO * N + col]);
            c[S_RHO * N + col] = scratch[j];
        }
    }
    if (threadIdx.x == 0) cr.counter[1 + chunk] = 0u;
}

// ---------------------------------------------------------------------------
// Asynchronous row pipeline.  Rows are copied global -> shared by cp.async
// (zero-filled outside the grid) into rings of kNS slots, kLA rows ahead of
// the row being computed, one commit group per row: at every step the block
// waits (a hardware wait on its own copies) until the rows it needs have
// landed, so about kLA rows per thread are in flight.
// ---------------------------------------------------------------------------
constexpr int kNS = 8;   // ring slots (power of two)
constexpr int kLA = 4;   // rows in flight beyond the three being used: kNS >= 3 + kLA + 1


__device__ __forceinline__ int sl8(int q) { return q & (kNS - 1); }

// Per-thread cursor over the rows of one [W x H][N] array at this thread's
// node column a and columns col..col+VEC: element offset of row r, and
// whether (a, r) lies on the grid.
struct Cursor {
    long base;   // offset of row 0 (may be off the grid; only used when valid)
    long rs;     // elements per grid row
    int H;
    bool a_ok;
    __device__ __forceinline__ long off(int r) const { return base + (long)r * rs; }
    __device__ __forceinline__ bool ok(int r) const { return a_ok && r >= 0 && r < H; }
};

__device__ __forceinline__ Cursor cursor(int W, int H, int N, int a, int col) {
    Cursor c;
    c.base = (long)a * N + col;
    c.rs = (long)W * N;
    c.H = H;
    c.a_ok = a >= 0 && a < W;
    return c;
}

template <int VEC>
__device__ __forceinline__ void issue_row(float* dst, const float* __restrict__ X, const Cursor& c, int r) {
    const bool ok = c.ok(r);
    cp_async<VEC * 4>(dst, ok ? X + c.off(r) : X, ok);
}

// the seven stencil neighbours of node slot ln at the rows in slots sS, sC, sN
template <int VEC>
__device__ __forceinline__ void nbrs(float* ring, int sS, int sC, int sN, int ln, int sx, int TT, int lc,
                                     float (&xc)[VEC], float (&xe)[VEC], float (&xw)[VEC], float (&xn)[VEC],
                                     float (&xs)[VEC], float (&xne)[VEC], float (&xsw)[VEC]) {
    lds<VEC>(srow<VEC>(ring, sC, ln, sx, TT, lc), xc);
    lds<VEC>(srow<VEC>(ring, sC, ln + 1, sx, TT, lc), xe);
    lds<VEC>(srow<VEC>(ring, sC, ln - 1, sx, TT, lc), xw);
    lds<VEC>(srow<VEC>(ring, sN, ln, sx, TT, lc), xn);
    lds<VEC>(srow<VEC>(ring, sS, ln, sx, TT, lc), xs);
    lds<VEC>(srow<VEC>(ring, sN, ln + 1, sx, TT, lc), xne);
    lds<VEC>(srow<VEC>(ring, sS, ln - 1, sx, TT, lc), xsw);
}

template <int VEC>
__device__ __forceinline__ float apply7(const A7& c, const float (&xc)[VEC], const float (&xe)[VEC],
                                        const float (&xw)[VEC], const float (&xn)[VEC], const float (&xs)[VEC],
                                        const float (&xne)[VEC], const float (&xsw)[VEC], int v) {
    return c.c * xc[v] + c.e * xe[v] + c.w * xw[v] + c.n * xn[v] + c.s * xs[v] + c.ne * xne[v] + c.sw * xsw[v];
}

// ---------------------------------------------------------------------------
// periodic residual (+ first GMG sweep), or its time restriction
// ---------------------------------------------------------------------------
// MODE 0: R = B - (A X^n - M X^{n-1}), Z0 = omega D^-1 R (if Z0 set)
// MODE 1: Yc^m = sum over n in {2m, 2m+1} of the same residual (N/2 columns)
// Rings: X rows y0-1 .. y1 (q = row - y0 + 1), with column col0 - 1 of each
// node (the tile's previous column, for X^{n-1}); B row q - 1 travels with X
// row q.
template <int VEC, int MODE>
__device__ __forceinline__ void st_presid_body(const StPresidArgs& p, const VGrid& g) {
    const StencilOp<float>& A = p.A;
    const int N = p.N, TT = p.TT, sy = p.sy, nseg = p.nseg;
    const float* __restrict__ X = p.X;
    const float* __restrict__ B = p.B;
    float* __restrict__ R = p.R;
    float* __restrict__ Z0 = p.Z0;
    const float omega = p.omega;
    const Skip& sk = p.sk;
    pdl_enter();
    if (skip_now(sk)) return;
    extern __shared__ float4 smem4[];
    const Lanes L = lanes<VEC>(TT, g.by);
    float* xr = reinterpret_cast<float*>(smem4);
    float* br = xr + kNS * (size_t)L.sx * TT;
    float* prev = br + kNS * (size_t)L.sx * TT;
    const int W = A.W, H = A.H;
    const int seg = g.bx % nseg, strip = g.bx / nseg;
    const int a0 = seg * (L.sx - 2) - 1;          // node slot 0 is a0; outputs at slots 1..sx-2
    const int y0 = strip * sy, y1 = min(H, y0 + sy);
    const int a = a0 + L.ln;
    const int pcol = (g.by * TT == 0 ? N : g.by * TT) - 1;   // previous column of the tile
    const Cursor cx = cursor(W, H, N, a, L.col);
    const long pdelta = (long)pcol - L.col;       // from this thread's column to the tile's previous one
    const int nrows = y1 - y0 + 2;
    float* xslot0 = srow<VEC>(xr, 0, L.ln, L.sx, TT, L.lc);
    float* bslot0 = srow<VEC>(br, 0, L.ln, L.sx, TT, L.lc);
    const size_t sstride = (size_t)L.sx * TT;     // floats per ring slot
    auto issue_q = [&](int q) {
        if (q < nrows) {
            const int r = y0 - 1 + q;
            issue_row<VEC>(xslot0 + sl8(q) * sstride, X, cx, r);
            if (L.lc == 0) {
                const bool ok = cx.ok(r);
                cp_async<4>(prev + sl8(q) * L.sx + L.ln, ok ? X + cx.off(r) + pdelta : X, ok);
            }
            if (q >= 2) issue_row<VEC>(bslot0 + sl8(q) * sstride, B, cx, r - 1);
        }
        cp_commit();
    };
    for (int q = 0; q < kLA + 2; ++q) issue_q(q);
    const bool out_lane = L.ln >= 1 && L.ln <= L.sx - 2 && a < W;
    const float* pre_base = xr + (size_t)L.lc * VEC - 1;       // column col - 1 within a slot row (lc > 0)
    // fused last PCG update (time restriction only): per-column scale xscale alpha[n]
    const bool upd = MODE == 1 && p.alpha != nullptr;
    float sv[VEC], sprev = 0.f;
    if (upd) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) sv[v] = p.xscale * p.alpha[L.col + v];
        sprev = p.xscale * p.alpha[L.lc > 0 ? L.col - 1 : pcol];
    }
    // this node's coefficients for the next row, loaded one row ahead
    A7 cn{}, mn{};
    float idn = 0.f;
    if (out_lane && y0 < y1) {
        load_a(A.acoef, (size_t)y0 * W + a, cn, idn);
        load_m(A.coef, (size_t)y0 * W + a, mn);
    }
    for (int b = y0; b < y1; ++b) {
        const int i = b - y0;
        const A7 c = cn, m = mn;
        const float idiag = idn;
        if (out_lane && b + 1 < y1) {
            load_a(A.acoef, (size_t)(b + 1) * W + a, cn, idn);
            load_m(A.coef, (size_t)(b + 1) * W + a, mn);
        }
        issue_q(i + kLA + 2);
        cp_wait<kLA>();
        __syncthreads();
        if (out_lane) {
            const int sS = sl8(i), sC = sl8(i + 1), sN = sl8(i + 2);
            float xc[VEC], xe[VEC], xw[VEC], xn[VEC], xs[VEC], xne[VEC], xsw[VEC];
            nbrs<VEC>(xr, sS, sC, sN, L.ln, L.sx, TT, L.lc, xc, xe, xw, xn, xs, xne, xsw);
            // column col - 1 of the seven nodes: from the lane to the left, or the tile's previous column
            auto before = [&](int slot, int nd) -> float {
                return L.lc > 0 ? pre_base[((size_t)slot * L.sx + nd) * TT] : prev[slot * L.sx + nd];
            };
            float p_c = before(sC, L.ln), p_e = before(sC, L.ln + 1), p_w = before(sC, L.ln - 1);
            float p_n = before(sN, L.ln), p_s = before(sS, L.ln), p_ne = before(sN, L.ln + 1),
                  p_sw = before(sS, L.ln - 1);
            if constexpr (MODE == 1) {
                if (upd) {   // the rings hold p: x = (xscale alpha) p, as the PCG update forms it
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {   // 0 + s p: the update's rounding, signed zeros included
                        xc[v] = 0.f + sv[v] * xc[v]; xe[v] = 0.f + sv[v] * xe[v]; xw[v] = 0.f + sv[v] * xw[v];
                        xn[v] = 0.f + sv[v] * xn[v]; xs[v] = 0.f + sv[v] * xs[v];
                        xne[v] = 0.f + sv[v] * xne[v]; xsw[v] = 0.f + sv[v] * xsw[v];
                    }
                    p_c = 0.f + sprev * p_c; p_e = 0.f + sprev * p_e; p_w = 0.f + sprev * p_w;
                    p_n = 0.f + sprev * p_n; p_s = 0.f + sprev * p_s; p_ne = 0.f + sprev * p_ne;
                    p_sw = 0.f + sprev * p_sw;
                    st_vec<float, VEC>(p.Xw + cx.off(b), xc);
                }
            }
            float bv[VEC], r[VEC];
            lds<VEC>(bslot0 + sN * sstride, bv);
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const float ax = apply7<VEC>(c, xc, xe, xw, xn, xs, xne, xsw, v);
                const float mx = m.c * p_c + m.e * p_e + m.w * p_w + m.n * p_n + m.s * p_s + m.ne * p_ne +
                                 m.sw * p_sw;
                r[v] = bv[v] - (ax - mx);
                p_c = xc[v]; p_e = xe[v]; p_w = xw[v]; p_n = xn[v]; p_s = xs[v]; p_ne = xne[v]; p_sw = xsw[v];
            }
            if constexpr (MODE == 0) {
                const long o = cx.off(b);
                st_vec<float, VEC>(R + o, r);
                if (Z0) {
                    const float w = omega * idiag;
                    float z[VEC];
#pragma unroll
                    for (int v = 0; v < VEC; ++v) z[v] = w * r[v];
                    st_vec<float, VEC>(Z0 + o, z);
                }
            } else {
                constexpr int HV = VEC / 2;
                float o[HV];
#pragma unroll
                for (int v = 0; v < HV; ++v) o[v] = r[2 * v] + r[2 * v + 1];
                const size_t node = (size_t)b * W + a;
                st_vec<float, HV>(R + node * (N / 2) + L.col / 2, o);
            }
        }
    }
    cp_wait<0>();
}

// ---------------------------------------------------------------------------
// GMG: residual on the fine level, restriction to the coarse level (+ sweep)
// ---------------------------------------------------------------------------
// Bc = P^T (Bf - Af Xf) with P the P1 interpolation of the nested grids:
//   coarse free node (A, B) sits on fine free node (2A+1, 2B+1) and takes the
//   fine residual there plus half of it at the six pattern neighbours.
// Xc = omega Dc^-1 Bc (the coarse level's first sweep from zero) if Xc is set.
// Rings: Xf rows f0-1 .. f1+1 (q = row - f0 + 1); Bf row q - 1 travels with
// Xf row q; the fine residual t in three rows.
template <int VEC>
__device__ __forceinline__ void st_resid_restrict_body(const StRestrictArgs& p, const VGrid& g) {
    const StencilOp<float>& Af = p.Af;
    const StencilOp<float>& Ac = p.Ac;
    const int N = p.N, TT = p.TT, cy = p.cy, nseg = p.nseg;
    const float* __restrict__ Xf = p.Xf;
    const float* __restrict__ Bf = p.Bf;
    float* __restrict__ Bc = p.Bc;
    float* __restrict__ Xc = p.Xc;
    const float omega = p.omega;
    const Skip& sk = p.sk;
    pdl_enter();
    if (skip_now(sk)) return;
    extern __shared__ float4 smem4[];
    const Lanes L = lanes<VEC>(TT, g.by);
    float* zr = reinterpret_cast<float*>(smem4);
    float* br = zr + kNS * (size_t)L.sx * TT;
    float* tr = br + kNS * (size_t)L.sx * TT;
    const int W = Af.W, H = Af.H, Wc = Ac.W, Hc = Ac.H;
    const int cxo = (L.sx - 3) / 2;                 // coarse nodes per block row segment
    const int seg = g.bx % nseg, strip = g.bx / nseg;
    const int A0 = seg * cxo;
    const int a = 2 * A0 - 1 + L.ln;                // fine node of slot ln
    const int B0 = strip * cy, B1 = min(Hc, B0 + cy);
    const int f0 = 2 * B0, f1 = 2 * B1;             // fine rows whose residual is needed: f0..f1
    const int nrows = f1 - f0 + 3;                  // Xf rows f0-1 .. f1+1
    const Cursor cf = cursor(W, H, N, a, L.col);
    const size_t sstride = (size_t)L.sx * TT;
    float* zslot0 = srow<VEC>(zr, 0, L.ln, L.sx, TT, L.lc);
    float* bslot0 = srow<VEC>(br, 0, L.ln, L.sx, TT, L.lc);
    auto issue_q = [&](int q) {
        if (q < nrows) {
            const int r = f0 - 1 + q;
            issue_row<VEC>(zslot0 + sl8(q) * sstride, Xf, cf, r);
            if (q >= 2) issue_row<VEC>(bslot0 + sl8(q) * sstride, Bf, cf, r - 1);
        }
        cp_commit();
    };
    for (int q = 0; q < kLA + 2; ++q) issue_q(q);
    const bool t_lane = L.ln >= 1 && L.ln <= 2 * cxo + 1 && a < W;
    // coarse output of this thread (slot ln < cxo): node (A0 + ln, Bq), fine centre slot 2 ln + 2
    const int Aq = A0 + L.ln;
    const bool c_lane = L.ln < cxo && Aq < Wc;
    const Cursor cc = cursor(Wc, Hc, N, Aq, L.col);
    const int sl = 2 * L.ln + 2;
    // fine coefficients one row ahead (rows f0..f1 on the grid)
    const bool t_ok = t_lane;
    A7 cn{};
    float idn = 0.f;
    auto fetch = [&](int f) {
        if (t_ok && f >= 0 && f < H) load_a(Af.acoef, (size_t)f * W + a, cn, idn);
    };
    fetch(f0);
    for (int f = f0; f <= f1; ++f) {
        const int k = f - f0;
        const A7 c = cn;
        if (f + 1 <= f1) fetch(f + 1);
        issue_q(k + kLA + 2);
        cp_wait<kLA>();
        __syncthreads();
        if (t_lane) {
            const int sS = sl8(k), sC = sl8(k + 1), sN = sl8(k + 2);
            float xc[VEC], xe[VEC], xw[VEC], xn[VEC], xs[VEC], xne[VEC], xsw[VEC], bv[VEC], t[VEC];
            nbrs<VEC>(zr, sS, sC, sN, L.ln, L.sx, TT, L.lc, xc, xe, xw, xn, xs, xne, xsw);
            lds<VEC>(bslot0 + sN * sstride, bv);
#pragma unroll
            for (int v = 0; v < VEC; ++v) t[v] = bv[v] - apply7<VEC>(c, xc, xe, xw, xn, xs, xne, xsw, v);
            sts<VEC>(srow<VEC>(tr, k % 3, L.ln, L.sx, TT, L.lc), t);
        }
        if (k >= 2 && (k & 1) == 0) {
            __syncthreads();
            // coarse row Bq: fine rows f-2 (S), f-1 (centre), f (N)
            const int Bq = B0 + (k - 2) / 2;
            if (c_lane && Bq < Hc) {
                const int tS = (k - 2) % 3, tC = (k - 1) % 3, tN = k % 3;
                float vc[VEC], ve[VEC], vw[VEC], vn[VEC], vs[VEC], vne[VEC], vsw[VEC], o[VEC];
                nbrs<VEC>(tr, tS, tC, tN, sl, L.sx, TT, L.lc, vc, ve, vw, vn, vs, vne, vsw);
#pragma unroll
                for (int v = 0; v < VEC; ++v)
                    o[v] = vc[v] + 0.5f * (ve[v] + vw[v] + vn[v] + vs[v] + vne[v] + vsw[v]);
                const long co = cc.off(Bq);
                st_vec<float, VEC>(Bc + co, o);
                if (Xc) {
                    const size_t cn = (size_t)Bq * Wc + Aq;
                    const float w = omega * __ldg(&Ac.acoef[2 * cn + 1].w);
#pragma unroll
                    for (int v = 0; v < VEC; ++v) o[v] *= w;
                    st_vec<float, VEC>(Xc + co, o);
                }
            }
        }
    }
    cp_wait<0>();
}

// ---------------------------------------------------------------------------
// GMG: interpolation of the coarse correction + one damped-Jacobi sweep
// ---------------------------------------------------------------------------
// x' = X + P Xc on the fine level, Out = x' + omega D^-1 (B - A x').
// DOTS 1: (B.Out, B.B) per column -> rho, bb, rr (first PCG direction);
// DOTS 2: B.Out -> beta, rho (later directions).  B is the PCG residual there.
// Rings: X rows y0-1 .. y1 (q = row - y0 + 1), turned into x' in place once
// they have landed; B row q - 1 travels with X row q; coarse rows by their
// own index c (slot c mod kNS), each issued with the first fine row that
// needs it.  Fine free row f uses coarse rows (f-1)/2 (f odd) or f/2 - 1 and
// f/2 (f even); fine free column a likewise.
template <int VEC, int DOTS>
__device__ __forceinline__ void st_interp_sweep_body(const StInterpArgs& p, const VGrid& g) {
    const StencilOp<float>& A = p.A;
    const int Wc = p.Wc, Hc = p.Hc, N = p.N, TT = p.TT, sy = p.sy, nseg = p.nseg;
    const float* __restrict__ Xc = p.Xc;
    const float* __restrict__ X = p.X;
    const float* __restrict__ B = p.B;
    float* __restrict__ Out = p.Out;
    const float omega = p.omega;
    const ColRed<float>& cr = p.cr;
    const Skip& sk = p.sk;
    pdl_enter();
    if (skip_now(sk)) return;
    extern __shared__ float4 smem4[];
    const Lanes L = lanes<VEC>(TT, g.by);
    const int cw = L.sx / 2 + 2;                    // coarse nodes per ring row
    float* xr = reinterpret_cast<float*>(smem4);
    float* br = xr + kNS * (size_t)L.sx * TT;
    float* cr8 = br + kNS * (size_t)L.sx * TT;      // coarse ring: kNS x cw x TT
    const int W = A.W, H = A.H;
    const int seg = g.bx % nseg, strip = g.bx / nseg;
    const int a0 = seg * (L.sx - 2) - 1;
    const int y0 = strip * sy, y1 = min(H, y0 + sy);
    const int a = a0 + L.ln;
    const int cA0 = (a0 >> 1) - 1;                  // first coarse column of the ring rows (a0 >= -1)
    const int nrows = y1 - y0 + 2;
    const Cursor cx = cursor(W, H, N, a, L.col);
    const Cursor cc = cursor(Wc, Hc, N, cA0 + L.ln, L.col);   // coarse loads by lanes ln < cw
    const bool c_issuer = L.ln < cw;
    const size_t sstride = (size_t)L.sx * TT, cstride = (size_t)cw * TT;
    float* xslot0 = srow<VEC>(xr, 0, L.ln, L.sx, TT, L.lc);
    float* bslot0 = srow<VEC>(br, 0, L.ln, L.sx, TT, L.lc);
    float* cslot0 = cr8 + (size_t)L.ln * TT + L.lc * VEC;
    int cnext = ((y0 - 1) >= 0 ? (y0 - 1) / 2 : 0) - 1;   // next coarse row to issue
    auto issue_q = [&](int q) {
        if (q < nrows) {
            const int r = y0 - 1 + q;
            issue_row<VEC>(xslot0 + sl8(q) * sstride, X, cx, r);
            if (q >= 2) issue_row<VEC>(bslot0 + sl8(q) * sstride, B, cx, r - 1);
            const int last = r >= 0 ? r / 2 : -1;
            for (; cnext <= last; ++cnext)
                if (c_issuer) issue_row<VEC>(cslot0 + sl8(cnext) * cstride, Xc, cc, cnext);
        }
        cp_commit();
    };
    // this thread's coarse columns for x': a odd -> (a-1)/2; a even -> a/2 - 1 and a/2
    const bool ao = a & 1;
    const int A1 = ao ? (a - 1) / 2 : a / 2 - 1, A2 = ao ? A1 : a / 2;
    const bool A1ok = A1 >= 0 && A1 < Wc, A2ok = A2 >= 0 && A2 < Wc;
    const float* c1base = cr8 + (size_t)(A1 - cA0) * TT + L.lc * VEC;
    const float* c2base = cr8 + (size_t)(A2 - cA0) * TT + L.lc * VEC;
    // x' = x + P xc in place for ring row q (fine row r)
    auto to_xprime = [&](int q) {
        const int r = y0 - 1 + q;
        if (q >= nrows || !cx.ok(r)) return;
        float* xp = xslot0 + sl8(q) * sstride;
        float v[VEC], c1[VEC], c2[VEC];
        lds<VEC>(xp, v);
        auto cval = [&](const float* base, bool aok, int Brow, float (&o)[VEC]) {
            if (!aok || Brow < 0 || Brow >= Hc) { zero_vec<VEC>(o); return; }
            lds<VEC>(base + sl8(Brow) * cstride, o);
        };
        if (r & 1) {                    // fine row on a coarse row: (r - 1) / 2
            const int Bo = (r - 1) / 2;
            cval(c1base, A1ok, Bo, c1);
            if (ao) {
#pragma unroll
                for (int k = 0; k < VEC; ++k) v[k] += c1[k];
            } else {
                cval(c2base, A2ok, Bo, c2);
#pragma unroll
                for (int k = 0; k < VEC; ++k) v[k] += 0.5f * (c1[k] + c2[k]);
            }
        } else {                        // between coarse rows r/2 - 1 and r/2
            cval(c1base, A1ok, r / 2 - 1, c1);
            if (ao) cval(c1base, A1ok, r / 2, c2);           // vertical edge midpoint
            else cval(c2base, A2ok, r / 2, c2);              // diagonal midpoint
#pragma unroll
            for (int k = 0; k < VEC; ++k) v[k] += 0.5f * (c1[k] + c2[k]);
        }
        sts<VEC>(xp, v);
    };
    // x' runs three rows ahead of the row being swept: one barrier per row
    // publishes x' of rows i..i+2 and frees slot i+3 for x' in the same phase
    for (int q = 0; q < kLA + 2; ++q) issue_q(q);
    cp_wait<kLA - 1>();      // rows q = 0, 1, 2 and their coarse rows have landed
    __syncthreads();
    to_xprime(0);
    to_xprime(1);
    to_xprime(2);
    constexpr int NQ = DOTS == 1 ? 2 : 1;
    float acc[NQ][VEC];
#pragma unroll
    for (int q = 0; q < NQ; ++q) zero_vec<VEC>(acc[q]);
    const bool out_lane = L.ln >= 1 && L.ln <= L.sx - 2 && a < W;
    A7 cn{};
    float idn = 0.f;
    if (out_lane && y0 < y1) load_a(A.acoef, (size_t)y0 * W + a, cn, idn);
    for (int b = y0; b < y1; ++b) {
        const int i = b - y0;
        const A7 c = cn;
        const float idiag = idn;
        if (out_lane && b + 1 < y1) load_a(A.acoef, (size_t)(b + 1) * W + a, cn, idn);
        issue_q(i + kLA + 2);
        cp_wait<kLA - 1>();  // row q = i + 3 has landed
        __syncthreads();
        to_xprime(i + 3);
        if (out_lane) {
            const int sS = sl8(i), sC = sl8(i + 1), sN = sl8(i + 2);
            float xc[VEC], xe[VEC], xw[VEC], xn[VEC], xs[VEC], xne[VEC], xsw[VEC], bv[VEC], o[VEC];
            nbrs<VEC>(xr, sS, sC, sN, L.ln, L.sx, TT, L.lc, xc, xe, xw, xn, xs, xne, xsw);
            lds<VEC>(bslot0 + sN * sstride, bv);
            const float w = omega * idiag;
#pragma unroll
            for (int v = 0; v < VEC; ++v) o[v] = xc[v] + w * (bv[v] - apply7<VEC>(c, xc, xe, xw, xn, xs, xne, xsw, v));
            st_vec<float, VEC>(Out + cx.off(b), o);
            if constexpr (DOTS > 0) {
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    acc[0][v] += bv[v] * o[v];
                    if constexpr (NQ == 2) acc[1][v] += bv[v] * bv[v];
                }
            }
        }
    }
    cp_wait<0>();
    __syncthreads();
    if constexpr (DOTS == 1) tile_reduce_finish<VEC, 2, FIN_RZ_FIRST>(acc, L, TT, N, xr, cr, g);
    if constexpr (DOTS == 2) tile_reduce_finish<VEC, 1, FIN_RZ_NEXT>(acc, L, TT, N, xr, cr, g);
}

// ---------------------------------------------------------------------------
// PCG step length: alpha = rho / (p . A p) per column, A p not written
// ---------------------------------------------------------------------------
template <int VEC>
__device__ __forceinline__ void st_apply_dot_body(const StApplyDotArgs& p, const VGrid& g) {
    const StencilOp<float>& A = p.A;
    const int N = p.N, TT = p.TT, sy = p.sy, nseg = p.nseg;
    const float* __restrict__ P = p.P;
    const ColRed<float>& cr = p.cr;
    const Skip& sk = p.sk;
    pdl_enter();
    if (skip_now(sk)) return;
    extern __shared__ float4 smem4[];
    const Lanes L = lanes<VEC>(TT, g.by);
    float* xr = reinterpret_cast<float*>(smem4);
    const int W = A.W, H = A.H;
    const int seg = g.bx % nseg, strip = g.bx / nseg;
    const int a0 = seg * (L.sx - 2) - 1;
    const int y0 = strip * sy, y1 = min(H, y0 + sy);
    const int a = a0 + L.ln;
    const int nrows = y1 - y0 + 2;
    const Cursor cx = cursor(W, H, N, a, L.col);
    const size_t sstride = (size_t)L.sx * TT;
    float* xslot0 = srow<VEC>(xr, 0, L.ln, L.sx, TT, L.lc);
    auto issue_q = [&](int q) {
        if (q < nrows) issue_row<VEC>(xslot0 + sl8(q) * sstride, P, cx, y0 - 1 + q);
        cp_commit();
    };
    for (int q = 0; q < kLA + 2; ++q) issue_q(q);
    float acc[1][VEC];
    zero_vec<VEC>(acc[0]);
    const bool out_lane = L.ln >= 1 && L.ln <= L.sx - 2 && a < W;
    A7 cn{};
    float idn = 0.f;
    if (out_lane && y0 < y1) load_a(A.acoef, (size_t)y0 * W + a, cn, idn);
    for (int b = y0; b < y1; ++b) {
        const int i = b - y0;
        const A7 c = cn;
        if (out_lane && b + 1 < y1) load_a(A.acoef, (size_t)(b + 1) * W + a, cn, idn);
        issue_q(i + kLA + 2);
        cp_wait<kLA>();
        __syncthreads();
        if (out_lane) {
            const int sS = sl8(i), sC = sl8(i + 1), sN = sl8(i + 2);
            float xc[VEC], xe[VEC], xw[VEC], xn[VEC], xs[VEC], xne[VEC], xsw[VEC];
            nbrs<VEC>(xr, sS, sC, sN, L.ln, L.sx, TT, L.lc, xc, xe, xw, xn, xs, xne, xsw);
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[0][v] += xc[v] * apply7<VEC>(c, xc, xe, xw, xn, xs, xne, xsw, v);
        }
    }
    cp_wait<0>();
    __syncthreads();
    tile_reduce_finish<VEC, 1, FIN_ALPHA>(acc, L, TT, N, xr, cr, g);
}

// ---------------------------------------------------------------------------
// launch shapes
// ---------------------------------------------------------------------------

inline bool al(const void* p, size_t a) { return p == nullptr || ((uintptr_t)p % a) == 0; }

// VEC (floats per thread) and TT (columns per time tile) for N columns
struct Shape {
    int vec, TT, tpn, sx, block;
};

// schedule of this host thread's launches (each context sets its autotuned one)
thread_local int g_st_tt = 32;      // largest time tile
thread_local int g_st_waves = 3;    // blocks per SM the strips aim at

Shape st_shape(int N, std::initializer_list<const void*> ptrs, bool need_even) {
    Shape s{};
    s.vec = 1;
    for (int v : {4, 2}) {
        if (N % v) continue;
        bool ok = true;
        for (const void* p : ptrs) ok = ok && al(p, v * sizeof(float));
        if (ok) { s.vec = v; break; }
    }
    if (need_even && s.vec < 2) throw Error(PTP_EINVAL, "stencil time restriction needs an even, aligned N");
    // the largest divisor of N up to the schedule's tile that VEC divides
    s.TT = s.vec;
    const int cap = std::min(g_st_tt, 32 * s.vec);   // at least 8 nodes per block row
    for (int d = std::min(N, cap); d >= s.vec; --d)
        if (N % d == 0 && d % s.vec == 0) { s.TT = d; break; }
    s.tpn = s.TT / s.vec;
    s.sx = kStBlock / s.tpn;
    s.block = s.sx * s.tpn;
    return s;
}

// Blocks of `kern` (with `smem` bytes of dynamic shared memory) that fit on
// one SM at once: the least of the thread, shared-memory and register limits.
int st_resident(const void* kern, int block, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<const void*, size_t>, int> memo;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(kern, smem);
    const auto it = memo.find(key);
    if (it != memo.end()) return it->second;
    cudaFuncAttributes fa{};
    PTP_CUDA(cudaFuncGetAttributes(&fa, kern));
    int dev = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0;
    PTP_CUDA(cudaGetDevice(&dev));
    PTP_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    PTP_CUDA(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
    PTP_CUDA(cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev));
    const size_t per_block = smem + fa.sharedSizeBytes + 1024;   // 1 KB of each block is reserved
    int r = thr_sm / block;
    r = std::min(r, (int)((size_t)smem_sm / per_block));
    const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;   // allocated per warp in units of 256
    if (regs_warp > 0) r = std::min(r, regs_sm / (regs_warp * ((block + 31) / 32)));
    r = std::max(1, r);
    memo[key] = r;
    return r;
}

// Rows per block strip.  A pass has nseg segments x nch time tiles x
// strips blocks, of which S = min(g_st_waves, resident) per SM run at once;
// each block walks its strip plus `halo` rows.  The strip height minimises
// waves x (rows + halo), waves = ceil(blocks / (S x SMs)): with few
// segments and tiles that is one wave of tall strips (every block of an SM
// starts and ends together), with many it is the fewest waves of shorter
// strips.  Memoised (the search is over H heights).
int strip_rows(int H, int nseg, int nch, int resident, double halo = 2.0, int min_rows = 2) {
    static std::mutex mu;
    static std::map<std::tuple<int, long, long, double, int>, int> memo;
    const long S = (long)std::max(1, std::min(g_st_waves, resident)) * num_sms();
    const long per = std::max(1L, (long)nseg * nch);
    const auto key = std::make_tuple(H, per, S, halo, min_rows);
    std::lock_guard<std::mutex> lock(mu);
    const auto it = memo.find(key);
    if (it != memo.end()) return it->second;
    double best = 1e300;
    long rows_best = std::max(1, H);
    for (long ns = 1; ns <= H; ++ns) {
        const long rows = (H + ns - 1) / ns;
        const long strips = (H + rows - 1) / rows;
        const long waves = (per * strips + S - 1) / S;
        const double t = (double)waves * ((double)rows + halo);
        if (t < best - 1e-9) {
            best = t;
            rows_best = rows;
        }
    }
    const int r = (int)std::max((long)min_rows, rows_best);
    memo[key] = r;
    return r;
}

}  // namespace

#define PTP_ST_VEC(vec, ...)                                     \
    switch (vec) {                                               \
        case 4: { constexpr int VEC = 4; __VA_ARGS__; } break;   \
        case 2: { constexpr int VEC = 2; __VA_ARGS__; } break;   \
        default: { constexpr int VEC = 1; __VA_ARGS__; } break;  \
    }

// Launch with `smem` bytes of dynamic shared memory; the kernel's limit is
// raised whenever a launch needs more than it was last granted (the ring
// sizes depend on the columns of the level).
template <typename... KArgs, typename... Args>
static void st_launch(void (*kernel)(KArgs...), dim3 grid, int block, size_t smem, cudaStream_t s, Args&&... args) {
    ensure_dynamic_smem((const void*)kernel, smem);
    launch_k_smem(kernel, grid, dim3(block), smem, s, std::forward<Args>(args)...);
}

void set_stencil_schedule(int tt, int waves) {
    g_st_tt = std::max(1, std::min(tt, 256));
    g_st_waves = std::max(1, std::min(waves, 16));
}

void launch_st_combine(int n, const float4* coef, float cm, float cl, float4* out, cudaStream_t s) {
    if (n <= 0) return;
    launch_k(k_st_combine, dim3(std::min(4096, (n + 255) / 256)), dim3(256), s, n, coef, cm, cl, out);
}

// ---------------------------------------------------------------------------
// start of a block-Jacobi sweep from x = 0: R = B, Z0 = omega D^-1 B
// ---------------------------------------------------------------------------
template <int VEC>
__device__ __forceinline__ void st_copy_sweep_body(const StCopyArgs& p, const VGrid& g) {
    pdl_enter();
    if (skip_now(p.sk)) return;
    const int N = p.N, NC = N / VEC;
    const size_t total = (size_t)p.n * NC;
    const float* __restrict__ B = p.B;
    for (size_t q = (size_t)g.bx * blockDim.x + threadIdx.x; q < total; q += (size_t)g.gx * blockDim.x) {
        const size_t node = q / NC;
        const size_t o = node * N + (q - node * NC) * VEC;
        float b[VEC];
        ldg_vec<float, VEC>(B + o, b);
        st_vec<float, VEC>(p.R + o, b);
        if (p.Z0) {
            const float w = p.omega * __ldg(&p.acoef[2 * node + 1].w);
            float z[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) z[v] = w * b[v];
            st_vec<float, VEC>(p.Z0 + o, z);
        }
    }
}

// ---- kernels: one single-instance and one batched entry per body ----
template <int VEC>
__global__ void __launch_bounds__(256) k_st_copy_sweep(StCopyArgs p) {
    st_copy_sweep_body<VEC>(p, native_grid());
}
template <int VEC>
__global__ void __launch_bounds__(256) k_st_copy_sweep_b(const StCopyArgs* __restrict__ ps, BatchMap m) {
    pdl_enter();
    int i;
    VGrid g;
    if (batch_block(m, i, g)) {
        const auto a_ = ps[i];   // a local copy: no store of the body aliases it
        st_copy_sweep_body<VEC>(a_, g);
    }
}
template <int VEC, int MODE>
__global__ void __launch_bounds__(kStBlock, 3) k_st_presid(StPresidArgs p) {
    st_presid_body<VEC, MODE>(p, native_grid());
}
template <int VEC, int MODE>
__global__ void __launch_bounds__(kStBlock, 3) k_st_presid_b(const StPresidArgs* __restrict__ ps, BatchMap m) {
    pdl_enter();
    int i;
    VGrid g;
    if (batch_block(m, i, g)) {
        const auto a_ = ps[i];   // a local copy: no store of the body aliases it
        st_presid_body<VEC, MODE>(a_, g);
    }
}
template <int VEC>
__global__ void __launch_bounds__(kStBlock) k_st_resid_restrict(StRestrictArgs p) {
    st_resid_restrict_body<VEC>(p, native_grid());
}
template <int VEC>
__global__ void __launch_bounds__(kStBlock) k_st_resid_restrict_b(const StRestrictArgs* __restrict__ ps, BatchMap m) {
    pdl_enter();
    int i;
    VGrid g;
    if (batch_block(m, i, g)) {
        const auto a_ = ps[i];   // a local copy: no store of the body aliases it
        st_resid_restrict_body<VEC>(a_, g);
    }
}
template <int VEC, int DOTS>
__global__ void __launch_bounds__(kStBlock) k_st_interp_sweep(StInterpArgs p) {
    st_interp_sweep_body<VEC, DOTS>(p, native_grid());
}
template <int VEC, int DOTS>
__global__ void __launch_bounds__(kStBlock) k_st_interp_sweep_b(const StInterpArgs* __restrict__ ps, BatchMap m) {
    pdl_enter();
    int i;
    VGrid g;
    if (batch_block(m, i, g)) {
        const auto a_ = ps[i];   // a local copy: no store of the body aliases it
        st_interp_sweep_body<VEC, DOTS>(a_, g);
    }
}
template <int VEC>
__global__ void __launch_bounds__(kStBlock) k_st_apply_dot(StApplyDotArgs p) {
    st_apply_dot_body<VEC>(p, native_grid());
}
template <int VEC>
__global__ void __launch_bounds__(kStBlock) k_st_apply_dot_b(const StApplyDotArgs* __restrict__ ps, BatchMap m) {
    pdl_enter();
    int i;
    VGrid g;
    if (batch_block(m, i, g)) {
        const auto a_ = ps[i];   // a local copy: no store of the body aliases it
        st_apply_dot_body<VEC>(a_, g);
    }
}

// ---- plans: arguments and shape of one call ----
StPresidArgs plan_st_presid(const StencilOp<float>& A, int N, const float* X, const float* B, float* R, float* Z0,
                            float omega, bool time_restrict, Skip sk, KShape& ks) {
    const Shape sh = st_shape(N, {X, B, R, Z0}, time_restrict);
    const int nseg = (A.W + sh.sx - 3) / (sh.sx - 2);
    const int nch = N / sh.TT;
    ks.smem = (2 * kNS * (size_t)sh.sx * sh.TT + kNS * (size_t)sh.sx) * sizeof(float);
    const void* kern = time_restrict ? (const void*)k_st_presid<4, 1> : (const void*)k_st_presid<4, 0>;
    const int sy = strip_rows(A.H, nseg, nch, st_resident(kern, sh.block, ks.smem));
    const int nstrip = (A.H + sy - 1) / sy;
    ks.gx = nseg * nstrip;
    ks.gy = nch;
    ks.block = sh.block;
    ks.vec = sh.vec;
    ks.variant = time_restrict ? 1 : 0;
    StPresidArgs a;
    a.A = A;
    a.N = N;
    a.TT = sh.TT;
    a.sy = sy;
    a.nseg = nseg;
    a.X = X;
    a.B = B;
    a.R = R;
    a.Z0 = Z0;
    a.omega = omega;
    a.sk = sk;
    return a;
}

StRestrictArgs plan_st_resid_restrict(const StencilOp<float>& Af, const StencilOp<float>& Ac, int N, const float* Xf,
                                      const float* Bf, float* Bc, float* Xc, float omega, Skip sk, KShape& ks) {
    PTP_REQUIRE(Af.W == 2 * Ac.W + 1 && Af.H == 2 * Ac.H + 1, "stencil restriction: grids are not nested");
    const Shape sh = st_shape(N, {Xf, Bf, Bc, Xc}, false);
    const int cxo = (sh.sx - 3) / 2;
    PTP_REQUIRE(cxo >= 1, "stencil restriction: block too narrow");
    const int nseg = (Ac.W + cxo - 1) / cxo;
    const int nch = N / sh.TT;
    ks.smem = (2 * kNS + 3) * (size_t)sh.sx * sh.TT * sizeof(float);
    // a strip of cy coarse rows walks 2 cy + 3 fine rows: 1.5 coarse rows of halo
    const int res = st_resident((const void*)k_st_resid_restrict<4>, sh.block, ks.smem);
    const int cy = strip_rows(Ac.H, nseg, nch, res, 1.5, 1);
    const int nstrip = (Ac.H + cy - 1) / cy;
    ks.gx = nseg * nstrip;
    ks.gy = nch;
    ks.block = sh.block;
    ks.vec = sh.vec;
    ks.variant = 0;
    return StRestrictArgs{Af, Ac, N, sh.TT, cy, nseg, Xf, Bf, Bc, Xc, omega, sk};
}

StInterpArgs plan_st_interp_sweep(const StencilOp<float>& A, int Wc, int Hc, int N, const float* Xc, const float* X,
                                  const float* B, float* Out, float omega, ColRed<float> cr, int dots, Skip sk,
                                  KShape& ks) {
    PTP_REQUIRE(A.W == 2 * Wc + 1 && A.H == 2 * Hc + 1, "stencil interpolation: grids are not nested");
    const Shape sh = st_shape(N, {Xc, X, B, Out}, false);
    const int nseg = (A.W + sh.sx - 3) / (sh.sx - 2);
    const int nch = N / sh.TT;
    ks.smem = (2 * kNS * (size_t)sh.sx + kNS * (size_t)(sh.sx / 2 + 2)) * sh.TT * sizeof(float);
    const int sy = strip_rows(A.H, nseg, nch, st_resident((const void*)k_st_interp_sweep<4, 1>, sh.block, ks.smem));
    const int nstrip = (A.H + sy - 1) / sy;
    ks.gx = nseg * nstrip;
    ks.gy = nch;
    ks.block = sh.block;
    ks.vec = sh.vec;
    ks.variant = dots;
    if (dots) {
        const size_t need = (size_t)ks.gx * ks.gy * 2 * sh.TT;
        PTP_REQUIRE(cr.partials != nullptr && need <= cr.capacity, "stencil reduction: partial buffer too small");
        PTP_REQUIRE(nch <= 254, "stencil reduction: too many time tiles");
    }
    return StInterpArgs{A, Wc, Hc, N, sh.TT, sy, nseg, Xc, X, B, Out, omega, cr, sk};
}

StApplyDotArgs plan_st_apply_dot(const StencilOp<float>& A, int N, const float* P, ColRed<float> cr, Skip sk,
                                 KShape& ks) {
    const Shape sh = st_shape(N, {P}, false);
    const int nseg = (A.W + sh.sx - 3) / (sh.sx - 2);
    const int nch = N / sh.TT;
    ks.smem = kNS * (size_t)sh.sx * sh.TT * sizeof(float);
    const int sy = strip_rows(A.H, nseg, nch, st_resident((const void*)k_st_apply_dot<4>, sh.block, ks.smem));
    const int nstrip = (A.H + sy - 1) / sy;
    ks.gx = nseg * nstrip;
    ks.gy = nch;
    ks.block = sh.block;
    ks.vec = sh.vec;
    ks.variant = 0;
    const size_t need = (size_t)ks.gx * ks.gy * sh.TT;
    PTP_REQUIRE(cr.partials != nullptr && need <= cr.capacity, "stencil reduction: partial buffer too small");
    PTP_REQUIRE(nch <= 254, "stencil reduction: too many time tiles");
    return StApplyDotArgs{A, N, sh.TT, sy, nseg, P, cr, sk};
}

// ---- single launches ----
int launch_st_presid_restrict_update(const StencilOp<float>& A, int N, const float* p, const float* alpha,
                                     float xscale, float* Xw, const float* B, float* Bc, Skip sk, cudaStream_t s) {
    KShape ks;
    StPresidArgs a = plan_st_presid(A, N, p, B, Bc, nullptr, 0.f, true, sk, ks);
    PTP_REQUIRE(alpha && Xw && ((uintptr_t)Xw % (ks.vec * sizeof(float))) == 0, "fused update: bad arguments");
    a.alpha = alpha;
    a.xscale = xscale;
    a.Xw = Xw;
    if (record_launch(launch_st_presid_batch, a, ks, body_id(BF_ST_PRESID, ks.vec, ks.variant))) return 1;
    const dim3 grid(ks.gx, ks.gy);
    if (ks.vec == 4) st_launch(k_st_presid<4, 1>, grid, ks.block, ks.smem, s, a);
    else st_launch(k_st_presid<2, 1>, grid, ks.block, ks.smem, s, a);
    return 1;
}

int launch_st_presid(const StencilOp<float>& A, int N, const float* X, const float* B, float* R, float* Z0,
                     float omega, bool time_restrict, Skip sk, cudaStream_t s) {
    KShape ks;
    const StPresidArgs a = plan_st_presid(A, N, X, B, R, Z0, omega, time_restrict, sk, ks);
    if (record_launch(launch_st_presid_batch, a, ks, body_id(BF_ST_PRESID, ks.vec, ks.variant))) return 1;
    const dim3 grid(ks.gx, ks.gy);
    if (time_restrict) {
        if (ks.vec == 4) st_launch(k_st_presid<4, 1>, grid, ks.block, ks.smem, s, a);
        else st_launch(k_st_presid<2, 1>, grid, ks.block, ks.smem, s, a);
    } else {
        PTP_ST_VEC(ks.vec, st_launch(k_st_presid<VEC, 0>, grid, ks.block, ks.smem, s, a));
    }
    return 1;
}

int launch_st_resid_restrict(const StencilOp<float>& Af, const StencilOp<float>& Ac, int N, const float* Xf,
                             const float* Bf, float* Bc, float* Xc, float omega, Skip sk, cudaStream_t s) {
    KShape ks;
    const StRestrictArgs a = plan_st_resid_restrict(Af, Ac, N, Xf, Bf, Bc, Xc, omega, sk, ks);
    if (record_launch(launch_st_resid_restrict_batch, a, ks, body_id(BF_ST_RESTRICT, ks.vec, 0))) return 1;
    PTP_ST_VEC(ks.vec, st_launch(k_st_resid_restrict<VEC>, dim3(ks.gx, ks.gy), ks.block, ks.smem, s, a));
    return 1;
}

int launch_st_interp_sweep(const StencilOp<float>& A, int Wc, int Hc, int N, const float* Xc, const float* X,
                           const float* B, float* Out, float omega, ColRed<float> cr, int dots, Skip sk,
                           cudaStream_t s) {
    KShape ks;
    const StInterpArgs a = plan_st_interp_sweep(A, Wc, Hc, N, Xc, X, B, Out, omega, cr, dots, sk, ks);
    if (record_launch(launch_st_interp_sweep_batch, a, ks, body_id(BF_ST_INTERP, ks.vec, ks.variant))) return 1;
    const dim3 grid(ks.gx, ks.gy);
    if (dots == 1) PTP_ST_VEC(ks.vec, st_launch(k_st_interp_sweep<VEC, 1>, grid, ks.block, ks.smem, s, a))
    else if (dots == 2) PTP_ST_VEC(ks.vec, st_launch(k_st_interp_sweep<VEC, 2>, grid, ks.block, ks.smem, s, a))
    else PTP_ST_VEC(ks.vec, st_launch(k_st_interp_sweep<VEC, 0>, grid, ks.block, ks.smem, s, a))
    return 1;
}

int launch_st_apply_dot(const StencilOp<float>& A, int N, const float* P, ColRed<float> cr, Skip sk, cudaStream_t s) {
    KShape ks;
    const StApplyDotArgs a = plan_st_apply_dot(A, N, P, cr, sk, ks);
    if (record_launch(launch_st_apply_dot_batch, a, ks, body_id(BF_ST_APPLYDOT, ks.vec, 0))) return 1;
    PTP_ST_VEC(ks.vec, st_launch(k_st_apply_dot<VEC>, dim3(ks.gx, ks.gy), ks.block, ks.smem, s, a));
    return 1;
}

int launch_st_copy_sweep_batch(const void* argv, BatchMap m, int blocks, const KShape& ks, cudaStream_t s) {
    const StCopyArgs* args = static_cast<const StCopyArgs*>(argv);
    PTP_ST_VEC(ks.vec, launch_k(k_st_copy_sweep_b<VEC>, dim3(blocks), dim3(256), s, args, m));
    return 1;
}

int launch_st_copy_sweep(const StencilOp<float>& A, int N, const float* B, float* R, float* Z0, float omega, Skip sk,
                         cudaStream_t s) {
    const StCopyArgs a{A.acoef, A.W * A.H, N, B, R, Z0, omega, sk};
    auto al = [](const void* p, size_t b) { return ((uintptr_t)p % b) == 0; };
    const bool a16 = al(B, 16) && al(R, 16) && (!Z0 || al(Z0, 16));
    const bool a8 = al(B, 8) && al(R, 8) && (!Z0 || al(Z0, 8));
    KShape ks;
    ks.vec = (N % 4 == 0 && a16) ? 4 : (N % 2 == 0 && a8) ? 2 : 1;
    const size_t total = (size_t)a.n * (N / ks.vec);
    ks.gx = (int)std::max<size_t>(1, std::min((total + 255) / 256, (size_t)num_sms() * 8));
    ks.gy = 1;
    ks.block = 256;
    if (record_launch(launch_st_copy_sweep_batch, a, ks, body_id(BF_ST_COPY, ks.vec, 0))) return 1;
    PTP_ST_VEC(ks.vec, launch_k(k_st_copy_sweep<VEC>, dim3(ks.gx), dim3(256), s, a));
    return 1;
}

// ---- batched launches: every instance's blocks in one 1-D grid ----
int launch_st_presid_batch(const void* argv, BatchMap m, int blocks, const KShape& ks, cudaStream_t s) {
    const StPresidArgs* args = static_cast<const StPresidArgs*>(argv);
    const dim3 grid(blocks);
    if (ks.variant == 1) {
        if (ks.vec == 4) st_launch(k_st_presid_b<4, 1>, grid, ks.block, ks.smem, s, args, m);
        else st_launch(k_st_presid_b<2, 1>, grid, ks.block, ks.smem, s, args, m);
    } else {
        PTP_ST_VEC(ks.vec, st_launch(k_st_presid_b<VEC, 0>, grid, ks.block, ks.smem, s, args, m));
    }
    return 1;
}

int launch_st_resid_restrict_batch(const void* argv, BatchMap m, int blocks, const KShape& ks,
                                   cudaStream_t s) {
    const StRestrictArgs* args = static_cast<const StRestrictArgs*>(argv);
    PTP_ST_VEC(ks.vec, st_launch(k_st_resid_restrict_b<VEC>, dim3(blocks), ks.block, ks.smem, s, args, m));
    return 1;
}

int launch_st_interp_sweep_batch(const void* argv, BatchMap m, int blocks, const KShape& ks, cudaStream_t s) {
    const StInterpArgs* args = static_cast<const StInterpArgs*>(argv);
    const dim3 grid(blocks);
    if (ks.variant == 1) PTP_ST_VEC(ks.vec, st_launch(k_st_interp_sweep_b<VEC, 1>, grid, ks.block, ks.smem, s, args, m))
    else if (ks.variant == 2) PTP_ST_VEC(ks.vec, st_launch(k_st_interp_sweep_b<VEC, 2>, grid, ks.block, ks.smem, s, args, m))
    else PTP_ST_VEC(ks.vec, st_launch(k_st_interp_sweep_b<VEC, 0>, grid, ks.block, ks.smem, s, args, m))
    return 1;
}

int launch_st_apply_dot_batch(const void* argv, BatchMap m, int blocks, const KShape& ks, cudaStream_t s) {
    const StApplyDotArgs* args = static_cast<const StApplyDotArgs*>(argv);
    PTP_ST_VEC(ks.vec, st_launch(k_st_apply_dot_b<VEC>, dim3(blocks), ks.block, ks.smem, s, args, m));
    return 1;
}


// ---------------------------------------------------------------------------
// Fused program of the coarse time levels.  Below a time level with few
// steps the V-cycle is a chain of small passes whose duration is launch and
// pipeline latency, not work.  It runs as one cooperative kernel: every
// phase is one recorded launch (body, virtual grid, argument struct); the
// kernel's blocks walk the phase's virtual blocks, and a grid-wide barrier
// separates the phases, as stream order separated the launches.  Every
// virtual block computes what the block of the separate launch computed, so
// the results are the same bit for bit.
// ---------------------------------------------------------------------------
namespace {

template <typename A>
__device__ __forceinline__ A load_args(const void* p) {
    return *static_cast<const A*>(p);
}

#define PTP_FUSED_BODIES(X)                                                                               \
    X(body_id(BF_ST_COPY, 4, 0), st_copy_sweep_body<4>(load_args<StCopyArgs>(args), g))                  \
    X(body_id(BF_ST_COPY, 2, 0), st_copy_sweep_body<2>(load_args<StCopyArgs>(args), g))                  \
    X(body_id(BF_ST_PRESID, 4, 0), (st_presid_body<4, 0>(load_args<StPresidArgs>(args), g)))             \
    X(body_id(BF_ST_PRESID, 2, 0), (st_presid_body<2, 0>(load_args<StPresidArgs>(args), g)))             \
    X(body_id(BF_ST_PRESID, 4, 1), (st_presid_body<4, 1>(load_args<StPresidArgs>(args), g)))             \
    X(body_id(BF_ST_PRESID, 2, 1), (st_presid_body<2, 1>(load_args<StPresidArgs>(args), g)))             \
    X(body_id(BF_ST_RESTRICT, 4, 0), st_resid_restrict_body<4>(load_args<StRestrictArgs>(args), g))      \
    X(body_id(BF_ST_RESTRICT, 2, 0), st_resid_restrict_body<2>(load_args<StRestrictArgs>(args), g))      \
    X(body_id(BF_ST_INTERP, 4, 0), (st_interp_sweep_body<4, 0>(load_args<StInterpArgs>(args), g)))       \
    X(body_id(BF_ST_INTERP, 2, 0), (st_interp_sweep_body<2, 0>(load_args<StInterpArgs>(args), g)))       \
    X(body_id(BF_ST_INTERP, 4, 1), (st_interp_sweep_body<4, 1>(load_args<StInterpArgs>(args), g)))       \
    X(body_id(BF_ST_INTERP, 2, 1), (st_interp_sweep_body<2, 1>(load_args<StInterpArgs>(args), g)))       \
    X(body_id(BF_ST_INTERP, 4, 2), (st_interp_sweep_body<4, 2>(load_args<StInterpArgs>(args), g)))       \
    X(body_id(BF_ST_INTERP, 2, 2), (st_interp_sweep_body<2, 2>(load_args<StInterpArgs>(args), g)))       \
    X(body_id(BF_ST_APPLYDOT, 4, 0), st_apply_dot_body<4>(load_args<StApplyDotArgs>(args), g))           \
    X(body_id(BF_ST_APPLYDOT, 2, 0), st_apply_dot_body<2>(load_args<StApplyDotArgs>(args), g))           \
    X(body_id(BF_DENSE_F, 0, 0), dense_apply_body<float>(load_args<DenseArgs<float>>(args), g))          \
    X(body_id(BF_XUPDATE_F, 4, 0), (pcg_xupdate_body<float, 4>(load_args<XUpdateArgs<float>>(args), g))) \
    X(body_id(BF_XUPDATE_F, 2, 0), (pcg_xupdate_body<float, 2>(load_args<XUpdateArgs<float>>(args), g))) \
    X(body_id(BF_PROLONG_F, 0, 0), time_prolong_add_body<float>(load_args<ProlongArgs<float>>(args), g)) \
    X(body_id(BF_DST_FD, 0, 0), (dst_body<float, double, false>(load_args<DstArgs>(args), g)))           \
    X(body_id(BF_DST_DD2, 0, 0), (dst_body<double, double, true>(load_args<DstArgs>(args), g)))          \
    X(body_id(BF_DST_DF, 0, 0), (dst_body<double, float, false>(load_args<DstArgs>(args), g)))

__device__ __forceinline__ void run_body(int body, const void* args, const VGrid& g) {
#define PTP_CASE(ID, CALL) \
    case ID:               \
        CALL;              \
        break;
    switch (body) { PTP_FUSED_BODIES(PTP_CASE) }
#undef PTP_CASE
}

__global__ void __launch_bounds__(kStBlock) k_fused_program(const FusedPhase* __restrict__ ph, int nph) {
    cooperative_groups::grid_group grid = cooperative_groups::this_grid();
    for (int p = 0; p < nph; ++p) {
        const FusedPhase P = ph[p];
        const int nb = P.gx * P.gy;
        for (int vb = blockIdx.x; vb < nb; vb += gridDim.x) {
            run_body(P.body, P.args, VGrid{vb % P.gx, vb / P.gx, P.gx, P.gy});
            __syncthreads();   // the next virtual block reuses the shared memory
        }
        grid.sync();
    }
}

}  // namespace

bool fused_body_supported(int body) {
#define PTP_CASE(ID, CALL) \
    case ID:               \
        return true;
    switch (body) { PTP_FUSED_BODIES(PTP_CASE) }
#undef PTP_CASE
    return false;
}

int fused_program_grid(size_t smem) {
    ensure_dynamic_smem((const void*)k_fused_program, smem);
    int per_sm = 0;
    PTP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_program, kStBlock, smem));
    return per_sm * num_sms();
}

int launch_fused_program(const FusedPhase* phases, int nphases, int grid, size_t smem, cudaStream_t s) {
    if (record_foreign()) return 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kStBlock);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    PTP_CUDA(cudaLaunchKernelEx(&cfg, k_fused_program, phases, nphases));
    return 1;
}

}  // namespace ptp
