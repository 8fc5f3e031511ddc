// Host-side set-up: free-node numbering, P1 geometry, the data of the fused
// residual kernel, sparse operators and the spatial / temporal hierarchies.
//
// Discretisation (Section 4, "Simulation setup"): P1 elements on triangles,
// homogeneous Dirichlet nodes removed, implicit Euler with tau = T/N.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

#include "common.h"
#include "kernels.h"

namespace ptp {

namespace {

// Gradients of the hat functions of vertices 1 and 2 and the area of a
// triangle: grad(phi_1) = (b11, -b01)/det, grad(phi_2) = (-b10, b00)/det with
// B = [p1 - p0, p2 - p0] = [[b00, b01], [b10, b11]]; grad(phi_0) = -(sum).
struct Geo {
    double g[3][2];
    double area;
};

Geo triangle_geo(const double* p0, const double* p1, const double* p2) {
    double b00 = p1[0] - p0[0], b10 = p1[1] - p0[1];
    double b01 = p2[0] - p0[0], b11 = p2[1] - p0[1];
    double det = b00 * b11 - b01 * b10;
    Geo G;
    if (!(det > 0.0)) throw Error(PTP_EINVAL, "triangle is clockwise or degenerate");
    G.g[1][0] = b11 / det;
    G.g[1][1] = -b01 / det;
    G.g[2][0] = -b10 / det;
    G.g[2][1] = b00 / det;
    G.g[0][0] = -(G.g[1][0] + G.g[2][0]);
    G.g[0][1] = -(G.g[1][1] + G.g[2][1]);
    G.area = 0.5 * det;
    return G;
}

// Row-wise accumulation into a CSR matrix with sorted columns.
struct RowAccum {
    std::vector<std::map<int, double>> rows;
    explicit RowAccum(int n) : rows(n) {}
    void add(int i, int j, double v) { rows[i][j] += v; }
    HostCSR finish(int cols, bool drop_zeros) const {
        HostCSR A;
        A.rows = (int)rows.size();
        A.cols = cols;
        A.ptr.assign(A.rows + 1, 0);
        for (int i = 0; i < A.rows; ++i) {
            for (auto& kv : rows[i]) {
                if (drop_zeros && kv.second == 0.0) continue;
                A.idx.push_back(kv.first);
                A.val.push_back(kv.second);
            }
            A.ptr[i + 1] = (int)A.idx.size();
        }
        return A;
    }
};

HostCSR transpose(const HostCSR& A) {
    HostCSR T;
    T.rows = A.cols;
    T.cols = A.rows;
    T.ptr.assign(T.rows + 1, 0);
    for (int k = 0; k < A.nnz(); ++k) T.ptr[A.idx[k] + 1]++;
    for (int i = 0; i < T.rows; ++i) T.ptr[i + 1] += T.ptr[i];
    T.idx.resize(A.nnz());
    T.val.resize(A.nnz());
    std::vector<int> pos(T.ptr.begin(), T.ptr.end() - 1);
    for (int i = 0; i < A.rows; ++i)
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
            int p = pos[A.idx[k]]++;
            T.idx[p] = i;
            T.val[p] = A.val[k];
        }
    return T;  // rows come out sorted because i increases
}

// C = A * B with a dense accumulator per row (Gustavson).
HostCSR matmul(const HostCSR& A, const HostCSR& B) {
    if (A.cols != B.rows) throw Error(PTP_EINVAL, "matmul size mismatch");
    HostCSR C;
    C.rows = A.rows;
    C.cols = B.cols;
    C.ptr.assign(C.rows + 1, 0);
    std::vector<double> acc(B.cols, 0.0);
    std::vector<int> mark(B.cols, -1), cols;
    for (int i = 0; i < A.rows; ++i) {
        cols.clear();
        for (int ka = A.ptr[i]; ka < A.ptr[i + 1]; ++ka) {
            int k = A.idx[ka];
            double a = A.val[ka];
            for (int kb = B.ptr[k]; kb < B.ptr[k + 1]; ++kb) {
                int j = B.idx[kb];
                if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; cols.push_back(j); }
                acc[j] += a * B.val[kb];
            }
        }
        std::sort(cols.begin(), cols.end());
        for (int j : cols) { C.idx.push_back(j); C.val.push_back(acc[j]); }
        C.ptr[i + 1] = (int)C.idx.size();
    }
    return C;
}

// Removes entries that are zero up to rounding (|a_ij| <= 1e-13 max_j |a_ij|):
// the Galerkin product of the nested P1 operators carries structural entries
// whose exact value is 0, which would widen every row for nothing.
HostCSR drop_small(const HostCSR& A) {
    HostCSR B;
    B.rows = A.rows;
    B.cols = A.cols;
    B.ptr.assign(A.rows + 1, 0);
    for (int i = 0; i < A.rows; ++i) {
        double m = 0.0;
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) m = std::max(m, std::fabs(A.val[k]));
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
            if (std::fabs(A.val[k]) > 1e-13 * m || A.idx[k] == i) {
                B.idx.push_back(A.idx[k]);
                B.val.push_back(A.val[k]);
            }
        B.ptr[i + 1] = (int)B.idx.size();
    }
    return B;
}

// Values of A on the pattern `pat` (pat must contain A's pattern).
std::vector<double> values_on(const HostCSR& pat, const HostCSR& A) {
    std::vector<double> v(pat.nnz(), 0.0);
    for (int i = 0; i < pat.rows; ++i) {
        int kp = pat.ptr[i];
        for (int ka = A.ptr[i]; ka < A.ptr[i + 1]; ++ka) {
            while (kp < pat.ptr[i + 1] && pat.idx[kp] < A.idx[ka]) ++kp;
            if (kp == pat.ptr[i + 1] || pat.idx[kp] != A.idx[ka])
                throw Error(PTP_EINVAL, "pattern does not contain matrix");
            v[kp] = A.val[ka];
        }
    }
    return v;
}

HostCSR pattern_union(const HostCSR& A, const HostCSR& B) {
    HostCSR U;
    U.rows = A.rows;
    U.cols = A.cols;
    U.ptr.assign(U.rows + 1, 0);
    for (int i = 0; i < A.rows; ++i) {
        int a = A.ptr[i], b = B.ptr[i];
        while (a < A.ptr[i + 1] || b < B.ptr[i + 1]) {
            int ja = a < A.ptr[i + 1] ? A.idx[a] : INT32_MAX;
            int jb = b < B.ptr[i + 1] ? B.idx[b] : INT32_MAX;
            int j = std::min(ja, jb);
            U.idx.push_back(j);
            U.val.push_back(0.0);
            if (ja == j) ++a;
            if (jb == j) ++b;
        }
        U.ptr[i + 1] = (int)U.idx.size();
    }
    return U;
}

// Dense inverse of an SPD matrix by Gauss-Jordan with partial pivoting
// (coarsest spatial level only, a few hundred unknowns).
std::vector<double> dense_inverse(const HostCSR& M, const HostCSR& L, double cm, double cl) {
    int n = M.rows;
    std::vector<double> a((size_t)n * n, 0.0), inv((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        for (int k = M.ptr[i]; k < M.ptr[i + 1]; ++k) a[(size_t)i * n + M.idx[k]] += cm * M.val[k];
        for (int k = L.ptr[i]; k < L.ptr[i + 1]; ++k) a[(size_t)i * n + L.idx[k]] += cl * L.val[k];
        inv[(size_t)i * n + i] = 1.0;
    }
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(a[(size_t)r * n + c]) > std::fabs(a[(size_t)piv * n + c])) piv = r;
        if (std::fabs(a[(size_t)piv * n + c]) == 0.0)
            throw Error(PTP_EINVAL, "singular coarsest spatial operator");
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(a[(size_t)piv * n + k], a[(size_t)c * n + k]);
                std::swap(inv[(size_t)piv * n + k], inv[(size_t)c * n + k]);
            }
        double d = 1.0 / a[(size_t)c * n + c];
        for (int k = 0; k < n; ++k) { a[(size_t)c * n + k] *= d; inv[(size_t)c * n + k] *= d; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double f = a[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                a[(size_t)r * n + k] -= f * a[(size_t)c * n + k];
                inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
            }
        }
    }
    return inv;
}

std::vector<float> to_float(const std::vector<double>& v) {
    return std::vector<float>(v.begin(), v.end());
}

}  // namespace

void upload_csr(DevCSR& d, const HostCSR& a, const HostCSR* b, bool diag, cudaStream_t s) {
    d.rows = a.rows;
    d.cols = a.cols;
    d.nnz = a.nnz();
    d.ptr.upload(a.ptr, s);
    d.idx.upload(a.idx, s);
    d.v1d.upload(a.val, s);
    d.v1f.upload(to_float(a.val), s);
    std::vector<double> bv;
    if (b) {
        bv = values_on(a, *b);
        d.v2d.upload(bv, s);
        d.v2f.upload(to_float(bv), s);
    }
    // padded ELL copy for rows of at most 8 entries (wider rows keep CSR)
    int wmax = 0;
    for (int i = 0; i < a.rows; ++i) wmax = std::max(wmax, a.ptr[i + 1] - a.ptr[i]);
    int w = wmax <= 2 ? 2 : wmax <= 4 ? 4 : wmax <= 8 ? 8 : 0;
    d.ell_w = w;
    if (w > 0) {
        std::vector<int> ei((size_t)a.rows * w);
        std::vector<double> e1((size_t)a.rows * w, 0.0), e2((size_t)a.rows * w, 0.0);
        for (int i = 0; i < a.rows; ++i) {
            int k = 0;
            for (int q = a.ptr[i]; q < a.ptr[i + 1]; ++q, ++k) {
                ei[(size_t)i * w + k] = a.idx[q];
                e1[(size_t)i * w + k] = a.val[q];
                if (b) e2[(size_t)i * w + k] = bv[q];
            }
            for (; k < w; ++k) ei[(size_t)i * w + k] = i < a.cols ? i : 0;
        }
        d.eidx.upload(ei, s);
        std::vector<int4> pk((size_t)a.rows * w);
        for (size_t q = 0; q < pk.size(); ++q) {
            float f1 = (float)e1[q], f2 = (float)e2[q];
            int b1, b2;
            std::memcpy(&b1, &f1, 4);
            std::memcpy(&b2, &f2, 4);
            pk[q] = make_int4(ei[q], b1, b2, 0);
        }
        d.pk.upload(pk, s);
        d.e1d.upload(e1, s);
        d.e1f.upload(to_float(e1), s);
        if (b) {
            d.e2d.upload(e2, s);
            d.e2f.upload(to_float(e2), s);
        }
    }
    if (diag) {
        std::vector<double> d1(a.rows, 0.0), d2(a.rows, 0.0);
        for (int i = 0; i < a.rows; ++i)
            for (int k = a.ptr[i]; k < a.ptr[i + 1]; ++k)
                if (a.idx[k] == i) {
                    d1[i] = a.val[k];
                    if (b) d2[i] = bv[k];
                }
        d.d1d.upload(d1, s);
        d.d1f.upload(to_float(d1), s);
        d.d2d.upload(d2, s);
        d.d2f.upload(to_float(d2), s);
    }
}

void make_structured_mesh(Ctx& c, int nx, int ny, double x0, double y0, double x1, double y1) {
    PTP_REQUIRE(nx >= 2 && ny >= 2, "structured grid needs nx, ny >= 2");
    PTP_REQUIRE((int64_t)nx * ny <= ((int64_t)1 << 28), "structured grid: at most 2^28 nodes");
    PTP_REQUIRE(x1 > x0 && y1 > y0 && std::isfinite(x0) && std::isfinite(x1) && std::isfinite(y0) &&
                    std::isfinite(y1),
                "structured grid needs finite x1 > x0 and y1 > y0");
    c.n_nodes = nx * ny;
    c.xy.assign(2 * (size_t)c.n_nodes, 0.0);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            c.xy[2 * ((size_t)j * nx + i) + 0] = x0 + (x1 - x0) * i / (nx - 1);
            c.xy[2 * ((size_t)j * nx + i) + 1] = y0 + (y1 - y0) * j / (ny - 1);
        }
    c.n_tri = 2 * (nx - 1) * (ny - 1);
    c.tri.assign(3 * (size_t)c.n_tri, 0);
    size_t e = 0;
    for (int j = 0; j < ny - 1; ++j)
        for (int i = 0; i < nx - 1; ++i) {
            int n00 = j * nx + i, n10 = n00 + 1, n11 = n00 + nx + 1, n01 = n00 + nx;
            int* t = &c.tri[3 * e];
            t[0] = n00; t[1] = n10; t[2] = n11;
            t[3] = n00; t[4] = n11; t[5] = n01;
            e += 2;
        }
    c.dirichlet.assign(c.n_nodes, 0);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            if (i == 0 || j == 0 || i == nx - 1 || j == ny - 1) c.dirichlet[(size_t)j * nx + i] = 1;
    c.structured = true;
    c.gnx = nx; c.gny = ny; c.gx0 = x0; c.gy0 = y0; c.gx1 = x1; c.gy1 = y1;
}

static void build_k1_structured(Ctx& c, const HostCSR& M, const std::vector<double>& mval, const HostCSR& Ll,
                                const std::vector<int>& iron_of, cudaStream_t s);
static void build_dst(Ctx& c, cudaStream_t s);

void build_problem(Ctx& c) {
    PTP_REQUIRE(c.n_nodes > 0 && c.n_tri > 0, "no mesh");
    PTP_REQUIRE(c.have_materials, "materials not set");
    PTP_REQUIRE(c.N >= 1 && c.T > 0, "time not set");
    PTP_REQUIRE((int)c.sigma.size() == c.n_tri, "materials do not match the mesh");
    PTP_REQUIRE((int)c.coil_of_elem.size() == c.n_tri || c.n_coils == 0, "sources do not match the mesh");
    PTP_REQUIRE((int)c.nonlinear.size() == c.n_tri, "materials do not match the mesh");
    PTP_REQUIRE(!c.law_exp || c.law_abcd.size() == 4 * (size_t)c.n_tri, "the exponential law does not match the mesh");
    PTP_REQUIRE(c.khat.empty() || (int)c.khat.size() == c.n_tri, "the K_hat weights do not match the mesh");
    cudaStream_t s = c.stream;
    const double tau = c.T / c.N;

    c.free_id.assign(c.n_nodes, -1);
    int n = 0;
    for (int i = 0; i < c.n_nodes; ++i)
        if (!c.dirichlet[i]) c.free_id[i] = n++;
    PTP_REQUIRE(n > 0, "mesh has no free node");
    c.n = n;

    // Residual data.  K(u) splits exactly into a linear part (elements with
    // constant nu_linear: a CSR stencil nu_linear * A_lin) and the iron
    // elements, whose fluxes nu(|g|^2)|T| g are computed per element.
    std::vector<int> iron_of(c.n_tri, -1);
    int n_iron = 0;
    for (int e = 0; e < c.n_tri; ++e)
        if (c.nonlinear[e]) iron_of[e] = n_iron++;
    std::vector<int> e_nodes(3 * (size_t)std::max(n_iron, 1), -1);
    std::vector<double> e_geo(6 * (size_t)std::max(n_iron, 1), 0.0);
    std::vector<double> e_area(std::max(n_iron, 1), 0.0);
    std::vector<double> e_law(c.law_exp ? 4 * (size_t)std::max(n_iron, 1) : 0, 0.0);
    const bool weighted = !c.khat.empty();
    std::vector<int> all_nodes(3 * (size_t)c.n_tri);
    std::vector<double> all_area(c.n_tri);
    std::vector<uint8_t> all_iron(c.n_tri);
    RowAccum MJa(n);
    std::vector<std::vector<std::pair<int, int>>> inc(n);  // (iron element, local vertex)
    std::vector<Geo> geo(c.n_tri);
    RowAccum Ma(n), Aa(n), Llin(n), Lw(weighted ? n : 0);
    std::vector<double> cb((size_t)std::max(c.n_coils, 1) * n, 0.0);
    const double dnu_c = (c.nu_max - c.nu_min) * c.s_sat * c.s_sat;
    for (int e = 0; e < c.n_tri; ++e) {
        const int* t = &c.tri[3 * (size_t)e];
        for (int a = 0; a < 3; ++a)
            PTP_REQUIRE(t[a] >= 0 && t[a] < c.n_nodes, "triangle vertex id out of range");
        Geo G = triangle_geo(&c.xy[2 * (size_t)t[0]], &c.xy[2 * (size_t)t[1]], &c.xy[2 * (size_t)t[2]]);
        geo[e] = G;
        const int ie = iron_of[e];
        for (int a = 0; a < 3; ++a) all_nodes[3 * (size_t)e + a] = c.free_id[t[a]];
        all_area[e] = G.area;
        all_iron[e] = ie >= 0 ? 1 : 0;
        if (ie >= 0) e_area[ie] = G.area;
        if (ie >= 0) {
            for (int a = 0; a < 3; ++a) e_nodes[3 * (size_t)ie + a] = c.free_id[t[a]];
            double* g = &e_geo[6 * (size_t)ie];
            g[0] = G.g[1][0]; g[1] = G.g[1][1]; g[2] = G.g[2][0]; g[3] = G.g[2][1];
            // nu |T| = |T| nu_max - |T| (nu_max - nu_min) s_sat^2 / (s^2 + s_sat^2)
            g[4] = G.area * c.nu_max;
            g[5] = G.area * dnu_c;
            if (c.law_exp) {
                const double* L = &c.law_abcd[4 * (size_t)e];
                double* w = &e_law[4 * (size_t)ie];
                w[0] = G.area * L[0];
                w[1] = L[1];
                w[2] = std::log(L[2]);
                w[3] = G.area * L[3];
            }
        }
        for (int a = 0; a < 3; ++a) {
            int i = c.free_id[t[a]];
            if (i < 0) continue;
            if (ie >= 0) inc[i].push_back({ie, a});
            for (int b = 0; b < 3; ++b) {
                int j = c.free_id[t[b]];
                if (j < 0) continue;
                // consistent mass sigma |T| / 12 (1 + delta_ab); unit stiffness
                const double k = G.area * (G.g[a][0] * G.g[b][0] + G.g[a][1] * G.g[b][1]);
                if (c.sigma[e] != 0.0) {
                    const double mv = c.sigma[e] * G.area * (a == b ? 2.0 : 1.0) / 12.0;
                    Ma.add(i, j, mv);
                    if (ie >= 0) MJa.add(i, j, mv);
                }
                Aa.add(i, j, k);
                if (weighted) Lw.add(i, j, c.khat[e] * k);
                if (ie < 0) Llin.add(i, j, c.nu_linear * k);
            }
            if (c.n_coils > 0 && c.coil_of_elem[e] >= 0)
                cb[(size_t)c.coil_of_elem[e] * n + i] += G.area / 3.0;
        }
    }
    c.n_iron = n_iron;
    c.e_nodes.upload(e_nodes, s);
    c.e_geo.upload(e_geo, s);
    if (c.law_exp) c.e_law.upload(e_law, s); else c.e_law.release();
    c.e_area.upload(e_area, s);
    c.all_nodes.upload(all_nodes, s);
    c.all_area.upload(all_area, s);
    c.all_iron.upload(all_iron, s);
    {
        HostCSR MJ = MJa.finish(n, true);
        c.mj_ptr.upload(MJ.ptr, s);
        c.mj_idx.upload(MJ.idx, s);
        c.mj_val.upload(MJ.val, s);
    }

    std::vector<int> ip(n + 1, 0), ie;
    std::vector<double> ig;
    for (int i = 0; i < n; ++i) {
        for (auto& pr : inc[i]) ie.push_back(pr.first);
        ip[i + 1] = (int)ie.size();
    }
    {
        std::vector<int> iron_elem(std::max(n_iron, 1), 0);
        for (int e = 0; e < c.n_tri; ++e)
            if (iron_of[e] >= 0) iron_elem[iron_of[e]] = e;
        for (int i = 0; i < n; ++i)
            for (auto& pr : inc[i]) {
                const Geo& G = geo[iron_elem[pr.first]];
                ig.push_back(G.g[pr.second][0]);
                ig.push_back(G.g[pr.second][1]);
            }
    }
    c.inc_ptr.upload(ip, s);
    c.inc_elem.upload(ie, s);
    c.inc_grad.upload(ig, s);

    HostCSR M = Ma.finish(n, true);
    HostCSR A = Aa.finish(n, false);
    {   // mass rows scaled by 1/tau and the linear-element stiffness, for the residual
        std::vector<double> mv(M.val);
        for (auto& v : mv) v /= tau;
        c.m_ptr.upload(M.ptr, s);
        c.zero_ptr.upload(std::vector<int>((size_t)n + 1, 0), s);
        c.m_idx.upload(M.idx, s);
        c.m_val.upload(mv, s);
        HostCSR Ll = Llin.finish(n, true);
        c.l_ptr.upload(Ll.ptr, s);
        c.l_idx.upload(Ll.idx, s);
        c.l_val.upload(Ll.val, s);
        build_k1_structured(c, M, mv, Ll, iron_of, s);
    }
    // K_hat: nu_max A, or sum_T khat_T A_T with the per-element weights
    HostCSR L = A;
    if (weighted) {
        HostCSR Lk = Lw.finish(n, false);
        L.val = values_on(A, Lk);
    } else {
        for (auto& v : L.val) v *= c.nu_max;
    }

    // spatial level 0
    c.sl.clear();
    c.sl.emplace_back();
    SpatialLevel& l0 = c.sl[0];
    l0.n = n;
    l0.nx = c.structured ? c.gnx : 0;
    l0.ny = c.structured ? c.gny : 0;
    l0.hM = M;
    l0.hL = L;

    // coils: loads and time factors amp sin(2 pi t^n / T + phase), t^n = n tau
    std::vector<double> cs((size_t)std::max(c.n_coils, 1) * c.N, 0.0), csin(cs.size(), 0.0);
    for (int k = 0; k < c.n_coils; ++k)
        for (int j = 0; j < c.N; ++j) {
            csin[(size_t)k * c.N + j] = std::sin(2.0 * M_PI * ((j + 1) * tau) / c.T + c.phase[k]);
            cs[(size_t)k * c.N + j] = c.amp[k] * csin[(size_t)k * c.N + j];
        }
    c.coil_b.upload(cb, s);
    c.coil_s.upload(cs, s);
    c.coil_sin.upload(csin, s);
}

// Data of the fused residual on a structured grid with the saturating law:
// per grid cell which of its two triangles are iron, per free node the rows
// of M / tau and of the linear-element stiffness as stencils (the P1 pattern
// of the grid), and the element constants, which are equal on every iron
// triangle of the uniform grid.  Leaves k1_struct false on any other mesh.
static void build_k1_structured(Ctx& c, const HostCSR& M, const std::vector<double>& mval, const HostCSR& Ll,
                                const std::vector<int>& iron_of, cudaStream_t s) {
    c.k1_struct = false;
    c.k1_cell.release(); c.k1_flag.release(); c.k1_mass.release(); c.k1_lin.release();
    if (!c.structured || c.law_exp || c.gnx < 3 || c.gny < 3) return;
    const int nx = c.gnx, ny = c.gny, W = nx - 2, H = ny - 2;
    if ((int64_t)W * H != c.n) return;
    const double hx = (c.gx1 - c.gx0) / (nx - 1), hy = (c.gy1 - c.gy0) / (ny - 1);
    std::vector<uint8_t> cell((size_t)(nx - 1) * (ny - 1), 0);
    for (int j = 0; j < ny - 1; ++j)
        for (int i = 0; i < nx - 1; ++i) {
            const size_t e = 2 * ((size_t)j * (nx - 1) + i);
            cell[(size_t)j * (nx - 1) + i] = (uint8_t)((iron_of[e] >= 0 ? 1 : 0) | (iron_of[e + 1] >= 0 ? 2 : 0));
        }
    auto slot = [&](int i, int j) -> int {
        const int da = j % W - i % W, db = j / W - i / W;
        const int off[7][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}};
        for (int k = 0; k < 7; ++k)
            if (off[k][0] == da && off[k][1] == db) return k;
        return -1;
    };
    std::vector<double> mass(8 * (size_t)c.n, 0.0), lin(8 * (size_t)c.n, 0.0);
    std::vector<uint8_t> flag(c.n, 0);
    for (int i = 0; i < c.n; ++i) {
        for (int k = M.ptr[i]; k < M.ptr[i + 1]; ++k) {
            const int sl = slot(i, M.idx[k]);
            if (sl < 0) return;
            mass[8 * (size_t)i + sl] = mval[k];
            if (mval[k] != 0.0) flag[i] |= 1;
        }
        for (int k = Ll.ptr[i]; k < Ll.ptr[i + 1]; ++k) {
            const int sl = slot(i, Ll.idx[k]);
            if (sl < 0 || sl > 4) return;   // right triangles: no diagonal coupling in the stiffness
            lin[8 * (size_t)i + sl] = Ll.val[k];
            if (Ll.val[k] != 0.0) flag[i] |= 2;
        }
    }
    const double area = 0.5 * hx * hy;
    c.k1_ihx2 = 1.0 / (hx * hx);
    c.k1_ihy2 = 1.0 / (hy * hy);
    c.k1_At = area * c.nu_max;
    c.k1_Bt = area * (c.nu_max - c.nu_min) * c.s_sat * c.s_sat;
    c.k1_cell.upload(cell, s);
    c.k1_flag.upload(flag, s);
    c.k1_mass.upload(mass, s);
    c.k1_lin.upload(lin, s);
    c.k1_struct = true;
}

// The exact tau_c L solve of the coarsest time level by sine transforms
// (k_poisson.cu): on a uniform structured grid with K_hat = nu_max A, and
// (nx - 1), (ny - 1) powers of two, the FFT twiddles, the inverse
// eigenvalues (with the transforms' normalisation) and two work arrays.
static void build_dst(Ctx& c, cudaStream_t s) {
    c.dst_ok = false;
    c.dst_wx.release(); c.dst_wy.release(); c.dst_scale.release(); c.dst_tmp.release(); c.dst_tmp2.release();
    if (!c.opts.coarse_direct || !c.structured || !c.khat.empty() || !c.coarse_ok || c.coarse_ops[0] < 0) return;
    const int W = c.gnx - 2, H = c.gny - 2;
    if (W < 1 || H < 1 || (int64_t)W * H != c.n) return;
    const int mx = W + 1, my = H + 1;
    if ((mx & (mx - 1)) || (my & (my - 1)) || 2 * mx > 65536 || 2 * my > 65536) return;
    const double hx = (c.gx1 - c.gx0) / (c.gnx - 1), hy = (c.gy1 - c.gy0) / (c.gny - 1);
    const double coef = c.ops[c.coarse_ops[0]].cl * c.nu_max;   // tau_c nu_max
    auto twiddles = [](int L) {
        std::vector<double2> w(L / 2);
        for (int j = 0; j < L / 2; ++j) w[j] = make_double2(std::cos(2.0 * M_PI * j / L), -std::sin(2.0 * M_PI * j / L));
        return w;
    };
    std::vector<double> sc((size_t)W * H);
    for (int k = 1; k <= W; ++k)
        for (int l = 1; l <= H; ++l) {
            const double lam = hy / hx * (2.0 - 2.0 * std::cos(M_PI * k / mx)) +
                               hx / hy * (2.0 - 2.0 * std::cos(M_PI * l / my));
            sc[(size_t)(k - 1) * H + (l - 1)] = (2.0 / mx) * (2.0 / my) / (coef * lam);
        }
    int lx = 0, ly = 0;
    while ((1 << lx) < 2 * mx) ++lx;
    while ((1 << ly) < 2 * my) ++ly;
    c.dst_wx.upload(twiddles(2 * mx), s);
    c.dst_wy.upload(twiddles(2 * my), s);
    c.dst_scale.upload(sc, s);
    c.dst_tmp.alloc((size_t)W * H);
    c.dst_tmp2.alloc((size_t)W * H);
    c.dst_logx = lx;
    c.dst_logy = ly;
    c.dst_ok = true;
}

// The operators M and L of a structured level as per-node 7-point stencils:
// for free node (a, b) (index b W + a) the coefficients of the neighbours
// C (a, b), E (a+1, b), W (a-1, b), N (a, b+1), S (a, b-1), NE (a+1, b+1),
// SW (a-1, b-1) -- the P1 pattern of the grid whose cells are split along
// (i, j)-(i+1, j+1).  Layout per node: M {C, E, W, N}, M {S, NE, SW, 0},
// L {C, E, W, N}, L {S, NE, SW, 0}.  Returns false if an entry lies outside
// the pattern (then the level has no stencil form).
static bool stencil_coefficients(const HostCSR& M, const HostCSR& L, int W, int H, std::vector<float>& out) {
    const int n = W * H;
    out.assign(16 * (size_t)n, 0.0f);
    auto slot = [&](int i, int j) -> int {
        const int ai = i % W, bi = i / W, aj = j % W, bj = j / W;
        const int da = aj - ai, db = bj - bi;
        if (da == 0 && db == 0) return 0;
        if (da == 1 && db == 0) return 1;
        if (da == -1 && db == 0) return 2;
        if (da == 0 && db == 1) return 3;
        if (da == 0 && db == -1) return 4;
        if (da == 1 && db == 1) return 5;
        if (da == -1 && db == -1) return 6;
        return -1;
    };
    for (int part = 0; part < 2; ++part) {
        const HostCSR& A = part == 0 ? M : L;
        if (A.rows != n) return false;
        for (int i = 0; i < n; ++i)
            for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
                const int sl = slot(i, A.idx[k]);
                if (sl < 0) {
                    if (A.val[k] != 0.0) return false;
                    continue;
                }
                out[16 * (size_t)i + 8 * part + sl] = (float)A.val[k];
            }
    }
    return true;
}

void build_hierarchy(Ctx& c) {
    cudaStream_t s = c.stream;
    const ptp_opts& o = c.opts;
    const int COARSE_MAX = 600;  // free nodes of the coarsest spatial level (dense inverse)

    // ---- spatial hierarchy on nested structured grids ----
    while (o.spatial_prec == PTP_PREC_GMG && c.structured) {
        SpatialLevel& f = c.sl.back();
        int nx = f.nx, ny = f.ny;
        if (f.n <= COARSE_MAX) break;
        if ((nx - 1) % 2 || (ny - 1) % 2 || nx < 5 || ny < 5) break;
        int cx = (nx - 1) / 2 + 1, cy = (ny - 1) / 2 + 1;
        // free numbering of both grids (interior nodes, row-major)
        auto fid = [&](int i, int j) { return (j - 1) * (nx - 2) + (i - 1); };
        auto cid = [&](int i, int j) -> int {
            if (i <= 0 || j <= 0 || i >= cx - 1 || j >= cy - 1) return -1;
            return (j - 1) * (cx - 2) + (i - 1);
        };
        int nc = (cx - 2) * (cy - 2);
        RowAccum Pa(f.n);
        for (int j = 1; j < ny - 1; ++j)
            for (int i = 1; i < nx - 1; ++i) {
                int r = fid(i, j);
                // P1 interpolation on the nested mesh (diagonal (i,j)-(i+1,j+1)):
                // coarse vertex, edge midpoints (horizontal, vertical, diagonal)
                int ci[2], cj[2], m;
                if (i % 2 == 0 && j % 2 == 0) { ci[0] = i / 2; cj[0] = j / 2; m = 1; }
                else if (j % 2 == 0) { ci[0] = (i - 1) / 2; cj[0] = j / 2; ci[1] = (i + 1) / 2; cj[1] = j / 2; m = 2; }
                else if (i % 2 == 0) { ci[0] = i / 2; cj[0] = (j - 1) / 2; ci[1] = i / 2; cj[1] = (j + 1) / 2; m = 2; }
                else { ci[0] = (i - 1) / 2; cj[0] = (j - 1) / 2; ci[1] = (i + 1) / 2; cj[1] = (j + 1) / 2; m = 2; }
                for (int k = 0; k < m; ++k) {
                    int q = cid(ci[k], cj[k]);
                    if (q >= 0) Pa.add(r, q, m == 1 ? 1.0 : 0.5);
                }
            }
        HostCSR P = Pa.finish(nc, true);
        HostCSR Rt = transpose(P);
        SpatialLevel cl;
        cl.n = nc;
        cl.nx = cx;
        cl.ny = cy;
        cl.hM = drop_small(matmul(Rt, matmul(f.hM, P)));
        cl.hL = drop_small(matmul(Rt, matmul(f.hL, P)));
        f.hP = P;
        c.sl.push_back(std::move(cl));
    }
    for (size_t k = 0; k < c.sl.size(); ++k) {
        SpatialLevel& L = c.sl[k];
        HostCSR pat = pattern_union(L.hM, L.hL);
        HostCSR vm = pat;
        vm.val = values_on(pat, L.hM);
        upload_csr(L.op, vm, &L.hL, true, s);
        if (k + 1 < c.sl.size()) {
            upload_csr(L.P, L.hP, nullptr, false, s);
            upload_csr(L.R, transpose(L.hP), nullptr, false, s);
        }
    }

    // ---- the same operators as 7-point stencils (structured hierarchy) ----
    c.stencil_ok = c.structured && o.spatial_prec == PTP_PREC_GMG && c.sl.size() > 1;
    for (auto& L : c.sl) {
        L.st_ok = false;
        L.st_coef.release();
        if (!c.stencil_ok) continue;
        if (L.nx < 3 || L.ny < 3 || (L.nx - 2) * (L.ny - 2) != L.n) { c.stencil_ok = false; continue; }
        std::vector<float> coef;
        if (!stencil_coefficients(L.hM, L.hL, L.nx - 2, L.ny - 2, coef)) { c.stencil_ok = false; continue; }
        std::vector<float4> packed(coef.size() / 4);
        std::memcpy(packed.data(), coef.data(), coef.size() * sizeof(float));
        L.st_coef.upload(packed, s);
        L.st_ok = true;
    }
    if (!c.stencil_ok)
        for (auto& L : c.sl) { L.st_ok = false; L.st_coef.release(); }

    // ---- time levels: coarsen by 2 while N_l is even and above N_c ----
    c.tl.clear();
    c.ops.clear();
    int Nl = c.N;
    int nc_target = o.coarse_steps == 2 ? 2 : 1;
    for (;;) {
        TimeLevel t;
        t.N = Nl;
        t.tau = c.T / Nl;
        c.tl.push_back(t);
        const bool can = (Nl % 2 == 0) && (Nl / 2 >= nc_target);
        if (!can) break;
        Nl /= 2;
    }
    const int Nc = c.tl.back().N;   // the exact coarse solve needs Nc in {1, 2}; checked by the solves
    auto add_op = [&](double cm, double cl) {
        OpPair p;
        p.cm = cm;
        p.cl = cl;
        c.ops.push_back(std::move(p));
        return (int)c.ops.size() - 1;
    };
    for (auto& t : c.tl) t.op = add_op(1.0, t.tau);
    double tc = c.tl.back().tau;
    c.coarse_ops[0] = add_op(0.0, tc);            // sum mode:        tau_c L
    c.coarse_ops[1] = Nc == 2 ? add_op(2.0, tc) : -1;  // difference:  2M + tau_c L
    c.coarse_ok = Nc == 1 || Nc == 2;
    build_dst(c, s);
    const int full = (int)c.tl.size();
    c.active_levels = o.time_levels > 0 ? std::min(o.time_levels, full) : full;
    // DFT in time on the last level used: preconditioner tau_l L, twiddles and mode shifts
    c.dft_level = -1;
    c.dft_op = -1;
    c.dft_W.release();
    c.dft_ck.release();
    if (o.coarse_solver == PTP_COARSE_DFT) {
        const int l = c.active_levels - 1;
        const int Nl = c.tl[l].N;
        PTP_REQUIRE(Nl >= 1 && Nl <= kMaxDftSteps, "DFT coarse solver: the last level needs 1..1022 steps");
        c.dft_level = l;
        c.dft_op = add_op(0.0, c.tl[l].tau);
        std::vector<double> W(2 * (size_t)Nl), ck(2 * (size_t)(Nl / 2 + 1));
        for (int j = 0; j < Nl; ++j) {
            const double th = 2.0 * M_PI * j / Nl;
            W[2 * j] = std::cos(th);
            W[2 * j + 1] = -std::sin(th);
        }
        for (int k = 0; k <= Nl / 2; ++k) {   // c_k = 1 - e^{-i theta_k}
            const double th = 2.0 * M_PI * k / Nl;
            ck[2 * k] = 1.0 - std::cos(th);
            ck[2 * k + 1] = std::sin(th);
        }
        c.dft_W.upload(W, s);
        c.dft_ck.upload(ck, s);
    }
    // precombined double operators cm M + cl L per spatial level (ELL values and diagonal)
    for (auto& p : c.ops) {
        p.comb.clear();
        p.dcomb.clear();
        p.comb.resize(c.sl.size());
        p.dcomb.resize(c.sl.size());
        for (size_t k = 0; k < c.sl.size(); ++k) {
            const DevCSR& d = c.sl[k].op;
            if (d.ell_w > 0) {
                const size_t m = (size_t)d.rows * d.ell_w;
                p.comb[k].alloc(m);
                launch_lincomb(m, p.cm, d.e1d.p, p.cl, d.e2d.p, p.comb[k].p, s);
            }
            p.dcomb[k].alloc((size_t)d.rows);
            launch_lincomb((size_t)d.rows, p.cm, d.d1d.p, p.cl, d.d2d.p, p.dcomb[k].p, s);
        }
    }
    // precombined float stencils cm M + cl L per op pair and structured level
    for (auto& p : c.ops) {
        p.st_a.clear();
        p.st_a.resize(c.sl.size());
        if (!c.stencil_ok) continue;
        for (size_t k = 0; k < c.sl.size(); ++k) {
            p.st_a[k].alloc((size_t)2 * c.sl[k].n);
            launch_st_combine(c.sl[k].n, c.sl[k].st_coef.p, (float)p.cm, (float)p.cl, p.st_a[k].p, s);
        }
    }
    // dense inverses on the coarsest spatial level
    const SpatialLevel& cs = c.sl.back();
    if (cs.n <= COARSE_MAX) {
        for (auto& p : c.ops) {
            std::vector<double> inv = dense_inverse(cs.hM, cs.hL, p.cm, p.cl);
            p.inv_d.upload(inv, s);
            p.inv_f.upload(to_float(inv), s);
        }
    }
}

}  // namespace ptp
