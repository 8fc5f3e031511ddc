// Choice of the block-Jacobi smoother of the multigrid-in-time cycle.
//
// On one spatial eigenmode of the pencil (L, M) with eigenvalue lambda, the
// periodic implicit-Euler system of time level l, (M + tau_l L) x^n - M x^{n-1}
// = b^n, becomes the scalar circulant system
//   P_l x = (1 + kappa_l) x^n - x^{n-1},   kappa_l = tau_l lambda,
// and the cycle of the solver acts on it mode by mode: damped Jacobi
// x += omega / (1 + kappa_l) (b - P_l x), restriction by pair sums
// r_c^m = r^{2m} + r^{2m+1}, injection x^{2m}, x^{2m+1} += x_c^m, and the
// Galerkin identity R P_l P = P_{l+1} (tau_{l+1} = 2 tau_l) holds exactly.
// Modes with small kappa (conducting regions, slow spatial modes, short
// steps) are pure transport in time, where the smoother barely damps and the
// coarse correction can amplify: the V(1,0) cycle with omega near 1, which is
// the cheapest and best cycle when kappa >= 1, has an error growth factor
// of several units when kappa -> 0.  So the damping and the post-smoothing
// are chosen per problem from the smallest kappa it has: the spectral radius
// of the cycle's error propagation on the scalar model is estimated by power
// iteration for each candidate and every kappa >= kappa_min, and the
// cheapest candidate with a radius below kRhoTarget is taken.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "common.h"

namespace ptp {

namespace {

constexpr double kRhoTarget = 0.6;

// exact solve of (1 + k) x^n - x^{n-1} = b^n, x^{-1} = x^{N-1}:
// x^n = (b^n + x^{n-1}) / (1 + k) unrolled over one period gives x^{N-1}
void exact_solve(const std::vector<double>& b, double k, std::vector<double>& x) {
    const int N = (int)b.size();
    const double q = 1.0 / (1.0 + k);
    // x^{N-1} = sum_{j=0}^{N-1} q^{j+1} b^{N-1-j} / (1 - q^N)
    double s = 0.0, qj = q;
    for (int j = 0; j < N; ++j) {
        s += qj * b[N - 1 - j];
        qj *= q;
    }
    const double denom = 1.0 - std::pow(q, N);
    double prev = denom > 0 ? s / denom : 0.0;
    x.assign(N, 0.0);
    for (int n = 0; n < N; ++n) {
        prev = q * (b[n] + prev);
        x[n] = prev;
    }
}

struct Model {
    std::vector<int> Nl;   // steps per level; the last level is solved exactly
    double kappa0;         // kappa of level 0
    int pre, post;
    double omega;

    double kappa(int l) const { return kappa0 * (double)Nl[0] / (double)Nl[l]; }

    void residual(int l, const std::vector<double>& x, const std::vector<double>& b, std::vector<double>& r) const {
        const int N = Nl[l];
        const double k = kappa(l);
        r.resize(N);
        for (int n = 0; n < N; ++n) r[n] = b[n] - ((1.0 + k) * x[n] - x[n == 0 ? N - 1 : n - 1]);
    }

    void smooth(int l, std::vector<double>& x, const std::vector<double>& b) const {
        std::vector<double> r;
        residual(l, x, b, r);
        const double w = omega / (1.0 + kappa(l));
        for (size_t n = 0; n < x.size(); ++n) x[n] += w * r[n];
    }

    // one V-cycle on level l for P_l x = b, improving x in place
    void cycle(int l, std::vector<double>& x, const std::vector<double>& b) const {
        const int L = (int)Nl.size();
        if (l == L - 1) {
            exact_solve(b, kappa(l), x);
            return;
        }
        for (int k = 0; k < pre; ++k) smooth(l, x, b);
        std::vector<double> r;
        residual(l, x, b, r);
        const int Nc = Nl[l + 1];
        std::vector<double> bc(Nc), xc(Nc, 0.0);
        for (int m = 0; m < Nc; ++m) bc[m] = r[2 * m] + r[2 * m + 1];
        cycle(l + 1, xc, bc);
        for (int m = 0; m < Nc; ++m) {
            x[2 * m] += xc[m];
            x[2 * m + 1] += xc[m];
        }
        for (int k = 0; k < post; ++k) smooth(l, x, b);
    }
};

double norm2(const std::vector<double>& v) {
    double s = 0.0;
    for (double a : v) s += a * a;
    return std::sqrt(s);
}

}  // namespace

// Asymptotic growth factor of the error under repeated cycles (b = 0):
// (||E^{2m} e|| / ||E^m e||)^{1/m} from a fixed pseudo-random start, which
// tends to the spectral radius of E (complex pairs included).
double tmg_cycle_rho(const std::vector<int>& Nl, double kappa0, int pre, int post, double omega) {
    if (Nl.empty() || Nl[0] < 1) return 0.0;
    for (size_t l = 1; l < Nl.size(); ++l)
        if (Nl[l - 1] != 2 * Nl[l]) return -1.0;   // not a halving hierarchy
    Model m{Nl, kappa0, pre, post, omega};
    std::vector<double> e(Nl[0]), zero(Nl[0], 0.0);
    uint64_t s = 0x9E3779B97F4A7C15ull;
    for (auto& v : e) {
        s = s * 6364136223846793005ull + 1442695040888963407ull;
        v = (double)(s >> 11) / 9007199254740992.0 - 0.5;
    }
    const int half = 200;
    double log_first = 0.0, log_total = 0.0;
    for (int it = 0; it < 2 * half; ++it) {
        m.cycle(0, e, zero);
        const double g = norm2(e);
        if (!(g > 1e-300) || !std::isfinite(g)) return g > 0 ? 1e300 : 0.0;
        const double lg = std::log(g);
        log_total += lg;
        if (it < half) log_first += lg;
        for (auto& v : e) v /= g;
    }
    return std::exp((log_total - log_first) / half);
}

// worst radius over kappa >= kappa_min, kappa doubled up to 1e3 (beyond it
// D^-1 P is the identity to 1e-3 and the smoother alone sets the rate);
// returns as soon as the radius exceeds stop_above
static double worst_rho(const std::vector<int>& Nl, double kappa_min, int pre, int post, double omega,
                        double stop_above) {
    double worst = 0.0;
    double k = std::max(kappa_min, 1e-12);
    do {
        worst = std::max(worst, tmg_cycle_rho(Nl, k, pre, post, omega));
        if (worst > stop_above) break;
        k *= 2.0;
    } while (k <= 1e3);
    return worst;
}

// Candidates in order of cost (V(pre, 0) first, then V(pre, 1)), largest
// damping first within each.  post < 0 or omega <= 0 leave that choice
// free; otherwise only candidates with the given value are considered.
TimeSmoother choose_time_smoother(const std::vector<int>& Nl, double kappa_min, int pre, int post, double omega) {
    static const double omegas[] = {0.95, 0.9, 0.8, 0.7, 0.6, 0.5};
    struct Cand { int post; double omega; };
    std::vector<Cand> cands;
    for (int q = 0; q <= 1; ++q) {
        if (post >= 0 && q != post) continue;
        if (omega > 0) cands.push_back({q, omega});
        else for (double w : omegas) cands.push_back({q, w});
    }
    if (post > 1) {
        if (omega > 0) cands.push_back({post, omega});
        else for (double w : omegas) cands.push_back({post, w});
    }
    for (const Cand& cd : cands) {
        const double rho = worst_rho(Nl, kappa_min, pre, cd.post, cd.omega, kRhoTarget);
        if (rho <= kRhoTarget) return TimeSmoother{cd.post, cd.omega, rho};
    }
    // none reaches the target: the least work per digit, (pre + post + 1) / -log rho
    TimeSmoother best{cands.back().post, cands.back().omega, 1e300};
    double best_cost = 1e300;
    for (const Cand& cd : cands) {
        const double rho = worst_rho(Nl, kappa_min, pre, cd.post, cd.omega, 1e300);
        const double cost = rho < 1.0 ? (double)(pre + cd.post + 1) / -std::log(rho) : 1e300;
        if (cost < best_cost || (best_cost >= 1e300 && rho < best.rho)) {
            best_cost = cost;
            best = TimeSmoother{cd.post, cd.omega, rho};
        }
    }
    return best;
}

}  // namespace ptp

extern "C" {

int ptp_time_cycle_rho(const int* Nl, int levels, double kappa0, int pre, int post, double omega, double* rho) {
    if (!Nl || levels < 1 || !rho || pre < 0 || post < 0 || !(omega > 0) || !(kappa0 >= 0)) return PTP_EINVAL;
    std::vector<int> v(Nl, Nl + levels);
    const double r = ptp::tmg_cycle_rho(v, kappa0, pre, post, omega);
    if (r < 0) return PTP_EINVAL;
    *rho = r;
    return PTP_OK;
}

int ptp_choose_time_smoother(const int* Nl, int levels, double kappa_min, int pre, int post, double omega,
                             int* post_out, double* omega_out, double* rho_out) {
    if (!Nl || levels < 1 || pre < 0 || !(kappa_min >= 0)) return PTP_EINVAL;
    std::vector<int> v(Nl, Nl + levels);
    for (int l = 1; l < levels; ++l)
        if (v[l - 1] != 2 * v[l]) return PTP_EINVAL;
    const ptp::TimeSmoother t = ptp::choose_time_smoother(v, kappa_min, pre, post, omega);
    if (post_out) *post_out = t.post;
    if (omega_out) *omega_out = t.omega;
    if (rho_out) *rho_out = t.rho;
    return PTP_OK;
}

}  // extern "C"
