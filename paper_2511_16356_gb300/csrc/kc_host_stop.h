// How many trees kc_estimate draws: the two stopping rules, host side.
//
// The paper fixes the number of trees through Hoeffding's inequality only
// (Theorem 5).  The default rule reads the same (eps, delta) guarantee through
// the normal approximation of the mean of f/2m: a pilot of max(64, batch)
// trees, then stop once w >= 64 and z_{1-delta/2} s / sqrt(w) <= eps K (1 - eps),
// else draw max(batch, ceil((z s / tol)^2) - w) more, never past the cap, for
// at most 64 rounds.  The Hoeffding rule draws Theorem 5's sample size once,
// with Delta read as ecc(r) (the proof bounds the tau0 path length) and
// kappa >= (n-1)^2/n.
//
// Plain C++ (no CUDA): the same header is compiled by the host tests.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>

namespace kc_host {

// z with P(Z > z) = p_upper for a standard normal Z, by bisection on erfc
// (monotone); 200 halvings of [-40, 40] reach the double's resolution.
inline double inv_normal_upper(double p_upper) {
    double lo = -40.0, hi = 40.0;
    for (int i = 0; i < 200; ++i) {
        const double mid = 0.5 * (lo + hi);
        const double tail = 0.5 * std::erfc(mid / std::sqrt(2.0));
        if (tail > p_upper) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// Pool moments: count trees, wf = sum w f/2m, w = sum w, x2 = sum (f/2m)^2.
struct Moments {
    int64_t count;
    double wf, w, x2;
};

// More trees the normal-approximation rule asks for after a pool of `pool`
// trees with moments s (0: stop).
inline int64_t clt_more(const Moments &s, double z, double eps, int64_t batch, int64_t cap,
                        int64_t pool) {
    const double w = (double)s.count;
    const double mean = s.wf / s.w;
    const double var = std::max(0.0, (s.x2 - w * mean * mean) / std::max(1.0, w - 1.0));
    const double sd = std::sqrt(var);
    const double tol = eps * mean * (1.0 - eps);
    if (w >= 64 && z * sd / std::sqrt(w) <= tol) return 0;
    if (pool >= cap) return 0;
    const double need = tol > 0 ? std::ceil((z * sd / tol) * (z * sd / tol)) : (double)cap;
    const int64_t more = (int64_t)std::min<double>(std::max<double>(need - w, (double)batch),
                                                   (double)(cap - pool));
    return more > 0 ? more : 0;
}

// The normal-approximation rule from a pool of pool0 trees: draw(k) appends k
// trees to the pool, moments() reads the pool's moments.
template <class Draw, class Read>
void run_clt(double delta, double eps, int64_t batch, int64_t cap, int64_t pool0, Draw draw,
             Read moments) {
    const double z = inv_normal_upper(delta / 2.0);
    int64_t pool = pool0;
    if (pool < 64) {
        const int64_t k = std::max<int64_t>(64, std::min(batch, cap)) - pool;
        draw(k);
        pool += k;
    }
    for (int round = 0; round < 64; ++round) {
        const int64_t more = clt_more(moments(), z, eps, batch, cap, pool);
        if (more <= 0) break;
        draw(more);
        pool += more;
    }
}

// Theorem 5's sample size, capped.
inline int64_t hoeffding_trees(int64_t n, int64_t m, int64_t ecc, double eps, double delta,
                               int64_t cap) {
    const double nn = (double)n, mm = (double)m, e = (double)ecc;
    const double kmin = (nn - 1) * (nn - 1) / nn;
    const double need = std::ceil(8.0 * mm * mm * e * e * std::log(2.0 / delta) /
                                  (kmin * kmin * eps * eps));
    return (int64_t)std::min<double>(need, (double)cap);
}

}  // namespace kc_host
