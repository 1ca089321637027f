/*
 * Seeded Chung-Lu graph generator (input synthesis only; no part of the
 * Kemeny-constant method lives here).
 *
 * Edge (i, j), i < j, is present independently with probability
 *     p_ij = min(1, w_i * w_j / W),   W = sum_k w_k,
 * where the weights w are sorted in non-increasing order.  The generator is
 * the O(n + m) geometric-skip scheme of Miller and Hagberg ("Efficient
 * generation of networks with given expected degrees", WAW 2011): for a fixed
 * row i the probabilities are non-increasing in j, so candidates are skipped
 * geometrically with the current upper bound p and accepted with q / p.
 *
 * Randomness: splitmix64 seeding a xoshiro256** stream (Blackman & Vigna),
 * doubles in [0, 1) from the top 53 bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct { uint64_t s[4]; } xo_t;

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t xo_next(xo_t *g) {
    uint64_t *s = g->s;
    uint64_t result = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
}

static double xo_double(xo_t *g) { return (double)(xo_next(g) >> 11) * 0x1.0p-53; }

/*
 * w: n weights, non-increasing.  Writes at most cap edges into (eu, ev).
 * Returns the number of edges generated, or -1 when cap was too small.
 */
int64_t synth_chung_lu(int64_t n, const double *w, uint64_t seed, int64_t cap,
                       int32_t *eu, int32_t *ev) {
    xo_t g;
    uint64_t sm = seed;
    for (int k = 0; k < 4; ++k) g.s[k] = splitmix64(&sm);
    double W = 0.0;
    for (int64_t i = 0; i < n; ++i) W += w[i];
    int64_t m = 0;
    for (int64_t u = 0; u + 1 < n; ++u) {
        int64_t v = u + 1;
        double p = w[u] * w[v] / W;
        if (p > 1.0) p = 1.0;
        while (v < n && p > 0.0) {
            if (p < 1.0) {
                double r = xo_double(&g);
                /* skip ~ Geometric(p): number of failures before a success */
                double skip = floor(log1p(-r) / log1p(-p));
                if (skip > (double)(n - v)) break;
                v += (int64_t)skip;
            }
            if (v >= n) break;
            double q = w[u] * w[v] / W;
            if (q > 1.0) q = 1.0;
            double r2 = xo_double(&g);
            if (r2 < q / p) {
                if (m >= cap) return -1;
                eu[m] = (int32_t)u;
                ev[m] = (int32_t)v;
                ++m;
            }
            p = q;
            ++v;
        }
    }
    return m;
}
