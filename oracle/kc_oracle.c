/*
 * CPU ORACLE for the 2-forest / tree-to-forest (TTF) Kemeny-constant method
 * (Li, Liao, Li, Wang, "Scalable and Provable Kemeny Constant Computation on
 * Static and Dynamic Graphs: A 2-Forest Sampling Approach").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code with the CUDA path and is deliberately plain, sequential and slow.
 *
 * Contents, each following the cited passage:
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Lemire's exact
 *     bounded integers: the random-number contract (the paper only asks for a
 *     uniformly random neighbour, Sec. 2.1 and the Wilson description, Sec. 2.2).
 *   - Root choice (highest degree, Exp-III of Sec. 5) and the BFS tree tau0
 *     (Algorithm 1, step "Generate tau0 using BFS").
 *   - Wilson's algorithm (Sec. 2.2; Algorithm 1 "wilson(G, r)") with the
 *     arrow of vertex u on its k-th departure keyed by (u, k), and the
 *     conditioned variant rooted at an edge (Algorithm 2, "Wilson(G', (u,v))").
 *   - Per-tree depth, subtree size, subtree volume and DFN (Algorithm 1 and
 *     Sec. 3.2 "Implementation Details").
 *   - f(tau) by the naive path comparison of Theorem 3 and by the DFS + BIT
 *     procedure of Algorithm 1 with the reverse-case undo written as the exact
 *     negation of the reverse-case add.
 *
 * Readings of the paper taken here (all listed with reasons in the design
 * notes): neighbours are indexed in ascending id order; ties in the root choice
 * go to the most central candidate (see orc_root_central), ties in the
 * BFS-parent choice to the smallest id; DFN visits children in ascending id;
 * the undo in the reverse case of Algorithm 1 negates its add.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: counter-based generator of Salmon et al. (SC'11).          */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/*
 * Uniform integer in [0, s) from the Philox block with counter
 * (c0, c1, c2, tag << 24 | retry) under key (seed low, seed high).
 * The four output words are tried in order with Lemire's multiply-and-reject
 * test (reject when the low half of x*s is below (2^32 - s) mod s); if all
 * four are rejected the retry field is incremented.
 */
uint32_t orc_bounded(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t tag,
                     uint32_t s) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t threshold = (uint32_t)(0u - s) % s;
    for (uint32_t retry = 0; retry < (1u << 24); ++retry) {
        uint32_t ctr[4] = {c0, c1, c2, (tag << 24) | retry};
        uint32_t out[4];
        orc_philox4x32_10(ctr, key, out);
        for (int j = 0; j < 4; ++j) {
            uint64_t m = (uint64_t)out[j] * (uint64_t)s;
            uint32_t low = (uint32_t)m;
            if (low < threshold) continue;
            return (uint32_t)(m >> 32);
        }
    }
    return 0; /* unreachable for any s < 2^32 in practice */
}

#define TAG_WALK 0u

/* ------------------------------------------------------------------------ */
/* Root and tau0                                                             */
/* ------------------------------------------------------------------------ */

/* Highest-degree vertex, smallest id among ties (Exp-III, Sec. 5). */
int32_t orc_root(int64_t n, const int64_t *row_off) {
    int32_t best = 0;
    int64_t bd = -1;
    for (int64_t v = 0; v < n; ++v) {
        int64_t d = row_off[v + 1] - row_off[v];
        if (d > bd) { bd = d; best = (int32_t)v; }
    }
    return best;
}

/* BFS levels from s (-1 when unreachable); returns the number of reached vertices */
static int64_t bfs_levels(int64_t n, const int64_t *row_off, const int32_t *col, int32_t s,
                          int32_t *level, int32_t *queue) {
    for (int64_t v = 0; v < n; ++v) level[v] = -1;
    int64_t head = 0, tail = 0;
    level[s] = 0;
    queue[tail++] = s;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = row_off[u]; e < row_off[u + 1]; ++e) {
            int32_t w = col[e];
            if (level[w] < 0) { level[w] = level[u] + 1; queue[tail++] = w; }
        }
    }
    return tail;
}

/* the smallest-id vertex of largest level */
static int32_t farthest(int64_t n, const int32_t *level) {
    int32_t best = 0;
    for (int64_t v = 0; v < n; ++v)
        if (level[v] > level[best]) best = (int32_t)v;
    return best;
}

/*
 * Highest-degree vertex, ties broken towards the centre of the graph (Exp-III
 * picks the highest degree because it shortens the walks; the paper gives no
 * tie-break).  With r0 the smallest-id highest-degree vertex: a = the vertex
 * farthest from r0, b = the vertex farthest from a, c = the vertex maximising
 * min(dist(a, .), dist(b, .)) (smallest id on ties); the root is the
 * highest-degree vertex minimising max(dist(a, .), dist(b, .), dist(c, .)),
 * smallest id among equals -- a three-source lower bound on the eccentricity.
 * A unique highest-degree vertex is returned directly.  Returns -1 for a
 * disconnected graph.
 */
int32_t orc_root_central(int64_t n, const int64_t *row_off, const int32_t *col) {
    int32_t r0 = orc_root(n, row_off);
    int64_t dmax = row_off[r0 + 1] - row_off[r0];
    int64_t ties = 0;
    for (int64_t v = 0; v < n; ++v) ties += (row_off[v + 1] - row_off[v]) == dmax;
    int32_t *la = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *lb = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *lc = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t r = -1;
    if (bfs_levels(n, row_off, col, r0, la, q) == n) {
        if (ties == 1) {
            r = r0;
        } else {
            int32_t a = farthest(n, la);
            bfs_levels(n, row_off, col, a, la, q);
            int32_t b = farthest(n, la);
            bfs_levels(n, row_off, col, b, lb, q);
            int32_t c = 0;
            for (int64_t v = 0; v < n; ++v) {
                int32_t mv = la[v] < lb[v] ? la[v] : lb[v];
                int32_t mc = la[c] < lb[c] ? la[c] : lb[c];
                if (mv > mc) c = (int32_t)v;
            }
            bfs_levels(n, row_off, col, c, lc, q);
            int32_t best = -1;
            for (int64_t v = 0; v < n; ++v) {
                if (row_off[v + 1] - row_off[v] != dmax) continue;
                int32_t e = la[v];
                if (lb[v] > e) e = lb[v];
                if (lc[v] > e) e = lc[v];
                if (r < 0 || e < best) { r = (int32_t)v; best = e; }
            }
        }
    }
    free(la); free(lb); free(lc); free(q);
    return r;
}

/*
 * BFS levels from r, and tau0 parent p0[v] = the smallest-id neighbour of v
 * one level closer to r.  p0[r] = -1.  Returns ecc(r) = max level, or -1 if
 * some vertex is unreachable.
 */
int32_t orc_bfs_tree(int64_t n, const int64_t *row_off, const int32_t *col, int32_t r,
                     int32_t *p0, int32_t *level) {
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t v = 0; v < n; ++v) level[v] = -1;
    int64_t head = 0, tail = 0;
    level[r] = 0;
    queue[tail++] = r;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = row_off[u]; e < row_off[u + 1]; ++e) {
            int32_t w = col[e];
            if (level[w] < 0) { level[w] = level[u] + 1; queue[tail++] = w; }
        }
    }
    free(queue);
    if (tail != n) return -1;
    int32_t ecc = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (level[v] > ecc) ecc = level[v];
        p0[v] = -1;
        if (v == r) continue;
        for (int64_t e = row_off[v]; e < row_off[v + 1]; ++e) {
            int32_t w = col[e];
            if (level[w] == level[v] - 1) { p0[v] = w; break; } /* rows ascend */
        }
    }
    return ecc;
}

/*
 * Depth-first spanning tree from r (the DFS path selection of Exp-II): the
 * recursive DFS that scans each adjacency row in ascending id and descends
 * into the first unvisited neighbour, run with an explicit stack of (vertex,
 * next row position).  p0 = DFS parent (-1 at r), level = depth in the DFS
 * tree.  Returns the largest depth, or -1 if some vertex is unreachable.
 */
int32_t orc_dfs_tree(int64_t n, const int64_t *row_off, const int32_t *col, int32_t r,
                     int32_t *p0, int32_t *level) {
    int32_t *sv = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *se = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t v = 0; v < n; ++v) { level[v] = -1; p0[v] = -1; }
    int64_t sp = 0, seen = 1;
    int32_t deepest = 0;
    level[r] = 0;
    sv[0] = r;
    se[0] = row_off[r];
    while (sp >= 0) {
        const int32_t u = sv[sp];
        if (se[sp] < row_off[u + 1]) {
            const int32_t w = col[se[sp]++];
            if (level[w] < 0) {
                p0[w] = u;
                level[w] = level[u] + 1;
                if (level[w] > deepest) deepest = level[w];
                ++seen;
                ++sp;
                sv[sp] = w;
                se[sp] = row_off[w];
            }
        } else {
            --sp;
        }
    }
    free(sv);
    free(se);
    return seen == n ? deepest : -1;
}

/* ------------------------------------------------------------------------ */
/* Wilson's algorithm                                                        */
/* ------------------------------------------------------------------------ */

/*
 * Uniform spanning tree rooted at r (Sec. 2.2).  Walks start from the
 * vertices in `order` (NULL: ascending id); the walk leaves u along the
 * neighbour with index bounded(seed, u, visits(u), sample, WALK, deg(u)),
 * overwriting next[u] (loop erasure by overwriting); on hitting the tree the
 * path from the start is retraced and added.  parent[r] = -1.
 * `pre_in_tree` (optional, n bytes) marks vertices already in the tree at the
 * start, with `pre_next` giving their fixed successors (used by the
 * conditioned sampler).  Returns 0, or 1 when the walk count exceeds cap.
 */
int orc_wilson_ex(int64_t n, const int64_t *row_off, const int32_t *col, int32_t r,
                  uint64_t seed, uint32_t sample, const int32_t *order,
                  const uint8_t *pre_in_tree, const int32_t *pre_next,
                  int32_t *parent, int64_t *steps, int64_t cap) {
    uint8_t *in_tree = (uint8_t *)calloc((size_t)n, 1);
    uint32_t *visits = (uint32_t *)calloc((size_t)n, sizeof(uint32_t));
    int32_t *next = parent;
    int64_t s_count = 0;
    int rc = 0;
    for (int64_t v = 0; v < n; ++v) next[v] = -1;
    in_tree[r] = 1;
    if (pre_in_tree) {
        for (int64_t v = 0; v < n; ++v)
            if (pre_in_tree[v]) { in_tree[v] = 1; next[v] = pre_next[v]; }
    }
    for (int64_t idx = 0; idx < n && !rc; ++idx) {
        int32_t s = order ? order[idx] : (int32_t)idx;
        int32_t u = s;
        while (!in_tree[u]) {
            uint32_t d = (uint32_t)(row_off[u + 1] - row_off[u]);
            uint32_t k = orc_bounded(seed, (uint32_t)u, visits[u], sample, TAG_WALK, d);
            visits[u] += 1;
            next[u] = col[row_off[u] + k];
            u = next[u];
            if (++s_count > cap) { rc = 1; break; }
        }
        if (rc) break;
        u = s;
        while (!in_tree[u]) { in_tree[u] = 1; u = next[u]; }
    }
    if (!pre_in_tree) next[r] = -1;
    *steps = s_count;
    free(in_tree);
    free(visits);
    return rc;
}

int orc_wilson(int64_t n, const int64_t *row_off, const int32_t *col, int32_t r, uint64_t seed,
               uint32_t sample, const int32_t *order, int32_t *parent, int64_t *steps,
               int64_t cap) {
    return orc_wilson_ex(n, row_off, col, r, seed, sample, order, NULL, NULL, parent, steps, cap);
}

/* ------------------------------------------------------------------------ */
/* Traversal: depth, size, volume, DFN (children in ascending id)            */
/* ------------------------------------------------------------------------ */
int orc_traverse(int64_t n, const int64_t *row_off, const int32_t *parent, int32_t r,
                 int32_t *depth, int32_t *size, int64_t *vol, int32_t *din, int32_t *dout) {
    /* children lists in ascending id: bucket v = 0..n-1 in order */
    int64_t *cstart = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *clist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 1 ? n : 1));
    int64_t *cfill = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int32_t *pre = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t v = 0; v < n; ++v)
        if (v != r) cstart[parent[v] + 1] += 1;
    for (int64_t v = 0; v < n; ++v) cstart[v + 1] += cstart[v];
    for (int64_t v = 0; v < n; ++v)
        if (v != r) { int32_t p = parent[v]; clist[cstart[p] + cfill[p]++] = (int32_t)v; }
    /* preorder by explicit stack; push children in reverse so the smallest id is visited first */
    int64_t sp = 0, cnt = 0;
    stack[sp++] = r;
    depth[r] = 0;
    while (sp > 0) {
        int32_t v = stack[--sp];
        din[v] = (int32_t)cnt;
        pre[cnt++] = v;
        for (int64_t k = cstart[v + 1] - 1; k >= cstart[v]; --k) {
            int32_t c = clist[k];
            depth[c] = depth[v] + 1;
            stack[sp++] = c;
        }
    }
    int rc = (cnt == n) ? 0 : 1;
    for (int64_t v = 0; v < n; ++v) { size[v] = 0; vol[v] = 0; }
    for (int64_t i = cnt - 1; i >= 0; --i) {
        int32_t v = pre[i];
        size[v] += 1;
        vol[v] += row_off[v + 1] - row_off[v];
        if (v != r) { size[parent[v]] += size[v]; vol[parent[v]] += vol[v]; }
    }
    for (int64_t v = 0; v < n; ++v) dout[v] = din[v] + size[v] - 1;
    free(cstart); free(clist); free(cfill); free(pre); free(stack);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* f(tau): naive path comparison (Theorem 3)                                 */
/* ------------------------------------------------------------------------ */
/*
 * For each u != r: mark the tau0 path P_u; walk the tau path from u to r; an
 * edge (y -> p(y)) of the tau path equal to the P_u edge (y -> p0(y))
 * contributes +vol(T1) (forward mapping), one equal to the reversed P_u edge
 * (p(y) -> y) contributes -vol(T1) (reverse mapping), where T1 is the part of
 * tau minus that edge containing r, vol(T1) = 2m - vol(Sub(tau, y)).
 * f = sum_u d(u) * (forward - reverse).
 */
int64_t orc_f_naive(int64_t n, const int64_t *row_off, int32_t r, const int32_t *parent,
                    const int64_t *vol, const int32_t *p0) {
    int64_t twom = row_off[n];
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t v = 0; v < n; ++v) mark[v] = -1;
    int64_t f = 0;
    for (int64_t u = 0; u < n; ++u) {
        if (u == r) continue;
        for (int32_t x = (int32_t)u; x != r; x = p0[x]) mark[x] = (int32_t)u;
        int64_t q = 0;
        for (int32_t y = (int32_t)u; y != r;) {
            int32_t py = parent[y];
            if (mark[y] == u && p0[y] == py) q += twom - vol[y];
            else if (py != r && mark[py] == u && p0[py] == y) q -= twom - vol[y];
            y = py;
        }
        f += (row_off[u + 1] - row_off[u]) * q;
    }
    free(mark);
    return f;
}

/* ------------------------------------------------------------------------ */
/* f(tau): Algorithm 1 (DFS over tau, BIT over the DFN of tau0)              */
/* ------------------------------------------------------------------------ */
static void bit_add(int64_t *bit, int64_t n, int64_t i1, int64_t val) {
    for (int64_t i = i1; i <= n; i += i & (-i)) bit[i] += val;
}
static void bit_range_add(int64_t *bit, int64_t n, int64_t l, int64_t r, int64_t val) {
    bit_add(bit, n, l + 1, val);
    if (r + 2 <= n) bit_add(bit, n, r + 2, -val);
}
static int64_t bit_point(const int64_t *bit, int64_t i0) {
    int64_t s = 0;
    for (int64_t i = i0 + 1; i > 0; i -= i & (-i)) s += bit[i];
    return s;
}

/*
 * Visiting v != r with tau parent p = p(v):
 *   (v, p) in tau0 with the same direction (p0(v) = p): add 2m - vol(v) on the
 *     tau0 DFN interval of v;
 *   (p, v) in tau0 (p0(p) = v): add vol(v) - 2m on the tau0 interval of p;
 * then f += d(v) * Query(in0(v)); recurse into the children; finally undo the
 * add by adding its negation.
 */
int64_t orc_f_alg1(int64_t n, const int64_t *row_off, int32_t r, const int32_t *parent,
                   const int64_t *vol, const int32_t *p0, const int32_t *in0,
                   const int32_t *out0) {
    int64_t twom = row_off[n];
    int64_t *bit = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *cstart = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *clist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 1 ? n : 1));
    int64_t *cfill = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int32_t *st_v = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *st_k = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t v = 0; v < n; ++v)
        if (v != r) cstart[parent[v] + 1] += 1;
    for (int64_t v = 0; v < n; ++v) cstart[v + 1] += cstart[v];
    for (int64_t v = 0; v < n; ++v)
        if (v != r) { int32_t p = parent[v]; clist[cstart[p] + cfill[p]++] = (int32_t)v; }

    int64_t f = 0;
    int64_t sp = 0;
    /* enter r: no add; its query is over an all-zero BIT */
    f += (row_off[r + 1] - row_off[r]) * bit_point(bit, in0[r]);
    st_v[sp] = r; st_k[sp] = cstart[r]; ++sp;
    while (sp > 0) {
        int32_t v = st_v[sp - 1];
        if (st_k[sp - 1] < cstart[v + 1]) {
            int32_t c = clist[st_k[sp - 1]++];
            /* enter c */
            int32_t p = v;
            if (p0[c] == p)
                bit_range_add(bit, n, in0[c], out0[c], twom - vol[c]);
            else if (p != r && p0[p] == c)
                bit_range_add(bit, n, in0[p], out0[p], vol[c] - twom);
            f += (row_off[c + 1] - row_off[c]) * bit_point(bit, in0[c]);
            st_v[sp] = c; st_k[sp] = cstart[c]; ++sp;
        } else {
            /* leave v: undo its add */
            --sp;
            if (v != r) {
                int32_t p = parent[v];
                if (p0[v] == p)
                    bit_range_add(bit, n, in0[v], out0[v], vol[v] - twom);
                else if (p != r && p0[p] == v)
                    bit_range_add(bit, n, in0[p], out0[p], twom - vol[v]);
            }
        }
    }
    free(bit); free(cstart); free(clist); free(cfill); free(st_v); free(st_k);
    return f;
}

/* ------------------------------------------------------------------------ */
/* Batch: trees with sample ids [id0, id0 + count), OpenMP across trees      */
/* ------------------------------------------------------------------------ */
/*
 * method 0: f by Algorithm 1; method 1: f by Theorem 3's naive comparison.
 * Returns 0, or 1 if any tree hit the step cap.
 */
int orc_sample_batch(int64_t n, const int64_t *row_off, const int32_t *col, int32_t r,
                     const int32_t *p0, const int32_t *in0, const int32_t *out0, uint64_t seed,
                     uint32_t id0, int64_t count, int method, int nthreads, int64_t cap,
                     int64_t *f_out, int64_t *steps_out) {
    int bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel reduction(| : bad)
#endif
    {
        int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        int32_t *depth = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        int32_t *size = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        int64_t *vol = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        int32_t *din = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        int32_t *dout = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t t = 0; t < count; ++t) {
            int64_t st = 0;
            int rc = orc_wilson(n, row_off, col, r, seed, id0 + (uint32_t)t, NULL, parent, &st,
                                cap);
            if (rc) { bad |= 1; f_out[t] = 0; steps_out[t] = st; continue; }
            orc_traverse(n, row_off, parent, r, depth, size, vol, din, dout);
            f_out[t] = method == 1 ? orc_f_naive(n, row_off, r, parent, vol, p0)
                                   : orc_f_alg1(n, row_off, r, parent, vol, p0, in0, out0);
            steps_out[t] = st;
        }
        free(parent); free(depth); free(size); free(vol); free(din); free(dout);
    }
    return bad;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
