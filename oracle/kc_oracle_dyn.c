/*
 * CPU ORACLE, dynamic part: the per-tree operations of the sample-maintenance
 * algorithms of Sec. 4 (BSM, Algorithm 2; ISM, Algorithm 3).
 *
 * TEST INFRASTRUCTURE ONLY (see kc_oracle.c).  Plain sequential code.
 *
 * Random choices use the same Philox4x32-10 / bounded-integer contract as the
 * walk (orc_bounded in kc_oracle.c) with their own tags:
 *   tag 1 (select):   counter (update seq, draw index, 0)          -- Floyd's sampling
 *   tag 2 (link-cut): counter (update seq, pool index, 0)          -- edge of the cycle to cut
 *   tag 3 (cut-link): counter (update seq, pool index, 0)          -- crossing edge to link
 * Conventions fixed here (the paper does not fix them):
 *   - the cycle edges of link-cut are numbered from u upwards to the lowest
 *     common ancestor, then from v upwards to it;
 *   - the crossing edges of cut-link are numbered by (preorder position of the
 *     inside endpoint in tau, then the outside endpoint ascending);
 *   - the replaced or transformed part is re-rooted so that every tree stays
 *     rooted at r (Algorithm 2 "Redirect edges in tau' to point towards r").
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

uint32_t orc_bounded(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t tag,
                     uint32_t s);
int orc_wilson_ex(int64_t n, const int64_t *row_off, const int32_t *col, int32_t r,
                  uint64_t seed, uint32_t sample, const int32_t *order,
                  const uint8_t *pre_in_tree, const int32_t *pre_next, int32_t *parent,
                  int64_t *steps, int64_t cap);
int orc_traverse(int64_t n, const int64_t *row_off, const int32_t *parent, int32_t r,
                 int32_t *depth, int32_t *size, int64_t *vol, int32_t *din, int32_t *dout);

#define TAG_SELECT 1u
#define TAG_LINKCUT 2u
#define TAG_CUTLINK 3u

/* Reverse the parent chain from x up to (and including) the old root y of its
 * tree part, then hang x below `attach` (attach = -1 makes x the new root). */
static void reroot_path(int32_t *parent, int32_t x, int32_t y, int32_t attach) {
    int32_t prev = attach, cur = x;
    while (1) {
        int32_t nxt = parent[cur];
        parent[cur] = prev;
        if (cur == y) break;
        prev = cur;
        cur = nxt;
    }
}

/*
 * Uniform spanning tree of G' conditioned on containing e = (u, v) (Algorithm
 * 2, "Wilson(G', (u,v))"): u and v start in the tree with the arrow u -> v and
 * Wilson's walks are absorbed there; the result is then re-rooted at r.
 */
int orc_cond_wilson(int64_t n, const int64_t *row_off, const int32_t *col, int32_t u, int32_t v,
                    int32_t r, uint64_t seed, uint32_t sample, int32_t *parent, int64_t *steps,
                    int64_t cap) {
    uint8_t *pre = (uint8_t *)calloc((size_t)n, 1);
    int32_t *pnext = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t x = 0; x < n; ++x) pnext[x] = -1;
    pre[u] = 1; pre[v] = 1;
    pnext[u] = v; pnext[v] = -1;
    int rc = orc_wilson_ex(n, row_off, col, v, seed, sample, NULL, pre, pnext, parent, steps, cap);
    free(pre);
    free(pnext);
    if (rc) return rc;
    parent[v] = -1;
    if (r != v) reroot_path(parent, r, v, -1);
    return 0;
}

/* Floyd's sampling of k distinct indices of [0, N), as the j-th selected set
 * member order of insertion.  out must hold k entries. */
void orc_select(uint64_t seed, uint32_t seq, int64_t N, int64_t k, int64_t *out) {
    uint8_t *taken = (uint8_t *)calloc((size_t)(N > 0 ? N : 1), 1);
    int64_t cnt = 0;
    for (int64_t j = N - k; j < N; ++j) {
        int64_t t = (int64_t)orc_bounded(seed, seq, (uint32_t)cnt, 0, TAG_SELECT, (uint32_t)(j + 1));
        if (taken[t]) t = j;
        taken[t] = 1;
        out[cnt++] = t;
    }
    free(taken);
}

/* tau-path length between a and b using depths */
static int64_t tree_dist(const int32_t *parent, const int32_t *depth, int32_t a, int32_t b) {
    int64_t d = 0;
    while (depth[a] > depth[b]) { a = parent[a]; ++d; }
    while (depth[b] > depth[a]) { b = parent[b]; ++d; }
    while (a != b) { a = parent[a]; b = parent[b]; d += 2; }
    return d;
}

/*
 * link-cut(tau, e) for e = (u, v) not in tau (Sec. 4.2): add e, cut the
 * k-th edge of the tau-path u..v (k uniform over its d(tau) edges, or k_force
 * when k_force >= 0, used to enumerate all neighbours), re-root the
 * detached part at the endpoint of e inside it.  Writes the new parent array,
 * d(tau) = path length and d(tau') = number of edges of G' other than e that
 * cross the two parts of tau' \ e (the link-cut bipartite degrees, Theorem 6).
 * row_off/col describe G' (which contains e).
 */
int orc_link_cut(int64_t n, const int64_t *row_off, const int32_t *col, const int32_t *parent,
                 int32_t r, int32_t u, int32_t v, uint64_t seed, uint32_t seq, uint32_t pool_idx,
                 int64_t k_force, int32_t *out, int64_t *d_old, int64_t *d_new) {
    int32_t *depth = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *size = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *vol = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *din = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *dout = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    orc_traverse(n, row_off, parent, r, depth, size, vol, din, dout);
    /* the cycle edges: (x, parent(x)) for x from u up to the LCA, then from v up */
    int32_t a = u, b = v;
    while (depth[a] > depth[b]) a = parent[a];
    while (depth[b] > depth[a]) b = parent[b];
    while (a != b) { a = parent[a]; b = parent[b]; }
    int32_t lca = a;
    int64_t du = depth[u] - depth[lca], dv = depth[v] - depth[lca];
    int64_t d = du + dv;
    *d_old = d;
    int64_t k = k_force >= 0 ? k_force
                             : (int64_t)orc_bounded(seed, seq, pool_idx, 0, TAG_LINKCUT, (uint32_t)d);
    int32_t x, side;  /* cut edge (x, parent(x)); side = endpoint of e below x */
    if (k < du) {
        x = u;
        for (int64_t i = 0; i < k; ++i) x = parent[x];
        side = u;
    } else {
        x = v;
        for (int64_t i = 0; i < k - du; ++i) x = parent[x];
        side = v;
    }
    memcpy(out, parent, sizeof(int32_t) * (size_t)n);
    reroot_path(out, side, x, side == u ? v : u);
    /* crossing edges of (Sub(tau, x), rest) in G' minus e */
    int64_t cross = 0;
    for (int64_t y = 0; y < n; ++y) {
        if (!(din[x] <= din[y] && din[y] <= dout[x])) continue;
        for (int64_t e = row_off[y]; e < row_off[y + 1]; ++e) {
            int32_t z = col[e];
            if (din[x] <= din[z] && din[z] <= dout[x]) continue;
            if ((y == u && z == v) || (y == v && z == u)) continue;
            ++cross;
        }
    }
    *d_new = cross;
    free(depth); free(size); free(vol); free(din); free(dout);
    return 0;
}

/*
 * cut-link(tau, e) for e = (u, v) in tau (Sec. 4.2): cut e, enumerate the
 * edges of G' (e already removed) crossing Sub(tau, c) (c the child endpoint
 * of e) and the rest in (preorder position of the inside endpoint, outside
 * endpoint ascending) order, link the k-th one (k uniform over all d(tau_e) of
 * them, or k_force when >= 0) and re-root the cut part at its inside endpoint.  d_old = number of
 * crossing edges (d(tau_e) in Theorem 7), d_new = tau'-path length u..v.
 * row_off/col describe G'.
 */
int orc_cut_link(int64_t n, const int64_t *row_off, const int32_t *col, const int32_t *parent,
                 int32_t r, int32_t u, int32_t v, uint64_t seed, uint32_t seq, uint32_t pool_idx,
                 int64_t k_force, int32_t *out, int64_t *d_old, int64_t *d_new) {
    int32_t c = (parent[u] == v) ? u : v;
    int32_t q = (c == u) ? v : u;  /* parent of c */
    int32_t *depth = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *size = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *vol = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *din = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *dout = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *pre = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    /* traverse tau on G' (degrees are irrelevant here; only DFN and depth are used) */
    orc_traverse(n, row_off, parent, r, depth, size, vol, din, dout);
    for (int64_t y = 0; y < n; ++y) pre[din[y]] = (int32_t)y;
    int64_t cross = 0;
    for (int32_t p = din[c]; p <= dout[c]; ++p) {
        int32_t y = pre[p];
        for (int64_t e = row_off[y]; e < row_off[y + 1]; ++e) {
            int32_t z = col[e];
            if (!(din[c] <= din[z] && din[z] <= dout[c])) ++cross;
        }
    }
    *d_old = cross;
    int64_t k = k_force >= 0 ? k_force
              : (cross > 0 ? (int64_t)orc_bounded(seed, seq, pool_idx, 0, TAG_CUTLINK, (uint32_t)cross)
                           : 0);
    int32_t ia = -1, ob = -1;
    int64_t idx = 0;
    for (int32_t p = din[c]; p <= dout[c] && ia < 0; ++p) {
        int32_t y = pre[p];
        for (int64_t e = row_off[y]; e < row_off[y + 1]; ++e) {
            int32_t z = col[e];
            if (din[c] <= din[z] && din[z] <= dout[c]) continue;
            if (idx == k) { ia = y; ob = z; break; }
            ++idx;
        }
    }
    memcpy(out, parent, sizeof(int32_t) * (size_t)n);
    reroot_path(out, ia, c, ob);
    /* new u..v distance: c..ia inside (depth difference in tau), the link, ob..q outside */
    *d_new = (int64_t)(depth[ia] - depth[c]) + 1 + tree_dist(parent, depth, ob, q);
    free(depth); free(size); free(vol); free(din); free(dout); free(pre);
    return 0;
}
