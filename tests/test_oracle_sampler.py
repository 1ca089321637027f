"""Pins of the oracle's Wilson sampler, random-number contract, root and tau0.

* Chi-square of sampled-tree frequencies over each tiny graph's enumerated
  (Kirchhoff-counted) tree set: uniform spanning trees (Sec. 2.2).
* Mean step count = Tr(I - P_r)^-1 (Sec. 2.2, proof of Theorem 8).
* Edge marginals P(e in tau) = R(e) (Sec. 4.1) and Foster's sum_e R(e) = n - 1.
* Start-order invariance of tree and step count (cycle popping with arrows
  keyed by (vertex, departure index)).
* Philox4x32-10 / bounded draws: exact special cases and uniformity.
* Root = highest degree, smallest id on ties; tau0 is a BFS tree (levels from
  scipy's shortest paths) whose parents are the smallest-id neighbour one level up;
  DFN intervals are a preorder with children in ascending id.
"""
import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import shortest_path
from scipy.stats import chi2

import oracle as O
from paper_2511_16356_gb300 import synth as S


def _tree_key(parent, r):
    return tuple(sorted((min(v, int(parent[v])), max(v, int(parent[v])))
                        for v in range(parent.shape[0]) if v != r))


@pytest.mark.parametrize("name,seed", [("K4", 1), ("grid3x3", 2), ("rc7", 3), ("rc7b", 4)])
def test_wilson_uniform_chi_square(name, seed):
    g = {"K4": S.complete(4), "grid3x3": S.grid(3, 3), "rc7": S.random_connected(7, 0.5, 3),
         "rc7b": S.random_connected(7, 0.45, 9)}[name]
    t0 = O.tau0(g)
    trees = O.spanning_trees(g)
    idx = {tuple(sorted(T)): i for i, T in enumerate(trees)}
    N = 200 * len(trees)
    cnt = np.zeros(len(trees))
    for k in range(N):
        par, _ = O.wilson(g, t0.r, 1000 + seed, k)
        cnt[idx[_tree_key(par, t0.r)]] += 1
    e = N / len(trees)
    stat = ((cnt - e) ** 2 / e).sum()
    assert chi2.sf(stat, len(trees) - 1) > 1e-3


@pytest.mark.parametrize("seed", [5, 6])
def test_mean_steps_is_trace_green(seed):
    g = S.random_connected(12, 0.3, seed)
    t0 = O.tau0(g)
    N = 20000
    st = np.array([O.wilson(g, t0.r, seed, k)[1] for k in range(N)], dtype=np.float64)
    want = O.trace_green(g, t0.r)
    assert abs(st.mean() - want) < 5 * st.std() / np.sqrt(N)


def test_edge_marginals_are_effective_resistance():
    g = S.random_connected(10, 0.4, 7)
    t0 = O.tau0(g)
    R = O.resistance_all_edges(g)
    assert sum(R.values()) == pytest.approx(g.n - 1, rel=1e-10)  # Foster
    N = 20000
    cnt = {e: 0 for e in R}
    for k in range(N):
        par, _ = O.wilson(g, t0.r, 77, k)
        for e in _tree_key(par, t0.r):
            cnt[e] += 1
    for e, r in R.items():
        p = cnt[e] / N
        assert abs(p - r) < 5 * np.sqrt(max(r * (1 - r), 0.0) / N) + 1e-9


def test_triangle_insert_resistance_example():
    """Sec. 4.1 example: closing the path v1-v3-v2 into a triangle, R(v1, v2) = 2/3 in G2,
    i.e. two of its three spanning trees contain (v1, v2)."""
    g = S.complete(3)
    assert O.resistance(g, 0, 1) == pytest.approx(2.0 / 3.0, rel=1e-14)
    trees = O.spanning_trees(g)
    assert sum((0, 1) in T for T in trees) == 2 and len(trees) == 3


@pytest.mark.parametrize("seed", [1, 2])
def test_start_order_invariance(seed):
    g = S.er_lcc(150, 0.04, seed)
    t0 = O.tau0(g)
    rng = np.random.default_rng(seed)
    for k in range(20):
        perm = rng.permutation(g.n).astype(np.int32)
        a, sa = O.wilson(g, t0.r, seed, k)
        b, sb = O.wilson(g, t0.r, seed, k, order=perm)
        c, sc = O.wilson(g, t0.r, seed, k, order=np.arange(g.n)[::-1].astype(np.int32))
        assert np.array_equal(a, b) and np.array_equal(a, c)
        assert sa == sb == sc


def test_step_cap_trips():
    g = S.grid(20, 20)
    t0 = O.tau0(g)
    with pytest.raises(RuntimeError):
        O.wilson(g, t0.r, 1, 0, cap=50)


# ------------------------------------------------------------------ RNG ----

def test_philox_is_a_function_of_counter_and_key():
    a = O.philox4x32_10([1, 2, 3, 4], [5, 6])
    assert np.array_equal(a, O.philox4x32_10([1, 2, 3, 4], [5, 6]))
    assert not np.array_equal(a, O.philox4x32_10([1, 2, 3, 5], [5, 6]))
    assert not np.array_equal(a, O.philox4x32_10([1, 2, 3, 4], [5, 7]))


def test_philox_bits_balanced():
    words = np.concatenate([O.philox4x32_10([i, 0, 0, 0], [123, 456]) for i in range(4000)])
    bits = np.unpackbits(words.view(np.uint8))
    n = bits.shape[0]
    assert abs(bits.mean() - 0.5) < 5 * 0.5 / np.sqrt(n)
    # byte histogram chi-square
    h = np.bincount(words.view(np.uint8), minlength=256)
    e = h.sum() / 256
    assert chi2.sf(((h - e) ** 2 / e).sum(), 255) > 1e-4


def test_bounded_special_cases():
    # s = 1 always 0; s = 2^k takes the top k bits of the first word (no rejection possible)
    for c in range(50):
        assert O.bounded(9, c, 0, 0, 0, 1) == 0
        w = O.philox4x32_10([c, 3, 4, 0], [9, 0])
        for k in [1, 3, 8]:
            assert O.bounded(9, c, 3, 4, 0, 1 << k) == int(w[0]) >> (32 - k)


@pytest.mark.parametrize("s", [3, 5, 6, 7, 1000])
def test_bounded_uniform(s):
    N = 30000
    x = np.array([O.bounded(42, i, 1, 2, 0, s) for i in range(N)])
    assert x.min() >= 0 and x.max() < s
    h = np.bincount(x, minlength=s)
    e = N / s
    assert chi2.sf(((h - e) ** 2 / e).sum(), s - 1) > 1e-4


def test_bounded_rejects_per_lemire():
    # For s = 2^31 + 1 about half of the words are rejected: the returned value must
    # equal the high half of x*s for the first accepted word x, in word order.
    s = (1 << 31) + 1
    thr = ((1 << 32) - s) % s
    for c in range(200):
        w = O.philox4x32_10([c, 0, 0, 0], [1, 0])
        want = None
        for x in w:
            m = int(x) * s
            if (m & 0xFFFFFFFF) >= thr:
                want = m >> 32
                break
        if want is not None:
            assert O.bounded(1, c, 0, 0, 0, s) == want


# ------------------------------------------------------------ root, tau0 ----

def test_root_highest_degree_smallest_id():
    g = S.csr_from_edges(6, [0, 1, 1, 2, 3, 3, 4], [5, 2, 4, 4, 4, 5, 5])
    deg = g.deg
    want = int(np.flatnonzero(deg == deg.max())[0])
    assert O.root_smallest_id(g) == want
    # a unique highest-degree vertex is the root under both tie rules
    st = S.star(7)
    assert O.root(st) == O.root_smallest_id(st) == 0


@pytest.mark.parametrize("n", [9, 10, 31])
def test_central_root_on_paths_is_a_middle_vertex(n):
    """All interior vertices of a path tie on degree; the centre (eccentricity
    minimiser) of a path is its middle vertex (one of the two middles for even n)."""
    g = S.path(n)
    r = O.root(g)
    assert r in ((n - 1) // 2, n // 2)
    assert O.root_smallest_id(g) == 1


def test_central_root_shortens_the_bfs_tree_on_grids():
    g = S.grid_perturbed(41, 41, 0.25, 3)
    near = O.tau0(g)
    far = O.tau0(g, O.root_smallest_id(g))
    assert g.deg[near.r] == g.deg.max()
    assert near.ecc < 0.7 * far.ecc


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tau0_is_min_id_bfs_tree(seed):
    g = S.er_lcc(400, 0.012, seed)
    t0 = O.tau0(g)
    A = csr_matrix((np.ones(g.col.shape[0]), g.col, g.row_off), shape=(g.n, g.n))
    dist = shortest_path(A, unweighted=True, indices=[t0.r])[0].astype(int)
    assert np.array_equal(dist, t0.level)
    assert t0.ecc == dist.max()
    for v in range(g.n):
        if v == t0.r:
            assert t0.p0[v] == -1
            continue
        cand = [w for w in g.neighbors(v) if dist[w] == dist[v] - 1]
        assert t0.p0[v] == min(cand)


def test_dfn_is_preorder_children_ascending():
    g = S.er_lcc(120, 0.05, 3)
    t0 = O.tau0(g)
    t = O.tree(g, t0, 5, 0)
    n, r = g.n, t0.r
    # brute force: ancestors by walking parents
    anc = [set() for _ in range(n)]
    for v in range(n):
        x = v
        while x != -1:
            anc[v].add(x)
            x = t.parent[x] if x != r else -1
    for v in range(n):
        sub = [u for u in range(n) if v in anc[u]]
        assert t.size[v] == len(sub)
        assert t.vol[v] == int(g.deg[sub].sum())
        assert t.depth[v] == len(anc[v]) - 1
        assert sorted(t.din[sub]) == list(range(t.din[v], t.dout[v] + 1))
    # children ascending: siblings ordered by id get increasing DFN
    for p in range(n):
        ch = sorted(v for v in range(n) if v != r and t.parent[v] == p)
        assert list(t.din[ch]) == sorted(t.din[ch])
    assert t.din[r] == 0 and t.dout[r] == n - 1


def _curand_host_philox(seed, words):
    """cuRAND's host-side Philox4_32_10 generator (no GPU needed).  Its i-th
    block of four 32-bit outputs is Philox4x32-10 with key (seed low 32, seed
    high 32) at counter (i // 65536, 0, i mod 65536, 0): 65536 subsequences in
    counter word 2, each advanced in word 0 once per sweep."""
    import ctypes
    import ctypes.util

    path = None
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if cand:
            try:
                lib = ctypes.CDLL(cand)
                path = cand
                break
            except OSError:
                continue
    if path is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:  # PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(words, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(words)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out.reshape(-1, 4)


@pytest.mark.parametrize("ctr,key,want", [
    ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
    ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
    ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
     [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
])
def test_philox_known_answer_vectors(ctr, key, want):
    """Philox4x32-10 known-answer vectors published with the generator's
    reference implementation (Salmon et al., SC'11): zero input, all-ones input,
    and the digits of pi as counter and key."""
    assert O.philox4x32_10(ctr, key).tolist() == want


@pytest.mark.parametrize("seed,blocks", [(0x123456789ABCDEF0, 250_000), (7, 4096),
                                         (2 ** 63 + 12345, 4096)])
def test_philox_matches_an_independent_implementation(seed, blocks):
    """The oracle's Philox4x32-10 (rounds, multipliers, key schedule, word
    order, key = seed split in two) equals NVIDIA's cuRAND generator block for
    block: one million 32-bit words for the first seed."""
    ref = _curand_host_philox(seed, 4 * blocks)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(blocks):
        ctr = [i // 65536, 0, i % 65536, 0]
        assert np.array_equal(O.philox4x32_10(ctr, key), ref[i]), i
