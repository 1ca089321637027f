"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs and the same Philox streams.

Integer outputs (tau0, parent, depth, DFN, subtree volume, Wilson step count and
f(tau)) must match bit for bit; K_hat is compared with 1e-12 relative
tolerance (it is a division of the same exact integer sum) and, against the
exact Kemeny constant, within the requested relative error.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2511_16356_gb300 import synth as S

pytestmark = pytest.mark.gpu

kc = pytest.importorskip("paper_2511_16356_gb300.kc")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2511_16356_gb300 import build as kbuild

    kbuild.build()
    kc.load()


def _cfg(variant=kc.KC_TTF_AUTO, **kw):
    c = kc.kc_config_default()
    c.ttf_variant = variant
    for k, v in kw.items():
        setattr(c, k, v)
    return c


SMALL = {
    "er300": lambda: S.er_lcc(300, 0.02, 7),
    "grid17x13": lambda: S.grid_perturbed(17, 13, 0.25, 3),
    "K7": lambda: S.complete(7),
    "C40": lambda: S.cycle(40),
    "star9": lambda: S.star(9),
    "path33": lambda: S.path(33),
    "K3,5": lambda: S.complete_bipartite(3, 5),
    "cl3000": lambda: S.chung_lu(3000, 2.1, 8.0, 5),
    # the smallest graphs: one edge (every tree is the graph, f = 1), the
    # triangle, the 3-vertex path rooted in its middle
    "K2": lambda: S.complete(2),
    "K3": lambda: S.complete(3),
    "P3": lambda: S.path(3),
}


@pytest.mark.parametrize("name", list(SMALL))
def test_tau0_matches_oracle(name):
    g = SMALL[name]()
    t0 = O.tau0(g)
    with kc.KemenyGraph.from_graph(g) as G:
        tau = G.tau0()
        assert tau["root"] == t0.r
        assert tau["ecc"] == t0.ecc
        assert np.array_equal(tau["p0"], t0.p0)
        assert np.array_equal(tau["level"], t0.level)
        assert np.array_equal(tau["in0"], t0.in0)
        assert np.array_equal(tau["out0"], t0.out0)


@pytest.mark.parametrize("walker", [kc.KC_WALK_LANE, kc.KC_WALK_WARP])
@pytest.mark.parametrize("variant", [kc.KC_TTF_SCAN, kc.KC_TTF_BIT])
@pytest.mark.parametrize("name", list(SMALL))
def test_trees_bit_exact(name, variant, walker):
    g = SMALL[name]()
    t0 = O.tau0(g)
    seed = 4242
    ntrees = 200
    with kc.KemenyGraph.from_graph(g, _cfg(variant, walker=walker)) as G:
        G.sample(seed, ntrees)
        got = G.samples()
        f_ref, st_ref = O.sample_batch(g, t0, seed, 0, ntrees)
        assert np.array_equal(got["sid"], np.arange(ntrees))
        assert np.array_equal(got["steps"], st_ref)
        assert np.array_equal(got["f"], f_ref)
        for k in [0, 1, ntrees // 2, ntrees - 1]:
            tr = G.tree(k)
            ref = O.tree(g, t0, seed, k)
            assert np.array_equal(tr["parent"], ref.parent)
            assert np.array_equal(tr["depth"], ref.depth)
            assert np.array_equal(tr["din"], ref.din)
            assert np.array_equal(tr["dout"], ref.dout)
            assert np.array_equal(tr["vol"], ref.vol)
            assert tr["f"] == ref.f and tr["steps"] == ref.steps


@pytest.mark.parametrize("prefix,tail", [(0, 0), (1, 1000), (250, 1000), (1000, 500),
                                         (400, 1)])
@pytest.mark.parametrize("name", ["er300", "grid17x13", "path33", "star9", "cl3000",
                                  "grid60x60"])
def test_hybrid_walker_bit_exact(name, prefix, tail):
    """Lane walkers for a prefix of the start order, or until a share of the
    wave has finished, then 32 walkers per tree from the saved state: the same
    trees and step counts as the sequential oracle.  prefix 1 hands every tree
    over before its first start; tail 1 hands over all but the first tree."""
    g = S.grid(60, 60) if name == "grid60x60" else SMALL[name]()
    t0 = O.tau0(g)
    seed = 77
    ntrees = 96
    cfg = _cfg(walker=kc.KC_WALK_HYBRID, hybrid_prefix_permille=prefix,
               hybrid_tail_permille=tail)
    with kc.KemenyGraph.from_graph(g, cfg) as G:
        assert G.stats()["walker"] == kc.KC_WALK_HYBRID
        G.sample(seed, ntrees)
        got = G.samples()
        f_ref, st_ref = O.sample_batch(g, t0, seed, 0, ntrees)
        assert np.array_equal(got["steps"], st_ref)
        assert np.array_equal(got["f"], f_ref)
        for k in [0, ntrees - 1]:
            tr = G.tree(k)
            ref = O.tree(g, t0, seed, k)
            assert np.array_equal(tr["parent"], ref.parent)
            assert np.array_equal(tr["depth"], ref.depth)
            assert np.array_equal(tr["din"], ref.din)


def test_launch_shape_does_not_change_trees():
    """Trees depend on (seed, sample id) only: one tree in flight or all of them,
    and sampling in several calls, give the same pool."""
    g = S.er_lcc(400, 0.015, 11)
    with kc.KemenyGraph.from_graph(g) as A, \
            kc.KemenyGraph.from_graph(g, _cfg(max_trees_in_flight=1)) as B, \
            kc.KemenyGraph.from_graph(g, _cfg(walker=kc.KC_WALK_LANE, max_trees_in_flight=7)) as C:
        A.reserve(64)  # capacity reserved ahead changes nothing in the results
        A.sample(9, 64)
        for _ in range(4):
            B.sample(9, 16)
        C.sample(9, 64)
        a, b, c = A.samples(), B.samples(), C.samples()
        assert np.array_equal(a["f"], b["f"]) and np.array_equal(a["steps"], b["steps"])
        assert np.array_equal(a["f"], c["f"]) and np.array_equal(a["steps"], c["steps"])


def test_estimate_equals_exact_integer_mean():
    g = S.er_lcc(500, 0.01, 2)
    t0 = O.tau0(g)
    with kc.KemenyGraph.from_graph(g) as G:
        G.sample(3, 300)
        k = G.estimate()
        f_ref, _ = O.sample_batch(g, t0, 3, 0, 300)
        want = float(int(f_ref.sum())) / (2 * g.m * 300)
        assert k == pytest.approx(want, rel=1e-12)
        st = G.stats()
        assert st["f_sum_hi"] * (1 << 64) + st["f_sum_lo"] == sum(int(x) for x in f_ref)


def test_er2000_full_config_parity_and_accuracy():
    """The small static configuration: ER G(2000, 8/1999) LCC, 2000 trees; every
    tree bit-exact, K within 1% of the FP64 eigendecomposition."""
    g = S.workload("er2000")
    t0 = O.tau0(g)
    k_exact = O.K_dense(g)
    with kc.KemenyGraph.from_graph(g) as G:
        G.sample(0, 2000)
        got = G.samples()
        f_ref, st_ref = O.sample_batch(g, t0, 0, 0, 2000)
        assert np.array_equal(got["f"], f_ref)
        assert np.array_equal(got["steps"], st_ref)
        k = G.estimate()
        assert abs(k - k_exact) / k_exact < 0.01


def test_estimate_to_eps_covers_exact():
    g = S.er_lcc(800, 0.01, 4)
    k_exact = O.K_dense(g)
    misses = 0
    for seed in range(8):
        with kc.KemenyGraph.from_graph(g) as G:
            G.sample(seed, 64)
            k = G.estimate(0.01, 0.05)
            misses += abs(k - k_exact) > 0.01 * k_exact
    assert misses <= 2


@pytest.mark.parametrize("name,eps,batch", [("er300", 0.01, 64), ("cl3000", 0.005, 64),
                                            ("grid17x13", 0.02, 100), ("er300", 0.01, 1024)])
def test_stopping_rule_matches_oracle(name, eps, batch):
    """kc_estimate on a fresh handle (seed 0) draws exactly the trees the
    oracle's stopping rule draws, batch by batch, and returns its K_hat.  The
    oracle decides with exact sums; the cases are chosen with every decision
    far from its threshold (margin), so the device's FP64 sums decide alike."""
    g = SMALL[name]()
    t0 = O.tau0(g)
    ref = O.estimate_clt(lambda a, c: O.sample_batch(g, t0, 0, a, c)[0], 2 * g.m, eps, 0.05,
                         batch=batch)
    assert ref.margin > 1e-9
    with kc.KemenyGraph.from_graph(g, _cfg(batch_trees=batch)) as G:
        k = G.estimate(eps, 0.05)
        assert G.stats()["pool_trees"] == ref.trees
    assert k == pytest.approx(ref.K, rel=1e-12)


@pytest.mark.parametrize("name,eps", [("K7", 0.5), ("C40", 1.0)])
def test_hoeffding_rule_draws_theorem5_trees(name, eps):
    """With the Hoeffding rule kc_estimate draws exactly Theorem 5's sample size
    (Delta read as ecc(r), kappa >= (n-1)^2/n), sample ids 0.., and K_hat is the
    oracle's mean over those trees; the sizes (1969, 13063) sit far from an
    integer boundary."""
    g = SMALL[name]()
    t0 = O.tau0(g)
    want = O.hoeffding_trees(g.n, g.m, t0.ecc, eps, 0.05)
    with kc.KemenyGraph.from_graph(g, _cfg(stop_rule=kc.KC_STOP_HOEFFDING)) as G:
        k = G.estimate(eps, 0.05)
        assert G.stats()["pool_trees"] == want
    f, _ = O.sample_batch(g, t0, 0, 0, want)
    assert k == pytest.approx(O.estimate_fixed(f, 2 * g.m), rel=1e-12)


@pytest.mark.parametrize("walker", ["warp", "lane"])
@pytest.mark.parametrize("name,trees", [("grid17x13", 500), ("er300", 500), ("cl3000", 500),
                                        ("cl80000", 96), ("grid300x300", 24)])
def test_rejection_by_walk_length_matches_oracle(name, trees, walker):
    """With reject_steps = X the pool holds the first sample ids whose Wilson
    step count is at most X, with the oracle's f and step counts (the oracle's
    accepted_samples); the other ids drawn are counted as rejected.  The
    80000-vertex graph and the 300x300 grid (BIT variant) take the pipelined
    waves, the others the plain ones; both walkers."""
    if name == "cl80000":
        g = S.chung_lu(80000, 2.1, 10.0, 6)
    elif name == "grid300x300":
        g = S.workload("grid300x300")
    else:
        g = SMALL[name]()
    t0 = O.tau0(g)
    probe = 4 * trees if name == "grid300x300" else 8 * trees  # oracle trees of the big grid are slow
    _, s_all = O.sample_batch(g, t0, 5, 0, probe)
    cap = int(np.quantile(s_all, 0.7))
    ids, f, steps = O.accepted_samples(lambda a, c: O.sample_batch(g, t0, 5, a, c), cap, trees,
                                       block=2 * trees)
    wk = kc.KC_WALK_WARP if walker == "warp" else kc.KC_WALK_LANE
    with kc.KemenyGraph.from_graph(g, _cfg(keep_trees=0, reject_steps=cap, walker=wk)) as G:
        G.sample(5, trees)
        got = G.samples()
        assert np.array_equal(got["sid"], ids)
        assert np.array_equal(got["f"], f) and np.array_equal(got["steps"], steps)
        st = G.stats()
        assert st["trees_rejected"] == int(ids[-1]) + 1 - trees
        assert st["next_sample_id"] == int(ids[-1]) + 1
        k = G.estimate()
    assert k == pytest.approx(O.estimate_fixed(f, 2 * g.m), rel=1e-12)


@pytest.mark.parametrize("bad", ["asym", "loop", "multi", "disconnected", "unsorted"])
def test_invalid_graphs_rejected(bad):
    g = S.cycle(6)
    ro, col = g.row_off.copy(), g.col.copy()
    want = {"asym": "KC_ERR_NOT_SYMMETRIC", "loop": "KC_ERR_SELF_LOOP",
            "multi": "KC_ERR_MULTI_EDGE", "disconnected": "KC_ERR_DISCONNECTED",
            "unsorted": "KC_ERR_MULTI_EDGE"}[bad]
    if bad == "asym":
        col[0] = 3  # 0 -> 3 without 3 -> 0 (row 0 becomes [3, 5])
    elif bad == "loop":
        col[0] = 0
    elif bad == "multi":
        col[1] = col[0]
    elif bad == "unsorted":
        col[0], col[1] = col[1], col[0]
    elif bad == "disconnected":
        g2 = S.csr_from_edges(6, [0, 1, 3, 4], [1, 2, 4, 5])
        ro, col = g2.row_off, g2.col
    st, h = kc.kc_graph_create(ro, col, check=False)
    assert kc.STATUS[st] == want
    assert not h


def test_empty_and_degenerate_calls():
    """Fewer than two vertices is rejected before any device work; zero trees
    is a no-op; an estimate of an empty pool reports NO_SAMPLES and leaves the
    handle unseeded; a single tree is the oracle's."""
    for n in (0, 1):
        st, h = kc.kc_graph_create(np.zeros(n + 1, np.int64), np.zeros(0, np.int32), check=False)
        assert kc.STATUS[st] == "KC_ERR_INVALID_ARG" and not h
    g = S.cycle(5)
    t0 = O.tau0(g)
    with kc.KemenyGraph.from_graph(g) as G:
        with pytest.raises(kc.KcError) as e:
            G.estimate()
        assert e.value.name == "KC_ERR_NO_SAMPLES"
        assert kc.kc_sample(G.h, 8, 0) == kc.KC_OK
        G.reserve(0)
        assert G.stats()["pool_trees"] == 0
        assert kc.STATUS[kc.kc_sample(G.h, 8, -1, check=False)] == "KC_ERR_INVALID_ARG"
        G.sample(8, 1)
        ref = O.tree(g, t0, 8, 0)
        got = G.samples()
        assert got["f"].tolist() == [ref.f] and got["steps"].tolist() == [ref.steps]
        assert G.estimate() == pytest.approx(ref.f / (2 * g.m), rel=1e-15)


@pytest.mark.parametrize("name", ["K2", "P3"])
def test_tree_graphs_estimate_is_exact(name):
    """A graph that is a tree has one spanning tree, so every f equals
    2m K and the estimate to any eps is exact: K2 = 1/2, P3 = 3/2."""
    g = SMALL[name]()
    want = {"K2": 0.5, "P3": 1.5}[name]
    with kc.KemenyGraph.from_graph(g) as G:
        k = G.estimate(0.01, 0.05)
        assert k == want
        assert set(G.samples()["f"].tolist()) == {int(2 * g.m * want)}


def test_step_cap_reports_error_and_keeps_handle():
    g = S.grid(30, 30)
    with kc.KemenyGraph.from_graph(g, _cfg(step_cap=100)) as G:
        st = kc.kc_sample(G.h, 1, 8, check=False)
        assert kc.STATUS[st] == "KC_ERR_STEP_LIMIT"
        assert G.stats()["pool_trees"] == 0


def test_seed_is_fixed_per_handle():
    g = S.cycle(10)
    with kc.KemenyGraph.from_graph(g) as G:
        assert G.stats()["resident_trees"] > 0  # SMs x resident 32-walker blocks
        G.sample(5, 4)
        assert kc.STATUS[kc.kc_sample(G.h, 6, 4, check=False)] == "KC_ERR_INVALID_ARG"
        G.sample(5, 4)
        assert np.array_equal(G.samples()["sid"], np.arange(8))


@pytest.mark.skipif(os.environ.get("KC_SKIP_LARGE") == "1", reason="large workload disabled")
def test_grid1000_sampled_ids_bit_exact():
    """Road-shaped full-size workload (1000x1000 grid, 25% edges deleted): the
    trees the benchmark draws, checked on sampled ids against the oracle."""
    g = S.workload("grid1000")
    t0 = O.tau0(g)
    with kc.KemenyGraph.from_graph(g, _cfg(keep_trees=0, step_cap=256 * g.n)) as G:
        tau = G.tau0()
        assert tau["ecc"] == t0.ecc and np.array_equal(tau["in0"], t0.in0)
        assert G.stats()["ttf_variant"] == kc.KC_TTF_BIT
        G.sample(1, 64)
        got = G.samples()
        ids = [0, 1, 17, 63]
        for k in ids:
            ref_f, ref_st = O.sample_batch(g, t0, 1, k, 1)
            assert got["f"][k] == ref_f[0] and got["steps"][k] == ref_st[0]
        tr = G.tree(17)
        ref = O.tree(g, t0, 1, 17)
        assert np.array_equal(tr["parent"], ref.parent)
        assert np.array_equal(tr["din"], ref.din)
        assert np.array_equal(tr["vol"], ref.vol)


@pytest.mark.parametrize("name", ["cl80000", "er70000"])
def test_large_shallow_graphs_bit_exact(name):
    """Graphs of at least 2^16 vertices with low eccentricity take the
    leaf-to-root traversal on the sampling path: f and step counts equal to the
    oracle's, and the tree read back (id-ordered DFN) too."""
    g = S.chung_lu(80000, 2.1, 10.0, 6) if name == "cl80000" else S.er_lcc(70000, 6.0 / 70000, 3)
    t0 = O.tau0(g)
    with kc.KemenyGraph.from_graph(g, _cfg()) as G:
        assert G.stats()["ttf_variant"] == kc.KC_TTF_SCAN
        G.sample(21, 96)
        got = G.samples()
        f_ref, st_ref = O.sample_batch(g, t0, 21, 0, 96)
        assert np.array_equal(got["steps"], st_ref)
        assert np.array_equal(got["f"], f_ref)
        tr = G.tree(5)
        ref = O.tree(g, t0, 21, 5)
        assert np.array_equal(tr["din"], ref.din) and np.array_equal(tr["vol"], ref.vol)


@pytest.mark.parametrize("name", ["er300", "grid17x13", "cl3000"])
def test_pipelined_chunks_bit_exact(name):
    """A workspace limit small enough for a handful of trees per traversal
    sub-wave makes the walk's finished trees go through several tree-mapped
    chunks on the second stream: trees and f unchanged."""
    g = SMALL[name]()
    t0 = O.tau0(g)
    with kc.KemenyGraph.from_graph(g, _cfg(keep_trees=0)) as G:
        kc.kc_graph_set_workspace_limit(G.h, 40 * 40 * g.n + 4096)
        G.sample(31, 120)
        st = G.stats()
        assert st["walker"] == kc.KC_WALK_WARP and st["trees_in_flight"] < 120
        got = G.samples()
        f_ref, st_ref = O.sample_batch(g, t0, 31, 0, 120)
        assert np.array_equal(got["steps"], st_ref)
        assert np.array_equal(got["f"], f_ref)


@pytest.mark.parametrize("kind,kname", [(kc.KC_TAU0_DFS, "dfs"), (kc.KC_TAU0_WILSON, "wilson")])
@pytest.mark.parametrize("name", ["er300", "grid17x13", "K3,5", "cl3000"])
def test_dfs_and_wilson_path_trees_bit_exact(name, kind, kname):
    """Exp-II path selections: tau0 built on the device as the depth-first tree
    or as the Wilson tree of sample id 0 under tau0_seed equals the oracle's,
    and so do the sampled trees' f and step counts."""
    g = SMALL[name]()
    t0 = O.tau0(g, kind=kname, seed=77)
    with kc.KemenyGraph.from_graph(g, _cfg(tau0_kind=kind, tau0_seed=77)) as G:
        tau = G.tau0()
        assert tau["root"] == t0.r and tau["ecc"] == t0.ecc
        assert np.array_equal(tau["p0"], t0.p0)
        assert np.array_equal(tau["level"], t0.level)
        assert np.array_equal(tau["in0"], t0.in0) and np.array_equal(tau["out0"], t0.out0)
        G.sample(5, 64)
        got = G.samples()
        f_ref, st_ref = O.sample_batch(g, t0, 5, 0, 64)
        assert np.array_equal(got["steps"], st_ref)
        assert np.array_equal(got["f"], f_ref)
        assert kc.STATUS[kc.kc_update(G.h, [(0, 1, 1)], kc.KC_UPDATE_ISM, check=False)] == \
            "KC_ERR_INVALID_ARG"


def test_sample_multi_equals_separate_calls_and_oracle():
    """One batched walker launch over graphs of uneven size and both TTF
    variants: every graph's pool equals the oracle's, as with kc_sample."""
    names = ["er300", "grid17x13", "K7", "path33", "cl3000", "star9"]
    gs = [SMALL[k]() for k in names]
    seeds = [3 + i for i in range(len(gs))]
    counts = [50, 37, 64, 10, 80, 1]
    Gs = [kc.KemenyGraph.from_graph(g, _cfg()) for g in gs]
    try:
        kc.kc_sample_multi([G.h for G in Gs], seeds, counts)
        kc.kc_sample_multi([G.h for G in Gs], seeds, [5] * len(gs))  # a second call appends
        for g, G, sd, k in zip(gs, Gs, seeds, counts):
            t0 = O.tau0(g)
            got = G.samples()
            assert np.array_equal(got["sid"], np.arange(k + 5))
            f_ref, st_ref = O.sample_batch(g, t0, sd, 0, k + 5)
            assert np.array_equal(got["steps"], st_ref)
            assert np.array_equal(got["f"], f_ref)
        # a seed that differs from a handle's fixed seed is refused and changes nothing
        st = kc.kc_sample_multi([G.h for G in Gs], [99] * len(gs), [4] * len(gs), check=False)
        assert kc.STATUS[st] == "KC_ERR_INVALID_ARG"
        assert Gs[0].stats()["pool_trees"] == counts[0] + 5
    finally:
        for G in Gs:
            G.close()


@pytest.mark.parametrize("name", ["er300", "grid17x13", "cl3000"])
def test_autotuner_pilots_keep_trees_bit_exact(name):
    """The autotuner's pilot waves (32 walkers + chunked traversal, then one
    walker per tree + leaf-to-root traversal) are real trees of the pool: the
    pool equals the oracle's, and a choice is recorded with its timings."""
    g = SMALL[name]()
    t0 = O.tau0(g)
    with kc.KemenyGraph.from_graph(g, _cfg(autotune=1)) as G:
        G.sample(13, 200)
        st = G.stats()
        assert st["tuned"] == 1
        assert st["walker"] in (kc.KC_WALK_WARP, kc.KC_WALK_LANE)
        assert st["tune_ms"][0] > 0 and st["tune_ms"][1] > 0 and st["tune_ms"][2] > 0
        G.sample(13, 50)  # after tuning: the chosen variant
        got = G.samples()
        f_ref, st_ref = O.sample_batch(g, t0, 13, 0, 250)
        assert np.array_equal(got["steps"], st_ref)
        assert np.array_equal(got["f"], f_ref)


@pytest.mark.parametrize("name,trees", [("cl80000", 96), ("grid300x300", 16)])
def test_lane_walker_pipelined_waves_bit_exact(name, trees):
    """One walker per tree on graphs large enough for pipelined waves: every
    lane flags its finished tree (depth + 1) for the traversal and TTF chunks
    on the second stream; f and step counts equal the oracle's, sample ids in
    order, and a retained tree's arrays equal the oracle's."""
    g = S.chung_lu(80000, 2.1, 10.0, 6) if name == "cl80000" else S.workload("grid300x300")
    t0 = O.tau0(g)
    seed = 31
    with kc.KemenyGraph.from_graph(g, _cfg(keep_trees=0, walker=kc.KC_WALK_LANE)) as G:
        G.sample(seed, trees)
        got = G.samples()
        assert G.stats()["walker"] == kc.KC_WALK_LANE
    f_ref, st_ref = O.sample_batch(g, t0, seed, 0, trees)
    assert np.array_equal(got["sid"], np.arange(trees))
    assert np.array_equal(got["steps"], st_ref)
    assert np.array_equal(got["f"], f_ref)


@pytest.mark.parametrize("k", [2, 3, 7, 64])
@pytest.mark.parametrize("name", ["grid17x13", "er300", "path33", "cl3000", "K3", "P3"])
def test_segmented_bit_evaluation_bit_exact(name, k):
    """Algorithm 1 split into k preorder segments a tree (ttf_segments = k), each
    warp starting from the DFS stack and Fenwick state rebuilt at its first
    position: f equals the oracle's bit for bit.  The cases cover segments of
    fewer than 32 positions and graphs with fewer vertices than segments."""
    g = SMALL[name]()
    t0 = O.tau0(g)
    seed = 4243
    with kc.KemenyGraph.from_graph(g, _cfg(kc.KC_TTF_BIT, ttf_segments=k)) as G:
        G.sample(seed, 150)
        got = G.samples()
    f_ref, st_ref = O.sample_batch(g, t0, seed, 0, 150)
    assert np.array_equal(got["steps"], st_ref)
    assert np.array_equal(got["f"], f_ref)


@pytest.mark.parametrize("k", [0, 1, 5])
def test_segmented_bit_evaluation_in_pipelined_and_rejection_waves(k):
    """The segmented evaluation inside the waves that use it: pipelined chunks
    forced by a small workspace (forced k: chunks evaluated while the walk
    runs take the handle buffer), and rejection waves whose rejected trees'
    walk arrays hold the segments once the walk has ended (automatic, k = 0).
    k = 1 never splits.  f and step counts equal the oracle's."""
    g = SMALL["grid17x13"]()
    t0 = O.tau0(g)
    with kc.KemenyGraph.from_graph(g, _cfg(kc.KC_TTF_BIT, keep_trees=0, ttf_segments=k)) as G:
        kc.kc_graph_set_workspace_limit(G.h, 40 * 40 * g.n + 4096)
        G.sample(31, 120)
        assert G.stats()["trees_in_flight"] < 120
        got = G.samples()
    f_ref, st_ref = O.sample_batch(g, t0, 31, 0, 120)
    assert np.array_equal(got["steps"], st_ref)
    assert np.array_equal(got["f"], f_ref)
    _, s_all = O.sample_batch(g, t0, 5, 0, 1000)
    cap = int(np.quantile(s_all, 0.6))
    ids, f, steps = O.accepted_samples(lambda a, c: O.sample_batch(g, t0, 5, a, c), cap, 300,
                                       block=600)
    for wk in (kc.KC_WALK_LANE, kc.KC_WALK_WARP):
        cfg = _cfg(kc.KC_TTF_BIT, keep_trees=0, reject_steps=cap, walker=wk, ttf_segments=k)
        with kc.KemenyGraph.from_graph(g, cfg) as G:
            G.sample(5, 300)
            got = G.samples()
        assert np.array_equal(got["sid"], ids)
        assert np.array_equal(got["f"], f) and np.array_equal(got["steps"], steps)


def test_pending_runtime_error_of_the_caller_is_not_reported():
    """An error that an unrelated runtime call left pending on the calling
    thread (here cudaSetDevice with an ordinal that does not exist, a plain
    argument error) is not reported as the failure of the library's next
    call: handle creation and sampling succeed and match the oracle."""
    import ctypes

    rt = None
    for name in ("libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so.13"):
        try:
            rt = ctypes.CDLL(name)
            break
        except OSError:
            continue
    if rt is None:
        pytest.skip("libcudart.so.13 not found")
    g = SMALL["er300"]()
    t0 = O.tau0(g)
    assert rt.cudaSetDevice(1 << 20) != 0  # leaves an error pending on this thread
    with kc.KemenyGraph.from_graph(g, _cfg()) as G:
        assert rt.cudaSetDevice(1 << 20) != 0
        G.sample(9, 40)
        got = G.samples()
    f_ref, _ = O.sample_batch(g, t0, 9, 0, 40)
    assert np.array_equal(got["f"], f_ref)
