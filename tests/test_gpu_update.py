"""GPU parity of sample maintenance (kc_update, Sec. 4) against the oracle's
sequential Algorithm 2 / Algorithm 3 semantics on the same Philox streams.

After every update: the pool's f (int64), sample ids, Wilson step counts and
parent arrays must match bit for bit; weights and K_hat within 1e-12
(relative).  R(u, v) is passed in (the oracle's exact FP64 value) so both sides
select the same number of trees; the device conjugate-gradient R is checked
separately against the exact value.
"""
import numpy as np
import pytest

import oracle as O
from oracle.dynamic import DynamicOracle
from paper_2511_16356_gb300 import synth as S

pytestmark = pytest.mark.gpu

kc = pytest.importorskip("paper_2511_16356_gb300.kc")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2511_16356_gb300 import build as kbuild

    kbuild.build()
    kc.load()


def _ops(g, rng, n_ops):
    """A deterministic mix of insertions of absent edges and deletions of
    non-bridge edges, valid against the evolving graph."""
    edges = {(int(a), int(b)) for a, b in g.edges()}
    out = []
    while len(out) < n_ops:
        if rng.random() < 0.5:
            a, b = sorted(int(x) for x in rng.choice(g.n, 2, replace=False))
            if (a, b) in edges:
                continue
            edges.add((a, b))
            out.append((a, b, 0))
        else:
            cand = sorted(edges)
            a, b = cand[int(rng.integers(len(cand)))]
            e2 = edges - {(a, b)}
            arr = np.array(sorted(e2))
            h = S.csr_from_edges(g.n, arr[:, 0], arr[:, 1])
            if h.n != g.n or np.any(h.deg == 0) or not S.is_connected(h):
                continue
            edges = e2
            out.append((a, b, 1))
    return out


def _compare(G, D, n):
    got = G.samples()
    assert np.array_equal(got["sid"], np.array(D.sid))
    assert np.array_equal(got["steps"], np.array(D.steps))
    assert np.array_equal(got["f"], np.array(D.f, dtype=np.int64))
    np.testing.assert_allclose(got["w"], np.array(D.w), rtol=1e-12, atol=0)
    for k in range(len(D.parents)):
        tr = G.tree(k)
        assert np.array_equal(tr["parent"], D.parents[k]), k
    assert G.estimate() == pytest.approx(D.estimate(), rel=1e-12)


@pytest.mark.parametrize("refresh", [0, 1])
@pytest.mark.parametrize("mode", [kc.KC_UPDATE_BSM, kc.KC_UPDATE_ISM])
@pytest.mark.parametrize("gname", ["er", "grid"])
def test_updates_bit_exact(gname, mode, refresh):
    g = {"er": lambda: S.er_lcc(160, 0.035, 5),
         "grid": lambda: S.grid_perturbed(12, 10, 0.2, 4)}[gname]()
    seed, T = 17, 48
    D = DynamicOracle(g, seed, T)
    cfg = kc.kc_config_default()
    cfg.keep_trees = 1
    cfg.r_source = kc.KC_R_GIVEN
    cfg.refresh_after_update = refresh
    with kc.KemenyGraph.from_graph(g, cfg) as G:
        G.sample(seed, T)
        _compare(G, D, g.n)
        rng = np.random.default_rng(100 + mode * 10 + refresh)
        for (a, b, op) in _ops(g, rng, 6):
            if op == 0:
                e2 = D.edges | {(a, b)}
                arr = np.array(sorted(e2))
                h = S.csr_from_edges(g.n, arr[:, 0], arr[:, 1])
                R = O.resistance(h, a, b)
                D.insert(a, b, mode, R=R, refresh=bool(refresh))
                G.update([(a, b, 0, R)], mode)
            else:
                D.delete(a, b, mode, refresh=bool(refresh))
                G.update([(a, b, 1)], mode)
            _compare(G, D, g.n)
        assert G.stats()["updates_applied"] == 6


def test_batch_is_all_or_nothing():
    g = S.er_lcc(120, 0.05, 3)
    cfg = kc.kc_config_default()
    cfg.r_source = kc.KC_R_GIVEN
    with kc.KemenyGraph.from_graph(g, cfg) as G:
        G.sample(3, 16)
        before = G.samples()
        for a, b in g.edges():  # an edge whose removal keeps the graph connected
            a, b = int(a), int(b)
            arr = np.array(sorted({(int(x), int(y)) for x, y in g.edges()} - {(a, b)}))
            h = S.csr_from_edges(g.n, arr[:, 0], arr[:, 1])
            if h.n == g.n and np.all(h.deg > 0) and S.is_connected(h):
                break
        # second op re-inserts an existing edge: nothing may be applied
        st = kc.kc_update(G.h, [(a, b, 1), (a, b, 1)], kc.KC_UPDATE_BSM, check=False)
        assert kc.STATUS[st] == "KC_ERR_EDGE_MISSING"
        st = kc.kc_update(G.h, [(a, b, 0, 0.5)], kc.KC_UPDATE_BSM, check=False)
        assert kc.STATUS[st] == "KC_ERR_EDGE_EXISTS"
        after = G.samples()
        assert np.array_equal(before["f"], after["f"]) and G.stats()["updates_applied"] == 0
    p = S.path(12)
    with kc.KemenyGraph.from_graph(p, cfg) as P:
        P.sample(1, 4)
        st = kc.kc_update(P.h, [(3, 4, 1)], kc.KC_UPDATE_ISM, check=False)
        assert kc.STATUS[st] == "KC_ERR_BRIDGE"
    cfg0 = kc.kc_config_default()
    cfg0.keep_trees = 0
    with kc.KemenyGraph.from_graph(g, cfg0) as G0:
        G0.sample(3, 4)
        st = kc.kc_update(G0.h, [(a, b, 1)], kc.KC_UPDATE_BSM, check=False)
        assert kc.STATUS[st] == "KC_ERR_NOT_RETAINED"


@pytest.mark.parametrize("gname", ["er", "grid"])
def test_cg_resistance_matches_exact(gname):
    g = {"er": lambda: S.er_lcc(300, 0.02, 9),
         "grid": lambda: S.grid_perturbed(15, 15, 0.25, 2)}[gname]()
    edges = {(int(a), int(b)) for a, b in g.edges()}
    rng = np.random.default_rng(1)
    while True:
        a, b = sorted(int(x) for x in rng.choice(g.n, 2, replace=False))
        if (a, b) not in edges:
            break
    arr = np.array(sorted(edges | {(a, b)}))
    h = S.csr_from_edges(g.n, arr[:, 0], arr[:, 1])
    want = O.resistance(h, a, b)
    with kc.KemenyGraph.from_graph(g) as G:  # default: R by device CG
        G.sample(5, 16)
        G.update([(a, b, 0)], kc.KC_UPDATE_BSM)
        st = G.stats()
        assert st["last_resistance"] == pytest.approx(want, rel=1e-9)
        assert st["last_cg_iters"] > 0


def _tau0_edge_deletable(g, p0, rng):
    """A tau0 edge (x, p0[x]) whose deletion keeps the graph connected."""
    xs = rng.permutation(np.flatnonzero(p0 >= 0))
    edges = {(int(a), int(b)) for a, b in g.edges()}
    for x in xs[:200]:
        a, b = sorted((int(x), int(p0[x])))
        arr = np.array(sorted(edges - {(a, b)}))
        h = S.csr_from_edges(g.n, arr[:, 0], arr[:, 1])
        if h.n == g.n and np.all(h.deg > 0) and S.is_connected(h):
            return a, b
    raise RuntimeError("no deletable tau0 edge")


@pytest.mark.parametrize("mode", [kc.KC_UPDATE_BSM, kc.KC_UPDATE_ISM])
def test_updates_bit_exact_on_a_large_power_law_graph(mode):
    """The device-resident update path (CSR edited on the device per op) on a
    Chung-Lu graph of about 10^5 vertices: a mixed stream of insertions and
    deletions, one of them an edge of tau0 (tau0 rebuilt, every f refreshed),
    every pool value and parent array bit for bit with the oracle after each
    op.  Deep subtrees and the crossing-count kernels meet sizes far beyond the
    small graphs above."""
    g = S.chung_lu(100000, 2.1, 8.0, 21)
    seed, T = 23, 16
    D = DynamicOracle(g, seed, T)
    cfg = kc.kc_config_default()
    cfg.keep_trees = 1
    cfg.r_source = kc.KC_R_GIVEN
    rng = np.random.default_rng(7 + mode)
    a0, b0 = _tau0_edge_deletable(g, D.t0.p0, rng)
    arr = np.array(sorted({(int(a), int(b)) for a, b in g.edges()} - {(a0, b0)}))
    g2 = S.csr_from_edges(g.n, arr[:, 0], arr[:, 1])
    ops = _ops(g2, rng, 9)
    ops.insert(0, (a0, b0, 1))  # first: an edge of tau0 (ops after it are valid on G - e)
    with kc.KemenyGraph.from_graph(g, cfg) as G:
        G.sample(seed, T)
        _compare(G, D, g.n)
        for (a, b, op) in ops:
            if op == 0:
                arr = np.array(sorted(D.edges | {(a, b)}))
                h = S.csr_from_edges(g.n, arr[:, 0], arr[:, 1])
                R = O.resistance_sparse(h, a, b)
                D.insert(a, b, mode, R=R)
                G.update([(a, b, 0, R)], mode)
            else:
                D.delete(a, b, mode)
                G.update([(a, b, 1)], mode)
            _compare(G, D, g.n)
        tau = G.tau0()
        assert np.array_equal(tau["p0"], D.t0.p0)  # rebuilt after the tau0 deletion
        assert G.stats()["updates_applied"] == len(ops)
        assert G.stats()["m"] == len(D.edges)


def test_batched_updates_equal_one_at_a_time():
    """A batch of ops in one kc_update call gives the pool, graph and tau0 that
    the same ops give one call at a time (the host copy of the CSR is refreshed
    once per batch, the device copy per op)."""
    g = S.chung_lu(20000, 2.1, 8.0, 5)
    rng = np.random.default_rng(3)
    ops = _ops(g, rng, 8)
    cfg = kc.kc_config_default()
    cfg.keep_trees = 1
    cfg.r_source = kc.KC_R_GIVEN
    Rs = {}
    edges = {(int(a), int(b)) for a, b in g.edges()}
    for (a, b, op) in ops:
        if op == 0:
            edges.add((a, b))
            arr = np.array(sorted(edges))
            Rs[(a, b)] = O.resistance_sparse(S.csr_from_edges(g.n, arr[:, 0], arr[:, 1]), a, b)
        else:
            edges.discard((a, b))
    full = [(a, b, 0, Rs[(a, b)]) if op == 0 else (a, b, 1) for (a, b, op) in ops]
    outs = []
    for batched in (True, False):
        with kc.KemenyGraph.from_graph(g, cfg) as G:
            G.sample(9, 24)
            if batched:
                G.update(full, kc.KC_UPDATE_ISM)
            else:
                for o in full:
                    G.update([o], kc.KC_UPDATE_ISM)
            outs.append((G.samples(), G.tau0(), G.stats()["m"],
                         [G.tree(k)["parent"] for k in range(24)]))
    (s1, t1, m1, p1), (s2, t2, m2, p2) = outs
    assert m1 == m2 == len(edges)
    assert np.array_equal(s1["f"], s2["f"]) and np.array_equal(s1["w"], s2["w"])
    assert np.array_equal(t1["p0"], t2["p0"])
    assert all(np.array_equal(a, b) for a, b in zip(p1, p2))
