"""GPU tests of the query server (continuous batching over resident graphs):
every result is the same alone and in a mix of concurrent traffic, and the
same as the plain one-graph-per-call path."""
import pytest

from paper_2511_16356_gb300 import synth as S

pytestmark = pytest.mark.gpu

kc = pytest.importorskip("paper_2511_16356_gb300.kc")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2511_16356_gb300 import build as kbuild

    kbuild.build()
    kc.load()


def _graphs():
    return [S.er_lcc(1500, 6.0 / 1500, 1), S.grid_perturbed(40, 30, 0.25, 2),
            S.chung_lu(5000, 2.1, 8.0, 3), S.er_lcc(3000, 4.0 / 3000, 4),
            S.grid_perturbed(60, 20, 0.2, 5), S.chung_lu(20000, 2.3, 10.0, 6)]


# (graph index, seed, eps, delta)
QUERIES = [(0, 11, 0.05, 0.05), (1, 12, 0.05, 0.05), (2, 13, 0.02, 0.05), (3, 14, 0.05, 0.1),
           (4, 15, 0.05, 0.05), (5, 16, 0.02, 0.05), (0, 17, 0.02, 0.05), (2, 11, 0.05, 0.05)]


def _plain(g, seed, eps, delta):
    with kc.KemenyGraph.from_graph(g, _static_cfg()) as G:
        G.sample(seed, 1024)
        return G.estimate(eps, delta), G.stats()["pool_trees"]


def _static_cfg():
    c = kc.kc_config_default()
    c.keep_trees = 0
    return c


def test_queries_same_alone_in_mix_and_plain():
    gs = _graphs()
    # alone: one worker, one request at a time
    alone = []
    with kc.Server(workers=1) as srv:
        ids = [srv.add_graph(g, _static_cfg()) for g in gs]
        for gi, seed, eps, delta in QUERIES:
            info = srv.wait(srv.query(ids[gi], seed, eps, delta))
            assert info["status"] == kc.KC_OK
            alone.append((info["K"], info["trees"]))
    # in the mix: four workers, everything submitted at once, twice over
    with kc.Server(workers=4) as srv:
        ids = [srv.add_graph(g, _static_cfg()) for g in gs]
        tickets = [srv.query(ids[gi], seed, eps, delta) for gi, seed, eps, delta in QUERIES * 2]
        srv.drain()
        infos = [srv.wait(t) for t in tickets]
    assert len({i["worker"] for i in infos}) > 1  # the work really spread over workers
    for k, info in enumerate(infos):
        assert info["status"] == kc.KC_OK
        assert (info["K"], info["trees"]) == alone[k % len(QUERIES)]
        assert info["t_submit_ms"] <= info["t_start_ms"] <= info["t_end_ms"]
    # the plain path: one handle per call
    for (gi, seed, eps, delta), (k, trees) in zip(QUERIES[:4], alone[:4]):
        assert _plain(gs[gi], seed, eps, delta) == (k, trees)


def _update_script(g, w):
    """Deletions of interior grid edges (never bridges) and insertions of
    diagonals, in batches."""
    ops = []
    for y in range(2, 8):
        x = 3 + y
        ops.append([(y * w + x, y * w + x + 1, 1), ((y + 1) * w + x, y * w + x + 1, 0)])
    return ops


def test_dynamic_graph_same_alone_and_in_mix():
    w = 16
    dyn = S.grid(w, 12)
    statics = _graphs()[:3]
    cfg = kc.kc_config_default()

    def run(workers, with_traffic):
        seq = []
        with kc.Server(workers=workers) as srv:
            d = srv.add_graph(dyn, cfg, pool_seed=5, pool_trees=256)
            sids = [srv.add_graph(g, _static_cfg()) for g in statics] if with_traffic else []
            tickets = []
            for b, batch in enumerate(_update_script(dyn, w)):
                for gi, sid in enumerate(sids):
                    srv.query(sid, 100 + b, 0.05, 0.05)
                tickets.append(("u", srv.update(d, batch, kc.KC_UPDATE_ISM)))
                tickets.append(("q", srv.pool_query(d, 0.05, 0.05)))
            srv.drain()
            for kind, t in tickets:
                info = srv.wait(t)
                assert info["status"] == kc.KC_OK, info
                seq.append((kind, info["K"], info["trees"]))
        return seq

    alone = run(1, False)
    mixed = run(4, True)
    assert alone == mixed
    # the plain path: one handle, the same calls in order
    with kc.KemenyGraph.from_graph(dyn, cfg) as G:
        G.sample(5, 256)
        plain = []
        for batch in _update_script(dyn, w):
            G.update(batch, kc.KC_UPDATE_ISM)
            plain.append(("u", 0.0, G.stats()["pool_trees"]))
            plain.append(("q", G.estimate(0.05, 0.05), G.stats()["pool_trees"]))
    assert plain == alone


def test_small_budget_queues_requests():
    """A budget that admits about one request at a time still serves every
    request, with the same results."""
    gs = _graphs()[:4]
    per = 4096 * (40 * max(g.n for g in gs) + 512)
    with kc.Server(workers=4, budget_bytes=per, request_bytes=per) as srv:
        ids = [srv.add_graph(g, _static_cfg()) for g in gs]
        tickets = [srv.query(ids[i], 7, 0.05, 0.05) for i in range(4)]
        infos = [srv.wait(t) for t in tickets]
    with kc.Server(workers=1) as srv:
        ids = [srv.add_graph(g, _static_cfg()) for g in gs]
        ref = [srv.wait(srv.query(ids[i], 7, 0.05, 0.05)) for i in range(4)]
    for a, b in zip(infos, ref):
        assert a["status"] == kc.KC_OK and a["K"] == b["K"]


def test_request_errors_are_reported():
    with kc.Server(workers=2) as srv:
        sid = srv.add_graph(S.grid(10, 10), _static_cfg())
        did = srv.add_graph(S.grid(10, 10), kc.kc_config_default(), pool_seed=1, pool_trees=32)
        with pytest.raises(kc.KcError):
            srv.pool_query(sid, 0.05, 0.05)  # static graph has no maintained pool
        with pytest.raises(kc.KcError):
            srv.query(did, 1, 0.05, 0.05)    # dynamic graph answers pool queries only
        with pytest.raises(kc.KcError):
            srv.query(sid, 1, 0.0, 0.05)
        t = srv.update(did, [(0, 1, 0)], kc.KC_UPDATE_ISM)  # (0, 1) exists: insert fails
        info = srv.wait(t)
        assert kc.STATUS[info["status"]] == "KC_ERR_EDGE_EXISTS"
        # the graph still serves
        assert srv.wait(srv.pool_query(did, 0.05, 0.05))["status"] == kc.KC_OK


@pytest.mark.parametrize("max_n", [0, 4000])
def test_coalesced_queries_same_as_alone(max_n):
    """With coalescing, queries on small graphs advance together (one
    kc_sample_multi launch per round) and still return exactly the K and tree
    count they get alone; with coalesce_max_n = 4000 the larger graphs stay
    with the workers while the small ones are coalesced, in the same mix."""
    gs = _graphs()
    alone = []
    with kc.Server(workers=1) as srv:
        ids = [srv.add_graph(g, _static_cfg()) for g in gs]
        for gi, seed, eps, delta in QUERIES:
            info = srv.wait(srv.query(ids[gi], seed, eps, delta))
            alone.append((info["K"], info["trees"]))
    with kc.Server(workers=2, coalesce=1, coalesce_max_n=max_n) as srv:
        ids = [srv.add_graph(g, _static_cfg()) for g in gs]
        tickets = [srv.query(ids[gi], seed, eps, delta) for gi, seed, eps, delta in QUERIES * 2]
        srv.drain()
        infos = [srv.wait(t) for t in tickets]
    limit = max_n or (1 << 18)
    shallow = []
    for g in gs:
        with kc.KemenyGraph.from_graph(g, _static_cfg()) as G:
            shallow.append(G.stats()["ttf_variant"] == kc.KC_TTF_SCAN)
    for k, info in enumerate(infos):
        gi = QUERIES[k % len(QUERIES)][0]
        assert info["status"] == kc.KC_OK
        assert (info["K"], info["trees"]) == alone[k % len(QUERIES)]
        if gs[gi].n <= limit and shallow[gi]:
            assert info["worker"] == -1  # run by the dispatcher
        else:
            assert info["worker"] >= 0  # large or deep graphs stay with the workers
