"""The seeded input generators shared by the tests, the oracle checks and the
benchmark: valid simple undirected CSR, connectivity, determinism, and the
shapes the workloads stand for."""
import numpy as np
import pytest

from paper_2511_16356_gb300 import synth as S


def _check_csr(g):
    n = g.n
    assert g.row_off.dtype == np.int64 and g.col.dtype == np.int32
    assert g.row_off[0] == 0 and g.row_off[-1] == g.col.shape[0] == 2 * g.m
    for v in range(n):
        row = g.col[g.row_off[v]:g.row_off[v + 1]]
        assert np.all(np.diff(row) > 0)  # ascending, no multi-edges
        assert not np.any(row == v)  # no self loops
    src = np.repeat(np.arange(n), np.diff(g.row_off))
    fwd = set(zip(src.tolist(), g.col.tolist()))
    assert all((b, a) in fwd for a, b in fwd)  # symmetric
    assert np.array_equal(g.deg, np.diff(g.row_off))


def _connected(g):
    seen = np.zeros(g.n, dtype=bool)
    stack = [0]
    seen[0] = True
    while stack:
        u = stack.pop()
        for w in g.col[g.row_off[u]:g.row_off[u + 1]]:
            if not seen[w]:
                seen[w] = True
                stack.append(int(w))
    return seen.all()


@pytest.mark.parametrize("make", [
    lambda: S.er_lcc(500, 0.01, 3), lambda: S.grid_perturbed(30, 20, 0.25, 4),
    lambda: S.chung_lu(3000, 2.1, 8.0, 5), lambda: S.torus(6, 5), lambda: S.hypercube(6),
    lambda: S.grid(7, 4), lambda: S.random_connected(9, 0.4, 2)])
def test_generators_give_connected_simple_csr(make):
    g = make()
    _check_csr(g)
    assert _connected(g)


def test_generators_are_deterministic_in_their_seed():
    for make in (lambda s: S.er_lcc(800, 0.01, s), lambda s: S.grid_perturbed(20, 20, 0.25, s),
                 lambda s: S.chung_lu(2000, 2.1, 8.0, s)):
        a, b, c = make(1), make(1), make(2)
        assert np.array_equal(a.col, b.col) and np.array_equal(a.row_off, b.row_off)
        assert not (a.n == c.n and np.array_equal(a.col, c.col))


def test_perturbed_grid_keeps_a_spanning_tree_and_deletes_the_share():
    w, h, frac = 40, 30, 0.25
    g = S.grid_perturbed(w, h, frac, 7)
    m0 = (w - 1) * h + w * (h - 1)
    assert g.n == w * h
    assert g.m == m0 - round(frac * m0)
    assert _connected(g)
    # only grid edges: neighbours differ by 1 in a row or by w between rows
    src = np.repeat(np.arange(g.n), g.deg)
    d = np.abs(src - g.col.astype(np.int64))
    assert np.all((d == 1) | (d == w))


def test_chung_lu_is_heavy_tailed():
    g = S.chung_lu(20000, 2.1, 10.0, 3)
    deg = np.sort(g.deg)
    assert deg[-1] > 20 * np.median(deg)  # hubs far above the typical degree
    assert 5.0 < deg.mean() < 15.0
