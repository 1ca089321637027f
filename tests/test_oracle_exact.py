"""Pins of the oracle's exact-K routines against closed forms and identities.

Eq. (1) (K = Tr of the pseudo-inverse of the normalised Laplacian) is computed
by a dense eigendecomposition; it is pinned here to spectra known in closed
form, to the single-spanning-tree case of the forest formula (Theorem 1) and
to the grounded-Laplacian identity (corrected Eq. (3)).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2511_16356_gb300 import synth as S


@pytest.mark.parametrize("n", [2, 3, 5, 17, 64])
def test_complete_graph(n):
    assert O.K_dense(S.complete(n)) == pytest.approx((n - 1) ** 2 / n, rel=1e-12)


@pytest.mark.parametrize("n", [3, 4, 7, 30, 101])
def test_cycle(n):
    assert O.K_dense(S.cycle(n)) == pytest.approx((n * n - 1) / 6.0, rel=1e-11)


@pytest.mark.parametrize("n", [3, 6, 40])
def test_star(n):
    assert O.K_dense(S.star(n)) == pytest.approx(n - 1.5, rel=1e-12)


@pytest.mark.parametrize("a,b", [(1, 4), (2, 3), (5, 7)])
def test_complete_bipartite(a, b):
    assert O.K_dense(S.complete_bipartite(a, b)) == pytest.approx(a + b - 1.5, rel=1e-12)


@pytest.mark.parametrize("a,b", [(3, 3), (4, 6), (7, 5)])
def test_torus(a, b):
    assert O.K_dense(S.torus(a, b)) == pytest.approx(O.K_torus(a, b), rel=1e-11)


@pytest.mark.parametrize("k", [1, 3, 6])
def test_hypercube(k):
    assert O.K_dense(S.hypercube(k)) == pytest.approx(O.K_hypercube(k), rel=1e-11)


def test_hypercube_closed_form_small_values():
    # Q1 = K2: K = 1/2 ; Q2 = C4: K = (16-1)/6
    assert O.K_hypercube(1) == pytest.approx(0.5)
    assert O.K_hypercube(2) == pytest.approx(15 / 6)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tree_graphs(seed):
    # random trees (Pruefer-like via random parent), K = (1/2m) sum_e vol_e (2m - vol_e)
    rng = np.random.default_rng(seed)
    n = 25
    par = [int(rng.integers(0, v)) for v in range(1, n)]
    g = S.csr_from_edges(n, np.arange(1, n), par)
    assert O.K_dense(g) == pytest.approx(O.K_tree_graph(g), rel=1e-11)
    p = S.path(9)
    assert O.K_dense(p) == pytest.approx(O.K_tree_graph(p), rel=1e-12)


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_grounded_formula_equals_eigen(seed):
    g = S.random_connected(30, 0.15, seed)
    k = O.K_dense(g)
    for r in [0, 7, 29]:
        assert O.K_grounded(g, r) == pytest.approx(k, rel=1e-10)


def test_eq3_sign_erratum():
    """Eq. (3) holds with a minus sign; as printed (plus) it gives 4 on K3 instead of 4/3."""
    g = S.complete(3)
    assert O.K_eq3(g, 0, -1.0) == pytest.approx(4.0 / 3.0, rel=1e-12)
    assert O.K_eq3(g, 0, +1.0) == pytest.approx(4.0, rel=1e-12)
    g = S.random_connected(12, 0.4, 8)
    assert O.K_eq3(g, 3, -1.0) == pytest.approx(O.K_dense(g), rel=1e-10)


@pytest.mark.parametrize("gname", ["K4", "grid3x3", "rc6"])
def test_forest_formula_theorem1(gname):
    g = {"K4": S.complete(4), "grid3x3": S.grid(3, 3), "rc6": S.random_connected(6, 0.6, 11)}[gname]
    k = O.K_dense(g)
    for r in range(g.n):
        assert O.K_forest_formula(g, r) == pytest.approx(k, rel=1e-12)


def test_kirchhoff_matches_enumeration():
    for g in [S.complete(5), S.grid(3, 3), S.random_connected(7, 0.5, 2), S.torus(3, 3)]:
        assert len(O.spanning_trees(g)) == round(O.kirchhoff_count(g))
    assert len(O.spanning_trees(S.complete(5))) == 5 ** 3  # Cayley


def test_hoeffding_sample_size_matches_theorem5_shape():
    # omega = ceil(8 m^2 ecc^2 ln(2/delta) / (kmin^2 eps^2)) with kmin = (n-1)^2/n
    n, m, ecc, eps, delta = 2000, 8000, 5, 0.01, 0.01
    kmin = (n - 1) ** 2 / n
    want = math.ceil(8 * m * m * ecc * ecc * math.log(2 / delta) / (kmin ** 2 * eps ** 2))
    assert O.hoeffding_trees(n, m, ecc, eps, delta) == want
    # kappa >= (n-1)^2/n holds with equality on K_n (the bound the proof needs)
    for n in [3, 6, 11]:
        assert O.K_dense(S.complete(n)) == pytest.approx((n - 1) ** 2 / n)


@pytest.mark.parametrize("w,h,frac,seed", [(12, 9, 0.25, 1), (30, 40, 0.25, 2), (45, 44, 0.0, 0),
                                           (7, 60, 0.3, 5)])
def test_block_tridiagonal_equals_eigen(w, h, frac, seed):
    """Selected inversion of the grounded grid Laplacian against the dense
    eigendecomposition of the normalised Laplacian (Eq. 1)."""
    g = S.grid_perturbed(w, h, frac, seed) if frac > 0 else S.grid(w, h)
    assert O.K_block_tridiagonal(g, w) == pytest.approx(O.K_dense(g), rel=1e-10)


def test_block_tridiagonal_path_is_tree_formula():
    """A path numbered in order is block tridiagonal for any block width; its
    only spanning tree is itself (closed form of Theorem 1 for trees)."""
    g = S.path(120)
    for w in (2, 5, 12, 40):
        assert O.K_block_tridiagonal(g, w) == pytest.approx(O.K_tree_graph(g), rel=1e-10)


def test_block_tridiagonal_rejects_other_layouts():
    with pytest.raises(ValueError):
        O.K_block_tridiagonal(S.torus(10, 10), 10)  # wrap-around rows
    with pytest.raises(ValueError):
        O.K_block_tridiagonal(S.grid(10, 10), 7)  # width does not divide n


@pytest.mark.parametrize("gname", ["er300", "cl800"])
def test_pinv_quadratic_form_matches_dense(gname):
    """CG solve of the normalised Laplacian against the dense pseudo-inverse,
    for Rademacher probes and for the unit vectors (whose sum is Tr N^+ = K)."""
    g = S.er_lcc(300, 0.02, 7) if gname == "er300" else S.chung_lu(800, 2.1, 8.0, 3)
    Nd = np.linalg.pinv(O.normalized_laplacian(g).toarray(), hermitian=True)
    rng = np.random.default_rng(1)
    Z = rng.integers(0, 2, size=(g.n, 5)).astype(np.float64) * 2 - 1
    got = O.quad_pinv(g, Z, tol=1e-12)
    want = np.einsum("ij,ij->j", Z, Nd @ Z)
    assert np.allclose(got, want, rtol=1e-8)
    unit = O.quad_pinv(g, np.eye(g.n), tol=1e-12)
    assert unit.sum() == pytest.approx(O.K_dense(g), rel=1e-8)


def test_hutchinson_mean_covers_exact_on_chung_lu():
    """Config-0-sized Chung-Lu graph: the probe mean lies within 4 standard
    errors of the exact K, and the standard error is small."""
    g = S.chung_lu(2000, 2.1, 17.0, 2)
    k = O.K_dense(g)
    mean, se, _ = O.K_hutchinson(g, 96, seed=5)
    assert abs(mean - k) <= 4 * se
    assert se / k < 0.01


def test_hutchinson_and_block_selected_inversion_agree_on_a_grid():
    """The two large-graph references cross-checked on a 60x50 perturbed grid
    (n = 3000): the Hutchinson mean lies within 4 standard errors of the exact
    value from block selected inversion, which itself equals dense Eq. 1."""
    g = S.grid_perturbed(60, 50, 0.25, 9)
    k = O.K_block_tridiagonal(g, 60)
    assert k == pytest.approx(O.K_dense(g), rel=1e-10)
    mean, se, _ = O.K_hutchinson(g, 64, seed=3)
    assert abs(mean - k) <= 4 * se


def _nx(g):
    nx = pytest.importorskip("networkx")
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    src = np.repeat(np.arange(g.n), g.deg)
    G.add_edges_from((int(a), int(b)) for a, b in zip(src, g.col) if a < b)
    return nx, G


@pytest.mark.parametrize("name", ["er300", "grid8x6", "cl500", "K2,7", "rc9"])
def test_exact_K_equals_networkx(name):
    """Eq. 1 as the oracle evaluates it (dense normalised-Laplacian spectrum,
    and the grounded-Laplacian form) against networkx's independent
    kemeny_constant."""
    g = {"er300": lambda: S.er_lcc(300, 0.02, 7), "grid8x6": lambda: S.grid(8, 6),
         "cl500": lambda: S.chung_lu(500, 2.1, 6.0, 2),
         "K2,7": lambda: S.complete_bipartite(2, 7),
         "rc9": lambda: S.random_connected(9, 0.4, 5)}[name]()
    nx, G = _nx(g)
    k = nx.kemeny_constant(G)
    assert O.K_dense(g) == pytest.approx(k, rel=1e-9)
    assert O.K_grounded(g, 0) == pytest.approx(k, rel=1e-9)


def test_resistance_and_tree_count_equal_networkx():
    g = S.random_connected(10, 0.4, 8)
    nx, G = _nx(g)
    for u, v in [(0, 1), (2, 7), (3, 9)]:
        assert O.resistance(g, u, v) == pytest.approx(nx.resistance_distance(G, u, v), rel=1e-9)
    assert O.kirchhoff_count(g) == pytest.approx(float(nx.number_of_spanning_trees(G)), rel=1e-9)


@pytest.mark.parametrize("seed", [1, 2])
def test_sparse_resistance_matches_dense_and_series_rule(seed):
    """The sparse CG resistance equals the dense grounded inverse on random
    graphs (both orientations, pairs at any distance), and on a path graph it
    is the hop distance (resistors in series)."""
    g = S.random_connected(40, 0.12, seed)
    rng = np.random.default_rng(seed)
    for _ in range(6):
        u, v = (int(x) for x in rng.choice(g.n, 2, replace=False))
        d = O.resistance(g, u, v)
        assert O.resistance_sparse(g, u, v) == pytest.approx(d, rel=1e-10)
        assert O.resistance_sparse(g, v, u) == pytest.approx(d, rel=1e-10)
    p = S.path(30)
    assert O.resistance_sparse(p, 3, 17) == pytest.approx(14.0, rel=1e-10)
