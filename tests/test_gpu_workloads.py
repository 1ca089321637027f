"""GPU tests at the workloads' full sizes: the estimate against exact or
reference Kemeny constants (within the requested relative error), coverage of
the stopping rule over 20 seeds, and bit-exact trees on sampled ids of the
road-shaped and power-law graphs.

Reference values: tests/golden/grid1000_K.txt (exact, block selected
inversion), tests/golden/cl4m_K.txt (Hutchinson mean and standard error),
closed forms for the torus and the hypercube (Eq. 1 with their spectra).
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2511_16356_gb300 import synth as S

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("KC_SKIP_LARGE") == "1",
                                 reason="large workloads disabled")]

kc = pytest.importorskip("paper_2511_16356_gb300.kc")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2511_16356_gb300 import build as kbuild

    kbuild.build()
    kc.load()


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    return [float(x) for x in rows[0]]


def _cfg(**kw):
    c = kc.kc_config_default()
    c.keep_trees = 0
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _estimate(g, eps, delta, seed, **kw):
    with kc.KemenyGraph.from_graph(g, _cfg(**kw)) as G:
        G.sample(seed, 64)
        k = G.estimate(eps, delta)
        return k, G.stats()["pool_trees"]


def test_grid1000_estimate_within_eps_of_exact():
    """Road-shaped workload: K_hat at eps = 1%, delta = 1% against the exact K."""
    g = S.workload("grid1000")
    (k_exact,) = _golden("grid1000_K.txt")
    k, trees = _estimate(g, 0.01, 0.01, 3, step_cap=256 * g.n)
    assert abs(k - k_exact) / k_exact <= 0.01, (k, k_exact, trees)


def test_cl4m_estimate_within_eps_of_reference():
    """Power-law workload: K_hat at eps = 1%, delta = 1% against the Hutchinson
    reference (its own standard error added to the tolerance)."""
    g = S.workload("cl4m")
    k_ref, se = _golden("cl4m_K.txt")
    k, trees = _estimate(g, 0.01, 0.01, 4)
    assert abs(k - k_ref) <= 0.01 * k_ref + 4 * se, (k, k_ref, se, trees)


@pytest.mark.parametrize("name", ["torus500x500", "Q20"])
def test_closed_form_graphs_at_scale(name):
    """2-D torus (high eccentricity) and hypercube Q_20 (low eccentricity, one
    million vertices): K_hat at eps = 1%, delta = 1% against closed forms."""
    if name == "Q20":
        g, k_exact = S.hypercube(20), O.K_hypercube(20)
    else:
        g, k_exact = S.torus(500, 500), O.K_torus(500, 500)
    k, trees = _estimate(g, 0.01, 0.01, 5, step_cap=256 * g.n)
    assert abs(k - k_exact) / k_exact <= 0.01, (k, k_exact, trees)


def test_er2000_coverage_over_20_seeds():
    """Small workload: over 20 seeds the eps = 1%, delta = 5% estimate misses
    the exact K at most 3 times (P[Binomial(20, 0.05) >= 4] < 2%)."""
    g = S.workload("er2000")
    k_exact = O.K_dense(g)
    errs = []
    for seed in range(20):
        k, _ = _estimate(g, 0.01, 0.05, 1000 + seed)
        errs.append(abs(k - k_exact) / k_exact)
    assert sum(e > 0.01 for e in errs) <= 3, errs


def _sampled_ids_parity(g, bases, per_base, step_cap):
    t0 = O.tau0(g)
    for base in bases:
        with kc.KemenyGraph.from_graph(g, _cfg(sample_id_base=base, step_cap=step_cap)) as G:
            G.sample(1, per_base)
            got = G.samples()
        assert np.array_equal(got["sid"], base + np.arange(per_base))
        f_ref, st_ref = O.sample_batch(g, t0, 1, base, per_base)
        assert np.array_equal(got["steps"], st_ref), base
        assert np.array_equal(got["f"], f_ref), base


def _random_bases(seed, count, per_base):
    rng = np.random.default_rng(seed)
    return [0] + [int(b) for b in rng.integers(1, (1 << 32) - per_base, size=count)]


def test_grid1000_ids_0_255_and_random_ids_bit_exact():
    """Road-shaped workload: sample ids 0..255 and 4 x 64 seeded-random ids,
    f and Wilson step counts equal to the oracle's."""
    g = S.workload("grid1000")
    bases = _random_bases(7, 4, 64)
    _sampled_ids_parity(g, bases[:1], 256, 256 * g.n)
    _sampled_ids_parity(g, bases[1:], 64, 256 * g.n)


def test_cl4m_ids_0_255_and_random_ids_bit_exact():
    """Power-law workload: sample ids 0..255 and 4 x 64 seeded-random ids."""
    g = S.workload("cl4m")
    bases = _random_bases(8, 4, 64)
    _sampled_ids_parity(g, bases[:1], 256, 0)
    _sampled_ids_parity(g, bases[1:], 64, 0)
