"""Pins of the oracle's stopping rule (oracle/estimate.py), the normal-
approximation reading of Theorem 5's (eps, delta) guarantee.

* The normal quantiles against printed table values.
* A sequence worked by hand: f alternating 900, 1100 with 2m = 1000.
* Degenerate runs: zero variance stops after the pilot; the cap bounds the pool.
* The guarantee itself: over 200 seeds on graphs with an exact Kemeny
  constant, the share of estimates off by more than eps K stays within three
  binomial standard deviations of delta.
"""
import math

import pytest

import oracle as O
from paper_2511_16356_gb300 import synth as S


def test_normal_quantiles_match_table_values():
    assert O.z_upper(0.025) == pytest.approx(1.959963984540054, rel=1e-12)
    assert O.z_upper(0.005) == pytest.approx(2.5758293035489004, rel=1e-12)
    assert O.z_upper(0.05) == pytest.approx(1.6448536269514722, rel=1e-12)
    assert abs(O.z_upper(0.5)) < 1e-15


def _alternating(first, count):
    return [900 if (first + i) % 2 == 0 else 1100 for i in range(count)]


def test_alternating_sequence_worked_by_hand():
    """2m = 1000, eps = 0.01, delta = 0.05 (z = 1.959964), batch 64.
    Pilot of 64: mean 1, variance 0.64 / 63, s = 0.100790; z s / 8 = 0.024693 is
    above tol = 0.01 * 1 * 0.99 = 0.0099, and (z s / tol)^2 = 398.17, so 399 - 64
    = 335 more trees.  At 399 trees (200 of 900, 199 of 1100): mean 0.99975,
    s = 0.100119, z s / sqrt(399) = 0.0098236 <= tol = 0.0098975: stop.
    K_hat = 398900 / 399000."""
    r = O.estimate_clt(_alternating, 1000, 0.01, 0.05, batch=64)
    assert r.sizes == [64, 335] and r.trees == 399 and r.rounds == 2
    assert r.K == 398900 / 399000


def test_zero_variance_stops_after_the_pilot():
    g = S.complete(2)  # one spanning tree: f = 1 always
    t0 = O.tau0(g)

    def draw(a, c):
        return O.sample_batch(g, t0, 3, a, c)[0]

    for batch, pilot in [(64, 64), (10, 64), (1024, 1024)]:
        r = O.estimate_clt(draw, 2 * g.m, 0.01, 0.05, batch=batch)
        assert r.trees == pilot and r.rounds == 1 and r.K == 0.5


def test_cap_bounds_the_pool():
    r = O.estimate_clt(_alternating, 1000, 0.001, 0.05, batch=64, cap=100)
    assert r.sizes == [64, 36] and r.trees == 100
    r = O.estimate_clt(_alternating, 1000, 0.001, 0.05, batch=64, cap=50)
    assert r.trees == 64  # the pilot is at least 64 trees


@pytest.mark.parametrize("name,eps,delta", [("er300", 0.01, 0.05), ("grid12x10", 0.02, 0.1)])
def test_coverage_over_seeds(name, eps, delta):
    g = {"er300": lambda: S.er_lcc(300, 0.02, 7),
         "grid12x10": lambda: S.grid_perturbed(12, 10, 0.2, 3)}[name]()
    t0 = O.tau0(g)
    k_exact = O.K_dense(g)
    runs = 200
    misses = 0
    trees = []
    for seed in range(runs):
        r = O.estimate_clt(lambda a, c: O.sample_batch(g, t0, seed, a, c)[0], 2 * g.m, eps, delta,
                           batch=64)
        misses += abs(r.K - k_exact) > eps * k_exact
        trees.append(r.trees)
    assert misses <= delta * runs + 3 * math.sqrt(delta * (1 - delta) * runs)
    # the pool size tracks the normal-approximation size (z sigma / (eps K))^2
    f, _ = O.sample_batch(g, t0, 10 ** 6, 0, 20000)
    x = f / (2 * g.m)
    want = (O.z_upper(delta / 2) * x.std() / (eps * k_exact * (1 - eps))) ** 2
    assert 0.8 * want < sum(trees) / runs < 1.25 * want + 64
