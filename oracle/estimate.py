"""The estimate K_hat and the rule that decides how many trees to draw.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Theorem 3 makes f(tau) / 2m an unbiased sample of the Kemeny constant, so the
estimate over w trees is their mean (Algorithm 1, last line), with the sum of
f kept as an exact integer.  The paper fixes the number of trees only through
Hoeffding's inequality (Theorem 5), which asks for far more trees than needed
in practice.  The rule used by default reads Theorem 5's (eps, delta)
guarantee through the normal approximation of the sample mean:

* draw a pilot of max(64, min(batch, cap)) trees;
* stop once w >= 64 and z s / sqrt(w) <= eps K_hat (1 - eps), where s is the
  sample standard deviation of f / 2m and z the upper delta/2 quantile of the
  standard normal (the factor 1 - eps keeps |K_hat - K| <= eps K when the
  interval holds around K rather than K_hat);
* otherwise draw max(batch, ceil((z s / tol)^2) - w) more trees, never past
  the cap, for at most 64 rounds.

Sums here are exact integers (Python ints and fractions), converted to floating
point only for the comparison and the square root, so each decision is the
exact one; ``margin`` reports how far the closest decision was from flipping.

``accepted_samples`` draws with rejection by walk length: trees whose Wilson
step count exceeds a cap are skipped, which leaves the accepted ones uniform
(its docstring gives the argument).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction
from statistics import NormalDist

import numpy as np

__all__ = ["z_upper", "EstimateRun", "estimate_clt", "estimate_fixed", "accepted_samples"]


def z_upper(p: float) -> float:
    """z with P(Z > z) = p for a standard normal Z (by symmetry, minus the
    lower p-quantile: 1 - p would round small tails away)."""
    return -NormalDist().inv_cdf(p)


@dataclass
class EstimateRun:
    K: float                 # K_hat = sum f / (2m w)
    trees: int               # w, trees drawn
    rounds: int              # stopping tests made
    margin: float = math.inf  # smallest relative distance of a decision from its threshold
    sizes: list = field(default_factory=list)  # trees drawn per batch


def estimate_fixed(f, twom: int) -> float:
    """K_hat of a fixed set of trees: the exact integer sum, divided once."""
    total = sum(int(x) for x in f)
    return total / (twom * len(f))


def estimate_clt(draw, twom: int, eps: float, delta: float, batch: int = 1024,
                 cap: int = 1 << 24) -> EstimateRun:
    """Run the normal-approximation stopping rule.

    draw(first, count) returns the f values of sample ids first .. first+count-1
    (any sampler keyed by sample id: the trees do not depend on the batching).
    """
    z = z_upper(delta / 2.0)
    f: list[int] = []
    sizes = []

    def more(count):
        vals = draw(len(f), count)
        f.extend(int(x) for x in np.asarray(vals).tolist())
        sizes.append(count)

    pilot = max(64, min(batch, cap))
    more(pilot)
    margin = math.inf
    rounds = 0
    for _ in range(64):
        rounds += 1
        w = len(f)
        sf = sum(f)
        sf2 = sum(x * x for x in f)
        mean = Fraction(sf, twom * w)
        var = Fraction(w * sf2 - sf * sf, twom * twom * w * max(1, w - 1))
        var = max(var, Fraction(0))
        sd = math.sqrt(float(var))
        tol = eps * float(mean) * (1.0 - eps)
        lhs = z * sd / math.sqrt(w)
        if tol > 0:
            margin = min(margin, abs(lhs - tol) / tol)
        if w >= 64 and lhs <= tol:
            break
        if w >= cap:
            break
        if tol > 0:
            q = (z * sd / tol) ** 2
            need = math.ceil(q)
            if need - w >= batch:  # the shortfall, not the batch, sets the next draw
                margin = min(margin, min(q - math.floor(q), math.ceil(q) - q) / max(q, 1.0))
        else:
            need = cap
        count = min(max(need - w, batch), cap - w)
        if count <= 0:
            break
        more(count)
    return EstimateRun(K=estimate_fixed(f, twom), trees=len(f), rounds=rounds, margin=margin,
                       sizes=sizes)


def accepted_samples(sample, cap: int, count: int, id0: int = 0, block: int = 1024):
    """Sampling with rejection by walk length: the first `count` sample ids,
    from id0 on, whose Wilson step count is at most `cap`, with their f and
    step counts.  sample(first, k) returns (f, steps) of ids first .. first+k-1.

    Rejection by step count leaves the accepted trees uniform.  Give every
    vertex a stack of independent uniform arrows; Wilson's walks pop cycles of
    arrows until the arrows on top form a tree T rooted at r (Sec. 2.2, with
    the cycle-popping view of Wilson's algorithm).  The probability that the
    popped cycles are C and the final tree is T is the product of the
    probabilities of the arrows involved: a factor for C times the product of
    1/d(v) over the non-root vertices, which is the same for every tree.  So T
    is uniform and independent of C, and the step count -- every popped arrow
    plus one arrow per non-root vertex -- is a function of C alone.  Any rule
    that accepts a tree according to its step count therefore keeps f(T)/2m an
    unbiased sample of K (Theorem 3)."""
    ids, fs, ss = [], [], []
    first = id0
    while len(ids) < count:
        f, steps = sample(first, block)
        for k in range(block):
            if steps[k] <= cap:
                ids.append(first + k)
                fs.append(int(f[k]))
                ss.append(int(steps[k]))
                if len(ids) == count:
                    break
        first += block
    return np.array(ids, dtype=np.int64), np.array(fs, dtype=np.int64), np.array(ss, dtype=np.int64)
