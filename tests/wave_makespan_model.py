"""Makespan of one wave of tree walks on the GPU's walker slots (test
infrastructure: a planning model, not a measurement).

Trees start in sample-id order on `slots` identical slots (resident one-warp
blocks of the 32-walker kernel) and each holds its slot for a time that grows
with its Wilson step count S as S^alpha (alpha > 1 because long walks keep few
walkers busy: tests/walker_protocol_model.py's tail study gives about 1.6 on a
100x100 grid).  With rejection by walk length, a tree whose S exceeds the cap X
stops at X departures and is replaced by the next sample id, until `need`
trees are accepted; oracle.accepted_samples and tests/test_oracle_rejection.py
show that the accepted trees stay uniform.

    python tests/wave_makespan_model.py 640      # S of 640 grid1000 trees from the oracle
"""
from __future__ import annotations

import heapq
import sys

import numpy as np


def makespan(durations, slots: int) -> float:
    """End of the last job when jobs start in order on the first free slot."""
    free = [0.0] * slots
    end = 0.0
    for d in durations:
        t = heapq.heappop(free) + float(d)
        end = max(end, t)
        heapq.heappush(free, t)
    return end


def wave_with_cap(s, need: int, slots: int, alpha: float, cap=None) -> float:
    """Makespan until `need` trees of the step counts s (in id order) are
    accepted; trees above `cap` cost cap^alpha and are not counted."""
    durations = []
    accepted = 0
    for v in s:
        if accepted >= need:
            break
        if cap is None or v <= cap:
            durations.append(v ** alpha)
            accepted += 1
        else:
            durations.append(cap ** alpha)
    if accepted < need:
        raise ValueError("not enough step counts for the accepted trees asked for")
    return makespan(durations, slots)


def main(trees: int):
    import oracle as O
    from paper_2511_16356_gb300 import synth as S

    g = S.workload("grid1000")
    t0 = O.tau0(g)
    _, steps = O.sample_batch(g, t0, 1, 0, trees)
    steps = steps.astype(np.float64)
    print(f"grid1000, {trees} trees: S median {np.median(steps):.3g}, q90 "
          f"{np.quantile(steps, 0.9):.3g}, max {steps.max():.3g}")
    rng = np.random.default_rng(0)
    for alpha in (1.0, 1.3, 1.6):
        ratios = {}
        for _ in range(5):
            s = rng.choice(steps, size=30000, replace=True)
            base = wave_with_cap(s, 10000, 3648, alpha)
            for q in (0.99, 0.95, 0.9, 0.8):
                ratios.setdefault(q, []).append(
                    wave_with_cap(s, 10000, 3648, alpha, np.quantile(steps, q)) / base)
        print(f"alpha {alpha}: walk time with the cap at the q-quantile of S, relative to no "
              f"cap: " + ", ".join(f"q{q:g} {np.mean(v):.2f}" for q, v in ratios.items()),
              flush=True)


if __name__ == "__main__":
    import os

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 640)
