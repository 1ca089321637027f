"""Writes cl4m_K.txt: a reference Kemeny constant of the power-law workload
graph (Chung-Lu, gamma 2.1, n = 4M, mean degree 17, largest component), by
Hutchinson's estimator on the pseudo-inverse of the normalised Laplacian
(oracle.K_hutchinson, 64 Rademacher probes, FP64 CG to 1e-10; pinned against
dense K by tests/test_oracle_exact.py), with its standard error.  No exact
method is affordable at this size.  Calls only the oracle and the seeded input
generator; a few minutes and ~10 GB of host memory.

    python tests/golden/make_cl4m_K.py
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2511_16356_gb300 import synth as S  # noqa: E402

PROBES, SEED = 64, 11


def main():
    g = S.workload("cl4m")
    t = time.time()
    mean, se, _ = O.K_hutchinson(g, PROBES, SEED)
    el = time.time() - t
    with open(os.path.join(HERE, "cl4m_K.txt"), "w") as f:
        f.write("# reference Kemeny constant of workload cl4m "
                f"(n = {g.n}, m = {g.m}): Hutchinson mean over {PROBES} Rademacher probes "
                f"(seed {SEED}) and its standard error\n")
        f.write(f"# computed in {el:.0f} s by tests/golden/make_cl4m_K.py\n")
        f.write(f"{mean!r} {se!r}\n")
    print(mean, se, el)


if __name__ == "__main__":
    main()
