"""Writes er2000_K.txt: the exact Kemeny constant of the small static workload
graph (Erdos-Renyi G(2000, 8/1999), seed 0, largest component) by Eq. 1, the
sum of the reciprocals of the nonzero eigenvalues of the normalised Laplacian
I - D^-1/2 A D^-1/2 from an FP64 dense eigendecomposition (oracle.K_dense,
pinned against closed forms by tests/test_oracle_exact.py).  Calls only the
oracle and the seeded input generator; a few seconds.

    python tests/golden/make_er2000_K.py
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2511_16356_gb300 import synth as S  # noqa: E402


def main():
    g = S.workload("er2000")
    t = time.time()
    K = O.K_dense(g)
    el = time.time() - t
    with open(os.path.join(HERE, "er2000_K.txt"), "w") as f:
        f.write(f"# exact Kemeny constant (Eq. 1) of workload er2000 (n = {g.n}, m = {g.m}), "
                "FP64 dense eigendecomposition of the normalised Laplacian\n")
        f.write(f"# computed in {el:.0f} s by tests/golden/make_er2000_K.py\n")
        f.write(f"{K!r}\n")
    print(K, el)


if __name__ == "__main__":
    main()
