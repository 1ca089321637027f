"""Writes grid1000_K.txt: the exact Kemeny constant (Eq. 1) of the 1000 x 1000
road-shaped workload graph, by FP64 block selected inversion of its grounded
Laplacian (oracle.K_block_tridiagonal; pinned against dense eigendecompositions
by tests/test_oracle_exact.py).  Calls only the oracle and the seeded input
generator.  About 10^13 flops and 9 GB of host memory.

    python tests/golden/make_grid1000_K.py
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2511_16356_gb300 import synth as S  # noqa: E402


def main():
    g = S.workload("grid1000")
    t = time.time()
    k = O.K_block_tridiagonal(g, 1000)
    el = time.time() - t
    with open(os.path.join(HERE, "grid1000_K.txt"), "w") as f:
        f.write("# exact Kemeny constant (Eq. 1) of workload grid1000 "
                f"(n = {g.n}, m = {g.m}), FP64 block selected inversion, r = n - 1\n")
        f.write(f"# computed in {el:.0f} s by tests/golden/make_grid1000_K.py\n")
        f.write(f"{k!r}\n")
    print(k, el)


if __name__ == "__main__":
    main()
