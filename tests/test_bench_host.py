"""Host-side pieces of bench.py that need no GPU: the algorithmic byte model,
the serving workload generator, the reference arm (the CPU oracle timed on the
host cores) and the shape of its JSON line."""
import json
import math
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_model():
    n, trees, steps = 1000, 10, 123456
    assert bench.algorithmic_bytes("wilson", n, 5, trees, steps) == 32 * (2 * steps + 3 * n * trees)
    assert bench.algorithmic_bytes("traverse", n, 5, trees, steps) == 32 * 6 * n * trees
    lg = math.log2(n)
    assert bench.algorithmic_bytes("ttf_bit", n, 5, trees, steps) == \
        32 * (3 * lg + 4) * n * trees
    assert bench.algorithmic_bytes("ttf_scan", n, 7, trees, steps) == 32 * 2 * 7 * n * trees
    assert bench.algorithmic_bytes("other", n, 7, trees, steps) == 0.0
    # the whole path: walk + traversal + the f variant in use
    assert bench.path_bytes(n, 5, True, trees, steps) == \
        32 * (2 * steps + 3 * n * trees) + 32 * 6 * n * trees + 32 * (3 * lg + 4) * n * trees
    assert bench.path_bytes(n, 7, False, trees, steps) == \
        32 * (2 * steps + 3 * n * trees) + 32 * 6 * n * trees + 32 * 2 * 7 * n * trees


def test_serving_workload_is_seeded_and_mixed():
    a = bench.serve_workload(6, 5000)
    b = bench.serve_workload(6, 5000)
    assert [g.n for g in a] == [g.n for g in b]
    assert all(np.array_equal(x.col, y.col) for x, y in zip(a, b))
    assert all(1 <= g.n <= 5000 for g in a)
    # ER, perturbed grid, Chung-Lu in turn: grids have maximum degree 4
    assert max(a[1].deg) <= 4 and max(a[2].deg) > 4
    # generation in spawned processes gives the same graphs
    c = bench.serve_workload(6, 5000, procs=2)
    assert all(np.array_equal(x.col, y.col) and np.array_equal(x.row_off, y.row_off)
               for x, y in zip(a, c))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "er2000", "--steps", "2", "--warmup", "3",
                          "--ref-trees", "8"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    d = json.loads(lines[-1])
    assert d["impl"] == "reference" and d["metric"] == "trees/sec" and d["unit"] == "trees/s"
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["higher_is_better"] is True


def test_single_core_oracle_baseline_and_cpu_model():
    from paper_2511_16356_gb300 import synth as S

    d = bench.single_core_baseline(S.workload("er2000"), 1, budget_s=0.5)
    assert d["cores"] == 1 and d["value"] > 0 and d["unit"] == "trees/s"
    assert isinstance(bench.host_cpu_model(), str) and bench.host_cpu_model()


def test_cpu_model_on_arm_hosts(tmp_path):
    info = tmp_path / "cpuinfo"
    info.write_text("processor\t: 0\nBogoMIPS\t: 2000.00\nCPU implementer\t: 0x41\n"
                    "CPU architecture: 8\nCPU variant\t: 0x0\nCPU part\t: 0xd4f\n\n")
    assert bench.host_cpu_model(str(info)).endswith("Arm Neoverse V2")
    info.write_text("processor\t: 0\nmodel name\t: Some x86 CPU @ 2.00GHz\n")
    assert bench.host_cpu_model(str(info)) == "Some x86 CPU @ 2.00GHz"


def test_reference_arm_under_torchrun_two_ranks():
    """The multi-rank launch of the reference arm: rank 0 alone prints one
    line (the other rank exits without work), and the oracle runs on every
    host core although the launcher sets OMP_NUM_THREADS=1."""
    import random

    port = str(random.randint(20000, 40000))
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                          "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                          "--master-port", port, os.path.join(ROOT, "bench.py"),
                          "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
                          "--ref-trees", "8", "--workload", "er2000"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["cores"] == bench.host_cores()


def test_update_stream_is_valid_against_the_evolving_graph():
    """Every insertion adds an absent edge and every deletion removes a present
    edge that is not a bridge (the graph stays connected); the stream is
    seeded and has the requested size."""
    from collections import deque

    from paper_2511_16356_gb300 import synth as S

    g = S.chung_lu(400, 2.1, 6.0, 4)
    a = bench.update_stream(g, 300, 40, seed=4)
    b = bench.update_stream(g, 300, 40, seed=4)
    assert a == b and sum(len(x) for x in a) == 300 and max(len(x) for x in a) <= 40
    adj = [set(g.col[g.row_off[v]:g.row_off[v + 1]].tolist()) for v in range(g.n)]

    def connected(u, v):
        seen, q = {u}, deque([u])
        while q:
            x = q.popleft()
            if x == v:
                return True
            for y in adj[x]:
                if y not in seen:
                    seen.add(y)
                    q.append(y)
        return False

    kinds = set()
    for batch in a:
        for u, v, op in batch:
            kinds.add(op)
            if op == 0:
                assert u != v and v not in adj[u]
                adj[u].add(v)
                adj[v].add(u)
            else:
                assert v in adj[u]
                adj[u].discard(v)
                adj[v].discard(u)
                assert connected(u, v)
    assert kinds == {0, 1}
