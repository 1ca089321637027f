"""Multi-rank host logic with two gloo ranks on the CPU: disjoint sample-id
ranges, exact combination of per-rank pool sums (the only cross-rank exchange
of the sharded path), max-over-ranks timing.  The per-rank pool values come
from the oracle, so no GPU is involved."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2511_16356_gb300 import dist as kd  # noqa: E402

PER_RANK = 40
IDS = 1000


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_sums(rank, world):
    import oracle as O
    from paper_2511_16356_gb300 import synth as S

    g = S.er_lcc(150, 0.04, 3)
    t0 = O.tau0(g)
    base = kd.rank_sample_base(rank, world, IDS)
    f, _ = O.sample_batch(g, t0, 9, base, PER_RANK, threads=1)
    twom = 2 * g.m
    x = f.astype(np.float64) / twom
    fs = int(sum(int(v) for v in f))
    return g, {"f_sum_hi": fs >> 64, "f_sum_lo": fs & ((1 << 64) - 1), "wf_sum": float(x.sum()),
               "w_sum": float(PER_RANK), "x2_sum": float((x * x).sum()), "count": PER_RANK}


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g, local = _rank_sums(rank, world)
    comb = kd.combine_pool_sums(local)
    k = kd.estimate_from_sums(comb, 2 * g.m)
    t = kd.max_over_ranks(float(rank + 1))
    q.put((rank, kd.f_sum(comb), comb["count"], k, t, kd.rank_sample_base(rank, world, IDS)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_exactly():
    import oracle as O
    from paper_2511_16356_gb300 import synth as S

    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    # both ranks agree on every combined value
    assert res[0][1:5] == res[1][1:5]
    assert res[0][4] == 2.0  # max over ranks
    assert [r[5] for r in res] == [0, IDS]
    # the combination equals the single-process computation over the union of ids
    g = S.er_lcc(150, 0.04, 3)
    t0 = O.tau0(g)
    fa, _ = O.sample_batch(g, t0, 9, 0, PER_RANK, threads=1)
    fb, _ = O.sample_batch(g, t0, 9, IDS, PER_RANK, threads=1)
    want = sum(int(v) for v in fa) + sum(int(v) for v in fb)
    assert res[0][1] == want and res[0][2] == 2 * PER_RANK
    assert res[0][3] == pytest.approx(want / (2 * g.m * 2 * PER_RANK), rel=1e-15)


def _sums(v, count=1, wf=0.0, w=1.0, x2=0.0):
    return {"f_sum_hi": v >> 64, "f_sum_lo": v & ((1 << 64) - 1), "wf_sum": wf, "w_sum": w,
            "x2_sum": x2, "count": count}


def test_c_combination_is_exact_for_negative_and_large_sums():
    """kc_combine_sums adds the int128 limbs exactly (carries across the low
    limb, negative values) and the counts; kc_estimate_from_sums divides the
    exact sum once."""
    from paper_2511_16356_gb300 import build as kbuild
    from paper_2511_16356_gb300 import kc

    kbuild.build()
    vals = [0, 1, -1, (1 << 100) + 12345, -(1 << 90) - 7, (1 << 64) - 1, 1 << 63]
    parts = [kd._as_struct(_sums(v, count=3)) for v in vals]
    arr = (kc.kc_pool_sums * len(parts))(*parts)
    out = kc.kc_pool_sums()
    import ctypes

    assert kc.load().kc_combine_sums(arr, len(parts), ctypes.byref(out)) == 0
    comb = kd._as_dict(out)
    assert kd.f_sum(comb) == sum(vals) and comb["count"] == 3 * len(vals)
    k = kd.estimate_from_sums(_sums(10 ** 20 + 7, count=9), 2 * 1000)
    assert k == (10 ** 20 + 7) / (2000 * 9)
    assert kd.estimate_from_sums(_sums(0, count=2, wf=3.0, w=4.0), 10, unit_weights=False) == 0.75
    # an int128 overflow is refused
    big = [kd._as_struct(_sums((1 << 126) + 1)), kd._as_struct(_sums((1 << 126) + 1))]
    arr2 = (kc.kc_pool_sums * 2)(*big)
    assert kc.load().kc_combine_sums(arr2, 2, ctypes.byref(out)) == 1


def test_rank_bases_are_disjoint_and_bounded():
    assert kd.rank_sample_base(3, 8) == 3 << 28
    with pytest.raises(ValueError):
        kd.rank_sample_base(0, 17)
