"""Multi-GPU plumbing: one process per GPU, trees sharded by sample id.

Trees are independent (Algorithm 1 samples them one by one), so ranks draw
disjoint sample-id ranges from the same seed and the graph is replicated; the
only exchange is combining the per-rank pool sums for a joint estimate
(exact int128 sum of f, FP64 sums of w f / 2m, w and (f / 2m)^2, tree count).
torch.distributed carries the exchange (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

IDS_PER_RANK = 1 << 28  # ranks' sample-id ranges [rank * IDS_PER_RANK, ...) below 2^32


def rank_sample_base(rank: int, world: int, ids_per_rank: int = IDS_PER_RANK) -> int:
    if world * ids_per_rank > (1 << 32):
        raise ValueError("sample ids must stay below 2^32")
    return rank * ids_per_rank


def pool_sums(stats: dict) -> dict:
    """The per-rank sums kc_stats reports (the fields of kc_pool_sums)."""
    return {k: stats[k] for k in ("f_sum_hi", "f_sum_lo", "wf_sum", "w_sum", "x2_sum")} | \
        {"count": int(stats["pool_trees"])}


def _as_struct(d: dict):
    from . import kc

    return kc.kc_pool_sums(int(d["f_sum_hi"]), int(d["f_sum_lo"]) & ((1 << 64) - 1),
                           float(d["wf_sum"]), float(d["w_sum"]), float(d["x2_sum"]),
                           int(d["count"]))


def _as_dict(s) -> dict:
    return {k: getattr(s, k) for k, _ in s._fields_}


def combine_pool_sums(local: dict, group=None) -> dict:
    """Every rank's kc_pool_sums gathered (the int128 f sum travels as its two
    64-bit limbs, the FP64 sums bit for bit) and combined by kc_combine_sums,
    which adds f exactly and the FP64 sums in rank order, so every rank gets the
    same bits.  Without an initialised process group: this rank's sums."""
    import ctypes

    import torch
    import torch.distributed as dist

    from . import kc

    if not dist.is_available() or not dist.is_initialized():
        parts = [_as_struct(local)]
    else:
        world = dist.get_world_size(group)
        ls = _as_struct(local)
        lo_signed = ls.f_sum_lo - (1 << 64) if ls.f_sum_lo >= (1 << 63) else ls.f_sum_lo
        t = torch.tensor([ls.f_sum_hi, lo_signed, ls.count], dtype=torch.int64)
        ft = torch.tensor([ls.wf_sum, ls.w_sum, ls.x2_sum], dtype=torch.float64)
        dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        t, ft = t.to(dev), ft.to(dev)
        gi = [torch.empty_like(t) for _ in range(world)]
        gf = [torch.empty_like(ft) for _ in range(world)]
        dist.all_gather(gi, t, group=group)
        dist.all_gather(gf, ft, group=group)
        parts = []
        for a, b in zip(gi, gf):
            hi, lo, cnt = (int(x) for x in a.cpu().tolist())
            wf, w, x2 = b.cpu().tolist()
            parts.append(kc.kc_pool_sums(hi, lo & ((1 << 64) - 1), wf, w, x2, cnt))
    arr = (kc.kc_pool_sums * len(parts))(*parts)
    out = kc.kc_pool_sums()
    kc._check(kc.load().kc_combine_sums(arr, len(parts), ctypes.byref(out)), "kc_combine_sums")
    return _as_dict(out)


def estimate_from_sums(sums: dict, twom: int, unit_weights: bool = True) -> float:
    """K_hat of (combined) pool sums, computed by kc_estimate_from_sums."""
    import ctypes

    from . import kc

    k = ctypes.c_double()
    kc._check(kc.load().kc_estimate_from_sums(ctypes.byref(_as_struct(sums)), int(twom),
                                             1 if unit_weights else 0, ctypes.byref(k)),
             "kc_estimate_from_sums")
    return k.value


def f_sum(sums: dict) -> int:
    """The exact int128 sum of f as a Python integer (for reporting)."""
    return int(sums["f_sum_hi"]) * (1 << 64) + (int(sums["f_sum_lo"]) & ((1 << 64) - 1))


def max_over_ranks(x: float, group=None) -> float:
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return x
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
