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
    """The per-rank sums kc_stats reports, as Python numbers."""
    hi, lo = int(stats["f_sum_hi"]), int(stats["f_sum_lo"])
    return {"f_sum": hi * (1 << 64) + (lo & ((1 << 64) - 1)), "wf": float(stats["wf_sum"]),
            "w": float(stats["w_sum"]), "x2": float(stats["x2_sum"]),
            "count": int(stats["pool_trees"])}


def combine_pool_sums(local: dict, group=None) -> dict:
    """Exact cross-rank combination: the int128 f sums are gathered as limbs and
    added as Python integers; the FP64 sums are gathered and added in rank
    order, so every rank gets the same bits."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return dict(local)
    world = dist.get_world_size(group)
    f = int(local["f_sum"])
    limbs = [(f >> (32 * k)) & 0xFFFFFFFF for k in range(4)]  # two's complement, 128 bits
    t = torch.tensor(limbs + [local["count"]], dtype=torch.int64)
    ft = torch.tensor([local["wf"], local["w"], local["x2"]], dtype=torch.float64)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t, ft = t.to(dev), ft.to(dev)
    gi = [torch.empty_like(t) for _ in range(world)]
    gf = [torch.empty_like(ft) for _ in range(world)]
    dist.all_gather(gi, t, group=group)
    dist.all_gather(gf, ft, group=group)
    out = {"f_sum": 0, "wf": 0.0, "w": 0.0, "x2": 0.0, "count": 0}
    for a, b in zip(gi, gf):
        a = [int(x) for x in a.cpu().tolist()]
        v = sum(a[k] << (32 * k) for k in range(4))
        if v >= 1 << 127:
            v -= 1 << 128
        out["f_sum"] += v
        out["count"] += a[4]
        bf = b.cpu().tolist()
        out["wf"] += bf[0]
        out["w"] += bf[1]
        out["x2"] += bf[2]
    return out


def estimate_from_sums(sums: dict, twom: int, unit_weights: bool = True) -> float:
    """K_hat = sum f / (2m omega) (exact numerator) or sum w f / (2m sum w)."""
    if unit_weights:
        return sums["f_sum"] / (twom * sums["count"])
    return sums["wf"] / sums["w"]


def max_over_ranks(x: float, group=None) -> float:
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return x
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
