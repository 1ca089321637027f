"""Benchmark of the TTF Kemeny-constant hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload grid1000] [--trees T]
    python bench.py --impl reference ...   # the CPU oracle on the host cores

A step is one pass of the sampling hot path over one batch of T trees: Wilson
walks, per-tree traversal (size, volume, DFN), f(tau) and the pool reduction
(kc_sample).  Metric: spanning trees per second, whole job (all ranks).  Multi-GPU
runs shard sample ids across ranks (weak scaling, no collective on the data
path); the time is the maximum over ranks.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L2_BYTES = 129 * 1024 * 1024
SECTOR = 32


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.t is not None:
            self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) < 9:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def algorithmic_bytes(phase: str, n: int, ecc: int, trees: int, steps: int) -> float:
    """Bytes the method must move per launch batch (32-byte sectors):
    wilson   2 sectors per departure (vertex record; walker word of u, whose line
             also answers the in-tree test of the next vertex) + 3 per committed vertex;
    traverse 6 sectors per vertex (three passes, two gathers each);
    ttf_bit  (3 log2 n + 4) sectors per vertex (query, add, undo chains);
    ttf_scan 2 ecc sectors per vertex (tau0 ancestor walk)."""
    lg = math.log2(max(n, 2))
    if phase == "wilson":
        return SECTOR * (2.0 * steps + 3.0 * n * trees)
    if phase == "traverse":
        return SECTOR * 6.0 * n * trees
    if phase == "ttf_bit":
        return SECTOR * (3.0 * lg + 4.0) * n * trees
    if phase == "ttf_scan":
        return SECTOR * 2.0 * ecc * n * trees
    return 0.0


def path_bytes(n: int, ecc: int, bit: bool, trees: int, steps: int) -> float:
    """Algorithmic bytes of the whole sampling path for `trees` trees with
    `steps` Wilson departures in all: walk, traversal and f(tau)."""
    ttf = "ttf_bit" if bit else "ttf_scan"
    return sum(algorithmic_bytes(ph, n, ecc, trees, steps) for ph in ("wilson", "traverse", ttf))


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        return dist, rank, ws, local
    return None, rank, ws, local


def reduce_max(dist, x: float) -> float:
    from paper_2511_16356_gb300.dist import max_over_ranks

    return x if dist is None else max_over_ranks(x)


def barrier(dist):
    if dist is not None:
        dist.barrier()


def host_cores() -> int:
    """Host cores this process may run on (launchers such as torchrun set
    OMP_NUM_THREADS=1, which would otherwise confine the oracle to one core)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_baseline(g, trees: int, seed: int, threads: int = 0, first: int = 0):
    """The CPU oracle as it stands: Wilson + traversal + Algorithm 1 over a
    bounded sample of sample ids, OpenMP across trees on all host cores
    (threads = 0) or on `threads` of them."""
    import oracle as O

    if threads <= 0:
        threads = host_cores()
    t0 = O.tau0(g)
    t = time.perf_counter()
    f, steps = O.sample_batch(g, t0, seed, first, trees, threads=threads)
    el = time.perf_counter() - t
    return trees / el, el, threads


# Arm cores by (implementer, part) of the main ID register, as /proc/cpuinfo
# prints them on aarch64 hosts, which give no model name
ARM_PARTS = {("0x41", "0xd0c"): "Arm Neoverse N1", ("0x41", "0xd40"): "Arm Neoverse V1",
             ("0x41", "0xd49"): "Arm Neoverse N2", ("0x41", "0xd4f"): "Arm Neoverse V2",
             ("0x41", "0xd84"): "Arm Neoverse V3"}


def host_cpu_model(cpuinfo: str = "/proc/cpuinfo") -> str:
    """The host CPU as /proc/cpuinfo names it: the model name on x86, the core
    type from the implementer and part numbers on Arm, else the architecture."""
    import platform

    fields = {}
    try:
        with open(cpuinfo) as f:
            for line in f:
                if ":" not in line:
                    continue
                key, val = (x.strip() for x in line.split(":", 1))
                fields.setdefault(key.lower(), val)
    except OSError:
        pass
    for key in ("model name", "cpu model", "hardware"):
        if fields.get(key):
            return fields[key]
    impl, part = fields.get("cpu implementer", "").lower(), fields.get("cpu part", "").lower()
    if impl and part:
        name = ARM_PARTS.get((impl, part), f"implementer {impl} part {part}")
        return f"{platform.machine()} {name}"
    return platform.machine()


def single_core_baseline(g, seed: int, budget_s: float = 5.0) -> dict:
    """The oracle on one core: a small calibration batch, then batches sized
    from the rate seen so far until about `budget_s` seconds of trees."""
    trees, el, batch = 0, 0.0, 2
    for _ in range(4):
        _, e, _ = oracle_baseline(g, batch, seed, threads=1, first=trees)
        trees, el = trees + batch, el + e
        if el >= budget_s / 2:
            break
        batch = int(min(1 << 20, max(1, batch / max(e, 1e-3) * (budget_s - el))))
    return {"value": trees / el, "unit": "trees/s", "cores": 1,
            "sample": f"{trees} trees (sample ids 0..{trees - 1}), {el:.1f} s"}


def run_reference(args):
    """--impl reference: the oracle timed on the host cores, same metric/config."""
    dist, rank, ws, _ = dist_setup()
    if rank != 0:
        return
    from paper_2511_16356_gb300 import synth as S

    g = S.workload(args.workload)
    per_step = args.ref_trees
    for _ in range(args.warmup):
        oracle_baseline(g, per_step, args.seed)
    times = []
    cores = 1
    for _ in range(args.steps):
        _, el, cores = oracle_baseline(g, per_step, args.seed)
        times.append(el)
    tot = sum(times)
    value = per_step * args.steps / tot
    line = {
        "impl": "reference",
        "metric": "trees/sec", "value": value, "unit": "trees/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": S.WORKLOADS.get(args.workload, args.workload),
                   "trees_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": "trees/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} trees (sample ids 0..{per_step - 1}) per step "
                                   f"of {args.workload}, OpenMP across trees",
                         "cpu": host_cpu_model()},
        "e2e": {"value": value, "unit": "trees/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


WALKER_NAMES = {1: "lane", 2: "warp", 3: "hybrid"}


def golden_K(workload: str):
    """The stored reference Kemeny constant of a workload (tests/golden/, written
    by committed scripts that call only the oracle): (K, standard error), the
    error 0 for exact values; None when no value is stored."""
    fn = os.path.join(ROOT, "tests", "golden", f"{workload}_K.txt")
    if not os.path.exists(fn):
        return None
    for line in open(fn):
        line = line.strip()
        if line and not line.startswith("#"):
            vals = [float(x) for x in line.split()]
            return vals[0], (vals[1] if len(vals) > 1 else 0.0)
    return None


def timed_sampling(G, T: int, steps: int, seed: int, stream, flush) -> list:
    """`steps` timed kc_sample calls of T trees each, L2 flushed before each;
    CUDA events on the handle's stream.  Returns the per-step milliseconds."""
    import torch

    step_ms = []
    for _ in range(steps):
        flush.fill_(1)  # evict L2 between timed steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G.sample(seed, T)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    return step_ms


def phase_roofline(kc, st: dict, n: int, trees: int, steps_total: int, tot_ms: float,
                   walker_traffic=None) -> tuple:
    """The dominant phase of the timed steps (kc_stats' CUDA-event phase timers)
    and its roofline object: algorithmic bytes per launch over the mean launch
    time, against the measured HBM copy peak; plus the whole path's fraction."""
    bit = st["ttf_variant"] == kc.KC_TTF_BIT
    phases = {
        "wilson": (st["ms_wilson"], st["launches_wilson"]),
        "traverse": (st["ms_traverse"], st["launches_traverse"]),
        "ttf_bit" if bit else "ttf_scan": (st["ms_ttf"], st["launches_ttf"]),
    }
    dom = max(phases, key=lambda k: phases[k][0])
    dom_ms, dom_launches = phases[dom]
    alg = algorithmic_bytes(dom, n, st["ecc"], trees, steps_total)
    peak, peak_kind = _peaks()
    per_launch_bytes = alg / max(1, dom_launches)
    per_launch_s = max(dom_ms, 1e-9) / 1000.0 / max(1, dom_launches)
    achieved = per_launch_bytes / per_launch_s / 1e9
    kernel_name = {"wilson": {kc.KC_WALK_LANE: "k_wilson", kc.KC_WALK_WARP: "k_wilson_warp",
                              kc.KC_WALK_HYBRID: "k_wilson+k_wilson_warp"}[st["walker"]],
                   "traverse": "traversal passes",
                   "ttf_bit": "k_ttf_bit", "ttf_scan": "k_ttf_scan"}[dom]
    traffic = None
    if walker_traffic is not None and dom == "wilson":
        traffic = walker_traffic * steps_total / max(1, dom_launches)
    roof = {"bound": "hbm", "kernel": kernel_name, "achieved": achieved, "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic,
            "algorithmic_bytes_per_launch": per_launch_bytes,
            "mean_launch_ms": per_launch_s * 1000.0,
            # the whole sampling path over the timed steps (walk, traversal,
            # f), against the same peak
            "path_frac": path_bytes(n, st["ecc"], bit, trees, steps_total)
                         / (tot_ms / 1000.0) / 1e9 / peak}
    phase_ms = {k: round(v[0], 3) for k, v in phases.items()}
    phase_ms["wave_init"] = round(st["ms_wave_init"], 3)
    phase_ms["reduce"] = round(st["ms_reduce"], 3)
    return dom, roof, phase_ms


def time_to_eps(kc, g, cfg, eps: float, delta: float, batch: int, stream, workload: str) -> dict:
    """Wall time of kc_estimate(eps, delta) on a fresh handle (tau0 precomputed,
    inputs resident), the trees it drew, K_hat and its error against the stored
    reference."""
    import torch

    cfg2 = kc.kc_config_default()
    for f, _ in kc.kc_config._fields_:
        setattr(cfg2, f, getattr(cfg, f))
    cfg2.batch_trees = batch
    H = kc.KemenyGraph.from_graph(g, cfg2, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t = time.perf_counter()
    k_hat = H.estimate(eps, delta)
    tte = time.perf_counter() - t
    sh = H.stats()
    drawn = H.samples(0, sh["pool_trees"])
    peak, _ = _peaks()
    tte_bytes = path_bytes(g.n, sh["ecc"], sh["ttf_variant"] == kc.KC_TTF_BIT,
                           sh["pool_trees"], int(drawn["steps"].sum()))
    H.close()
    out = {"value": tte, "unit": "s", "eps": eps, "delta": delta, "trees": sh["pool_trees"],
           "K": k_hat, "batch_trees": int(batch),
           "roofline_frac": tte_bytes / tte / 1e9 / peak,
           "rule": "CLT: z s/sqrt(w) <= eps K (1-eps)"}
    ref = golden_K(workload)
    if ref is not None:
        out["K_ref"] = ref[0]
        out["K_ref_se"] = ref[1]
        out["rel_err"] = (k_hat - ref[0]) / ref[0]
    return out


def other_workload_leg(args, kc, stream, flush, name: str, T: int, steps: int, warmup: int,
                       delta: float) -> dict:
    """A further static workload at its stated size: trees/s over `steps` timed
    kc_sample calls of T trees (after `warmup` untimed ones), the dominant
    kernel's roofline, and time to eps with K_hat against the stored reference."""
    import torch

    from paper_2511_16356_gb300 import synth as S

    g = S.workload(name)
    cfg = kc.kc_config_default()
    cfg.keep_trees = 0
    cfg.autotune = 1  # the first warm-up call times both walkers and keeps the faster
    G = kc.KemenyGraph.from_graph(g, cfg, stream=stream.cuda_stream)
    G.reserve(T * (warmup + steps))
    for _ in range(warmup):
        G.sample(args.seed, T)
    torch.cuda.synchronize()
    kc.kc_reset_timers(G.h)
    pool0 = G.stats()["pool_trees"]
    step_ms = timed_sampling(G, T, steps, args.seed, stream, flush)
    tot_ms = float(sum(step_ms))
    st = G.stats()
    smp = G.samples(pool0, st["pool_trees"] - pool0)
    steps_total = int(smp["steps"].sum())
    dom, roof, phase_ms = phase_roofline(kc, st, g.n, T * steps, steps_total, tot_ms)
    G.close()
    out = {"workload": S.WORKLOADS.get(name, name), "n": g.n, "m": g.m, "ecc": st["ecc"],
           "trees_per_step": T, "steps": steps, "warmup": warmup,
           "value": T * steps / (tot_ms / 1000.0), "unit": "trees/s",
           "ms_per_step": tot_ms / steps, "roofline": roof, "phase_ms": phase_ms,
           "steps_per_tree": steps_total / (T * steps),
           "ttf": "BIT" if st["ttf_variant"] == kc.KC_TTF_BIT else "SCAN",
           "walker": WALKER_NAMES[st["walker"]], "autotune_ms": st["tune_ms"]}
    # time to eps with the walker the autotuner chose (no tuning inside the timing)
    cfg.autotune = 0
    cfg.walker = st["walker"]
    out["time_to_eps"] = time_to_eps(kc, g, cfg, args.eps, delta, 1024, stream, name)
    return out



def _serve_graph(spec):
    """One graph of the serving mix (module level, so a spawned pool can run it)."""
    from paper_2511_16356_gb300 import synth as S

    kind, n, seed = spec
    if kind == 0:
        return S.er_lcc(n, 8.0 / n, seed)
    if kind == 1:
        w = max(8, int(np.sqrt(n)))
        return S.grid_perturbed(w, max(8, n // w), 0.25, seed)
    return S.chung_lu(n, 2.1, 10.0, seed)


def serve_workload(n_graphs: int, n_max: float, seed: int = 3, procs: int = 0):
    """Mixed resident graphs: ER, perturbed grids and Chung-Lu graphs in turn,
    with n log-uniform on [1e3, n_max] (seeded).  procs > 1 generates them in a
    pool of spawned processes (spawn: the parent may already hold a CUDA
    context, which a forked child must not inherit)."""
    rng = np.random.default_rng(seed)
    specs = [(i % 3, int(np.exp(rng.uniform(np.log(1e3), np.log(n_max)))), 100 + i)
             for i in range(n_graphs)]
    if procs > 1:
        import multiprocessing as mp

        with mp.get_context("spawn").Pool(procs) as pool:
            return pool.map(_serve_graph, specs, chunksize=1)
    return [_serve_graph(sp) for sp in specs]


def batched_leg(args, kc):
    """Many small graphs: one kc_sample_multi call (all walks in one launch)
    against one kc_sample call per graph, same trees."""
    gs = serve_workload(args.batched_graphs, args.batched_nmax)
    T = args.batched_trees
    cfg = kc.kc_config_default()
    cfg.keep_trees = 0

    def run(batched):
        hs = [kc.KemenyGraph.from_graph(g, cfg) for g in gs]
        kc.kc_sample_multi([h.h for h in hs], [1] * len(hs), [8] * len(hs))  # warm-up
        import torch

        torch.cuda.synchronize()
        t = time.perf_counter()
        if batched:
            kc.kc_sample_multi([h.h for h in hs], [1] * len(hs), [T] * len(hs))
        else:
            for h in hs:
                h.sample(1, T)
        torch.cuda.synchronize()
        el = time.perf_counter() - t
        f = [h.samples()["f"] for h in hs]
        for h in hs:
            h.close()
        return len(gs) * T / el, f

    v_b, f_b = run(True)
    v_s, f_s = run(False)
    return {"workload": f"{len(gs)} graphs of the serving mix with n log-uniform on [1e3, "
                        f"{args.batched_nmax:.0e}], {T} trees each",
            "batched_trees_per_s": v_b, "separate_calls_trees_per_s": v_s,
            "identical_results": all(np.array_equal(a, b) for a, b in zip(f_b, f_s))}


def update_stream(g, n_updates: int, bmax: int, seed: int = 4):
    """Seeded edge-update batches against the evolving graph: half insertions of
    absent pairs, half deletions of edges that lie on a triangle (never a
    bridge), batch sizes uniform on [1, bmax].  The first k ops of a longer
    stream are the stream of length k (only the last batch is cut short).  The
    evolving graph is the CSR plus small sets of added and removed edges, so a
    prefix of a stream on a 10^7-edge graph costs no per-vertex Python state."""
    rng = np.random.default_rng(seed)
    ro, col = g.row_off, g.col
    added, removed = set(), set()
    extra = {}  # vertex -> neighbours added by the stream

    def key(u, v):
        return (u, v) if u < v else (v, u)

    def has(u, v):
        k = key(u, v)
        if k in added:
            return True
        if k in removed:
            return False
        a, b = ro[u], ro[u + 1]
        i = a + int(np.searchsorted(col[a:b], v))
        return i < b and int(col[i]) == v

    def nbrs(u):
        base = col[ro[u]:ro[u + 1]].tolist()
        out = {x for x in base if key(u, x) not in removed}
        return out | extra.get(u, set())

    added_list = []
    batches, done = [], 0
    while done < n_updates:
        b = int(min(rng.integers(1, bmax + 1), n_updates - done))
        ops = []
        while len(ops) < b:
            if rng.random() < 0.5:
                u, v = (int(x) for x in rng.choice(g.n, 2, replace=False))
                if has(u, v):
                    continue
                k = key(u, v)
                if k in removed:
                    removed.discard(k)
                else:
                    added.add(k)
                    added_list.append(k)
                extra.setdefault(u, set()).add(v)
                extra.setdefault(v, set()).add(u)
                ops.append((u, v, 0))
            else:
                e = int(rng.integers(len(col) // 2 + len(added_list)))
                if e < len(col) // 2:  # the e-th edge (u < v) of the base graph
                    x = int(rng.integers(len(col)))
                    u = int(np.searchsorted(ro, x, side="right") - 1)
                    v = int(col[x])
                else:
                    u, v = added_list[e - len(col) // 2]
                if not has(u, v) or not (nbrs(u) & nbrs(v)):
                    continue
                k = key(u, v)
                if k in added:
                    added.discard(k)
                else:
                    removed.add(k)
                extra.get(u, set()).discard(v)
                extra.get(v, set()).discard(u)
                ops.append((u, v, 1))
        batches.append(ops)
        done += b
    return batches


def dynamic_leg(args, kc):
    """Dynamic serving at its stated size: a Chung-Lu graph (gamma 2.1, mean
    degree 20), a pool of `--dyn-trees` retained trees maintained on the device,
    and the first `--dyn-updates` ops of the seeded update stream (batches
    uniform on 1..`--dyn-batch`; only a prefix fits a bench run), with a Kemeny
    query at eps after each batch.  ISM (Algorithm 3) against BSM (Algorithm 2)
    on the same pool and ops; R(u, v) by device CG.  K error: the maintained
    estimates against a fresh pool of the same size drawn on the final graph."""
    import torch

    from paper_2511_16356_gb300 import synth as S

    g = S.chung_lu(args.dyn_n, 2.1, 20.0, 4)
    t = time.perf_counter()
    batches = update_stream(g, args.dyn_updates, args.dyn_batch)
    gen_s = time.perf_counter() - t
    out = {"workload": f"Chung-Lu gamma 2.1, mean degree 20, seed 4 (n = {g.n:,}, m = {g.m:,}); "
                       f"the first {args.dyn_updates} ops of the seeded update stream (batches "
                       f"uniform on 1..{args.dyn_batch}: {len(batches)} batch(es) here), half "
                       f"insertions of absent pairs, half deletions of edges on a triangle (never "
                       f"a bridge); pool of {args.dyn_trees} trees; a query at eps {args.eps} "
                       f"after each batch", "ops": args.dyn_updates, "stream_gen_s": gen_s}
    finals = {}
    for name, mode in (("ism", kc.KC_UPDATE_ISM), ("bsm", kc.KC_UPDATE_BSM)):
        cfg = kc.kc_config_default()
        cfg.keep_trees = 1
        G = kc.KemenyGraph.from_graph(g, cfg)
        t = time.perf_counter()
        G.sample(args.seed, args.dyn_trees)
        torch.cuda.synchronize()
        pool_s = time.perf_counter() - t
        k0 = G.estimate()
        upd_ms, q_ms = [], []
        k_hat = k0
        for ops in batches:
            t = time.perf_counter()
            G.update(ops, mode)
            upd_ms.append(1000.0 * (time.perf_counter() - t) / len(ops))
            t = time.perf_counter()
            k_hat = G.estimate(args.eps, args.delta)
            q_ms.append(1000.0 * (time.perf_counter() - t))
        st = G.stats()
        finals[name] = k_hat
        G.close()
        ops_n = sum(len(b) for b in batches)
        out[name] = {"update_ms_per_op": float(np.average(upd_ms, weights=[len(b) for b in batches])),
                     "update_ms_per_op_device": st["ms_update"] / max(1, ops_n),
                     "query_p50_ms": float(np.percentile(q_ms, 50)),
                     "query_p99_ms": float(np.percentile(q_ms, 99)),
                     "trees_resampled": int(st["trees_resampled"]),
                     "pool_trees": int(st["pool_trees"]), "pool_build_s": pool_s,
                     "K_before": k0, "K_after": k_hat, "last_cg_iters": int(st["last_cg_iters"]),
                     "ms_per_op_by_part": {
                         k: st[f"ms_update_{k}"] / max(1, ops_n)
                         for k in ("graph", "resistance", "trees", "refresh")}}
    # reference: a fresh pool of the same size on the final graph
    ins = {(min(u, v), max(u, v)) for b in batches for u, v, op in b if op == 0}
    dele = {(min(u, v), max(u, v)) for b in batches for u, v, op in b if op == 1}
    e = {(int(a), int(b)) for a, b in g.edges()}
    e = (e | ins) - dele if len(ins & dele) == 0 else None
    if e is not None:
        arr = np.array(sorted(e))
        g2 = S.csr_from_edges(g.n, arr[:, 0], arr[:, 1])
        cfg = kc.kc_config_default()
        cfg.keep_trees = 0
        F = kc.KemenyGraph.from_graph(g2, cfg)
        F.sample(args.seed + 1, args.dyn_trees)
        k_ref = F.estimate()
        F.close()
        out["K_fresh_pool"] = k_ref
        for name in ("ism", "bsm"):
            out[name]["rel_diff_vs_fresh"] = (finals[name] - k_ref) / k_ref
    return out


def serve_leg(args, kc):
    """Served (continuous batching on `--serve-workers` streams, small-graph
    queries coalesced into one launch per round) against the plain
    one-graph-per-call path on the same Poisson streams of Kemeny queries, at
    each offered load of `--serve-loads` (multiples of the plain path's closed-
    loop capacity: below 1 the plain path keeps up, above it queues).  Both
    paths give every request the same workspace cap; every K must agree."""
    import torch

    t = time.perf_counter()
    gs = serve_workload(args.serve_graphs, args.serve_nmax,
                        procs=min(host_cores(), 16) if args.serve_graphs > 64 else 0)
    gen_s = time.perf_counter() - t
    rng = np.random.default_rng(7)
    Q = args.serve_queries
    q_graph = rng.integers(0, len(gs), size=Q)
    q_eps = rng.choice([0.05, 0.02, 0.01], size=Q)
    q_seed = 1000 + np.arange(Q)
    delta = 0.05
    cfg = kc.kc_config_default()
    cfg.keep_trees = 0
    free, _ = torch.cuda.mem_get_info()
    budget = int(free * 0.5)
    per_req = budget // args.serve_workers
    handles = [kc.KemenyGraph.from_graph(g, cfg) for g in gs]
    resident = sum(int(g.row_off.nbytes + g.col.nbytes) + 52 * g.n for g in gs)

    def plain_one(i):
        G = handles[int(q_graph[i])]
        kc.kc_graph_set_workspace_limit(G.h, per_req - per_req // 8)
        G.reset(int(q_seed[i]))
        k = G.estimate(float(q_eps[i]), delta)
        kc.kc_graph_release_workspace(G.h)
        return k

    for i in range(min(8, Q)):  # warm-up
        plain_one(i)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for i in range(Q):
        plain_one(i)
    torch.cuda.synchronize()
    closed = time.perf_counter() - t
    capacity = Q / closed

    def summ(lat, span):
        a = np.asarray(lat) * 1000.0
        return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
                "qps": Q / span}

    loads = {}
    identical = True
    srv = kc.Server(workers=args.serve_workers, budget_bytes=budget, request_bytes=per_req,
                    coalesce=1)
    ids = [srv.add_graph(g, cfg) for g in gs]
    for i in range(min(8, Q)):  # warm-up
        srv.wait(srv.query(ids[int(q_graph[i])], int(q_seed[i]), float(q_eps[i]), delta))
    for load in args.serve_loads:
        rate = load * capacity
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=Q))
        # plain: one query at a time in arrival order (latency includes queueing)
        lat_p, k_p = [], []
        t0 = time.perf_counter()
        for i in range(Q):
            now = time.perf_counter() - t0
            if now < arrivals[i]:
                time.sleep(arrivals[i] - now)
            k_p.append(plain_one(i))
            lat_p.append(time.perf_counter() - t0 - arrivals[i])
        span_p = time.perf_counter() - t0
        # served: submit at arrival, requests overlap on the device
        lat_s, k_s, tickets = [], [], []
        t0 = time.perf_counter()
        for i in range(Q):
            now = time.perf_counter() - t0
            if now < arrivals[i]:
                time.sleep(arrivals[i] - now)
            tickets.append((time.perf_counter() - t0,
                            srv.query(ids[int(q_graph[i])], int(q_seed[i]), float(q_eps[i]),
                                      delta)))
        coal = 0
        for i, (t_sub, tk) in enumerate(tickets):
            info = srv.wait(tk)
            k_s.append(info["K"])
            coal += info["worker"] < 0
            lat_s.append((info["t_end_ms"] - info["t_submit_ms"]) / 1000.0 + t_sub - arrivals[i])
        span_s = time.perf_counter() - t0
        identical = identical and bool(np.array_equal(np.asarray(k_s), np.asarray(k_p)))
        loads[f"{load:g}x"] = {"offered_qps": rate, "served": summ(lat_s, span_s),
                               "plain": summ(lat_p, span_p), "coalesced_queries": int(coal)}
    srv.close()
    for G in handles:
        G.close()
    ns = np.array([g.n for g in gs])
    return {
        "workload": f"{len(gs)} resident graphs (ER / perturbed grid / Chung-Lu in turn, n "
                    f"log-uniform on [1e3, {args.serve_nmax:.0e}]: total n {int(ns.sum()):,}, "
                    f"largest {int(ns.max()):,}), {Q} Kemeny queries per load, Poisson "
                    f"arrivals, eps in {{5%, 2%, 1%}}, delta {delta}",
        "graph_gen_s": gen_s, "resident_graph_bytes": resident,
        "budget_bytes": budget, "request_bytes": per_req, "workers": args.serve_workers,
        "coalesce_max_n": 1 << 18, "plain_capacity_qps": capacity, "loads": loads,
        "identical_results": identical,
    }


# DRAM bytes per Wilson departure of the walkers on road-shaped grids, from ncu
# captures (dram__bytes_read.sum + dram__bytes_write.sum) on the 300x300
# perturbed grid with 1000 trees in flight (profiles/); a full-size launch runs
# for seconds, too long to capture, so its traffic is this figure times its
# departures.  k_wilson_warp: 10.213 GB, k_wilson: 4.648 GB, each for the
# same 1,133,364,358 departures.
WALKER_GRID_DRAM_BYTES_PER_STEP = {"warp": 10.213e9 / 1133364358, "lane": 4.648e9 / 1133364358}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="grid1000")
    ap.add_argument("--trees", type=int, default=10000)
    ap.add_argument("--warmup-trees", type=int, default=-1,
                    help="trees per warm-up step (0: same as --trees; default 16, or --trees "
                         "with rejection, whose wave sizes learn the acceptance rate)")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--eps", type=float, default=0.01)
    ap.add_argument("--delta", type=float, default=0.05)
    ap.add_argument("--ref-trees", type=int, default=32)
    ap.add_argument("--step-cap-per-n", type=int, default=256,
                    help="Wilson departures allowed per tree, in units of n")
    ap.add_argument("--walker", default="auto", choices=["auto", "warp", "lane", "hybrid"])
    ap.add_argument("--hybrid-prefix", type=int, default=0,
                    help="hybrid walker: lane-phase starts in thousandths of n (0: library default)")
    ap.add_argument("--hybrid-tail", type=int, default=0,
                    help="hybrid walker: hand-off share of finished trees, in thousandths "
                         "(0: library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tte", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-other", action="store_true",
                    help="skip the other static workloads (er2000, cl4m)")
    ap.add_argument("--serve-graphs", type=int, default=512)
    ap.add_argument("--serve-nmax", type=float, default=1e6)
    ap.add_argument("--serve-queries", type=int, default=64)
    ap.add_argument("--serve-workers", type=int, default=8)
    ap.add_argument("--serve-loads", type=lambda x: [float(v) for v in x.split(",")],
                    default=[0.8, 1.5],
                    help="offered loads, as multiples of the plain path's capacity")
    ap.add_argument("--batched-trees", type=int, default=256,
                    help="trees per graph in the batched multi-graph leg")
    ap.add_argument("--batched-graphs", type=int, default=48)
    ap.add_argument("--batched-nmax", type=float, default=3e4)
    ap.add_argument("--reject-quantile", type=float, default=0.65,
                    help="rejection by walk length with the cap at this quantile of a probe "
                         "batch's step counts (0: off)")
    ap.add_argument("--mem-fraction", type=float, default=0.9,
                    help="share of free device memory for the sampling workspaces")
    ap.add_argument("--reject-probe", type=int, default=256,
                    help="trees of the probe batch that sets the rejection cap")
    ap.add_argument("--no-dynamic", action="store_true",
                    help="skip the dynamic-serving leg (ISM against BSM under an update stream)")
    ap.add_argument("--dyn-n", type=int, default=1000000)
    ap.add_argument("--dyn-updates", type=int, default=32,
                    help="ops of the seeded update stream processed (a prefix)")
    ap.add_argument("--dyn-batch", type=int, default=1000)
    ap.add_argument("--dyn-trees", type=int, default=5000)
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch

    from paper_2511_16356_gb300 import kc
    from paper_2511_16356_gb300 import synth as S

    dist, rank, ws, local = dist_setup()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    kc.load()
    g = S.workload(args.workload)
    n = g.n
    T = args.trees
    if args.warmup_trees < 0:
        args.warmup_trees = 0 if args.reject_quantile > 0 else 16
    WT = args.warmup_trees or T
    from paper_2511_16356_gb300.dist import rank_sample_base

    cfg = kc.kc_config_default()
    cfg.keep_trees = 0
    cfg.sample_id_base = rank_sample_base(rank, ws)
    cfg.step_cap = args.step_cap_per_n * n
    cfg.walker = {"auto": kc.KC_WALK_AUTO, "warp": kc.KC_WALK_WARP,
                  "lane": kc.KC_WALK_LANE, "hybrid": kc.KC_WALK_HYBRID}[args.walker]
    cfg.hybrid_prefix_permille = args.hybrid_prefix
    cfg.hybrid_tail_permille = args.hybrid_tail
    cfg.mem_fraction = args.mem_fraction
    reject = None
    if args.reject_quantile > 0:
        # rejection by walk length: the cap is a quantile of the step counts of
        # a probe batch (a rule on step counts only, so the trees stay uniform)
        pcfg = kc.kc_config_default()
        for f, _ in kc.kc_config._fields_:
            setattr(pcfg, f, getattr(cfg, f))
        pcfg.walker = kc.KC_WALK_WARP  # a few hundred trees: 32 walkers each finish sooner
        P = kc.KemenyGraph.from_graph(g, pcfg, stream=stream.cuda_stream)
        P.sample(args.seed, args.reject_probe)
        probe_steps = P.samples()["steps"]
        P.close()
        cfg.reject_steps = max(int(np.quantile(probe_steps, args.reject_quantile)), n - 1)
        # the probe's quantile estimates the acceptance rate with a standard
        # error of sqrt(q (1 - q) / probe); a hint three errors lower makes a
        # fresh handle's first wave (time to eps, end to end) rarely fall short
        se = math.sqrt(args.reject_quantile * (1 - args.reject_quantile) / args.reject_probe)
        cfg.reject_accept_hint = max(0.05, args.reject_quantile - 3 * se)
        reject = {"quantile": args.reject_quantile, "probe_trees": args.reject_probe,
                  "reject_steps": int(cfg.reject_steps),
                  "accept_hint": float(cfg.reject_accept_hint)}
    G = kc.KemenyGraph.from_graph(g, cfg, stream=stream.cuda_stream)
    st0 = G.stats()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")

    # pool capacity and workspace for every tree of the run, outside the timing
    G.reserve(WT * args.warmup + T * args.steps)
    for _ in range(args.warmup):
        G.sample(args.seed, WT)
    torch.cuda.synchronize()
    kc.kc_reset_timers(G.h)
    pool0 = G.stats()["pool_trees"]
    rej0 = G.stats()["trees_rejected"]
    clocks = ClockSampler(local)
    barrier(dist)
    torch.cuda.synchronize()
    clocks.start()
    step_ms = timed_sampling(G, T, args.steps, args.seed, stream, flush)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(dist)
    tot_ms = reduce_max(dist, float(sum(step_ms)))
    ms_per_step = tot_ms / args.steps
    value = T * ws * args.steps / (tot_ms / 1000.0)
    st = G.stats()
    samples = G.samples(pool0, st["pool_trees"] - pool0)
    steps_total = int(samples["steps"].sum())
    trees_timed = T * args.steps
    traffic_per_step = (WALKER_GRID_DRAM_BYTES_PER_STEP.get(WALKER_NAMES[st["walker"]])
                        if args.workload.startswith("grid") else None)
    dom, roof, phase_ms = phase_roofline(kc, st, n, trees_timed, steps_total, tot_ms,
                                         traffic_per_step)
    roof["traffic_basis"] = (None if roof["traffic"] is None else
                             "ncu dram bytes per departure on grid300x300 (1000 trees) x "
                             "departures")
    launches = sum(st[k] for k in st if k.startswith("launches_") and k != "launches_setup")

    out = {
        "metric": "trees/sec", "value": value, "unit": "trees/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": S.WORKLOADS.get(args.workload, args.workload),
                   "n": n, "m": g.m, "ecc": st["ecc"], "trees_per_step": T,
                   "trees_per_rank_per_step": T, "parallelism": f"sample-sharded x{ws}",
                   "l2": "flushed between timed steps (258 MB write); per-step working set "
                         f"{st['workspace_bytes'] / 1e9:.1f} GB",
                   "ttf": "BIT" if st["ttf_variant"] == kc.KC_TTF_BIT else "SCAN",
                   "walker": WALKER_NAMES[st["walker"]],
                   "trees_in_flight": st["trees_in_flight"]},
        "roofline": roof,
        "phase_ms": phase_ms,
        "rejection": None if reject is None else
        dict(reject, trees_rejected=int(st["trees_rejected"] - rej0),
             note="trees/s counts accepted trees; the roofline counts their steps only"),
        "steps_per_tree": steps_total / trees_timed,
        "step_ms": [round(x, 1) for x in step_ms],
        "gpu_launches": int(launches),
        "clocks": clk,
    }

    G.close()  # release its workspace before the other measurements

    # ---- time to eps on a fresh handle (tau0 precomputed, inputs resident)
    if not args.no_tte and rank == 0:
        # batches of one resident wave where trees are long (deep tau0: a wave
        # lasts about as long as its slowest tree, so a wave of 1024 costs
        # about what a full one does), 1024 trees where waves are throughput-bound
        # (with one walker per tree every tree of a wave is in flight at once, so
        # a pilot large enough for the usual answer costs one wave as well)
        deep = st["ttf_variant"] == kc.KC_TTF_BIT
        if deep and st["walker"] == kc.KC_WALK_LANE:
            batch = 4096
        elif deep:
            batch = max(1024, st["resident_trees"])
        else:
            batch = 1024
        out["time_to_eps"] = time_to_eps(kc, g, cfg, args.eps, args.delta, batch, stream,
                                         args.workload)

    # ---- the other static workloads at their stated sizes (rank 0)
    if not args.no_other and rank == 0:
        out["other_workloads"] = {
            "er2000": other_workload_leg(args, kc, stream, flush, "er2000", 2000, 20, 5, 0.05),
            "cl4m": other_workload_leg(args, kc, stream, flush, "cl4m", 10000, 2, 2, 0.01),
        }

    # ---- end to end through the C ABI with host buffers
    if not args.no_e2e:
        ro = torch.from_numpy(g.row_off).pin_memory().numpy()
        co = torch.from_numpy(g.col).pin_memory().numpy()
        fbuf = torch.empty(T, dtype=torch.int64).pin_memory().numpy()

        def e2e_step():
            st_, h = kc.kc_graph_create(ro, co, cfg)
            kc.kc_graph_set_stream(h, stream.cuda_stream)
            kc.kc_sample(h, args.seed, T)
            kc.load().kc_get_samples(h, 0, T, fbuf.ctypes.data, None, None, None)
            kc.kc_graph_destroy(h)

        e2e_step()
        torch.cuda.synchronize()
        barrier(dist)
        k_e2e = max(1, args.steps)  # the same step count as the device-timed value
        t = time.perf_counter()
        for _ in range(k_e2e):
            e2e_step()
        torch.cuda.synchronize()
        el = reduce_max(dist, time.perf_counter() - t)
        out["e2e"] = {"value": T * ws * k_e2e / el, "unit": "trees/s",
                      "h2d_bytes_per_step": int(ro.nbytes + co.nbytes),
                      "d2h_bytes_per_step": int(fbuf.nbytes),
                      "steps": k_e2e,
                      "includes": "kc_graph_create from pinned host CSR (validation, "
                                  "records, BFS tau0, DFN), kc_sample, f read back, destroy"}

    # ---- served p50/p99 against the plain path (rank 0)
    if not args.no_serve and rank == 0:
        out["serve"] = serve_leg(args, kc)
        out["batched"] = batched_leg(args, kc)

    # ---- sample maintenance under an update stream (rank 0, on request)
    if not args.no_dynamic and rank == 0:
        out["dynamic"] = dynamic_leg(args, kc)

    # ---- the CPU oracle on the host cores (rank 0, N = 1 only)
    if not args.no_cpu_baseline and rank == 0 and ws == 1:
        # a calibration batch, then batches sized from the rate seen so far
        # until about 15 s of work (small batches overstate the per-tree time,
        # so one correction may not reach it)
        cores = host_cores()
        trees, el, used = 0, 0.0, cores
        batch = max(2 * cores, 16)
        for _ in range(4):
            _, e, used = oracle_baseline(g, batch, args.seed, first=trees)
            trees, el = trees + batch, el + e
            if el >= 10.0:
                break
            rate = batch / max(e, 1e-3)
            batch = int(min(1 << 22, max(cores, rate * (15.0 - el))))
            batch = (batch + cores - 1) // cores * cores
        out["cpu_baseline"] = {"value": trees / el, "unit": "trees/s", "cores": used,
                               "kind": "oracle",
                               "sample": f"{trees} trees (sample ids 0..{trees - 1}) of "
                                         f"{args.workload}, {el:.1f} s, OpenMP across trees",
                               "cpu": host_cpu_model(),
                               "single_core": single_core_baseline(g, args.seed)}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
