"""Python binding of libkc (include/kc.h): argument marshalling only.

Every function keeps the C name and forwards to the CUDA library; there is no
Python or CPU implementation of any step behind it.  Loading fails loudly when
the in-tree ``libkc.so`` is missing or no sm_103 device is present.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkc.so")

KC_OK = 0
STATUS = {
    0: "KC_OK", 1: "KC_ERR_INVALID_ARG", 2: "KC_ERR_NOT_SYMMETRIC", 3: "KC_ERR_SELF_LOOP",
    4: "KC_ERR_MULTI_EDGE", 5: "KC_ERR_DISCONNECTED", 6: "KC_ERR_OVERFLOW",
    7: "KC_ERR_OUT_OF_MEMORY", 8: "KC_ERR_CUDA", 9: "KC_ERR_STEP_LIMIT",
    10: "KC_ERR_EDGE_EXISTS", 11: "KC_ERR_EDGE_MISSING", 12: "KC_ERR_BRIDGE",
    13: "KC_ERR_NO_SAMPLES", 14: "KC_ERR_NO_DEVICE", 15: "KC_ERR_NOT_RETAINED",
    16: "KC_ERR_SCRATCH_LIMIT",
}
KC_TTF_AUTO, KC_TTF_SCAN, KC_TTF_BIT = 0, 1, 2
KC_STOP_CLT, KC_STOP_HOEFFDING = 0, 1
KC_UPDATE_BSM, KC_UPDATE_ISM = 0, 1
KC_R_CG, KC_R_GIVEN = 0, 1
KC_WALK_AUTO, KC_WALK_LANE, KC_WALK_WARP, KC_WALK_HYBRID = 0, 1, 2, 3
KC_TAU0_BFS, KC_TAU0_DFS, KC_TAU0_WILSON = 0, 1, 2
KC_OP_INSERT, KC_OP_DELETE = 0, 1


class kc_config(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32), ("root", ctypes.c_int32),
        ("ttf_variant", ctypes.c_int32), ("keep_trees", ctypes.c_int32),
        ("stop_rule", ctypes.c_int32), ("refresh_after_update", ctypes.c_int32),
        ("inputs_on_device", ctypes.c_int32), ("r_source", ctypes.c_int32),
        ("walker", ctypes.c_int32), ("autotune", ctypes.c_int32),
        ("max_trees_in_flight", ctypes.c_int64), ("batch_trees", ctypes.c_int64),
        ("max_trees", ctypes.c_int64), ("step_cap", ctypes.c_int64),
        ("mem_fraction", ctypes.c_double), ("sample_id_base", ctypes.c_int64),
        ("hybrid_prefix_permille", ctypes.c_int32), ("hybrid_tail_permille", ctypes.c_int32),
        ("tau0_kind", ctypes.c_int32), ("reserved1", ctypes.c_int32),
        ("tau0_seed", ctypes.c_uint64), ("reject_steps", ctypes.c_int64),
        ("reject_accept_hint", ctypes.c_double),
        ("ttf_segments", ctypes.c_int32), ("reserved2", ctypes.c_int32),
    ]


class kc_edge_op(ctypes.Structure):
    _fields_ = [("u", ctypes.c_int32), ("v", ctypes.c_int32), ("op", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("r", ctypes.c_double)]


_STATS_FIELDS = [
    ("n", ctypes.c_int64), ("m", ctypes.c_int64), ("root", ctypes.c_int32),
    ("ecc", ctypes.c_int32), ("ttf_variant", ctypes.c_int32), ("walker", ctypes.c_int32),
    ("pool_trees", ctypes.c_int64), ("next_sample_id", ctypes.c_int64),
    ("total_steps", ctypes.c_int64), ("trees_in_flight", ctypes.c_int64),
    ("pool_bytes", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
    ("updates_applied", ctypes.c_int64), ("trees_resampled", ctypes.c_int64),
    ("ms_wilson", ctypes.c_double), ("ms_traverse", ctypes.c_double),
    ("ms_ttf", ctypes.c_double), ("ms_reduce", ctypes.c_double),
    ("ms_update", ctypes.c_double), ("ms_setup", ctypes.c_double),
    ("ms_wave_init", ctypes.c_double),
    ("launches_wilson", ctypes.c_int64), ("launches_traverse", ctypes.c_int64),
    ("launches_ttf", ctypes.c_int64), ("launches_reduce", ctypes.c_int64),
    ("launches_update", ctypes.c_int64), ("launches_setup", ctypes.c_int64),
    ("launches_wave_init", ctypes.c_int64),
    ("f_sum_hi", ctypes.c_int64), ("f_sum_lo", ctypes.c_uint64),
    ("wf_sum", ctypes.c_double), ("w_sum", ctypes.c_double), ("x2_sum", ctypes.c_double),
    ("last_resistance", ctypes.c_double), ("last_cg_iters", ctypes.c_int64),
    ("traversal", ctypes.c_int32), ("tuned", ctypes.c_int32),
    ("tune_ms", ctypes.c_double * 4), ("trees_rejected", ctypes.c_int64),
    ("resident_trees", ctypes.c_int64),
    ("ms_update_graph", ctypes.c_double), ("ms_update_resistance", ctypes.c_double),
    ("ms_update_trees", ctypes.c_double), ("ms_update_refresh", ctypes.c_double),
]


class kc_stats_t(ctypes.Structure):
    _fields_ = _STATS_FIELDS

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in _STATS_FIELDS}
        d["tune_ms"] = list(d["tune_ms"])
        return d


class kc_pool_sums(ctypes.Structure):
    _fields_ = [("f_sum_hi", ctypes.c_int64), ("f_sum_lo", ctypes.c_uint64),
                ("wf_sum", ctypes.c_double), ("w_sum", ctypes.c_double),
                ("x2_sum", ctypes.c_double), ("count", ctypes.c_int64)]


class kc_server_config(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("workers", ctypes.c_int32),
                ("budget_bytes", ctypes.c_int64), ("request_bytes", ctypes.c_int64),
                ("coalesce", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("coalesce_max_n", ctypes.c_int64)]


class kc_request_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("kind", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("worker", ctypes.c_int32), ("K", ctypes.c_double), ("trees", ctypes.c_int64),
                ("t_submit_ms", ctypes.c_double), ("t_start_ms", ctypes.c_double),
                ("t_end_ms", ctypes.c_double), ("workspace_bytes", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


KC_REQ_QUERY, KC_REQ_POOL_QUERY, KC_REQ_UPDATE = 0, 1, 2

# The C prototypes, in header order (kc.h, then kc_serve.h).
_P = ctypes.c_void_p
_SIGS = {
    "kc_config_default": (None, [ctypes.POINTER(kc_config)]),
    "kc_graph_create": (ctypes.c_int, [ctypes.c_int64, _P, _P, ctypes.POINTER(kc_config),
                                       ctypes.POINTER(_P)]),
    "kc_graph_destroy": (ctypes.c_int, [_P]),
    "kc_graph_set_stream": (ctypes.c_int, [_P, _P]),
    "kc_graph_set_workspace_limit": (ctypes.c_int, [_P, ctypes.c_int64]),
    "kc_graph_release_workspace": (ctypes.c_int, [_P]),
    "kc_graph_reset": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int64]),
    "kc_sample": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int64]),
    "kc_reserve": (ctypes.c_int, [_P, ctypes.c_int64]),
    "kc_sample_multi": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_uint64),
                                       ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]),
    "kc_estimate": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_double)]),
    "kc_update": (ctypes.c_int, [_P, ctypes.POINTER(kc_edge_op), ctypes.c_int64, ctypes.c_int32]),
    "kc_get_tree": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P]),
    "kc_get_samples": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P]),
    "kc_get_tau0": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "kc_wilson_noalloc": (ctypes.c_int, [ctypes.c_int64, _P, _P, ctypes.c_int32, ctypes.c_uint64,
                                         ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _P, _P,
                                         _P, _P]),
    "kc_stats": (ctypes.c_int, [_P, ctypes.POINTER(kc_stats_t)]),
    "kc_reset_timers": (ctypes.c_int, [_P]),
    "kc_get_pool_sums": (ctypes.c_int, [_P, ctypes.POINTER(kc_pool_sums)]),
    "kc_combine_sums": (ctypes.c_int, [ctypes.POINTER(kc_pool_sums), ctypes.c_int32,
                                       ctypes.POINTER(kc_pool_sums)]),
    "kc_estimate_from_sums": (ctypes.c_int, [ctypes.POINTER(kc_pool_sums), ctypes.c_int64,
                                             ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "kc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "kc_last_error": (ctypes.c_char_p, [_P]),
    "kc_server_config_default": (None, [ctypes.POINTER(kc_server_config)]),
    "kc_server_create": (ctypes.c_int, [ctypes.POINTER(kc_server_config), ctypes.POINTER(_P)]),
    "kc_server_destroy": (ctypes.c_int, [_P]),
    "kc_server_add_graph": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, ctypes.POINTER(kc_config),
                                           ctypes.c_uint64, ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_int32)]),
    "kc_server_submit_query": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint64,
                                              ctypes.c_double, ctypes.c_double,
                                              ctypes.POINTER(ctypes.c_int64)]),
    "kc_server_submit_pool_query": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double,
                                                   ctypes.c_double,
                                                   ctypes.POINTER(ctypes.c_int64)]),
    "kc_server_submit_update": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(kc_edge_op),
                                               ctypes.c_int64, ctypes.c_int32,
                                               ctypes.POINTER(ctypes.c_int64)]),
    "kc_server_wait": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(kc_request_info)]),
    "kc_server_poll": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(kc_request_info)]),
    "kc_server_drain": (ctypes.c_int, [_P]),
}
EXPORTED = tuple(_SIGS)

_lib = None


def load(path: str = LIB_PATH):
    """Load libkc.so and attach the prototypes (no device needed for loading)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libkc.so not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class KcError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.name}" + (f" ({detail})" if detail else ""))


def _ptr(a):
    return None if a is None else a.ctypes.data


def _check(st: int, where: str, g=None):
    if st != KC_OK:
        detail = ""
        if g is not None:
            try:
                detail = (load().kc_last_error(g) or b"").decode()
            except Exception:
                detail = ""
        raise KcError(st, where, detail)


def kc_config_default() -> kc_config:
    c = kc_config()
    load().kc_config_default(ctypes.byref(c))
    return c


def kc_status_string(st: int) -> str:
    return load().kc_status_string(st).decode()


def kc_graph_create(row_off: np.ndarray, col: np.ndarray, cfg: kc_config | None = None,
                    check: bool = True):
    """Returns (status, handle).  Host arrays: int64[n+1], int32[2m]."""
    row_off = np.ascontiguousarray(row_off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = row_off.shape[0] - 1
    h = _P()
    st = load().kc_graph_create(n, _ptr(row_off), _ptr(col),
                                None if cfg is None else ctypes.byref(cfg), ctypes.byref(h))
    if check:
        _check(st, "kc_graph_create")
    return st, h


def kc_graph_destroy(g) -> None:
    _check(load().kc_graph_destroy(g), "kc_graph_destroy")


def kc_graph_set_stream(g, stream_ptr: int) -> None:
    _check(load().kc_graph_set_stream(g, _P(stream_ptr)), "kc_graph_set_stream", g)


def kc_sample(g, seed: int, n_trees: int, check: bool = True) -> int:
    st = load().kc_sample(g, seed, n_trees)
    if check:
        _check(st, "kc_sample", g)
    return st


def kc_sample_multi(handles, seeds, n_trees, check: bool = True) -> int:
    k = len(handles)
    hs = (_P * k)(*[h.value if isinstance(h, _P) else h for h in handles])
    ss = (ctypes.c_uint64 * k)(*[int(x) for x in seeds])
    ns = (ctypes.c_int64 * k)(*[int(x) for x in n_trees])
    st = load().kc_sample_multi(hs, ss, ns, k)
    if check:
        _check(st, "kc_sample_multi")
    return st


def kc_estimate(g, eps: float, delta: float) -> float:
    k = ctypes.c_double(0.0)
    _check(load().kc_estimate(g, eps, delta, ctypes.byref(k)), "kc_estimate", g)
    return float(k.value)


def kc_update(g, ops, mode: int, check: bool = True) -> int:
    """ops: iterable of (u, v, op[, r])."""
    ops = list(ops)
    arr = (kc_edge_op * max(1, len(ops)))()
    for i, o in enumerate(ops):
        arr[i].u, arr[i].v, arr[i].op = int(o[0]), int(o[1]), int(o[2])
        arr[i].r = float(o[3]) if len(o) > 3 else 0.0
    st = load().kc_update(g, arr, len(ops), mode)
    if check:
        _check(st, "kc_update", g)
    return st


def kc_get_tree(g, sample: int, n: int) -> dict:
    out = {
        "parent": np.empty(n, dtype=np.int32), "depth": np.empty(n, dtype=np.int32),
        "din": np.empty(n, dtype=np.int32), "dout": np.empty(n, dtype=np.int32),
        "vol": np.empty(n, dtype=np.int64),
    }
    f = np.zeros(1, dtype=np.int64)
    steps = np.zeros(1, dtype=np.int64)
    _check(load().kc_get_tree(g, sample, _ptr(out["parent"]), _ptr(out["depth"]),
                              _ptr(out["din"]), _ptr(out["dout"]), _ptr(out["vol"]), _ptr(f),
                              _ptr(steps)), "kc_get_tree", g)
    out["f"] = int(f[0])
    out["steps"] = int(steps[0])
    return out


def kc_get_samples(g, first: int, count: int) -> dict:
    f = np.empty(count, dtype=np.int64)
    w = np.empty(count, dtype=np.float64)
    steps = np.empty(count, dtype=np.int64)
    sid = np.empty(count, dtype=np.int64)
    _check(load().kc_get_samples(g, first, count, _ptr(f), _ptr(w), _ptr(steps), _ptr(sid)),
           "kc_get_samples", g)
    return {"f": f, "w": w, "steps": steps, "sid": sid}


def kc_get_tau0(g, n: int) -> dict:
    p0 = np.empty(n, dtype=np.int32)
    level = np.empty(n, dtype=np.int32)
    in0 = np.empty(n, dtype=np.int32)
    out0 = np.empty(n, dtype=np.int32)
    root = ctypes.c_int32(0)
    ecc = ctypes.c_int32(0)
    _check(load().kc_get_tau0(g, _ptr(p0), _ptr(level), _ptr(in0), _ptr(out0),
                              ctypes.addressof(root), ctypes.addressof(ecc)), "kc_get_tau0", g)
    return {"p0": p0, "level": level, "in0": in0, "out0": out0, "root": root.value,
            "ecc": ecc.value}


def kc_stats(g) -> dict:
    s = kc_stats_t()
    _check(load().kc_stats(g, ctypes.byref(s)), "kc_stats", g)
    return s.as_dict()


def kc_graph_reset(g, seed: int, sample_id_base: int = 0) -> None:
    _check(load().kc_graph_reset(g, seed, sample_id_base), "kc_graph_reset", g)


def kc_graph_set_workspace_limit(g, nbytes: int) -> None:
    _check(load().kc_graph_set_workspace_limit(g, nbytes), "kc_graph_set_workspace_limit", g)


def kc_graph_release_workspace(g) -> None:
    _check(load().kc_graph_release_workspace(g), "kc_graph_release_workspace", g)


def kc_reset_timers(g) -> None:
    _check(load().kc_reset_timers(g), "kc_reset_timers", g)


class KemenyGraph:
    """Owning wrapper around a kc_graph handle."""

    def __init__(self, row_off, col, cfg: kc_config | None = None, stream: int | None = None):
        _, self.h = kc_graph_create(row_off, col, cfg)
        self.n = int(np.asarray(row_off).shape[0] - 1)
        if stream is not None:
            kc_graph_set_stream(self.h, stream)

    @classmethod
    def from_graph(cls, g, cfg=None, stream=None):
        return cls(g.row_off, g.col, cfg, stream)

    def sample(self, seed: int, n_trees: int):
        kc_sample(self.h, seed, n_trees)

    def reserve(self, n_trees: int):
        _check(load().kc_reserve(self.h, n_trees), "kc_reserve", self.h)

    def estimate(self, eps: float = 0.0, delta: float = 0.05) -> float:
        return kc_estimate(self.h, eps, delta)

    def update(self, ops, mode: int = KC_UPDATE_BSM):
        kc_update(self.h, ops, mode)

    def tree(self, sample: int) -> dict:
        return kc_get_tree(self.h, sample, self.n)

    def samples(self, first: int = 0, count: int | None = None) -> dict:
        if count is None:
            count = self.stats()["pool_trees"] - first
        return kc_get_samples(self.h, first, count)

    def tau0(self) -> dict:
        return kc_get_tau0(self.h, self.n)

    def reset(self, seed: int, sample_id_base: int = 0):
        kc_graph_reset(self.h, seed, sample_id_base)

    def stats(self) -> dict:
        return kc_stats(self.h)

    def pool_sums(self) -> dict:
        s = kc_pool_sums()
        _check(load().kc_get_pool_sums(self.h, ctypes.byref(s)), "kc_get_pool_sums", self.h)
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if getattr(self, "h", None):
            kc_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _edge_ops(ops):
    ops = list(ops)
    arr = (kc_edge_op * max(1, len(ops)))()
    for i, o in enumerate(ops):
        arr[i].u, arr[i].v, arr[i].op = int(o[0]), int(o[1]), int(o[2])
        arr[i].r = float(o[3]) if len(o) > 3 else 0.0
    return arr, len(ops)


class Server:
    """Owning wrapper around a kc_server (resident graphs, continuous batching)."""

    def __init__(self, workers: int = 4, budget_bytes: int = 0, request_bytes: int = 0,
                 coalesce: int = 0, coalesce_max_n: int = 0):
        c = kc_server_config()
        load().kc_server_config_default(ctypes.byref(c))
        c.workers, c.budget_bytes, c.request_bytes = workers, budget_bytes, request_bytes
        c.coalesce, c.coalesce_max_n = coalesce, coalesce_max_n
        self.h = _P()
        _check(load().kc_server_create(ctypes.byref(c), ctypes.byref(self.h)), "kc_server_create")

    def add_graph(self, g, cfg: kc_config | None = None, pool_seed: int = 0,
                  pool_trees: int = 0) -> int:
        row_off = np.ascontiguousarray(g.row_off, dtype=np.int64)
        col = np.ascontiguousarray(g.col, dtype=np.int32)
        gid = ctypes.c_int32(-1)
        _check(load().kc_server_add_graph(self.h, row_off.shape[0] - 1, _ptr(row_off), _ptr(col),
                                          None if cfg is None else ctypes.byref(cfg), pool_seed,
                                          pool_trees, ctypes.byref(gid)), "kc_server_add_graph")
        return gid.value

    def query(self, graph: int, seed: int, eps: float, delta: float) -> int:
        t = ctypes.c_int64(-1)
        _check(load().kc_server_submit_query(self.h, graph, seed, eps, delta, ctypes.byref(t)),
               "kc_server_submit_query")
        return t.value

    def pool_query(self, graph: int, eps: float, delta: float) -> int:
        t = ctypes.c_int64(-1)
        _check(load().kc_server_submit_pool_query(self.h, graph, eps, delta, ctypes.byref(t)),
               "kc_server_submit_pool_query")
        return t.value

    def update(self, graph: int, ops, mode: int = KC_UPDATE_ISM) -> int:
        arr, k = _edge_ops(ops)
        t = ctypes.c_int64(-1)
        _check(load().kc_server_submit_update(self.h, graph, arr, k, mode, ctypes.byref(t)),
               "kc_server_submit_update")
        return t.value

    def wait(self, ticket: int) -> dict:
        info = kc_request_info()
        _check(load().kc_server_wait(self.h, ticket, ctypes.byref(info)), "kc_server_wait")
        return info.as_dict()

    def poll(self, ticket: int):
        info = kc_request_info()
        done = ctypes.c_int32(0)
        _check(load().kc_server_poll(self.h, ticket, ctypes.byref(done), ctypes.byref(info)),
               "kc_server_poll")
        return info.as_dict() if done.value else None

    def drain(self):
        _check(load().kc_server_drain(self.h), "kc_server_drain")

    def close(self):
        if getattr(self, "h", None):
            load().kc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
