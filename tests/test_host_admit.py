"""Admission in the query server (paper_2511_16356_gb300/csrc/kc_host_admit.h),
compiled with the host C++ compiler and driven by an event simulation of
workers, arrivals and completions: every request is served; requests on one
graph start in submission order and never overlap; the running reservations
stay within the budget unless a single request runs.  Direct cases: a request
that fits passes one that does not, the earliest request of a graph is the one
that starts, and a request larger than the budget runs when nothing else
does."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2511_16356_gb300", "csrc")

SHIM = r"""
#include "kc_host_admit.h"
#include <algorithm>
#include <deque>
#include <vector>
// index of the admissible ticket among tickets 0..n-1 (graph[k], busy[g],
// reserve[g]), or -1
extern "C" int ha_pick(int n, const int32_t *graph, int n_graphs, const char *busy,
                       const int64_t *reserve, int64_t reserved, int64_t budget) {
    std::vector<int64_t> q;
    for (int k = 0; k < n; ++k) q.push_back(k);
    int64_t b = 0;
    auto it = kc_host::first_admissible(
        q.begin(), q.end(), (size_t)n_graphs, [&](int64_t k) { return graph[k]; },
        [&](size_t gi) { return busy[gi] != 0; }, [&](size_t gi) { return reserve[gi]; },
        reserved, budget, &b);
    return it == q.end() ? -1 : (int)*it;
}

// requests in arrival order; writes start/end times
extern "C" void ha_simulate(int n_req, const int32_t *graph, const double *arrival,
                           const double *duration, int n_graphs, const int64_t *reserve,
                           int64_t budget, int workers, double *start, double *end) {
    std::deque<int64_t> queue;
    std::vector<char> busy(n_graphs, 0);
    struct Run { double end; int64_t ticket; int64_t bytes; };
    std::vector<Run> running;
    int64_t reserved = 0;
    int next = 0, done = 0;
    double t = 0.0;
    while (done < n_req) {
        while (next < n_req && arrival[next] <= t) queue.push_back(next++);
        // admit while a worker is free
        while ((int)running.size() < workers) {
            int64_t b = 0;
            auto it = kc_host::first_admissible(
                queue.begin(), queue.end(), (size_t)n_graphs,
                [&](int64_t k) { return graph[k]; }, [&](size_t gi) { return busy[gi] != 0; },
                [&](size_t gi) { return reserve[gi]; }, reserved, budget, &b);
            if (it == queue.end()) break;
            const int64_t k = *it;
            queue.erase(it);
            busy[graph[k]] = 1;
            reserved += b;
            start[k] = t;
            end[k] = t + duration[k];
            running.push_back({end[k], k, b});
        }
        // next event: the earliest completion or arrival
        double tn = 1e300;
        for (const Run &r : running) tn = std::min(tn, r.end);
        if (next < n_req) tn = std::min(tn, arrival[next]);
        t = tn;
        for (size_t i = 0; i < running.size();) {
            if (running[i].end <= t) {
                busy[graph[running[i].ticket]] = 0;
                reserved -= running[i].bytes;
                running[i] = running.back();
                running.pop_back();
                ++done;
            } else {
                ++i;
            }
        }
    }
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("hostadmit")
    (d / "shim.cpp").write_text(SHIM)
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(d / "shim.cpp"),
                    "-o", str(d / "shim.so")], check=True, capture_output=True)
    h = ctypes.CDLL(str(d / "shim.so"))
    h.ha_simulate.restype = None
    h.ha_pick.restype = ctypes.c_int
    h.ha_pick.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                          ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64]
    h.ha_simulate.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_void_p,
                                                                        ctypes.c_int64, ctypes.c_int,
                                                                        ctypes.c_void_p,
                                                                        ctypes.c_void_p]
    return h


@pytest.mark.parametrize("seed,workers,budget", [(1, 4, 10), (2, 8, 6), (3, 2, 100), (4, 4, 3)])
def test_admission_invariants(lib, seed, workers, budget):
    rng = np.random.default_rng(seed)
    n_graphs, n_req = 12, 400
    graph = rng.integers(0, n_graphs, n_req).astype(np.int32)
    arrival = np.sort(rng.exponential(0.3, n_req).cumsum())
    duration = rng.exponential(1.0, n_req) + 0.01
    reserve = rng.integers(1, 5, n_graphs).astype(np.int64)
    reserve[0] = budget + 2  # one graph whose requests exceed the budget: they must run alone
    start = np.full(n_req, -1.0)
    end = np.full(n_req, -1.0)
    lib.ha_simulate(n_req, graph.ctypes.data, arrival.ctypes.data, duration.ctypes.data,
                           n_graphs, reserve.ctypes.data, budget, workers, start.ctypes.data,
                           end.ctypes.data)
    assert np.all(start >= arrival - 1e-12) and np.all(end > start)
    for gi in range(n_graphs):
        idx = np.flatnonzero(graph == gi)           # submission order
        assert np.all(np.diff(start[idx]) >= 0)     # started in order
        assert np.all(start[idx][1:] >= end[idx][:-1] - 1e-12)  # one at a time
    # at every start instant: running reservations within budget, unless alone
    for k in range(n_req):
        t = start[k]
        run = (start <= t) & (end > t)
        assert run.sum() <= workers
        if run.sum() > 1:
            assert reserve[graph[run]].sum() <= budget


def _pick(lib, graph, busy, reserve, reserved, budget):
    graph = np.ascontiguousarray(graph, dtype=np.int32)
    busy = np.ascontiguousarray(busy, dtype=np.int8)
    reserve = np.ascontiguousarray(reserve, dtype=np.int64)
    return lib.ha_pick(len(graph), graph.ctypes.data, len(busy), busy.ctypes.data,
                       reserve.ctypes.data, reserved, budget)


def test_direct_cases(lib):
    # graph 0 runs (6 of 10 reserved); waiting: graph 1 (6, does not fit), graph 2 (3, fits)
    assert _pick(lib, [1, 2], [1, 0, 0], [6, 6, 3], 6, 10) == 1
    # of two requests on one graph, the earlier is the one that starts
    assert _pick(lib, [2, 1, 1], [1, 0, 0], [6, 4, 9], 6, 10) == 1
    # a busy graph's requests wait; the next graph's first request starts
    assert _pick(lib, [0, 0, 2], [1, 0, 0], [6, 6, 3], 6, 10) == 2
    # larger than the budget: runs when nothing else does
    assert _pick(lib, [1], [0, 0, 0], [6, 50, 3], 0, 10) == 0
    assert _pick(lib, [1], [0, 0, 0], [6, 50, 3], 1, 10) == -1
