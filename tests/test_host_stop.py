"""The stopping rules of kc_estimate (paper_2511_16356_gb300/csrc/kc_host_stop.h),
compiled with the host C++ compiler and compared with the oracle's restatement
(oracle/estimate.py): the normal quantile, Theorem 5's sample size, and the
batch sizes the normal-approximation rule draws on the same f sequences, with
the pool moments summed in double as the device reduction does."""
import ctypes
import os
import shutil
import subprocess
from statistics import NormalDist

import numpy as np
import pytest

import oracle as O
from paper_2511_16356_gb300 import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2511_16356_gb300", "csrc")

SHIM = r"""
#include "kc_host_stop.h"
extern "C" double hs_z(double p) { return kc_host::inv_normal_upper(p); }
extern "C" int64_t hs_hoeffding(int64_t n, int64_t m, int64_t ecc, double eps, double delta,
                                int64_t cap) {
    return kc_host::hoeffding_trees(n, m, ecc, eps, delta, cap);
}
extern "C" int hs_run(const int64_t *f, int64_t nf, int64_t twom, double eps, double delta,
                      int64_t batch, int64_t cap, int64_t *sizes, int max_sizes) {
    int64_t pool = 0;
    double wf = 0, w = 0, x2 = 0;
    int ns = 0;
    bool over = false;
    const double inv = 1.0 / (double)twom;
    auto draw = [&](int64_t k) {
        if (ns < max_sizes) sizes[ns] = k;
        ++ns;
        for (int64_t i = 0; i < k; ++i) {
            if (pool >= nf) { over = true; return; }
            const double x = (double)f[pool] * inv;
            wf += x; w += 1.0; x2 += x * x; ++pool;
        }
    };
    auto read = [&] { return kc_host::Moments{pool, wf, w, x2}; };
    kc_host::run_clt(delta, eps, batch, cap, 0, draw, read);
    return over ? -1 : ns;
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("hoststop")
    (d / "shim.cpp").write_text(SHIM)
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(d / "shim.cpp"),
                    "-o", str(d / "shim.so")], check=True, capture_output=True)
    h = ctypes.CDLL(str(d / "shim.so"))
    h.hs_z.restype = ctypes.c_double
    h.hs_z.argtypes = [ctypes.c_double]
    h.hs_hoeffding.restype = ctypes.c_int64
    h.hs_hoeffding.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                               ctypes.c_double, ctypes.c_int64]
    h.hs_run.restype = ctypes.c_int
    h.hs_run.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                         ctypes.c_double, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                         ctypes.c_int]
    return h


def test_normal_quantile(lib):
    # -inv_cdf(p) rather than inv_cdf(1 - p): 1 - p would round away the tail
    for p in (0.025, 0.005, 0.05, 0.3, 1e-6):
        assert lib.hs_z(p) == pytest.approx(-NormalDist().inv_cdf(p), rel=1e-12)


def test_hoeffding_size(lib):
    for n, m, ecc, eps, delta in [(7, 21, 1, 0.5, 0.05), (40, 40, 20, 1.0, 0.05),
                                  (2000, 8020, 5, 0.01, 0.01)]:
        want = min(O.hoeffding_trees(n, m, ecc, eps, delta), 1 << 24)
        assert lib.hs_hoeffding(n, m, ecc, eps, delta, 1 << 24) == want
    assert lib.hs_hoeffding(2000, 8020, 5, 0.01, 0.01, 5000) == 5000


def _sizes(lib, f, twom, eps, delta, batch, cap=1 << 24):
    f = np.ascontiguousarray(f, dtype=np.int64)
    out = np.zeros(128, dtype=np.int64)
    ns = lib.hs_run(f.ctypes.data, f.shape[0], twom, eps, delta, batch, cap, out.ctypes.data, 128)
    assert ns > 0, "the f sequence ran out"
    return out[:ns].tolist()


def test_alternating_sequence(lib):
    f = [900 if i % 2 == 0 else 1100 for i in range(5000)]
    assert _sizes(lib, f, 1000, 0.01, 0.05, 64) == [64, 335]
    assert _sizes(lib, f, 1000, 0.001, 0.05, 64, cap=100) == [64, 36]


@pytest.mark.parametrize("name,eps,batch", [("er300", 0.01, 64), ("cl3000", 0.005, 64),
                                            ("grid17x13", 0.02, 100), ("er300", 0.01, 1024),
                                            ("grid17x13", 0.01, 64)])
def test_batches_match_the_oracle(lib, name, eps, batch):
    g = {"er300": lambda: S.er_lcc(300, 0.02, 7), "cl3000": lambda: S.chung_lu(3000, 2.1, 8.0, 5),
         "grid17x13": lambda: S.grid_perturbed(17, 13, 0.25, 3)}[name]()
    t0 = O.tau0(g)
    f, _ = O.sample_batch(g, t0, 0, 0, 20000)
    ref = O.estimate_clt(lambda a, c: f[a:a + c], 2 * g.m, eps, 0.05, batch=batch)
    assert ref.margin > 1e-9
    assert _sizes(lib, f, 2 * g.m, eps, 0.05, batch) == ref.sizes
