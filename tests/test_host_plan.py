"""Wave planning of kc_sample (paper_2511_16356_gb300/csrc/kc_host_plan.h),
compiled with the host C++ compiler: the planned workspace fits the budget
(up to 256-byte alignment), waves hold at least one tree and never more than
asked for or allowed, sub-waves never exceed waves, more budget never gives
smaller waves, and the BIT split gives the walk about 70% of the budget."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2511_16356_gb300", "csrc")

SHIM = r"""
#include "kc_host_plan.h"
extern "C" void hp_plan(int64_t n, int64_t ntrees, int bit, int canon, double budget,
                        int64_t max_in_flight, double share, int64_t *bw, int64_t *bt,
                        uint64_t *bytes) {
    const kc_host::Plan p = kc_host::plan_waves(n, ntrees, bit != 0, canon != 0, budget,
                                                max_in_flight, share);
    *bw = p.BW;
    *bt = p.BT;
    *bytes = kc_host::ws_bytes(n, p);
}
extern "C" int64_t hp_reject(int64_t need, int64_t drawn, int64_t accepted, double hint) {
    return kc_host::reject_wave_size(need, drawn, accepted, hint);
}
"""


@pytest.fixture(scope="module")
def plan(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("hostplan")
    (d / "shim.cpp").write_text(SHIM)
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(d / "shim.cpp"),
                    "-o", str(d / "shim.so")], check=True, capture_output=True)
    lib = ctypes.CDLL(str(d / "shim.so"))
    lib.hp_plan.restype = None
    lib.hp_plan.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                            ctypes.c_double, ctypes.c_int64, ctypes.c_double] + \
        [ctypes.c_void_p] * 3

    def run(n, ntrees, bit, canon, budget, cap=0, share=0.7):
        bw, bt, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_uint64()
        lib.hp_plan(n, ntrees, int(bit), int(canon), float(budget), cap, share, ctypes.byref(bw),
                    ctypes.byref(bt), ctypes.byref(b))
        return bw.value, bt.value, b.value
    lib.hp_reject.restype = ctypes.c_int64
    lib.hp_reject.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double]
    run.reject = lib.hp_reject
    return run


SLACK = 256 * 12  # at most 12 aligned regions


@pytest.mark.parametrize("share", [0.7, 0.9])
@pytest.mark.parametrize("bit", [False, True])
@pytest.mark.parametrize("canon", [False, True])
@pytest.mark.parametrize("n", [2, 2000, 10 ** 6, 4 * 10 ** 6])
def test_plans_fit_the_budget(plan, n, bit, canon, share):
    one = plan(n, 1, bit, canon, 0.0)[2]  # what a single tree needs
    for budget in (one, 3.7 * one, 1e9, 4e10, 2.3e11):
        for ntrees in (1, 64, 10000):
            bw, bt, b = plan(n, ntrees, bit, canon, budget, share=share)
            assert 1 <= bt <= bw <= min(ntrees, 1 << 20) and bt <= 65535
            if budget >= one:
                assert b <= budget + SLACK, (budget, bw, bt, b)
            if not bit:
                assert bt == min(bw, 65535)


def test_caps_and_monotone_budget(plan):
    n = 10 ** 6
    assert plan(n, 10000, True, False, 2.3e11, cap=500)[0] == 500
    prev = 0
    for budget in (1e9, 1e10, 5e10, 1e11, 2e11):
        bw = plan(n, 10 ** 6, False, False, budget)[0]
        assert bw >= prev
        prev = bw
    # long-diameter graphs: about 70% of the budget to walker waves by default,
    # the requested share otherwise
    bw, bt, b = plan(n, 10 ** 6, True, False, 1e11)
    walk = bw * 12 * n
    assert 0.68 < walk / 1e11 <= 0.7
    bw, bt, b = plan(n, 10 ** 6, True, False, 2.2e11, share=0.9)
    assert 0.88 < bw * 12 * n / 2.2e11 <= 0.9 and bt >= 1


def test_rejection_wave_size_rarely_falls_short(plan):
    """A rejection wave draws need / rate plus three standard deviations: at the
    assumed rate the chance that it accepts fewer than `need` trees is about
    the normal tail beyond 3 sd (checked by binomial sampling), it grows as the
    rate falls, uses the hint before any tree is seen, and the observed rate
    afterwards."""
    import numpy as np

    rs = plan.reject
    rng = np.random.default_rng(0)
    for rate in (0.9, 0.65, 0.3):
        for need in (100, 4096, 10000):
            B = rs(need, 0, 0, rate)
            assert B >= need / rate
            short = (rng.binomial(B, rate, size=20000) < need).mean()
            assert short < 0.005, (rate, need, B, short)
    assert rs(10000, 0, 0, 0.5) > rs(10000, 0, 0, 0.8)
    # the observed rate replaces the hint
    assert rs(10000, 20000, 10000, 0.9) == rs(10000, 0, 0, 10001 / 20001)
    assert rs(10000, 1000, 0, 0.9) == rs(10000, 0, 0, 1 / 64)  # floor on the rate
