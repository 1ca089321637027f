"""Memory carving of the segmented BIT evaluation
(paper_2511_16356_gb300/csrc/kc_host_seg.h), compiled with the host C++
compiler and checked on random, disjoint regions at random alignments: every
Fenwick array (n int64, entries 1 .. n, 8-byte aligned) and every stack
(stack_cap int4, 16-byte aligned) lies inside one region, no two slots
overlap, a successful carve returns exactly the slots asked for, and
fit_segments returns the largest k <= kmax that carves (0 below two); and the
segment-count policy of ttf_segments."""
import ctypes
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2511_16356_gb300", "csrc")

SHIM = r"""
#include "kc_host_seg.h"
static std::vector<kc_host::SegRegion> regs(const uint64_t *p, const uint64_t *bytes, int nr) {
    std::vector<kc_host::SegRegion> r;
    for (int i = 0; i < nr; ++i) r.push_back({(uintptr_t)p[i], (size_t)bytes[i]});
    return r;
}
extern "C" int hs_carve(const uint64_t *p, const uint64_t *bytes, int nr, uint64_t need,
                        uint64_t bit_bytes, uint64_t stk_bytes, uint64_t *bits, uint64_t *stks) {
    std::vector<uintptr_t> b, s;
    const bool ok = kc_host::carve_segments(regs(p, bytes, nr), need, bit_bytes, stk_bytes, b, s);
    for (size_t i = 0; i < b.size() && i < need; ++i) bits[i] = b[i];
    for (size_t i = 0; i < s.size() && i < need; ++i) stks[i] = s[i];
    return ok ? 1 : 0;
}
extern "C" int hs_limit(int cfgk, int64_t b, int walk_over, int64_t sms) {
    return kc_host::seg_limit(cfgk, b, walk_over != 0, sms);
}
extern "C" int hs_fit(const uint64_t *p, const uint64_t *bytes, int nr, int64_t b, int kmax,
                      uint64_t bit_bytes, uint64_t stk_bytes) {
    std::vector<uintptr_t> x, y;
    return kc_host::fit_segments(regs(p, bytes, nr), b, kmax, bit_bytes, stk_bytes, x, y);
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("hostseg")
    (d / "shim.cpp").write_text(SHIM)
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(d / "shim.cpp"),
                    "-o", str(d / "shim.so")], check=True, capture_output=True)
    L = ctypes.CDLL(str(d / "shim.so"))
    u64p = ctypes.POINTER(ctypes.c_uint64)
    L.hs_carve.restype = ctypes.c_int
    L.hs_carve.argtypes = [u64p, u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                           ctypes.c_uint64, u64p, u64p]
    L.hs_limit.restype = ctypes.c_int
    L.hs_limit.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int64]
    L.hs_fit.restype = ctypes.c_int
    L.hs_fit.argtypes = [u64p, u64p, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                         ctypes.c_uint64, ctypes.c_uint64]
    return L


def _arr(xs):
    return (ctypes.c_uint64 * max(1, len(xs)))(*xs)


def _regions(rng, nr, bit_bytes):
    p, out = 1 << 40, []
    for _ in range(nr):
        p += rng.randrange(0, 4096)             # gap, any alignment
        size = rng.choice([rng.randrange(1, 64), rng.randrange(1, 3 * bit_bytes + 200),
                           rng.randrange(bit_bytes, 9 * bit_bytes)])
        out.append((p, size))
        p += size
    return out


def test_random_carves_are_inside_aligned_and_disjoint(lib):
    rng = random.Random(7)
    for _ in range(400):
        n = rng.randrange(2, 3000)
        cap = rng.randrange(2, 400)
        bit_bytes, stk_bytes = 8 * n, 16 * cap
        regs = _regions(rng, rng.randrange(1, 12), bit_bytes)
        need = rng.randrange(1, 40)
        bits = (ctypes.c_uint64 * need)()
        stks = (ctypes.c_uint64 * need)()
        ok = lib.hs_carve(_arr([a for a, _ in regs]), _arr([b for _, b in regs]), len(regs),
                          need, bit_bytes, stk_bytes, bits, stks)
        if not ok:
            continue
        spans = [(b + 8, b + 8 + bit_bytes) for b in bits] + [(s, s + stk_bytes) for s in stks]
        assert all((b + 8) % 8 == 0 for b in bits)
        assert all(s % 16 == 0 for s in stks)
        for lo, hi in spans:
            assert any(a <= lo and hi <= a + size for a, size in regs), (lo, hi)
        spans.sort()
        for (l0, h0), (l1, h1) in zip(spans, spans[1:]):
            assert h0 <= l1  # no overlap


def test_fit_returns_the_largest_k_that_carves(lib):
    rng = random.Random(11)
    for _ in range(200):
        n = rng.randrange(2, 2000)
        cap = rng.randrange(2, 300)
        bit_bytes, stk_bytes = 8 * n, 16 * cap
        regs = _regions(rng, rng.randrange(1, 10), bit_bytes)
        P, Bs = _arr([a for a, _ in regs]), _arr([b for _, b in regs])
        b = rng.randrange(1, 12)
        kmax = rng.randrange(2, 17)
        k = lib.hs_fit(P, Bs, len(regs), b, kmax, bit_bytes, stk_bytes)
        assert k == 0 or 2 <= k <= kmax

        def carves(kk):
            need = b * kk
            x = (ctypes.c_uint64 * need)()
            y = (ctypes.c_uint64 * need)()
            return lib.hs_carve(P, Bs, len(regs), need, bit_bytes, stk_bytes, x, y) == 1
        if k:
            assert carves(k)
        for kk in range(max(k + 1, 2), kmax + 1):
            assert not carves(kk)


def test_exact_fit_and_shortfall(lib):
    """One region of exactly two Fenwick arrays and two stacks (8-byte aligned
    start, the stacks 16-byte aligned after them) holds two segments, one byte
    less holds none."""
    n, cap = 10, 3
    base = (1 << 40) + 16
    size = 2 * 8 * n + 2 * 16 * cap
    bits = (ctypes.c_uint64 * 2)()
    stks = (ctypes.c_uint64 * 2)()
    assert lib.hs_carve(_arr([base]), _arr([size]), 1, 2, 8 * n, 16 * cap, bits, stks) == 1
    assert list(bits) == [base - 8, base + 8 * n - 8]
    assert list(stks) == [base + 16 * n, base + 16 * n + 16 * cap]
    assert lib.hs_carve(_arr([base]), _arr([size - 1]), 1, 2, 8 * n, 16 * cap, bits, stks) == 0
    assert lib.hs_fit(_arr([base]), _arr([size]), 1, 1, 16, 8 * n, 16 * cap) == 2
    assert lib.hs_fit(_arr([base]), _arr([size]), 1, 2, 16, 8 * n, 16 * cap) == 0


def test_segment_limit_policy(lib):
    """ttf_segments = k >= 2 forces k whatever the chunk; 1 never splits; 0
    splits only after the walk, to about 32 segment warps an SM and at most
    16 segments a tree."""
    sms = 152
    for k in (2, 5, 64):
        for b in (1, 1000, 100000):
            for over in (0, 1):
                assert lib.hs_limit(k, b, over, sms) == k
    for b in (1, 300, 5000):
        assert lib.hs_limit(1, b, 1, sms) == 0
        assert lib.hs_limit(0, b, 0, sms) == 0            # walk still running
    assert lib.hs_limit(0, 1, 1, sms) == 16               # capped at 16
    assert lib.hs_limit(0, 2400, 1, sms) == 2             # 4864 resident warps
    assert lib.hs_limit(0, 1000, 1, sms) == 4
    assert lib.hs_limit(0, 4864, 1, sms) == 1             # one a tree: no split below 2
    assert lib.hs_limit(0, 5000, 1, sms) == 0
    assert lib.hs_limit(0, 0, 1, sms) == 0
    assert lib.hs_limit(0, 3, 1, 0) == 10                 # unknown SM count: one SM's worth
