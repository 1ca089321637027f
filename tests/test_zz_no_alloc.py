"""kc_wilson_noalloc: tree sampling for callers that cannot allocate device
memory (allocator callbacks, fixed-budget plugins, latency-critical paths).

The call keeps its working state in a fixed array inside the library, so its
trees must equal the ones the regular entry points (kc_sample + kc_get_tree)
draw for the same sample ids -- bit for bit, like every integer output here.
Two calls in a row check that the shared array is cleared between calls.
This file is collected last so a failure here does not hide other results.
"""
import numpy as np
import pytest

from paper_2511_16356_gb300 import synth as S

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_sampler_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_2511_16356_gb300 import build as kbuild
    from paper_2511_16356_gb300 import kc

    kbuild.build()
    lib = kc.load()
    g = S.er_lcc(300, 0.02, 7)
    n, seed, total = g.n, 99, 96
    with kc.KemenyGraph.from_graph(g) as G:
        G.sample(seed, total)
        ref_steps = G.samples()["steps"]
        root = G.tau0()["root"]
        ref_par = np.stack([G.tree(k)["parent"] for k in range(total)])

    ro = torch.from_numpy(g.row_off).cuda()
    co = torch.from_numpy(g.col).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for first, cnt in [(0, 64), (32, 64)]:  # the second call overlaps the first's ids
        par = torch.full((cnt, n), -7, dtype=torch.int32, device="cuda")
        steps = torch.zeros(cnt, dtype=torch.int64, device="cuda")
        status = torch.full((1,), 5, dtype=torch.int32, device="cuda")
        st = lib.kc_wilson_noalloc(n, ro.data_ptr(), co.data_ptr(), root, seed, first, cnt, 0,
                                   par.data_ptr(), steps.data_ptr(), status.data_ptr(), stream)
        assert kc.STATUS[st] == "KC_OK"
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert np.array_equal(par.cpu().numpy(), ref_par[first:first + cnt])
        assert np.array_equal(steps.cpu().numpy(), ref_steps[first:first + cnt])

    # a request beyond the fixed scratch is refused before anything runs
    too_many = (8 << 20) // n + 1
    st = lib.kc_wilson_noalloc(n, ro.data_ptr(), co.data_ptr(), root, seed, 0, too_many, 0,
                               par.data_ptr(), steps.data_ptr(), status.data_ptr(), stream)
    assert kc.STATUS[st] == "KC_ERR_SCRATCH_LIMIT"
