"""The C-ABI library loads and exports every entry point include/*.h declares
(no compute calls: these run without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("kc.h", "kc_serve.h")]


def _declared():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names.update(re.findall(r"\b(kc_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2511_16356_gb300 import build as kbuild
    from paper_2511_16356_gb300 import kc

    kbuild.build()
    return kc.load()


def test_header_parses():
    names = _declared()
    for must in ["kc_graph_create", "kc_sample", "kc_estimate", "kc_update", "kc_get_tree",
                 "kc_stats", "kc_status_string", "kc_graph_set_stream", "kc_graph_destroy"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_mirrors_header():
    from paper_2511_16356_gb300 import kc

    assert sorted(kc.EXPORTED) == _declared()


def test_status_strings(lib):
    from paper_2511_16356_gb300 import kc

    for code in kc.STATUS:
        assert kc.kc_status_string(code)
    assert kc.kc_status_string(9999) == "unknown status"


def test_config_defaults(lib):
    from paper_2511_16356_gb300 import kc

    c = kc.kc_config_default()
    assert c.struct_size == __import__("ctypes").sizeof(kc.kc_config)
    assert c.root == -1 and c.keep_trees == 1 and c.step_cap == 0


def test_null_arguments_are_rejected(lib):
    import ctypes

    from paper_2511_16356_gb300 import kc

    h = ctypes.c_void_p()
    assert lib.kc_graph_create(1, None, None, None, ctypes.byref(h)) == 1
    assert lib.kc_sample(None, 0, 1) == 1
    assert lib.kc_graph_destroy(None) == 0
    assert lib.kc_estimate(None, 0.1, 0.1, None) == 1
    assert kc.STATUS[lib.kc_update(None, None, 0, 0)] == "KC_ERR_INVALID_ARG"


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="checks the no-device path")
def test_no_device_is_reported(lib):
    import numpy as np

    from paper_2511_16356_gb300 import kc
    from paper_2511_16356_gb300 import synth as S

    g = S.cycle(5)
    st, h = kc.kc_graph_create(g.row_off, g.col, check=False)
    assert kc.STATUS[st] == "KC_ERR_NO_DEVICE" and not h
    assert np.all(g.deg == 2)


def test_rejection_config_is_checked_before_any_device_work(lib):
    """Rejection by walk length needs the 32-walker kernel, static pools, no
    autotune and a cap of at least n - 1 departures (each non-root vertex
    departs once): anything else is INVALID_ARG before the device is touched;
    a valid setting passes on to the device check."""
    from paper_2511_16356_gb300 import kc
    from paper_2511_16356_gb300 import synth as S

    g = S.cycle(12)

    def status(**kw):
        c = kc.kc_config_default()
        c.keep_trees = 0
        for k, v in kw.items():
            setattr(c, k, v)
        st, h = kc.kc_graph_create(g.row_off, g.col, c, check=False)
        if h:
            kc.kc_graph_destroy(h)
        return kc.STATUS[st]

    assert kc.kc_config_default().reject_steps == 0
    assert status(reject_steps=-1) == "KC_ERR_INVALID_ARG"
    assert status(reject_steps=10) == "KC_ERR_INVALID_ARG"            # below n - 1 = 11
    assert status(reject_steps=100, keep_trees=1) == "KC_ERR_INVALID_ARG"
    assert status(reject_steps=100, autotune=1) == "KC_ERR_INVALID_ARG"
    assert status(reject_steps=100, walker=kc.KC_WALK_HYBRID) == "KC_ERR_INVALID_ARG"
    if not os.path.exists("/dev/nvidia0"):
        assert status(reject_steps=11) == "KC_ERR_NO_DEVICE"
        assert status(reject_steps=100, walker=kc.KC_WALK_LANE) == "KC_ERR_NO_DEVICE"


def test_ttf_segments_config_is_checked_before_any_device_work(lib):
    """ttf_segments: 0 (automatic, the default), 1 (never) or 2 .. 64 segments a
    tree; anything else is INVALID_ARG before the device is touched."""
    from paper_2511_16356_gb300 import kc
    from paper_2511_16356_gb300 import synth as S

    g = S.cycle(12)

    def status(k):
        c = kc.kc_config_default()
        c.ttf_segments = k
        st, h = kc.kc_graph_create(g.row_off, g.col, c, check=False)
        if h:
            kc.kc_graph_destroy(h)
        return kc.STATUS[st]

    assert kc.kc_config_default().ttf_segments == 0
    assert status(-1) == "KC_ERR_INVALID_ARG"
    assert status(65) == "KC_ERR_INVALID_ARG"
    if not os.path.exists("/dev/nvidia0"):
        for k in (0, 1, 2, 64):
            assert status(k) == "KC_ERR_NO_DEVICE"


def test_server_config_defaults(lib):
    import ctypes

    from paper_2511_16356_gb300 import kc

    c = kc.kc_server_config()
    lib.kc_server_config_default(ctypes.byref(c))
    assert c.struct_size == ctypes.sizeof(kc.kc_server_config)
    assert c.workers == 4 and c.budget_bytes == 0 and c.request_bytes == 0


def _struct_fields(header, name):
    """Field names, in order, of `typedef struct { ... } name;` in a header."""
    import re as _re

    src = open(os.path.join(ROOT, "include", header)).read()
    src = _re.sub(r"/\*.*?\*/", "", src, flags=_re.S)
    end = _re.search(r"\}\s*" + name + r"\s*;", src)
    assert end, name
    start = src.rfind("typedef struct", 0, end.start())
    body = src[src.index("{", start) + 1:end.start()]
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            tok = part.strip().split()[-1]
            fields.append(_re.sub(r"\[.*\]", "", tok).lstrip("*"))
    return fields


@pytest.mark.parametrize("header,name,pyname", [
    ("kc.h", "kc_config", "kc_config"), ("kc.h", "kc_edge_op", "kc_edge_op"),
    ("kc.h", "kc_stats_t", "kc_stats_t"), ("kc_serve.h", "kc_server_config", "kc_server_config"),
    ("kc_serve.h", "kc_request_info", "kc_request_info")])
def test_binding_structs_match_header_field_order(header, name, pyname):
    from paper_2511_16356_gb300 import kc

    assert [f for f, _ in getattr(kc, pyname)._fields_] == _struct_fields(header, name)


def test_binding_struct_sizes_match_the_c_compiler(tmp_path):
    """sizeof of every ABI struct as gcc lays it out equals the ctypes size."""
    import ctypes
    import shutil
    import subprocess

    from paper_2511_16356_gb300 import kc

    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    names = ["kc_config", "kc_edge_op", "kc_stats_t", "kc_server_config", "kc_request_info"]
    prog = tmp_path / "sizes.c"
    prog.write_text('#include <stdio.h>\n#include "kc_serve.h"\nint main(void) {\n' +
                    "".join(f'  printf("%zu\\n", sizeof({n}));\n' for n in names) +
                    "  return 0;\n}\n")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == [ctypes.sizeof(getattr(kc, n)) for n in names]


def test_noalloc_rejects_bad_arguments_before_device_work(lib):
    """kc_wilson_noalloc validates its sizes before it touches a device: sample
    ids past 2^32 (including a count whose sum with the first id would overflow
    int64), negative counts and oversized requests are refused, and zero trees
    is a no-op.  The pointers are never dereferenced on these paths."""
    from paper_2511_16356_gb300 import kc

    p = 256  # a non-null dummy address, never read
    call = lambda n, first, cnt: kc.STATUS[lib.kc_wilson_noalloc(n, p, p, 0, 1, first, cnt, 0,
                                                                  p, p, p, None)]
    assert call(10, (1 << 32) - 4, 5) == "KC_ERR_INVALID_ARG"
    assert call(10, 1 << 40, 1) == "KC_ERR_INVALID_ARG"
    assert call(10, 7, (1 << 63) - 2) == "KC_ERR_INVALID_ARG"
    assert call(10, 0, -1) == "KC_ERR_INVALID_ARG"
    assert call(1, 0, 1) == "KC_ERR_INVALID_ARG"
    assert call(10, 0, 0) == "KC_OK"
    assert call(1 << 20, 0, 9) == "KC_ERR_SCRATCH_LIMIT"
