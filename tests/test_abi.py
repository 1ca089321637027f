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


def test_server_config_defaults(lib):
    import ctypes

    from paper_2511_16356_gb300 import kc

    c = kc.kc_server_config()
    lib.kc_server_config_default(ctypes.byref(c))
    assert c.struct_size == ctypes.sizeof(kc.kc_server_config)
    assert c.workers == 4 and c.budget_bytes == 0 and c.request_bytes == 0
