"""The C-ABI library loads and exports every function include/gsm.h declares;
host-side argument validation needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "gsm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|int64_t|size_t|const char\*)\s+(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2006_04391_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("gsm_create", "gsm_update", "gsm_destroy", "ms_solve", "ms_create", "ms_run"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_the_same_symbols():
    import paper_2006_04391_gb300 as G
    assert sorted(G.EXPORTS) == declared_functions()


def test_create_validates_parameters(lib):
    import paper_2006_04391_gb300 as G
    G.load()
    G.norton(70.0, 0.3, 0.1, 1.0, 5.0)
    G.elastic(400.0, 0.2, precision=G.GSM_FP32)
    for bad in [(70.0, 0.3, 0.0, 1.0, 5.0), (70.0, 0.3, 0.1, -1.0, 5.0), (70.0, 0.3, 0.1, 1.0, 0.0),
                (-70.0, 0.3, 0.1, 1.0, 5.0), (70.0, 0.5, 0.1, 1.0, 5.0), (70.0, float("nan"), 0.1, 1.0, 5.0)]:
        with pytest.raises(G.GsmError) as ei:
            G.norton(*bad)
        assert ei.value.code == G.GSM_EINVAL
    with pytest.raises(G.GsmError):
        G.gsm_create(G.GSM_PSI_ELASTIC, G.GSM_PHI_NORTON, (1.0, 0.2), 0)
    with pytest.raises(G.GsmError):
        G.gsm_create(G.GSM_PSI_ELASTIC, G.GSM_PHI_NONE, (1.0, 0.2), 7)


def test_ms_create_rejects_bad_problems(lib):
    import paper_2006_04391_gb300 as G
    G.load()
    h = ctypes.c_void_p()
    prob = G.ms_problem(1, None, 1, None, 0)
    assert lib.ms_create(ctypes.byref(h), ctypes.byref(prob), None) == G.GSM_EINVAL
    assert G.ms_workspace_bytes(1) == 0
    assert G.ms_workspace_bytes(64) > 6 * 8 * 64 ** 3 * 4


def test_strerror(lib):
    lib.gsm_strerror.restype = ctypes.c_char_p
    assert lib.gsm_strerror(0) == b"ok"
    assert lib.gsm_strerror(-4) == b"iteration cap reached"
