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


def test_peak_probe_validates_arguments(lib):
    """The FMA-throughput probe refuses bad arguments before any CUDA call."""
    f = ctypes.c_double()
    lib.gsm_peak_probe.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                   ctypes.c_void_p]
    for prec, iters, bps, out in [(2, 10, 1, ctypes.byref(f)), (0, 0, 1, ctypes.byref(f)),
                                  (1, 1 << 33, 1, ctypes.byref(f)), (0, 10, 0, ctypes.byref(f)),
                                  (0, 10, 65, ctypes.byref(f)), (0, 10, 1, None)]:
        assert lib.gsm_peak_probe(prec, iters, bps, out, None) == -1


def test_update_entries_validate_before_any_device_work(lib):
    """Argument checks of the update entry points that return before any CUDA
    call: no handle, negative sizes, an unknown integrator, a negative chunk,
    the Michel-Suquet law on the implicit path, its parameter ranges."""
    import paper_2006_04391_gb300 as G
    L = G.load()
    nor = G.norton(70.0, 0.3, 0.1, 1.0, 5.0)
    ms = G.michel_suquet(55.0, 0.33, 0.025, 1.8, 1.0, 0.13, 3.6)
    x = ctypes.c_void_p(16)  # never dereferenced: every call below returns before touching it
    d = ctypes.c_double
    assert L.gsm_update(None, 4, x, x, 4, d(0.1), x, x, None, None, None) == G.GSM_EINVAL
    assert L.gsm_update(nor.handle, -1, x, x, 4, d(0.1), x, x, None, None, None) == G.GSM_EINVAL
    assert L.gsm_update(nor.handle, 8, x, x, 4, d(0.1), x, x, None, None, None) == G.GSM_EINVAL  # ld < n
    assert L.gsm_update(nor.handle, 0, x, x, 4, d(0.1), x, x, None, None, None) == G.GSM_OK  # no-op
    assert L.gsm_update(ms.handle, 4, x, x, 4, d(0.1), x, x, None, None, None) == G.GSM_ENOTSUP
    assert L.gsm_update_host(nor.handle, 4, x, x, 4, d(0.1), x, x, None, None, -1, None) == G.GSM_EINVAL
    assert L.gsm_update_host(ms.handle, 4, x, x, 4, d(0.1), x, x, None, None, 0, None) == G.GSM_ENOTSUP
    for method in (-1, 3, 7):
        assert L.gsm_update_ode(nor.handle, method, 4, x, x, x, 4, d(0.1), d(1e-3), d(1e-6), 100, x, x, None, None,
                                None) == G.GSM_EINVAL
    el = G.elastic(70.0, 0.3)
    assert L.gsm_update_ode(el.handle, G.GSM_ODE23, 4, x, x, x, 4, d(0.1), d(1e-3), d(1e-6), 100, x, x, None, None,
                            None) == G.GSM_ENOTSUP
    for bad in [(55.0, 0.33, -0.025, 1.8, 1.0, 0.13, 3.6), (55.0, 0.33, 0.025, -1.8, 1.0, 0.13, 3.6),
                (55.0, 0.33, 0.025, 1.8, 0.0, 0.13, 3.6), (55.0, 0.33, 0.025, 1.8, 1.0, 0.0, 3.6),
                (55.0, 0.33, 0.025, 1.8, 1.0, 0.13, 0.5)]:
        with pytest.raises(G.GsmError):
            G.michel_suquet(*bad)


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


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the header's size and
    field offsets (compiled with the host C compiler; no GPU needed)."""
    import ctypes
    import os
    import subprocess

    import paper_2006_04391_gb300 as G
    src = os.path.join(os.path.dirname(__file__), "native", "abi_layout.c")
    exe = str(tmp_path / "abi_layout")
    subprocess.run(["gcc", "-std=c11", "-o", exe, src], check=True)
    layout = {}
    for line in subprocess.run([exe], check=True, capture_output=True, text=True).stdout.splitlines():
        struct, field, value = line.split()
        layout[(struct, field)] = int(value)
    structs = {"ms_problem": G.ms_problem, "ms_load": G.ms_load, "ms_state": G.ms_state,
               "ms_result": G.ms_result, "serve_job": G.serve_job}
    for name, cls in structs.items():
        assert ctypes.sizeof(cls) == layout[(name, ".")], name
        fields = [f[0] for f in cls._fields_]
        c_fields = [f for (s, f) in layout if s == name and f != "."]
        assert fields == c_fields, name
        for f in fields:
            assert getattr(cls, f).offset == layout[(name, f)], (name, f)
