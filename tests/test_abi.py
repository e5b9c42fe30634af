"""CPU checks of the C ABI library: it builds, loads, exports every function
declared in include/*.h, and validates arguments on the host (no GPU call)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2301_05451_gb300 import build
    build.build()
    from paper_2301_05451_gb300 import _abi
    return _abi


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(tdq_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "tdq_execute" in names and len(names) >= 10
    L = lib.lib()
    for n in sorted(names):
        assert hasattr(L, n), n
    # and the Python binding covers the same set
    assert names == set(lib.SIGNATURES), names ^ set(lib.SIGNATURES)


def test_circuit_validation_on_host(lib):
    h = ctypes.c_void_p()
    L = lib.lib()
    assert L.tdq_circuit_create(0, ctypes.byref(h)) == lib.TDQ_ERR_ARG
    assert L.tdq_circuit_create(65, ctypes.byref(h)) == lib.TDQ_ERR_ARG
    assert L.tdq_circuit_create(3, ctypes.byref(h)) == lib.TDQ_OK
    bad_q = lib.int_array([3])
    assert L.tdq_circuit_gate(h, lib.GATES["RX"], bad_q, 1, lib.int_array([0]), None) == lib.TDQ_ERR_ARG
    assert b"qubit" in L.tdq_last_error()
    assert L.tdq_circuit_gate(h, 99, lib.int_array([0]), 1, None, None) == lib.TDQ_ERR_ARG
    assert L.tdq_circuit_gate(h, lib.GATES["CNOT"], lib.int_array([1, 1]), 2, None, None) == lib.TDQ_ERR_ARG
    assert L.tdq_circuit_gate(h, lib.GATES["RY"], lib.int_array([0]), 1, lib.int_array([lib.TDQ_FIXED]),
                              lib.double_array([float("nan")])) == lib.TDQ_ERR_NONFINITE
    assert L.tdq_circuit_gate(h, lib.GATES["RY"], lib.int_array([0]), 1, lib.int_array([4]), None) == lib.TDQ_OK
    assert L.tdq_circuit_gate(h, lib.GATES["RX"], lib.int_array([2]), 1,
                              lib.int_array([lib.TDQ_INPUT(2)]), None) == lib.TDQ_OK
    assert L.tdq_circuit_observable(h, lib.int_array([0, 0]), 2, 1.0, 0) == lib.TDQ_ERR_ARG
    assert L.tdq_circuit_observable(h, lib.int_array([0, 2]), 2, 0.5, 1) == lib.TDQ_OK
    bits = (ctypes.c_uint8 * 3)(0, 2, 0)
    assert L.tdq_circuit_amplitude(h, bits) == lib.TDQ_ERR_ARG
    vals = [ctypes.c_int() for _ in range(6)]
    assert L.tdq_circuit_info(h, *[ctypes.byref(v) for v in vals]) == lib.TDQ_OK
    assert [v.value for v in vals] == [2, 5, 3, 2, 1, 0]
    assert L.tdq_circuit_destroy(h) == lib.TDQ_OK


def test_compile_argument_errors_before_device(lib):
    L = lib.lib()
    h = ctypes.c_void_p()
    L.tdq_circuit_create(2, ctypes.byref(h))
    out = ctypes.c_void_p()
    opts = lib.CompileOpts(0, 0, 0, 0, 0, 0)
    assert L.tdq_compile_sweep(h, ctypes.byref(opts), ctypes.byref(out)) == lib.TDQ_ERR_ARG
    opts = lib.CompileOpts(1, 1, 1, 0, 0, 0)  # gradients of amplitudes
    assert L.tdq_compile_sweep(h, ctypes.byref(opts), ctypes.byref(out)) == lib.TDQ_ERR_UNSUPPORTED
    opts = lib.CompileOpts(1, 0, 0, 0, 0, 0)  # no observable
    assert L.tdq_compile_sweep(h, ctypes.byref(opts), ctypes.byref(out)) == lib.TDQ_ERR_STATE
    L.tdq_circuit_destroy(h)


def test_package_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2301_05451_gb300 import _abi
    monkeypatch.setattr(_abi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_abi, "_lib", None)
    with pytest.raises(ImportError):
        _abi.lib()


def test_plan_compile_option_errors_before_device(lib):
    """Tree-plan launch options are checked on the host before any device call."""
    from paper_2301_05451_gb300 import api, workloads as W
    C = api.Circuit(W.hea6()[0])
    P = api.Plan(api.Network(C, "expval", 0))
    L = lib.lib()
    out = ctypes.c_void_p()
    for field, bad in (("subtree_log2", 14), ("subtree_log2", -1), ("tc_min_log2", 65), ("tc_min_log2", -2)):
        opts = lib.CompileOpts(1, 0, 0, 0, 0, 0)
        setattr(opts, field, bad)
        assert L.tdq_plan_compile(P.h, ctypes.byref(opts), ctypes.byref(out)) == lib.TDQ_ERR_ARG, (field, bad)


def test_multi_compile_argument_errors_before_device(lib):
    """tdq_compile_multi checks its arguments on the host before any device call."""
    from paper_2301_05451_gb300 import api, workloads as W
    small = api.Circuit(W.hea6()[0])
    big = api.Circuit(W.random_circuit(14, 20, 5)[0])
    bare = W.CircuitSpec(3)
    bare.add("H", [0])
    noobs = api.Circuit(bare)
    L = lib.lib()
    out = ctypes.c_void_p()

    def call(circs, batch, **kw):
        o = lib.CompileOpts(1, lib.TDQ_OUT_EXPVAL, kw.pop("grad", lib.TDQ_GRAD_NONE), 0, 0, 0)
        for k, v in kw.items():
            setattr(o, k, v)
        hs = (ctypes.c_void_p * max(len(circs), 1))(*[c.h.value for c in circs])
        return L.tdq_compile_multi(hs, lib.int_array(batch or [0]), len(circs), ctypes.byref(o), ctypes.byref(out))

    assert call([], []) == lib.TDQ_ERR_ARG
    assert call([small], [0]) == lib.TDQ_ERR_ARG
    assert call([small], [1], output=lib.TDQ_OUT_AMPLITUDE) == lib.TDQ_ERR_ARG
    assert call([small], [1], interpret=1) == lib.TDQ_ERR_ARG
    assert call([small], [1], fwd_reg_bits=5) == lib.TDQ_ERR_ARG
    assert call([small], [1], autotune=1, rev_reg_bits=2) == lib.TDQ_ERR_ARG
    assert call([small, big], [1, 1], grad=lib.TDQ_GRAD_ADJOINT) == lib.TDQ_ERR_UNSUPPORTED
    assert call([small, noobs], [1, 1]) == lib.TDQ_ERR_STATE
    assert L.tdq_multi_layout(None, 0, None, None, None, None) == lib.TDQ_ERR_ARG
