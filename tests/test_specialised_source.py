"""CPU checks of the specialised whole-state kernels: the source the library
generates for a circuit (tdq_sweep_source) compiles for sm_103a with NVRTC,
for every gate kind and register-bit placement, with and without the reverse
program.  (Running them, and their parity with the oracle, needs a GPU:
tests/test_gpu_sweep.py.)"""
import ctypes
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", "tdq.h")] + [
    os.path.join(ROOT, "paper_2301_05451_gb300", "csrc", f) for f in ("sweep_common.cuh", "engine.cuh", "k1_body.cuh", "k2_body.cuh")]


@pytest.fixture(scope="module")
def nvrtc():
    from paper_2301_05451_gb300 import build
    build.build()
    try:
        lib = ctypes.CDLL(os.path.join(build.CUDA_LIB, "libnvrtc.so"))
    except OSError as e:
        pytest.skip("libnvrtc not loadable: %s" % e)
    return lib


def _compile(nvrtc, src):
    prog = ctypes.c_void_p()
    names = (ctypes.c_char_p * len(HEADERS))(*[os.path.basename(h).encode() for h in HEADERS])
    bodies = (ctypes.c_char_p * len(HEADERS))(*[open(h, "rb").read() for h in HEADERS])
    assert nvrtc.nvrtcCreateProgram(ctypes.byref(prog), src.encode(), b"spec.cu", len(HEADERS), bodies, names) == 0
    opts = [b"-arch=sm_103a", b"-std=c++17", b"-default-device"]
    r = nvrtc.nvrtcCompileProgram(prog, len(opts), (ctypes.c_char_p * len(opts))(*opts))
    n = ctypes.c_size_t()
    nvrtc.nvrtcGetProgramLogSize(prog, ctypes.byref(n))
    log = ctypes.create_string_buffer(n.value + 1)
    nvrtc.nvrtcGetProgramLog(prog, log)
    nvrtc.nvrtcDestroyProgram(ctypes.byref(prog))
    return r, log.value.decode(errors="replace")


def _circuits():
    from paper_2301_05451_gb300 import workloads as W
    spec7 = W.random_circuit(7, 70, seed=41)[0]
    for q in range(7):  # Y and Z too
        spec7.add("Y", [q])
        spec7.add("Z", [(q + 3) % 7])
    spec16 = W.random_circuit(16, 120, seed=44)[0]
    for q in range(16):
        spec16.add("Y", [q])
        spec16.add("Z", [(q + 5) % 16])
    # (name, circuit, gradient, tile bits: 0 = whole state in one CTA)
    return [("hea6", W.hea6()[0], "adjoint", 0), ("random7", spec7, "adjoint", 0),
            ("random3", W.random_circuit(3, 25, seed=42)[0], "adjoint", 0),
            ("random5_value", W.random_circuit(5, 40, seed=43)[0], "none", 0),
            ("ladder20_tiled", W.ladder20()[0], "adjoint", 12),
            ("random16_tiled", spec16, "adjoint", 8),
            ("random16_tiled_value", spec16, "none", 10)]


def _share_tables(src):
    """The gradient-share index tables of a generated source: (size, entries,
    the row stride of the grad_share_multi call that reads the table)."""
    import re
    tabs = {name: (int(k), [int(v) for v in body.split(",")])
            for name, k, body in re.findall(r"__constant__ int (tdq_gi_\d+)\[(\d+)\] = \{([^}]*)\}", src)}
    calls = re.findall(r"grad_share_multi<(\d+)>\(gpart, (\d+), (tdq_gi_\d+), gs\d+\)", src)
    assert len(calls) == len(tabs)
    out = []
    for k, stride, name in calls:
        assert tabs[name][0] == int(k)
        out.append((int(k), tabs[name][1], int(stride)))
    return out


@pytest.mark.parametrize("case", ["random7", "ladder20_tiled", "tied5", "tied7_tiled", "tied3_two_params"])
def test_gradient_share_tables_never_repeat_an_index(case):
    """A table's K lanes add to one shared-memory word each in one
    instruction, so an index held twice would lose an addition (tied
    parameters made real entries repeat; padding repeated entry 0)."""
    from paper_2301_05451_gb300 import api, build
    from paper_2301_05451_gb300 import workloads as W
    build.build()
    circuits = {n: (c, t) for n, c, g, t in _circuits()}
    spec, tile = {"random7": circuits["random7"], "ladder20_tiled": circuits["ladder20_tiled"],
                  "tied5": (W.random_circuit_tied(5, 60, 4, 7)[0], 0),
                  "tied7_tiled": (W.random_circuit_tied(7, 84, 6, 8)[0], 5),
                  "tied3_two_params": (W.random_circuit_tied(3, 36, 2, 9)[0], 0)}[case]
    tables = _share_tables(api.Circuit(spec).specialised_source("adjoint", tile_qubits=tile))
    assert tables
    for k, idx, stride in tables:
        assert len(idx) == k and k & (k - 1) == 0 and k <= 32
        assert len(set(idx)) == k, idx
        # inside the warp's row: padding never reaches the next warp's
        assert 0 <= min(idx) and max(idx) < stride, (idx, stride)


@pytest.mark.parametrize("case", range(7))
def test_generated_source_compiles(nvrtc, case):
    from paper_2301_05451_gb300 import api
    name, spec, grad, tile = _circuits()[case]
    src = api.Circuit(spec).specialised_source(grad, tile_qubits=tile)
    assert 'extern "C" __global__' in src
    if tile == 0:
        assert "tdq_k2_specialised" in src
        assert ("// reverse pass" in src) == (grad == "adjoint")
    else:
        assert "tdq_k1f_0" in src
        assert ("tdq_k1r_0" in src) == (grad == "adjoint")
    r, log = _compile(nvrtc, src)
    assert r == 0, name + "\n" + log[:3000]


def test_source_rejects_bad_arguments():
    from paper_2301_05451_gb300 import _abi as A, api, workloads as W
    C = api.Circuit(W.hea6()[0])
    n = ctypes.c_size_t()
    L = A.lib()
    assert L.tdq_sweep_source(C.h, A.TDQ_GRAD_PARAM_SHIFT, 0, None, 0, ctypes.byref(n)) == A.TDQ_ERR_ARG
    assert L.tdq_sweep_source(C.h, A.TDQ_GRAD_NONE, 0, None, 0, ctypes.byref(n)) == A.TDQ_OK
    buf = ctypes.create_string_buffer(8)
    assert L.tdq_sweep_source(C.h, A.TDQ_GRAD_NONE, 0, buf, 8, ctypes.byref(n)) == A.TDQ_ERR_ARG
    assert L.tdq_sweep_source(C.h, A.TDQ_GRAD_NONE, 4, None, 0, ctypes.byref(n)) == A.TDQ_ERR_ARG
    assert L.tdq_sweep_source(C.h, A.TDQ_GRAD_NONE, 14, None, 0, ctypes.byref(n)) == A.TDQ_ERR_ARG
    big = api.Circuit(W.random_circuit(15, 10, seed=1)[0])
    assert L.tdq_sweep_source(big.h, A.TDQ_GRAD_NONE, 0, None, 0, ctypes.byref(n)) == A.TDQ_ERR_UNSUPPORTED
    assert L.tdq_sweep_source(big.h, A.TDQ_GRAD_NONE, 9, None, 0, ctypes.byref(n)) == A.TDQ_OK


def _compile_rdc(nvrtc, src, maxrreg=0):
    """Relocatable cubin of one module (NVRTC -rdc=true), or (None, log)."""
    prog = ctypes.c_void_p()
    names = (ctypes.c_char_p * len(HEADERS))(*[os.path.basename(h).encode() for h in HEADERS])
    bodies = (ctypes.c_char_p * len(HEADERS))(*[open(h, "rb").read() for h in HEADERS])
    assert nvrtc.nvrtcCreateProgram(ctypes.byref(prog), src.encode(), b"mod.cu", len(HEADERS), bodies, names) == 0
    opts = [b"-arch=sm_103a", b"-std=c++17", b"-default-device", b"-rdc=true"]
    if maxrreg:
        opts.append(b"--maxrregcount=%d" % maxrreg)
    r = nvrtc.nvrtcCompileProgram(prog, len(opts), (ctypes.c_char_p * len(opts))(*opts))
    n = ctypes.c_size_t()
    nvrtc.nvrtcGetProgramLogSize(prog, ctypes.byref(n))
    log = ctypes.create_string_buffer(n.value + 1)
    nvrtc.nvrtcGetProgramLog(prog, log)
    cubin = None
    if r == 0:
        nvrtc.nvrtcGetCUBINSize(prog, ctypes.byref(n))
        cubin = ctypes.create_string_buffer(n.value)
        nvrtc.nvrtcGetCUBIN(prog, cubin)
    nvrtc.nvrtcDestroyProgram(ctypes.byref(prog))
    return cubin, log.value.decode(errors="replace")


def test_multi_circuit_modules_compile_and_link(nvrtc):
    """The persistent multi-circuit kernel (tdq_multi_source: the modules
    tdq_compile_multi compiles) for circuits of 3..9 qubits, every gate kind,
    with and without the reverse programs: every module compiles as
    relocatable device code and nvJitLink links them into one kernel."""
    from paper_2301_05451_gb300 import _abi as A, api, build, workloads as W
    try:
        jl = ctypes.CDLL(os.path.join(build.CUDA_LIB, "libnvJitLink.so"))
    except OSError as e:
        pytest.skip("libnvJitLink not loadable: %s" % e)
    specs = [W.hea6()[0], W.random_circuit(3, 20, seed=51)[0], W.random_circuit(9, 40, seed=52)[0]]
    C = [api.Circuit(s) for s in specs]
    hs = (ctypes.c_void_p * len(C))(*[c.h.value for c in C])
    L = A.lib()
    mark = "// ==== tdq module "
    for grad, threads, bits in ((A.TDQ_GRAD_ADJOINT, 128, 2), (A.TDQ_GRAD_NONE, 256, 3), (A.TDQ_GRAD_ADJOINT, 512, 3)):
        n = ctypes.c_size_t()
        assert L.tdq_multi_source(hs, len(C), grad, threads, bits, bits, None, 0, ctypes.byref(n)) == A.TDQ_OK
        buf = ctypes.create_string_buffer(n.value)
        assert L.tdq_multi_source(hs, len(C), grad, threads, bits, bits, buf, n.value, ctypes.byref(n)) == A.TDQ_OK
        mods = [m.split("\n", 1)[1] for m in buf.value.decode().split(mark)[1:]]
        assert len(mods) == len(C) + 1
        assert 'extern "C" __global__' in mods[0] and "atomicAdd(next, 1)" in mods[0]
        assert all("__noinline__ void tdq_multi_row_%d(" % c in mods[c + 1] for c in range(len(C)))
        h = ctypes.c_void_p()
        opts = (ctypes.c_char_p * 1)(b"-arch=sm_103a")
        assert jl.nvJitLinkCreate(ctypes.byref(h), 1, opts) == 0
        for i, m in enumerate(mods):  # row functions within the kernel's launch bounds, as the library does
            cubin, log = _compile_rdc(nvrtc, m, min(255, 65536 // threads))
            assert cubin is not None, "module %d\n%s" % (i, log[:3000])
            assert jl.nvJitLinkAddData(h, 1, cubin, ctypes.c_size_t(len(cubin.raw)), b"m%d" % i) == 0
        r = jl.nvJitLinkComplete(h)
        size = ctypes.c_size_t()
        jl.nvJitLinkGetLinkedCubinSize(h, ctypes.byref(size))
        jl.nvJitLinkDestroy(ctypes.byref(h))
        assert r == 0 and size.value > 0
    n = ctypes.c_size_t()
    assert L.tdq_multi_source(hs, len(C), A.TDQ_GRAD_NONE, 100, 2, 2, None, 0, ctypes.byref(n)) == A.TDQ_ERR_ARG
    assert L.tdq_multi_source(hs, 0, A.TDQ_GRAD_NONE, 128, 2, 2, None, 0, ctypes.byref(n)) == A.TDQ_ERR_ARG
