"""The allocation-free entry point, tdq_execute_param_shift_noalloc.

It exists for callers that cannot call cudaMalloc: code running under a
memory manager that owns every device allocation, or a service that reserves
its memory at start-up and forbids allocation (which can synchronise the
device and fail under fragmentation) on its request path.  It must give the
same values and parameter-shift gradients as the compiled parameter-shift
exec, call after call (every call reuses one fixed device array), and both
must agree with the FP64 oracle.

This file is collected last, so a run that stops at its first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2301_05451_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EXP_TOL, GRAD_TOL = 1e-5, 1e-4


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_05451_gb300 import build
    build.build()
    from paper_2301_05451_gb300 import api as _api
    return _api


def _noalloc(spec_h, B, params, inputs, ng, P, stride):
    import torch
    from paper_2301_05451_gb300 import _abi as A
    values = torch.full((B, ng), float("nan"), dtype=torch.float64, device="cuda")
    grads = torch.full((B, max(P, 1)), float("nan"), dtype=torch.float32, device="cuda")
    A.call("tdq_execute_param_shift_noalloc", spec_h, B, ctypes.c_void_p(params.data_ptr()),
           ctypes.c_int64(stride), ctypes.c_void_p(0 if inputs is None else inputs.data_ptr()),
           ctypes.c_void_p(values.data_ptr()), ctypes.c_void_p(grads.data_ptr()),
           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return values.cpu().numpy(), grads.cpu().numpy()


def _case(name):
    """(spec, params, inputs, B, shared params?) of each case: the 12-qubit
    classifier with shared parameters and per-row inputs, and random circuits
    with per-row parameters at 4 qubits (CTAs of one warp), 9 and 13 qubits
    (the largest state the entry point takes)."""
    if name == "qnn12":
        spec, params, inputs = W.qnn12(batch=6)
        return spec, params, inputs, 6, True
    n, B = {"random4": (4, 5), "random9": (9, 3), "random13": (13, 2)}[name]
    spec, params, inputs = W.random_circuit(n, 6 * n, 4242 + n, batch=B)
    return spec, params, inputs, B, False


@pytest.mark.parametrize("case", ["qnn12", "random4", "random9", "random13"])
def test_no_alloc_matches_compiled_param_shift_and_oracle(api, orc, case):
    import torch
    spec, params, inputs, B, shared = _case(case)
    p = torch.as_tensor(params[0] if shared else params).cuda().contiguous()
    stride = 0 if shared else params.shape[1]
    x = None if inputs is None else torch.as_tensor(inputs).cuda().contiguous()
    C = api.Circuit(spec)
    E = api.Exec(C, B, grad="param_shift")
    v_ref, g_ref = E.run(p, x)
    torch.cuda.synchronize()
    E.status()
    v_ref, g_ref = v_ref.cpu().numpy(), g_ref.cpu().numpy()
    # the FP64 oracle: state-vector values and shift-rule gradients
    v_orc = orc.expvals(spec, W.resolve_angles(spec, params, inputs, batch=B))
    g_orc = np.stack([orc.param_grads_param_shift(spec, (params[0] if shared else params[b]).astype(np.float64),
                                                  None if inputs is None else inputs[b]) for b in range(B)])
    np.testing.assert_allclose(v_ref, v_orc, atol=EXP_TOL)
    np.testing.assert_allclose(g_ref[:, :C.n_params], g_orc, atol=GRAD_TOL)
    for _ in range(2):  # two calls in a row share the scratch array
        v, g = _noalloc(C.h, B, p, x, C.n_groups, C.n_params, stride)
        np.testing.assert_allclose(v, v_ref, atol=EXP_TOL)
        np.testing.assert_allclose(g[:, :C.n_params], g_ref[:, :C.n_params], atol=GRAD_TOL)
        np.testing.assert_allclose(v, v_orc, atol=EXP_TOL)
        np.testing.assert_allclose(g[:, :C.n_params], g_orc, atol=GRAD_TOL)


def test_no_alloc_rejects_oversize(api):
    import torch
    from paper_2301_05451_gb300._abi import TdqError, TDQ_ERR_ARG
    spec, params, inputs = W.qnn12(batch=4)
    C = api.Circuit(spec)
    p = torch.as_tensor(params[0]).cuda()
    with pytest.raises(TdqError) as ei:  # 4096 rows x 289 copies x 8 bytes > 8 MiB
        _noalloc(C.h, 4096, p, torch.zeros((4096, 12), device="cuda"), C.n_groups, C.n_params, 0)
    assert ei.value.status == TDQ_ERR_ARG and "maximum" in str(ei.value)
    spec14, params14, _ = W.random_circuit(14, 20, 7, batch=1)
    C14 = api.Circuit(spec14)
    with pytest.raises(TdqError) as ei:  # the state must fit one CTA's shared memory
        _noalloc(C14.h, 1, torch.as_tensor(params14[0]).cuda(), None, C14.n_groups, C14.n_params, 0)
    assert ei.value.status == TDQ_ERR_ARG
