"""The allocation-free entry point (for callers that cannot call cudaMalloc,
e.g. under a memory manager that owns every device allocation) must give the
same values and parameter-shift gradients as the compiled parameter-shift
exec, call after call.  Kept in a file collected last."""
import ctypes

import numpy as np
import pytest

from paper_2301_05451_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("case", ["qnn12", "random9"])
def test_no_alloc_matches_compiled_param_shift(api, case):
    import torch
    if case == "qnn12":
        spec, params, inputs = W.qnn12(batch=6)
        p = torch.as_tensor(params[0]).cuda()
        stride = 0
    else:
        spec, params, inputs = W.random_circuit(9, 60, 4242, batch=3)
        p = torch.as_tensor(params).cuda().contiguous()
        stride = params.shape[1]
    x = None if inputs is None else torch.as_tensor(inputs).cuda().contiguous()
    B = 6 if case == "qnn12" else 3
    C = api.Circuit(spec)
    E = api.Exec(C, B, grad="param_shift")
    v_ref, g_ref = E.run(p, x)
    torch.cuda.synchronize()
    E.status()
    v_ref, g_ref = v_ref.cpu().numpy(), g_ref.cpu().numpy()
    for _ in range(2):  # two calls in a row share the scratch array
        v, g = _noalloc(C.h, B, p, x, C.n_groups, C.n_params, stride)
        np.testing.assert_allclose(v, v_ref, atol=1e-5)
        np.testing.assert_allclose(g[:, :C.n_params], g_ref[:, :C.n_params], atol=1e-4)


def test_no_alloc_rejects_oversize(api):
    import torch
    from paper_2301_05451_gb300._abi import TdqError, TDQ_ERR_ARG
    spec, params, inputs = W.qnn12(batch=4)
    C = api.Circuit(spec)
    p = torch.as_tensor(params[0]).cuda()
    x = torch.as_tensor(inputs).cuda()
    with pytest.raises(TdqError) as ei:  # 4096 rows x 289 copies x 8 bytes > 8 MiB
        _noalloc(C.h, 4096, p, torch.zeros((4096, 12), device="cuda"), C.n_groups, C.n_params, 0)
    assert ei.value.status == TDQ_ERR_ARG and "maximum" in str(ei.value)
