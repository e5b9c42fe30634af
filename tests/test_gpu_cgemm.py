"""Kernel-level parity of the tcgen05 3xTF32 complex product (K3) with an
FP64 host product on random complex operands; the bound is the 3xTF32 error
of an FP32-accumulated dot product: relative 2e-6 of the entry scale."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_05451_gb300 import build
    build.build()
    from paper_2301_05451_gb300 import _abi
    return _abi


@pytest.mark.parametrize("batch,I,J,K", [(1, 128, 64, 8), (2, 256, 128, 64), (3, 128, 192, 520), (1, 512, 512, 256)])
def test_cgemm_nt_matches_fp64(lib, batch, I, J, K):
    import torch
    r = np.random.default_rng(I + J + K)
    X = (r.normal(size=(batch, I, K)) + 1j * r.normal(size=(batch, I, K))).astype(np.complex64)
    Y = (r.normal(size=(batch, J, K)) + 1j * r.normal(size=(batch, J, K))).astype(np.complex64)
    ref = np.einsum("bik,bjk->bij", X.astype(np.complex128), Y.astype(np.complex128))
    dX = torch.as_tensor(X.view(np.float32)).cuda()
    dY = torch.as_tensor(Y.view(np.float32)).cuda()
    dD = torch.zeros((batch, I, 2 * J), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    lib.call("tdq_cgemm_nt", batch, I, J, K, ctypes.c_void_p(dX.data_ptr()), ctypes.c_void_p(dY.data_ptr()),
             ctypes.c_void_p(dD.data_ptr()), ctypes.c_void_p(st.data_ptr()),
             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    D = dD.cpu().numpy().view(np.complex64).reshape(batch, I, J).astype(np.complex128)
    scale = np.sqrt(K) * 2
    assert np.max(np.abs(D - ref)) <= 2e-6 * scale * 4, np.max(np.abs(D - ref))


def test_cgemm_nt_rejects_bad_shapes(lib):
    from paper_2301_05451_gb300._abi import TdqError, TDQ_ERR_ARG
    with pytest.raises(TdqError) as ei:
        lib.call("tdq_cgemm_nt", 1, 100, 64, 8, ctypes.c_void_p(1), ctypes.c_void_p(1), ctypes.c_void_p(1),
                 ctypes.c_void_p(1), ctypes.c_void_p(0))
    assert ei.value.status == TDQ_ERR_ARG
