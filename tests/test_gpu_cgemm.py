"""Kernel-level parity of the tcgen05 3xTF32 complex product (K3) with an
FP64 host product on random complex operands.

The bound is on every entry, relative to the Cauchy-Schwarz scale of that
entry's dot product: |D_ij - ref_ij| <= 1e-6 |x_i| |y_j| (x_i row i of X,
y_j row j of Y, 2-norms).  3xTF32 drops only the lo*lo term of each
product (relative 2^-22) and the FP32 running sums round at 2^-24 of their
size, which never exceeds |x_i||y_j|; for random operands these errors add
like a random walk and stay a small multiple of 2^-24 of that scale.
Measured on GB300: at most 1.8e-7 of it for K = 8..4096."""
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


REL_BOUND = 1e-6


@pytest.mark.parametrize("batch,I,J,K", [(1, 128, 64, 8), (2, 256, 128, 64), (3, 128, 192, 520), (1, 512, 512, 256),
                                         (1, 1024, 1024, 4096)])
def test_cgemm_nt_matches_fp64(lib, batch, I, J, K):
    import torch
    r = np.random.default_rng(I + J + K)
    X = (r.normal(size=(batch, I, K)) + 1j * r.normal(size=(batch, I, K))).astype(np.complex64)
    Y = (r.normal(size=(batch, J, K)) + 1j * r.normal(size=(batch, J, K))).astype(np.complex64)
    # FP64 product on the host (a library matmul as the definition of the product)
    Xd, Yd = torch.as_tensor(X.astype(np.complex128)), torch.as_tensor(Y.astype(np.complex128))
    ref = torch.matmul(Xd, Yd.transpose(1, 2)).numpy()
    scale = np.linalg.norm(X.astype(np.complex128), axis=2)[:, :, None] * \
        np.linalg.norm(Y.astype(np.complex128), axis=2)[:, None, :]
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
    rel = np.abs(D - ref) / scale
    assert np.max(rel) <= REL_BOUND, np.max(rel)


def test_cgemm_nt_rejects_bad_shapes(lib):
    from paper_2301_05451_gb300._abi import TdqError, TDQ_ERR_ARG
    with pytest.raises(TdqError) as ei:
        lib.call("tdq_cgemm_nt", 1, 100, 64, 8, ctypes.c_void_p(1), ctypes.c_void_p(1), ctypes.c_void_p(1),
                 ctypes.c_void_p(1), ctypes.c_void_p(0))
    assert ei.value.status == TDQ_ERR_ARG


def test_cgemm_wait_bound_runs_out_and_recovers(lib):
    """Failure detection without a fault: with the main-loop wait bound at 0
    ns the issuing thread's first wait for a staged k-block gives up before
    any tensor-core product is issued; the kernel must report
    TDQ_ERR_TIMEOUT in its status word, wait for nothing left in flight,
    free its tensor memory and return, so that a normal call right after it
    (on the same SMs, which must be able to allocate tensor memory again)
    gives the FP64 product with a clean status."""
    import torch
    from paper_2301_05451_gb300._abi import TDQ_ERR_TIMEOUT
    batch, I, J, K = 2, 256, 128, 512
    r = np.random.default_rng(77)
    X = (r.normal(size=(batch, I, K)) + 1j * r.normal(size=(batch, I, K))).astype(np.complex64)
    Y = (r.normal(size=(batch, J, K)) + 1j * r.normal(size=(batch, J, K))).astype(np.complex64)
    dX = torch.as_tensor(X.view(np.float32)).cuda()
    dY = torch.as_tensor(Y.view(np.float32)).cuda()
    dD = torch.zeros((batch, I, 2 * J), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (batch, I, J, K, ctypes.c_void_p(dX.data_ptr()), ctypes.c_void_p(dY.data_ptr()),
            ctypes.c_void_p(dD.data_ptr()), ctypes.c_void_p(st.data_ptr()))
    lib.call("tdq_cgemm_nt_bounded", *args, ctypes.c_int64(0), s)
    torch.cuda.synchronize()
    assert int(st.item()) & (1 << TDQ_ERR_TIMEOUT)
    st.zero_()
    for _ in range(2):
        lib.call("tdq_cgemm_nt", *args, s)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    D = dD.cpu().numpy().view(np.complex64).reshape(batch, I, J).astype(np.complex128)
    Xd, Yd = torch.as_tensor(X.astype(np.complex128)), torch.as_tensor(Y.astype(np.complex128))
    ref = torch.matmul(Xd, Yd.transpose(1, 2)).numpy()
    scale = np.linalg.norm(X.astype(np.complex128), axis=2)[:, :, None] * \
        np.linalg.norm(Y.astype(np.complex128), axis=2)[:, None, :]
    assert np.max(np.abs(D - ref) / scale) <= REL_BOUND
    from paper_2301_05451_gb300._abi import TdqError, TDQ_ERR_ARG
    with pytest.raises(TdqError) as ei:
        lib.call("tdq_cgemm_nt_bounded", *args, ctypes.c_int64(-1), s)
    assert ei.value.status == TDQ_ERR_ARG
