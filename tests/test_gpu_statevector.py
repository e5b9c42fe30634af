"""State-vector mode of the state sweep (Sec. 3.1): the final state and the
probabilities as outputs, and a caller-given initial state in place of
|0...0>, against the FP64 oracle, through the C ABI, on every kernel form
(whole state in one CTA or tiled through HBM; specialised to the circuit or
generic).

Tolerances: state entries 1e-4 relative plus 2e-6 absolute (FP32 rounding is
relative to the unit-norm state), probabilities the same; expectations 1e-5,
gradients 1e-4 absolute."""
import ctypes

import numpy as np
import pytest

from paper_2301_05451_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EXP_TOL, GRAD_TOL = 1e-5, 1e-4
PATHS = {"smem": {}, "smem_interp": {"interpret": True},
         "tiled": {"max_smem_qubits": 1}, "tiled_interp": {"max_smem_qubits": 1, "interpret": True}}


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_05451_gb300 import build
    build.build()
    from paper_2301_05451_gb300 import api as _api
    return _api


def _random_states(r, rows, n):
    v = r.normal(size=(rows, 1 << n)) + 1j * r.normal(size=(rows, 1 << n))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _kw(path, n):
    kw = dict(PATHS[path])
    if path.startswith("tiled"):
        kw["tile_qubits"] = max(5, n - 3)
    return kw


def _close(got, ref):
    assert np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref) + 2e-6), np.abs(got - ref).max()


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("n", [5, 9, 13])
def test_state_and_probabilities(api, orc, path, n):
    import torch
    if path.startswith("tiled") and n < 6:
        pytest.skip("tile needs at least 5 bits")
    spec, params, _ = W.random_circuit(n, 8 * n, 900 + n, batch=3)
    ang = W.resolve_angles(spec, params)
    C = api.Circuit(spec)
    p = torch.as_tensor(params, dtype=torch.float32).cuda()
    for out in ("state", "probs"):
        E = api.Exec(C, 3, output=out, **_kw(path, n))
        v, _ = E.run(p)
        torch.cuda.synchronize()
        E.status()
        v = v.cpu().numpy()
        for b in range(3):
            ref = orc.statevector(spec, ang[b])
            if out == "state":
                _close(v[b, 0::2] + 1j * v[b, 1::2], ref)
            else:
                _close(v[b], np.abs(ref) ** 2)


@pytest.mark.parametrize("path", list(PATHS))
def test_initial_states_values_and_adjoint_gradients(api, orc, path):
    """Per-row and shared initial states; expectations and adjoint gradients
    against the oracle's expectations and shift rule from the same states."""
    import torch
    n = 11
    r = np.random.default_rng(910)
    spec, params, _ = W.random_circuit(n, 70, 911, batch=3)
    ang = W.resolve_angles(spec, params)
    init = _random_states(r, 3, n)
    C = api.Circuit(spec)
    E = api.Exec(C, 3, grad="adjoint", **_kw(path, n))
    p = torch.as_tensor(params, dtype=torch.float32).cuda()
    for rows in (init, init[1]):  # one state per row, then one shared state
        psi0 = torch.as_tensor(rows.astype(np.complex64)).cuda().contiguous()
        E.set_initial_state(psi0)
        v, g = E.run(p)
        torch.cuda.synchronize()
        E.status()
        ref = orc.expvals(spec, ang, init=rows)
        np.testing.assert_allclose(v.cpu().numpy(), ref, atol=EXP_TOL)
        g = g.cpu().numpy()
        for b in (0, 2):
            row0 = rows[b] if rows.ndim == 2 else rows
            gr = orc.param_grads_param_shift(spec, params[b].astype(np.float64), init=row0)
            np.testing.assert_allclose(g[b], gr, atol=GRAD_TOL)
    # back to |0...0>
    E.set_initial_state(None)
    v, _ = E.run(p)
    torch.cuda.synchronize()
    np.testing.assert_allclose(v.cpu().numpy(), orc.expvals(spec, ang), atol=EXP_TOL)


@pytest.mark.parametrize("path", ["smem", "tiled"])
def test_initial_state_parameter_shift_and_state_output(api, orc, path):
    import torch
    n = 10
    r = np.random.default_rng(920)
    spec, params, _ = W.ladder20(batch=2, n=n, layers=2)
    init = _random_states(r, 2, n)
    psi0 = torch.as_tensor(init.astype(np.complex64)).cuda().contiguous()
    C = api.Circuit(spec)
    p = torch.as_tensor(params, dtype=torch.float32).cuda()
    E = api.Exec(C, 2, grad="param_shift", **_kw(path, n))
    E.set_initial_state(psi0)
    v, g = E.run(p)
    torch.cuda.synchronize()
    ang = W.resolve_angles(spec, params)
    np.testing.assert_allclose(v.cpu().numpy(), orc.expvals(spec, ang, init=init), atol=EXP_TOL)
    gr = orc.param_grads_param_shift(spec, params[1].astype(np.float64), init=init[1])
    np.testing.assert_allclose(g.cpu().numpy()[1], gr, atol=GRAD_TOL)
    S = api.Exec(C, 2, output="state", **_kw(path, n))
    S.set_initial_state(psi0)
    s, _ = S.run(p)
    torch.cuda.synchronize()
    s = s.cpu().numpy()
    for b in range(2):
        _close(s[b, 0::2] + 1j * s[b, 1::2], orc.statevector(spec, ang[b], init=init[b]))


def test_hea20_neel_probabilities_full_size(api, orc):
    """20 qubits from the Neel state |0101...>, the tiled kernels at their
    default launch shape: the probabilities of two rows against the oracle."""
    import torch
    n = 20
    spec, params, _ = W.hea_sv(n=n, batch=4)
    neel = np.zeros(1 << n, np.complex64)
    neel[int("01" * (n // 2), 2)] = 1
    C = api.Circuit(spec)
    E = api.Exec(C, 4, output="probs")
    E.set_initial_state(torch.as_tensor(neel).cuda())
    v, _ = E.run(torch.as_tensor(params, dtype=torch.float32).cuda())
    torch.cuda.synchronize()
    E.status()
    v = v.cpu().numpy()
    ang = W.resolve_angles(spec, params)
    for b in (0, 3):
        ref = np.abs(orc.statevector(spec, ang[b], init=neel.astype(np.complex128))) ** 2
        _close(v[b], ref)
        assert abs(v[b].sum() - 1) < 1e-4


def test_initial_state_argument_errors(api):
    import torch
    from paper_2301_05451_gb300 import _abi as A
    spec, params, _ = W.hea6()
    C = api.Circuit(spec)
    E = api.Exec(C, 1, grad="none")
    buf = torch.zeros(64, dtype=torch.complex64, device="cuda")
    L = A.lib()
    assert L.tdq_exec_set_initial_state(E.h, ctypes.c_void_p(buf.data_ptr()), ctypes.c_int64(10)) == A.TDQ_ERR_ARG
    assert L.tdq_exec_set_initial_state(E.h, ctypes.c_void_p(buf.data_ptr()), ctypes.c_int64(64)) == A.TDQ_OK
    assert L.tdq_exec_set_initial_state(E.h, None, ctypes.c_int64(0)) == A.TDQ_OK
    N = api.Network(C, "expval", 0, False, False)
    T = api.TreeExec(api.Plan(N, method="greedy"), 1)
    assert L.tdq_exec_set_initial_state(T.h, ctypes.c_void_p(buf.data_ptr()), ctypes.c_int64(0)) == \
        A.TDQ_ERR_UNSUPPORTED
