"""Parity of the CUDA state-sweep contraction (values, amplitudes, adjoint and
parameter-shift gradients) with the FP64 oracle, through the C ABI.

Tolerances (the error budget of FP32 complex arithmetic over a few hundred
gates): |expectation| 1e-5 absolute, gradients 1e-4 absolute, amplitudes
1e-4 relative to the amplitude plus 2e-6 absolute (FP32 rounding is relative
to the unit-norm state, not to one small amplitude)."""
import math

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


def _dev(x):
    import torch
    return None if x is None else torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32).cuda()


def _oracle_values(orc, spec, params, inputs, B):
    ang = W.resolve_angles(spec, params, inputs, batch=B)
    return orc.expvals(spec, ang)


def _oracle_grads(orc, spec, params, inputs, rows, weights=None):
    out = []
    for b in rows:
        p = params[b] if params.shape[0] > 1 else params[0]
        x = inputs[b] if inputs is not None else None
        w = None if weights is None else weights[b]
        out.append(orc.param_grads_param_shift(spec, p.astype(np.float64), x, weights=w))
    return np.stack(out)


def _run(api, spec, params, inputs, B, grad="none", output="expval", gw=None, **kw):
    import torch
    C = api.Circuit(spec)
    E = api.Exec(C, B, output=output, grad=grad, **kw)
    p = _dev(params if params.shape[0] > 1 else params[0])
    gwt = None if gw is None else torch.as_tensor(gw, dtype=torch.float64).cuda()
    vals, grads = E.run(p, _dev(inputs), grad_weights=gwt)
    torch.cuda.synchronize()
    E.status()
    return vals.cpu().numpy(), (None if grads is None else grads.cpu().numpy()), E


def test_worked_example(api, orc):
    """Sec. 3.2.1 two-qubit example: <Z_1> = -cos(theta)."""
    c = W.CircuitSpec(2)
    c.add("X", [0]); c.add("RY", [1], ("p", 0)); c.add("CNOT", [0, 1]); c.z([1])
    th = np.linspace(-3, 6, 16).astype(np.float32)[:, None]
    v, g, _ = _run(api, c, th, None, 16, grad="adjoint")
    np.testing.assert_allclose(v[:, 0], -np.cos(th[:, 0].astype(np.float64)), atol=EXP_TOL)
    np.testing.assert_allclose(g[:, 0], np.sin(th[:, 0].astype(np.float64)), atol=GRAD_TOL)


def test_c1_hea6(api, orc):
    spec, params, _ = W.hea6()
    v, g, _ = _run(api, spec, params, None, 1, grad="adjoint")
    np.testing.assert_allclose(v, _oracle_values(orc, spec, params, None, 1), atol=EXP_TOL)
    np.testing.assert_allclose(g, _oracle_grads(orc, spec, params, None, [0]), atol=GRAD_TOL)


@pytest.mark.parametrize("interpret", [False, True])
def test_c2_qnn12_full_batch(api, orc, interpret):
    """The 12-qubit classifier at its full batch of 256 (one launch), with the
    kernel specialised to the circuit and with the generic kernel."""
    spec, params, inputs = W.qnn12()
    v, g, E = _run(api, spec, params, inputs, 256, grad="adjoint", interpret=interpret)
    np.testing.assert_allclose(v, _oracle_values(orc, spec, params, inputs, 256), atol=EXP_TOL)
    # every row's gradient with the specialised kernel (the benchmark's), a
    # sample with the generic one
    rows = list(range(256)) if not interpret else [0, 1, 77, 128, 255]
    np.testing.assert_allclose(g[rows], _oracle_grads(orc, spec, params, inputs, rows), atol=GRAD_TOL)
    assert E.launches() == 1


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("path", ["smem", "smem_interp", "smem_b43", "smem_b11", "tiled", "tiled_interp", "tiled_b32"])
def test_random_circuits(api, orc, seed, path):
    """Every gate kind, several output groups, gradient weights, every kernel:
    whole state and tiled, each specialised to the circuit and generic."""
    n = [3, 5, 7, 9, 10, 11, 12, 13][seed]
    spec, params, _ = W.random_circuit(n, 10 * n, 500 + seed, batch=3)
    for q in range(0, n, 2):  # Y and Z as well
        spec.add("Y", [q])
        spec.add("Z", [(q + 1) % n])
    tile = {"max_smem_qubits": 1, "tile_qubits": max(5, n - 3)}
    kw = {"smem": {}, "smem_interp": {"interpret": True},
          "smem_b43": {"fwd_reg_bits": 4, "rev_reg_bits": 3}, "smem_b11": {"fwd_reg_bits": 1, "rev_reg_bits": 1},
          "tiled": tile, "tiled_interp": dict(tile, interpret=True),
          "tiled_b32": dict(tile, fwd_reg_bits=3, rev_reg_bits=2)}[path]
    if path.startswith("tiled") and n < 6:
        pytest.skip("tile needs at least 5 bits")
    B = 3
    gw = np.random.default_rng(seed).normal(size=(B, spec.n_groups))
    v, g, _ = _run(api, spec, params, None, B, grad="adjoint", gw=gw, **kw)
    np.testing.assert_allclose(v, _oracle_values(orc, spec, params, None, B), atol=EXP_TOL)
    np.testing.assert_allclose(g, _oracle_grads(orc, spec, params, None, range(B), gw), atol=GRAD_TOL)


@pytest.mark.parametrize("path", ["smem", "smem_interp", "smem_b11", "tiled", "tiled_b32"])
@pytest.mark.parametrize("n", [3, 7])
def test_tied_parameters(api, orc, n, path):
    """Parameters shared by several gates (and by the angles of one gate): a
    parameter's gradient sums the shares of every angle it feeds.  Shares of
    one parameter inside a reverse register pass meet in one accumulator."""
    spec, params, _ = W.random_circuit_tied(n, 12 * n, max(2, n - 2), 600 + n, batch=3)
    if path.startswith("tiled") and n < 6:
        pytest.skip("tile needs at least 5 bits")
    tile = {"max_smem_qubits": 1, "tile_qubits": 5}
    kw = {"smem": {}, "smem_interp": {"interpret": True}, "smem_b11": {"fwd_reg_bits": 1, "rev_reg_bits": 1},
          "tiled": tile, "tiled_b32": dict(tile, fwd_reg_bits=3, rev_reg_bits=2)}[path]
    v, g, _ = _run(api, spec, params, None, 3, grad="adjoint", **kw)
    np.testing.assert_allclose(v, _oracle_values(orc, spec, params, None, 3), atol=EXP_TOL)
    np.testing.assert_allclose(g, _oracle_grads(orc, spec, params, None, range(3)), atol=GRAD_TOL)


@pytest.mark.parametrize("n,tile,interpret", [(14, 8, False), (16, 12, False), (15, 13, False), (14, 8, True)])
def test_tiled_ladder_multi_pass(api, orc, n, tile, interpret):
    spec, params, _ = W.ladder20(batch=5, n=n, layers=3)
    v, g, _ = _run(api, spec, params, None, 5, grad="adjoint", tile_qubits=tile, interpret=interpret)
    np.testing.assert_allclose(v, _oracle_values(orc, spec, params, None, 5), atol=EXP_TOL)
    np.testing.assert_allclose(g[[0, 4]], _oracle_grads(orc, spec, params, None, [0, 4]), atol=GRAD_TOL)


def test_c3_ladder20_full_size(api, orc):
    """20 qubits, B = 64, value + adjoint gradient in the launch configuration
    the benchmark times.  Every row's value, and the full 240-entry gradients
    of the first and the last row, against the FP64 oracle (state vector and
    shift rule, Sec. 4.2, Eq. 10) stored by tests/golden/make_golden.py; a few
    values are recomputed by the oracle here as well."""
    import json
    import os
    spec, params, _ = W.ladder20()
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c3_ladder20.json")))
    assert gold["params_sha256"] == _params_digest(params), "stored values belong to other parameters"
    v, g, _ = _run(api, spec, params, None, 64, grad="adjoint")
    np.testing.assert_allclose(v[:, 0], np.asarray(gold["values"]), atol=EXP_TOL)
    for b, ref in gold["grads"].items():
        np.testing.assert_allclose(g[int(b)], np.asarray(ref), atol=GRAD_TOL)
    rows = [5, 31]
    np.testing.assert_allclose(v[rows], _oracle_values(orc, spec, params[rows], None, 2), atol=EXP_TOL)


def _params_digest(params):
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(params, dtype=np.float32).tobytes()).hexdigest()


@pytest.mark.parametrize("path", ["smem", "smem_interp", "tiled", "tiled_interp"])
def test_param_shift_mode(api, orc, path):
    spec, params, _ = W.ladder20(batch=2, n=14 if path.startswith("tiled") else 8, layers=2)
    kw = {"smem": {}, "smem_interp": {"interpret": True}, "tiled": {"tile_qubits": 9},
          "tiled_interp": {"tile_qubits": 9, "interpret": True}}[path]
    v, g, E = _run(api, spec, params, None, 2, grad="param_shift", **kw)
    np.testing.assert_allclose(v, _oracle_values(orc, spec, params, None, 2), atol=EXP_TOL)
    np.testing.assert_allclose(g, _oracle_grads(orc, spec, params, None, [0, 1]), atol=GRAD_TOL)
    _, ga, _ = _run(api, spec, params, None, 2, grad="adjoint", **kw)
    np.testing.assert_allclose(g, ga, atol=GRAD_TOL)


def test_adjoint_vs_finite_difference(api, orc):
    spec, params, inputs = W.qnn12(batch=2)
    _, g, _ = _run(api, spec, params, inputs, 2, grad="adjoint")
    fd = orc.param_grads_finite_difference(spec, params[0].astype(np.float64), inputs[1])
    np.testing.assert_allclose(g[1], fd, atol=GRAD_TOL)


@pytest.mark.parametrize("path", ["smem", "smem_interp", "tiled"])
def test_amplitudes(api, orc, path):
    n = 11
    spec, params, _ = W.random_circuit(n, 80, 77, batch=4, observables=False, amplitudes=5)
    spec.amplitude([0] * n)
    kw = {"smem": {}, "smem_interp": {"interpret": True}, "tiled": {"max_smem_qubits": 1, "tile_qubits": 7}}[path]
    v, _, _ = _run(api, spec, params, None, 4, output="amplitude", **kw)
    ref = orc.amplitudes(spec, W.resolve_angles(spec, params))
    got = v[:, 0::2] + 1j * v[:, 1::2]
    assert np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref) + 2e-6)


def test_ghz_and_mirror_amplitudes(api, orc):
    n = 10
    c = W.CircuitSpec(n)
    c.add("H", [0])
    for q in range(n - 1):
        c.add("CNOT", [q, q + 1])
    c.amplitude([0] * n); c.amplitude([1] * n); c.amplitude([0, 1] + [0] * (n - 2))
    v, _, _ = _run(api, c, np.zeros((1, 1), np.float32), None, 1, output="amplitude")
    np.testing.assert_allclose(v[0], [2 ** -0.5, 0, 2 ** -0.5, 0, 0, 0], atol=1e-6)
    m, p, _ = W.grid_u3cz_mirror(rows=3, cols=4, depth=3)
    v, _, _ = _run(api, m, p, None, 1, output="amplitude")
    assert abs(complex(v[0, 0], v[0, 1]) - 1) < 1e-5


def test_batch_edges(api, orc):
    spec, params, inputs = W.qnn12(batch=257)
    for B in (1, 257):
        v, g, _ = _run(api, spec, params, inputs[:B], B, grad="adjoint")
        ref = _oracle_values(orc, spec, params, inputs[:B], B)
        np.testing.assert_allclose(v, ref, atol=EXP_TOL)


def test_nonfinite_parameter_reported(api):
    import torch
    spec, params, _ = W.hea6()
    C = api.Circuit(spec)
    E = api.Exec(C, 1, grad="adjoint")
    p = _dev(params[0]).clone()
    p[3] = float("nan")
    E.run(p)
    torch.cuda.synchronize()
    from paper_2301_05451_gb300._abi import TdqError, TDQ_ERR_NONFINITE
    with pytest.raises(TdqError) as ei:
        E.status()
    assert ei.value.status == TDQ_ERR_NONFINITE
    E.run(_dev(params[0]))
    E.status()  # cleared


def test_argument_errors(api):
    import torch
    from paper_2301_05451_gb300._abi import TdqError, TDQ_ERR_ARG
    spec, params, _ = W.hea6()
    C = api.Circuit(spec)
    E = api.Exec(C, 1, grad="none")
    vals = torch.empty((1, 1), dtype=torch.float64, device="cuda")
    grads = torch.empty((1, 36), dtype=torch.float32, device="cuda")
    with pytest.raises(TdqError) as ei:
        E.run(_dev(params[0]), values=vals, grads=grads)
    assert ei.value.status == TDQ_ERR_ARG


def test_autograd_function(api, orc):
    import torch
    spec, params, inputs = W.qnn12(batch=8)
    layer = api.QuantumLayer(spec, 8, init=params[0])
    x = _dev(inputs)
    out = layer(x)
    w = torch.linspace(-1, 1, 8, device="cuda", dtype=torch.float64)[:, None]
    (out * w).sum().backward()
    ref = np.zeros(spec.n_params)
    for b in range(8):
        ref += orc.param_grads_param_shift(spec, params[0].astype(np.float64), inputs[b],
                                           weights=[w[b, 0].item()])
    np.testing.assert_allclose(layer.weight.grad.cpu().numpy(), ref, atol=8 * GRAD_TOL)
