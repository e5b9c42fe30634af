"""Edge cases of the state-sweep and tree paths against the FP64 oracle or
closed forms: one qubit, no parameters, constant observable terms, circuits
that are all Clifford tail after their first gate, angles at the period's
edges, the largest whole-state sizes (13 qubits with gradients, 14 without),
the first sizes that go to the tiled path, and 30 qubits (the sweep's
maximum) against closed forms."""
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


def _run(api, spec, params, B, grad="adjoint", output="expval", **kw):
    import torch
    E = api.Exec(api.Circuit(spec), B, output=output, grad=grad, **kw)
    p = torch.as_tensor(np.ascontiguousarray(params if params.shape[0] > 1 else params[0]),
                        dtype=torch.float32).cuda()
    v, g = E.run(p)
    torch.cuda.synchronize()
    E.status()
    return v.cpu().numpy(), (None if g is None else g.cpu().numpy())


def _check(api, orc, spec, params, B, **kw):
    v, g = _run(api, spec, params, B, **kw)
    np.testing.assert_allclose(v, orc.expvals(spec, W.resolve_angles(spec, params, batch=B)), atol=EXP_TOL)
    for b in range(B):
        ref = orc.param_grads_param_shift(spec, (params[b] if params.shape[0] > 1 else params[0]).astype(np.float64))
        np.testing.assert_allclose(g[b][:spec.n_params], ref, atol=GRAD_TOL)
    return v, g


def test_one_qubit_and_period_edges(api, orc):
    """One qubit, RY then RZ then RX, at angles 0, +-pi, 2 pi and near them."""
    c = W.CircuitSpec(1)
    c.add("RY", [0], ("p", 0)); c.add("RZ", [0], ("p", 1)); c.add("RX", [0], ("p", 2))
    c.z([0])
    th = np.array([[0, 0, 0], [math.pi, -math.pi, math.pi], [2 * math.pi, 1e-7, -2 * math.pi],
                   [math.pi / 2, math.pi / 2, -math.pi / 2]], np.float32)
    _check(api, orc, c, th, 4)


def test_no_parameters_and_constant_terms(api, orc):
    """A circuit of fixed gates only (no gradient columns) and an observable
    with a constant (identity) term beside Z terms, in two groups."""
    c = W.CircuitSpec(5)
    for q in range(5):
        c.add("H", [q])
    c.add("CNOT", [0, 1]); c.add("RZ", [2], ("c", 0.4)); c.add("CZ", [2, 3]); c.add("RY", [4], ("c", 1.1))
    c.z([], 0.5, 0); c.z([2], -1.25, 0); c.z([3, 4], 2.0, 1)
    v, _ = _run(api, c, np.zeros((1, 1), np.float32), 3, grad="none")
    ref = orc.expvals(c, W.resolve_angles(c, np.zeros((1, 1), np.float32), batch=3))
    np.testing.assert_allclose(v, ref, atol=EXP_TOL)


@pytest.mark.parametrize("n,kw", [(6, {}), (16, {"tile_qubits": 10})])
def test_all_clifford_after_the_first_gate(api, orc, n, kw):
    """Everything after the first gate is a Clifford tail (CNOT, CZ, X, Y, Z):
    the sweep keeps the first gate and folds the rest into the observable;
    values and gradients as the oracle applies every gate.  Whole state and
    tiled."""
    c = W.CircuitSpec(n)
    c.add("RY", [0], ("p", 0))
    for q in range(n - 1):
        c.add("CNOT", [q, q + 1])
    c.add("X", [1]); c.add("Y", [n - 1]); c.add("CZ", [0, 2]); c.add("Z", [3])
    for q in range(n - 1):
        c.z([q, q + 1], 1.0 + 0.1 * q, q % 2)
    c.z([0], 0.3, 0)
    th = np.array([[0.3], [1.7], [-2.4]], np.float32)
    _check(api, orc, c, th, 3, **kw)


def test_largest_whole_state_sizes(api, orc):
    """13 qubits with adjoint gradients and 14 without stay whole-state in one
    CTA's shared memory; 14 with gradients goes tiled."""
    spec, params, _ = W.random_circuit(13, 60, 6013, batch=2)
    _check(api, orc, spec, params, 2)
    spec, params, _ = W.random_circuit(14, 60, 6014, batch=2)
    v, _ = _run(api, spec, params, 2, grad="none")
    np.testing.assert_allclose(v, orc.expvals(spec, W.resolve_angles(spec, params)), atol=EXP_TOL)
    _check(api, orc, spec, params, 2)


def test_thirty_qubits_closed_forms(api):
    """The sweep's largest state (2^30 amplitudes, 8 GiB per row): a product
    of RY(t_q) on every qubit, then its mirror on qubits 0..14 and a CNOT
    chain on 15..29; <Z_q> = 1 on the mirrored qubits, and on the others the
    chain gives <Z_q> = prod_{r=15..q} cos t_r.  Values only."""
    n = 30
    c = W.CircuitSpec(n)
    for q in range(n):
        c.add("RY", [q], ("p", q))
    for q in range(15):
        c.add("RY", [q], ("p", n + q))
    for q in range(15, n - 1):
        c.add("CNOT", [q, q + 1])
    for q in (0, 7, 14, 15, 16, 22, 29):
        c.z([q], 1.0, len(c.terms))
    r = np.random.default_rng(30)
    t = r.uniform(-1.2, 1.2, size=n).astype(np.float32)
    params = np.concatenate([t, -t[:15]])[None, :].astype(np.float32)
    v, _ = _run(api, c, params, 1, grad="none")
    td = t.astype(np.float64)
    want = []
    for q in (0, 7, 14, 15, 16, 22, 29):
        want.append(1.0 if q < 15 else float(np.prod(np.cos(td[15:q + 1]))))
    np.testing.assert_allclose(v[0], want, atol=EXP_TOL)
