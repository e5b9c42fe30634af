"""Many circuits of uneven qubit counts and depths in one persistent launch
(tdq_compile_multi): every circuit's rows -- data samples, parameter sets and
parameter-shift copies -- against the FP64 oracle, through the C ABI.
Tolerances: expectations 1e-5, gradients 1e-4 (absolute)."""
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


def _workload(seed=0):
    """(spec, params [B][P], inputs [B][F] or None) of circuits of 4..12 qubits."""
    r = np.random.default_rng(3000 + seed)
    out = []
    spec, p, x = W.qnn12(batch=3)
    out.append((spec, np.repeat(p, 3, axis=0), x))
    spec, p, _ = W.hea6()
    out.append((spec, (r.random((2, p.shape[1])) * 2 * np.pi).astype(np.float32), None))
    spec, p, _ = W.ladder20(batch=4, n=10, layers=2)
    out.append((spec, p, None))
    spec, p, _ = W.random_circuit(9, 80, 3100 + seed, batch=5)
    out.append((spec, p, None))
    spec, p, _ = W.random_circuit(4, 30, 3200 + seed, batch=1)
    out.append((spec, p, None))
    return out


def _pack(M, wl, torch):
    params = M.pack([p for _, p, _ in wl])
    xs = [x if x is not None else np.zeros((p.shape[0], 0), np.float32) for _, p, x in wl]
    inputs = M.pack(xs) if M.n_inputs_total > 0 else None
    return params, inputs


def _check_values(orc, M, wl, vals):
    for (spec, p, x), v in zip(wl, M.unpack(vals, "values")):
        ref = orc.expvals(spec, W.resolve_angles(spec, p, x))
        np.testing.assert_allclose(v.cpu().numpy(), ref, atol=EXP_TOL)


@pytest.mark.parametrize("grad", ["none", "adjoint", "param_shift"])
def test_uneven_circuits_one_launch(api, orc, grad):
    import torch
    wl = _workload()
    C = [api.Circuit(s) for s, _, _ in wl]
    M = api.MultiExec(C, [p.shape[0] for _, p, _ in wl], grad=grad)
    params, inputs = _pack(M, wl, torch)
    vals, grads = M.run(params, inputs)
    torch.cuda.synchronize()
    M.status()
    assert M.launches() == (2 if grad == "param_shift" else 1)
    _check_values(orc, M, wl, vals)
    if grad == "none":
        return
    for (spec, p, x), g in zip(wl, M.unpack(grads, "grads")):
        for b in (0, p.shape[0] - 1):
            ref = orc.param_grads_param_shift(spec, p[b].astype(np.float64), None if x is None else x[b])
            np.testing.assert_allclose(g[b].cpu().numpy(), ref, atol=GRAD_TOL)


def test_graph_replay_follows_new_parameters(api, orc):
    """Repeated calls with the same buffers are replayed from a CUDA graph;
    new parameters written into the same buffer reach every circuit."""
    import torch
    wl = _workload(1)
    C = [api.Circuit(s) for s, _, _ in wl]
    M = api.MultiExec(C, [p.shape[0] for _, p, _ in wl], grad="adjoint")
    params, inputs = _pack(M, wl, torch)
    vals, grads = M.alloc_outputs()
    r = np.random.default_rng(3300)
    for it in range(4):
        wl = [(s, (r.random(p.shape) * 2 * np.pi).astype(np.float32), x) for s, p, x in wl]
        params.copy_(M.pack([p for _, p, _ in wl]))
        M.run(params, inputs, values=vals, grads=grads)
        torch.cuda.synchronize()
        M.status()
        _check_values(orc, M, wl, vals)


def test_autotuned_launch(api, orc):
    """The autotuner times CTA sizes and register widths on the workload;
    whatever it keeps computes the same values and gradients."""
    import torch
    wl = _workload(2)[1:4]
    C = [api.Circuit(s) for s, _, _ in wl]
    M = api.MultiExec(C, [p.shape[0] for _, p, _ in wl], grad="adjoint", autotune=True)
    cfg = M.config()
    assert cfg["threads"] in (128, 256, 512) and cfg["fwd_reg_bits"] in (2, 3)
    assert 1 <= cfg["ctas"] <= sum(p.shape[0] for _, p, _ in wl)
    params, inputs = _pack(M, wl, torch)
    vals, grads = M.run(params, inputs)
    torch.cuda.synchronize()
    M.status()
    _check_values(orc, M, wl, vals)
    for (spec, p, x), g in zip(wl, M.unpack(grads, "grads")):
        ref = orc.param_grads_param_shift(spec, p[0].astype(np.float64))
        np.testing.assert_allclose(g[0].cpu().numpy(), ref, atol=GRAD_TOL)



@pytest.mark.parametrize("path", ["smem", "tiled"])
def test_autotuned_single_circuit_sweep(api, orc, path):
    """tdq_compile_sweep with autotune: whole-state kernels try CTA sizes and
    register bits, tiled sweeps tile widths; the kept configuration is within
    the candidates and computes the oracle's values and gradients."""
    import torch
    n = 11 if path == "smem" else 12
    spec, params, _ = W.random_circuit(n, 8 * n, 3400 + n, batch=4)
    C = api.Circuit(spec)
    E = api.Exec(C, 4, grad="adjoint", autotune=True, max_smem_qubits=(1 if path == "tiled" else 0))
    cfg = E.config()
    if path == "smem":
        assert cfg["threads"] in (128, 256, 512) and cfg["fwd_reg_bits"] in (2, 3) and cfg["tile_qubits"] == 0
    else:
        assert 10 <= cfg["tile_qubits"] <= 12
    p = torch.as_tensor(params).cuda().contiguous()
    v, g = E.run(p)
    torch.cuda.synchronize()
    E.status()
    ang = W.resolve_angles(spec, params)
    np.testing.assert_allclose(v.cpu().numpy(), orc.expvals(spec, ang), atol=EXP_TOL)
    for b in (0, 3):
        ref = orc.param_grads_param_shift(spec, params[b].astype(np.float64))
        np.testing.assert_allclose(g[b].cpu().numpy(), ref, atol=GRAD_TOL)


def test_gradient_weights_per_circuit(api, orc):
    """Packed gradient weights [batch_c][groups_c]: each circuit's gradient is
    the weighted sum of its groups' gradients (the vector-Jacobian product)."""
    import torch
    wl = _workload(4)[1:4]
    C = [api.Circuit(s) for s, _, _ in wl]
    M = api.MultiExec(C, [p.shape[0] for _, p, _ in wl], grad="adjoint")
    params, inputs = _pack(M, wl, torch)
    r = np.random.default_rng(3500)
    ws = [r.normal(size=(p.shape[0], s.n_groups)) for s, p, _ in wl]
    gw = torch.cat([torch.as_tensor(w, dtype=torch.float64).reshape(-1) for w in ws]).cuda().contiguous()
    vals, grads = M.run(params, inputs, grad_weights=gw)
    torch.cuda.synchronize()
    M.status()
    _check_values(orc, M, wl, vals)
    for (spec, p, x), w, g in zip(wl, ws, M.unpack(grads, "grads")):
        b = p.shape[0] - 1
        ref = orc.param_grads_param_shift(spec, p[b].astype(np.float64), weights=list(w[b]))
        np.testing.assert_allclose(g[b].cpu().numpy(), ref, atol=GRAD_TOL)
