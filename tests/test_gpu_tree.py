"""Parity of the tree executor (any pairwise path, slicing, FP64 slice sum)
with the FP64 oracle, through the C ABI.  Tolerances: expectations 1e-5
absolute; amplitudes 1e-4 relative (plus 2e-6 absolute for amplitudes of
small circuits, whose FP32 rounding scales with the unit-norm state)."""
import json
import os

import numpy as np
import pytest

from paper_2301_05451_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_05451_gb300 import build
    build.build()
    from paper_2301_05451_gb300 import api as _api
    return _api


def _run_tree(api, spec, params, output, index=0, lightcone=False, split=False, method="greedy",
              target=0, plain=False, seed=0, repeats=1, B=None, inputs=None, hyper=False, rank_simplify=False):
    import torch
    C = api.Circuit(spec)
    N = api.Network(C, output, index, lightcone, split, hyper)
    P = api.Plan(N, method=method, seed=seed, temperature=0.3, target_log2=target, repeats=repeats,
                 rank_simplify=rank_simplify)
    B = B or params.shape[0]
    E = api.TreeExec(P, B, plain=plain)
    p = torch.as_tensor(params if params.shape[0] > 1 else params[0]).cuda()
    x = None if inputs is None else torch.as_tensor(inputs).cuda()
    v, _ = E.run(p, x)
    torch.cuda.synchronize()
    E.status()
    v = v.cpu().numpy()
    return (v[:, 0] if output == "expval" else v[:, 0] + 1j * v[:, 1]), P


def test_worked_example_tree(api, orc):
    c = W.CircuitSpec(2)
    c.add("X", [0]); c.add("RY", [1], ("p", 0)); c.add("CNOT", [0, 1]); c.z([1])
    th = np.linspace(-3, 6, 8).astype(np.float32)[:, None]
    for split in (False, True):
        for plain in (False, True):
            v, _ = _run_tree(api, c, th, "expval", split=split, plain=plain)
            np.testing.assert_allclose(v, -np.cos(th[:, 0].astype(np.float64)), atol=1e-5)


@pytest.mark.parametrize("plain", [False, True])
def test_c1_hea6_greedy_path(api, orc, plain):
    """The 6-qubit ansatz contracted along the greedy path, batch 1."""
    spec, params, _ = W.hea6()
    v, P = _run_tree(api, spec, params, "expval", plain=plain)
    ref = orc.expvals(spec, W.resolve_angles(spec, params))[0, 0]
    assert abs(v[0] - ref) < 1e-5


@pytest.mark.parametrize("seed", range(6))
def test_random_circuit_terms_and_amplitudes(api, orc, seed):
    n = 4 + seed
    spec, params, _ = W.random_circuit(n, 8 * n, 900 + seed, batch=3, amplitudes=2)
    ang = W.resolve_angles(spec, params)
    ev = orc.expvals(spec, ang)
    amps = orc.amplitudes(spec, ang)
    for t, (qs, coeff, g) in enumerate(spec.terms[:3]):
        for split in (False, True):
            v, _ = _run_tree(api, spec, params, "expval", index=t, split=split, target=6 if seed % 2 else 0,
                             plain=bool(seed % 3 == 0), lightcone=bool(t % 2))
            np.testing.assert_allclose(v, ev[:, g], atol=1e-5)
    for a in range(2):
        v, _ = _run_tree(api, spec, params, "amplitude", index=a, split=True, method="random_greedy",
                         seed=seed, target=4, plain=bool(seed % 2))
        assert np.all(np.abs(v - amps[:, a]) <= 1e-4 * np.abs(amps[:, a]) + 2e-6)
        # the hypergraph-partition path, unsplit and split networks, sliced
        v, _ = _run_tree(api, spec, params, "amplitude", index=a, split=bool(a), method="partition",
                         seed=seed, repeats=3, target=4 + a)
        assert np.all(np.abs(v - amps[:, a]) <= 1e-4 * np.abs(amps[:, a]) + 2e-6)
    v, _ = _run_tree(api, spec, params, "expval", index=0, lightcone=bool(seed % 2), method="partition",
                     seed=seed, repeats=3, target=8)
    np.testing.assert_allclose(v, ev[:, spec.terms[0][2]], atol=1e-5)


def test_slices_sum_to_unsliced(api, orc):
    """Sec. 3.2.3, Eq. 8: the sum over slices equals the unsliced contraction."""
    spec, params, _ = W.grid_u3cz(rows=3, cols=4, depth=6, seed=11)
    vals = []
    for target in (0, 6, 4, 3):
        v, P = _run_tree(api, spec, params, "amplitude", split=True, target=target)
        vals.append(v[0])
        if target:
            assert P.stats()["n_sliced"] > 0
    ref = orc.amplitudes(spec, W.resolve_angles(spec, params))[0, 0]
    for v in vals:
        assert abs(v - ref) <= 1e-4 * abs(ref) + 1e-7


@pytest.mark.parametrize("grad", ["none", "adjoint"])
def test_slice_ranges_shard_the_sum(api, orc, grad):
    """Slice sharding (Sec. 3.2.3): an exec restricted to disjoint slice
    ranges (as the ranks of a sharded run are) gives partial values and
    gradients whose FP64 sum -- what the one all-reduce forms -- equals the
    full contraction and the oracle; an empty range gives zeros; the full
    range restores the unrestricted result (after a graph replay)."""
    import torch
    from paper_2301_05451_gb300 import shard
    from paper_2301_05451_gb300._abi import TdqError, TDQ_ERR_ARG
    if grad == "none":
        spec, params, _ = W.grid_u3cz(rows=3, cols=4, depth=6, seed=11)
        out, target = "amplitude", 4
    else:  # sliced to 2^4 entries: 2^5 slices
        spec, params, _ = W.random_circuit(10, 60, 31, batch=2)
        out, target = "expval", 4
    C = api.Circuit(spec)
    N = api.Network(C, out, 0, False, True, False)
    P = api.Plan(N, method="greedy", target_log2=target)
    ns = 1 << P.stats()["n_sliced"]
    assert ns >= 4
    B = params.shape[0]
    E = api.TreeExec(P, B, grad=grad)
    p = torch.as_tensor(params if B > 1 else params[0]).cuda()
    full_v, full_g = E.run(p)
    full_v, full_g = full_v.double().cpu(), None if full_g is None else full_g.double().cpu()
    for world in (2, 3):
        acc_v, acc_g = 0, 0
        for r in range(world):
            lo, hi = shard.share(ns, r, world)
            E.set_slice_range(lo, hi - lo)
            v, g = E.run(p)
            torch.cuda.synchronize()
            E.status()
            acc_v = acc_v + v.double().cpu()
            if g is not None:
                acc_g = acc_g + g.double().cpu()
        np.testing.assert_allclose(acc_v.numpy(), full_v.numpy(), rtol=1e-5, atol=1e-7)
        if full_g is not None:
            np.testing.assert_allclose(acc_g.numpy(), full_g.numpy(), atol=1e-5)
    E.set_slice_range(1, 0)
    v, _ = E.run(p)
    assert float(v.abs().max()) == 0.0
    with pytest.raises(TdqError) as ei:
        E.set_slice_range(ns - 1, 2)
    assert ei.value.status == TDQ_ERR_ARG
    E.set_slice_range(0, ns)
    for _ in range(3):  # direct launch, capture, replay
        v, _ = E.run(p)
    torch.cuda.synchronize()
    np.testing.assert_allclose(v.double().cpu().numpy(), full_v.numpy(), rtol=1e-6, atol=1e-9)
    ang = W.resolve_angles(spec, params)
    if out == "amplitude":
        ref = orc.amplitudes(spec, ang)[:, 0]
        got = full_v.numpy()[:, 0] + 1j * full_v.numpy()[:, 1]
        assert np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref) + 1e-7)
    else:
        np.testing.assert_allclose(full_v.numpy()[:, 0], orc.expvals(spec, ang)[:, 0], atol=1e-5)


def test_c4a_lightcone_5x10(api, orc):
    """<Z_25> of the 5x10 RZZ/RX brickwork through its 16-qubit light cone."""
    gold = json.load(open(os.path.join(GOLDEN, "c4_values.json")))["brickwork_5x10_l4_z25"]["1003"]
    spec, params, _ = W.grid_brickwork()
    v, P = _run_tree(api, spec, params, "expval", lightcone=True)
    assert abs(v[0] - gold) < 1e-5
    v2, _ = _run_tree(api, spec, params, "expval", lightcone=True, plain=True, split=True)
    assert abs(v2[0] - gold) < 1e-5


def test_grid_5x5_amplitude(api, orc):
    spec, params, _ = W.grid_u3cz(rows=5, cols=5, depth=8)
    gold = json.load(open(os.path.join(GOLDEN, "c4_values.json")))["grid_u3cz_5x5_d8"]["1004"]
    v, _ = _run_tree(api, spec, params, "amplitude", split=True, target=12)
    g = complex(*gold)
    assert abs(v[0] - g) <= 1e-4 * abs(g)


@pytest.mark.parametrize("seed", [1004, 1005, 1006])
def test_c4b_7x7_depth8_sliced_amplitude(api, orc, seed):
    """The 49-qubit amplitude: random-greedy path on the split network,
    sliced to 2^17 entries, slices batched, FP64 slice sum; against the
    oracle's loop-nest contraction (stored)."""
    gold = json.load(open(os.path.join(GOLDEN, "c4_values.json")))["grid_u3cz_7x7_d8"][str(seed)]
    spec, params, _ = W.grid_u3cz(seed=seed)
    v, P = _run_tree(api, spec, params, "amplitude", split=True, method="random_greedy", seed=1,
                     repeats=16, target=17)
    st = P.stats()
    assert st["max_log2_width"] <= 17 and st["n_sliced"] >= 1
    g = complex(*gold)
    assert abs(v[0] - g) <= 1e-4 * abs(g), (v[0], g, st)


@pytest.mark.parametrize("seed", [1004, 1005, 1006])
def test_c4b_7x7_depth8_partition_path(api, orc, seed):
    """The same 49-qubit amplitudes along the hypergraph-partition path
    (Sec. 3.2.2) with two-phase slicing to 2^15 entries."""
    gold = json.load(open(os.path.join(GOLDEN, "c4_values.json")))["grid_u3cz_7x7_d8"][str(seed)]
    spec, params, _ = W.grid_u3cz(seed=seed)
    v, P = _run_tree(api, spec, params, "amplitude", split=True, method="partition", seed=1,
                     repeats=64, target=15)
    st = P.stats()
    assert st["max_log2_width"] <= 15 and st["n_sliced"] >= 1
    g = complex(*gold)
    assert abs(v[0] - g) <= 1e-4 * abs(g), (v[0], g, st)


def test_mirror_7x7(api, orc):
    spec, params, _ = W.grid_u3cz_mirror(rows=7, cols=7, depth=4)
    v, _ = _run_tree(api, spec, params, "amplitude", split=True, method="random_greedy", seed=2,
                     repeats=8, target=22)
    assert abs(v[0] - 1) < 1e-4


@pytest.mark.parametrize("plain", [False, True])
def test_tree_adjoint_hea6_greedy_path(api, orc, plain):
    """Reverse tree of the greedy path: value and gradient of the 6-qubit
    ansatz against the shift rule in FP64."""
    import torch
    spec, params, _ = W.hea6()
    C = api.Circuit(spec)
    N = api.Network(C, "expval", 0)
    P = api.Plan(N)
    E = api.TreeExec(P, 1, grad="adjoint", plain=plain)
    v, g = E.run(torch.as_tensor(params[0]).cuda())
    torch.cuda.synchronize()
    E.status()
    ref_v = orc.expvals(spec, W.resolve_angles(spec, params))[0, 0]
    ref_g = orc.param_grads_param_shift(spec, params[0].astype(np.float64))
    assert abs(v[0, 0].item() - ref_v) < 1e-5
    np.testing.assert_allclose(g[0].cpu().numpy(), ref_g, atol=1e-4)


@pytest.mark.parametrize("seed", range(4))
def test_tree_adjoint_random_terms(api, orc, seed):
    """Every gate kind (U3, RZZ, CNOT, CZ ...), split and unsplit networks,
    light cone, slices, batch rows with weights."""
    import torch
    n = 4 + seed
    spec, params, _ = W.random_circuit(n, 7 * n, 1300 + seed, batch=3)
    ang = W.resolve_angles(spec, params)
    for t in (0, len(spec.terms) - 1):
        qs, coeff, grp = spec.terms[t]
        C = api.Circuit(spec)
        N = api.Network(C, "expval", t, lightcone=bool(seed % 2), split_2q=bool(seed >= 2))
        P = api.Plan(N, method="random_greedy", seed=seed, temperature=0.3, target_log2=4 if seed == 3 else 0)
        E = api.TreeExec(P, 3, grad="adjoint", plain=(seed == 1))
        w = torch.tensor([0.5, -1.0, 2.0], dtype=torch.float64, device="cuda")
        v, g = E.run(torch.as_tensor(params).cuda().contiguous(), grad_weights=w)
        torch.cuda.synchronize()
        E.status()
        ev = orc.expvals(spec, ang)[:, grp]
        # the network of one term: coeff * <Z..>; ev groups sum terms of a group
        single = W.CircuitSpec(spec.n_qubits)
        single.gates, single.terms, single.n_groups = spec.gates, [(qs, coeff, 0)], 1
        sv = orc.expvals(single, ang)[:, 0]
        np.testing.assert_allclose(v[:, 0].cpu().numpy(), sv, atol=1e-5)
        for b in range(3):
            ref = orc.param_grads_param_shift(single, params[b].astype(np.float64), weights=[w[b].item()])
            np.testing.assert_allclose(g[b].cpu().numpy(), ref, atol=1e-4)


def test_tree_adjoint_partition_path(api, orc):
    """Reverse tree along a hypergraph-partition path with slices."""
    import torch
    spec, params, _ = W.random_circuit(7, 49, 1400, batch=2)
    ang = W.resolve_angles(spec, params)
    qs, coeff, grp = spec.terms[0]
    single = W.CircuitSpec(spec.n_qubits)
    single.gates, single.terms, single.n_groups = spec.gates, [(qs, coeff, 0)], 1
    C = api.Circuit(spec)
    N = api.Network(C, "expval", 0, lightcone=False, split_2q=True)
    P = api.Plan(N, method="partition", seed=4, repeats=4, target_log2=5)
    assert P.stats()["n_sliced"] >= 1
    E = api.TreeExec(P, 2, grad="adjoint")
    v, g = E.run(torch.as_tensor(params).cuda().contiguous())
    torch.cuda.synchronize()
    E.status()
    np.testing.assert_allclose(v[:, 0].cpu().numpy(), orc.expvals(single, ang)[:, 0], atol=1e-5)
    for b in range(2):
        ref = orc.param_grads_param_shift(single, params[b].astype(np.float64))
        np.testing.assert_allclose(g[b].cpu().numpy(), ref, atol=1e-4)


def test_tree_graph_replay_follows_inputs(api, orc):
    """A call that repeats the previous call's pointers is captured as a CUDA
    graph and replayed: new parameter values written into the same buffer,
    and a switch of output buffer, give the oracle's values every time."""
    import torch
    spec, params, _ = W.random_circuit(8, 64, 1500, batch=2)
    C = api.Circuit(spec)
    qs, coeff, grp = spec.terms[0]
    single = W.CircuitSpec(spec.n_qubits)
    single.gates, single.terms, single.n_groups = spec.gates, [(qs, coeff, 0)], 1
    P = api.Plan(api.Network(C, "expval", 0, split_2q=True), method="partition", seed=2, repeats=4, target_log2=6)
    E = api.TreeExec(P, 2)
    p = torch.zeros(params.shape, dtype=torch.float32, device="cuda")
    outs = [E.alloc_outputs()[0], E.alloc_outputs()[0]]
    r = np.random.default_rng(1501)
    for it in range(6):
        x = (r.random(params.shape) * 2 * np.pi).astype(np.float32)
        p.copy_(torch.as_tensor(x))
        vals = outs[1] if it == 4 else outs[0]
        E.run(p, values=vals)
        torch.cuda.synchronize()
        E.status()
        ref = orc.expvals(single, W.resolve_angles(spec, x))[:, 0]
        np.testing.assert_allclose(vals[:, 0].cpu().numpy(), ref, atol=1e-5)



HYPER_GATES = ("H", "X", "Y", "Z", "RX", "RY", "RZ", "U3", "CNOT", "CZ", "RZZ")


@pytest.mark.parametrize("seed", range(6))
def test_hyper_networks_terms_and_amplitudes(api, orc, seed):
    """Diagonal reduction (hyperedges): expectations and amplitudes of random
    circuits over every gate kind, greedy and partition paths, sliced
    hyperedges, the fused and the one-launch-per-step forms."""
    n = 4 + seed
    spec, params, _ = W.random_circuit(n, 9 * n, 1600 + seed, batch=3, amplitudes=2, gates=HYPER_GATES)
    ang = W.resolve_angles(spec, params)
    ev = orc.expvals(spec, ang)
    amps = orc.amplitudes(spec, ang)
    method = "partition" if seed % 2 else "greedy"
    for t, (qs, coeff, g) in enumerate(spec.terms[:2] + spec.terms[-1:]):
        ti = spec.terms.index((qs, coeff, g))
        single = W.CircuitSpec(spec.n_qubits)
        single.gates, single.terms, single.n_groups = spec.gates, [(qs, coeff, 0)], 1
        ref = orc.expvals(single, ang)[:, 0]
        v, P = _run_tree(api, spec, params, "expval", index=ti, lightcone=bool(t % 2), method=method, seed=seed,
                         repeats=3, target=(5 if seed % 3 else 0), plain=(seed == 2), hyper=True)
        np.testing.assert_allclose(v, ref, atol=1e-5)
    for a in range(2):
        v, _ = _run_tree(api, spec, params, "amplitude", index=a, method=method, seed=seed, repeats=3,
                         target=3 + a, plain=(seed == 4), hyper=True)
        assert np.all(np.abs(v - amps[:, a]) <= 1e-4 * np.abs(amps[:, a]) + 2e-6)


@pytest.mark.parametrize("plain", [False, True])
def test_hyper_adjoint_gradients(api, orc, plain):
    """Reverse tree through diagonal (RZ, RZZ, CZ, Z) and controlled leaves:
    values and parameter gradients against the FP64 shift rule."""
    import torch
    spec, params, _ = W.random_circuit(6, 48, 1700 + int(plain), batch=2, gates=HYPER_GATES)
    ang = W.resolve_angles(spec, params)
    for t in (0, len(spec.terms) - 1):
        qs, coeff, grp = spec.terms[t]
        single = W.CircuitSpec(spec.n_qubits)
        single.gates, single.terms, single.n_groups = spec.gates, [(qs, coeff, 0)], 1
        C = api.Circuit(spec)
        N = api.Network(C, "expval", t, lightcone=bool(t), hyper=True)
        P = api.Plan(N, method="partition", seed=3, repeats=3, target_log2=4 if t else 0)
        E = api.TreeExec(P, 2, grad="adjoint", plain=plain)
        v, g = E.run(torch.as_tensor(params).cuda().contiguous())
        torch.cuda.synchronize()
        E.status()
        np.testing.assert_allclose(v[:, 0].cpu().numpy(), orc.expvals(single, ang)[:, 0], atol=1e-5)
        for b in range(2):
            ref = orc.param_grads_param_shift(single, params[b].astype(np.float64))
            np.testing.assert_allclose(g[b].cpu().numpy(), ref, atol=1e-4)


@pytest.mark.parametrize("seed", [0, 1])
def test_anti_diagonal_reduction_gpu(api, orc, seed):
    """X / Y-heavy circuits on hyper networks, where X and Y leave no gate
    tensor (complemented indices, Y's phases as a one-index tensor): sliced
    amplitudes, and expectation values with adjoint gradients through the
    complemented leaves, against the oracle."""
    import torch
    spec, params, _ = W.random_circuit(7, 50, 3400 + seed, batch=2, amplitudes=1,
                                       gates=("X", "Y", "RX", "RY", "RZ", "CNOT", "CZ", "RZZ"))
    for q in range(7):
        spec.add("X" if (q + seed) % 2 else "Y", [q])
    C = api.Circuit(spec)
    Na = api.Network(C, "amplitude", 0, False, False, True)
    assert any(Na.tensor(i)["flip"] for i in range(Na.n_tensors))
    ang = W.resolve_angles(spec, params)
    v, P = _run_tree(api, spec, params, "amplitude", method="greedy", target=3, hyper=True)
    assert P.stats()["n_sliced"] >= 1
    ref = orc.amplitudes(spec, ang)[:, 0]
    assert np.all(np.abs(v - ref) <= 1e-4 * np.abs(ref) + 2e-6)
    for t in (0, len(spec.terms) - 1):
        qs, coeff, grp = spec.terms[t]
        single = W.CircuitSpec(spec.n_qubits)
        single.gates, single.terms, single.n_groups = spec.gates, [(qs, coeff, 0)], 1
        N = api.Network(C, "expval", t, lightcone=bool(t), hyper=True)
        E = api.TreeExec(api.Plan(N, method="greedy", target_log2=4), 2, grad="adjoint")
        vv, g = E.run(torch.as_tensor(params).cuda().contiguous())
        torch.cuda.synchronize()
        E.status()
        np.testing.assert_allclose(vv[:, 0].cpu().numpy(), orc.expvals(single, ang)[:, 0], atol=1e-5)
        for b in range(2):
            gref = orc.param_grads_param_shift(single, params[b].astype(np.float64))
            np.testing.assert_allclose(g[b].cpu().numpy(), gref, atol=1e-4)


@pytest.mark.parametrize("seed", [1004, 1005, 1006])
def test_c4b_7x7_depth8_hyper_partition(api, orc, seed):
    """The 49-qubit amplitudes on the diagonally reduced network (CZ as
    hyperedges) along a partition path sliced to 2^13 entries."""
    gold = json.load(open(os.path.join(GOLDEN, "c4_values.json")))["grid_u3cz_7x7_d8"][str(seed)]
    spec, params, _ = W.grid_u3cz(seed=seed)
    v, P = _run_tree(api, spec, params, "amplitude", method="partition", seed=1, repeats=64, target=13,
                     hyper=True)
    st = P.stats()
    assert st["max_log2_width"] <= 13 and st["n_sliced"] >= 1
    g = complex(*gold)
    assert abs(v[0] - g) <= 1e-4 * abs(g), (v[0], g, st)


@pytest.mark.parametrize("method", ["greedy", "partition"])
def test_rank_simplified_plans(api, orc, method):
    """Rank simplification before the path search (Sec. 3.2.1): the 7x7
    amplitude on the diagonally reduced network, sliced, against its golden
    value; expectations and adjoint gradients of a random circuit (hyper
    network) against the FP64 oracle and its shift rule."""
    import torch
    gold = json.load(open(os.path.join(GOLDEN, "c4_values.json")))["grid_u3cz_7x7_d8"]["1004"]
    spec, params, _ = W.grid_u3cz(seed=1004)
    v, P = _run_tree(api, spec, params, "amplitude", method=method, seed=1, repeats=16, target=13, hyper=True,
                     rank_simplify=True)
    g = complex(*gold)
    assert abs(v[0] - g) <= 1e-4 * abs(g), (v[0], g, P.stats())
    spec, params, _ = W.random_circuit(6, 48, 1750, batch=2, gates=HYPER_GATES)
    ang = W.resolve_angles(spec, params)
    for t in (0, len(spec.terms) - 1):
        qs, coeff, grp = spec.terms[t]
        single = W.CircuitSpec(spec.n_qubits)
        single.gates, single.terms, single.n_groups = spec.gates, [(qs, coeff, 0)], 1
        N = api.Network(api.Circuit(spec), "expval", t, lightcone=bool(t), hyper=True)
        P = api.Plan(N, method=method, seed=3, repeats=3, target_log2=4 if t else 0, rank_simplify=True)
        E = api.TreeExec(P, 2, grad="adjoint")
        v, gr = E.run(torch.as_tensor(params).cuda().contiguous())
        torch.cuda.synchronize()
        E.status()
        np.testing.assert_allclose(v.cpu().numpy()[:, 0], orc.expvals(single, ang)[:, 0], atol=1e-5)
        for b in range(2):
            ref = orc.param_grads_param_shift(single, params[b].astype(np.float64))
            np.testing.assert_allclose(gr[b].cpu().numpy(), ref, atol=1e-4)


def test_c4a_lightcone_5x10_hyper(api, orc):
    gold = json.load(open(os.path.join(GOLDEN, "c4_values.json")))["brickwork_5x10_l4_z25"]["1003"]
    spec, params, _ = W.grid_brickwork()
    for plain in (False, True):
        v, _ = _run_tree(api, spec, params, "expval", lightcone=True, plain=plain, hyper=True)
        assert abs(v[0] - gold) < 1e-5


@pytest.mark.parametrize("hyper", [False, True])
def test_tree_adjoint_recomputes_when_hbm_is_short(api, orc, hyper):
    """With a workspace budget below what keeping every value (and cotangent)
    of the reverse tree needs, the compile switches to recomputing the values
    region by region from checkpoints; values and gradients still match the
    FP64 shift rule and the workspace stays within the budget."""
    import torch
    spec, params, _ = W.random_circuit(9, 90, 1800 + int(hyper), batch=2,
                                       gates=HYPER_GATES if hyper else ("H", "RX", "RY", "RZ", "U3", "CNOT", "CZ",
                                                                        "RZZ"))
    ang = W.resolve_angles(spec, params)
    qs, coeff, grp = spec.terms[0]
    single = W.CircuitSpec(spec.n_qubits)
    single.gates, single.terms, single.n_groups = spec.gates, [(qs, coeff, 0)], 1
    C = api.Circuit(spec)
    N = api.Network(C, "expval", 0, split_2q=not hyper, hyper=hyper)
    P = api.Plan(N, method="greedy")
    B = 2
    full = api.TreeExec(P, B, grad="adjoint", plain=True)
    cfg = full.config()
    assert cfg["reverse"] == 2
    budget = int(cfg["workspace_entries"] * 8 * B * 0.8)
    E = api.TreeExec(P, B, grad="adjoint", plain=True, workspace_bytes=budget)
    rc = E.config()
    assert rc["reverse"] == 3 and rc["regions"] >= 2, rc
    assert rc["workspace_entries"] * 8 * B <= budget
    p = torch.as_tensor(params).cuda().contiguous()
    for ex in (full, E):
        v, g = ex.run(p)
        torch.cuda.synchronize()
        ex.status()
        np.testing.assert_allclose(v[:, 0].cpu().numpy(), orc.expvals(single, ang)[:, 0], atol=1e-5)
        for b in range(B):
            ref = orc.param_grads_param_shift(single, params[b].astype(np.float64))
            np.testing.assert_allclose(g[b].cpu().numpy(), ref, atol=1e-4)


def test_concurrent_schedule_over_several_slice_batches(api, orc):
    """A workspace budget that holds only part of the slices: the concurrent
    large steps and the graph replay run batch after batch of slices; the
    5x5 amplitude still matches the stored oracle value."""
    import torch
    gold = complex(*json.load(open(os.path.join(GOLDEN, "c4_values.json")))["grid_u3cz_5x5_d8"]["1004"])
    spec, params, _ = W.grid_u3cz(rows=5, cols=5, depth=8)
    C = api.Circuit(spec)
    N = api.Network(C, "amplitude", 0, hyper=True)
    P = api.Plan(N, method="partition", seed=3, repeats=8, target_log2=7)
    assert P.stats()["n_sliced"] >= 3
    whole = api.TreeExec(P, 1)
    per_slice = whole.config()["workspace_entries"] * 8
    E = api.TreeExec(P, 1, workspace_bytes=per_slice * 3)
    cfg = E.config()
    assert 1 <= cfg["chunk"] < 2 ** P.stats()["n_sliced"], cfg
    p = torch.as_tensor(params[0]).cuda()
    vals, _ = E.alloc_outputs()
    for _ in range(3):  # direct, captured, replayed
        E.run(p, values=vals)
        torch.cuda.synchronize()
        E.status()
        v = complex(*vals[0].cpu().numpy())
        assert abs(v - gold) <= 1e-4 * abs(gold), (v, gold, cfg)
