"""Contraction paths and slicing on the host (Sec. 3.2.2-3.2.3), no device
work: every path finder returns a valid SSA path over all tensors, whose
FLOPs p(2q - 1) per step (Eq. 5) and widths -- recomputed here from the
network's index sets -- are the plan's statistics; slicing meets its width
target; the two-phase slicing-aware search never ends above the single
greedy slicing of the same trees; the hypergraph-partition finder beats the
greedy finders on deep grid networks."""
import ctypes

import numpy as np
import pytest

from paper_2301_05451_gb300 import workloads as W

METHODS = ("greedy", "random_greedy", "partition")


@pytest.fixture(scope="module")
def api():
    from paper_2301_05451_gb300 import build
    build.build()
    from paper_2301_05451_gb300 import api as _api
    return _api


def _networks(api):
    single = W.CircuitSpec(3)  # no two-qubit gate: three disconnected pieces
    for q in range(3):
        single.add("RX", [q], ("p", q))
    single.z([0])
    single.amplitude([0, 1, 0])
    bare = W.CircuitSpec(1)  # two tensors: |0> and <0|
    bare.z([0])
    bare.amplitude([0])
    r6 = W.random_circuit(6, 40, 77, amplitudes=1)[0]
    out = []
    for name, spec, kind, lc, split, hyper in [
            ("random6_expval", r6, "expval", False, False, False),
            ("random6_expval_split_cone", r6, "expval", True, True, False),
            ("random6_amp", r6, "amplitude", False, True, False),
            ("random6_expval_hyper", r6, "expval", False, False, True),
            ("random6_amp_hyper_cone", r6, "amplitude", True, False, True),
            ("grid4x4", W.grid_u3cz(rows=4, cols=4, depth=6)[0], "amplitude", False, True, False),
            ("grid4x4_hyper", W.grid_u3cz(rows=4, cols=4, depth=6)[0], "amplitude", False, False, True),
            ("brickwork_hyper", W.grid_brickwork(rows=3, cols=4, layers=4, observed=5)[0], "expval", True, False,
             True),
            ("disconnected", single, "amplitude", False, False, False),
            ("disconnected_hyper", single, "amplitude", False, False, True),
            ("two_tensors", bare, "amplitude", False, False, False),
            ("two_tensors_hyper", bare, "expval", False, False, True)]:
        C = api.Circuit(spec)
        out.append((name, C, api.Network(C, kind, 0, lc, split, hyper)))
    return out


def _recount(N, path, sliced):
    """FLOPs over all slices, log2 width: from the index sets, sliced indices
    removed.  An index on both operands is summed unless a third live tensor
    holds it (a hyperedge); an index on one tensor only is open and stays."""
    cut = set(sliced)
    full = [N.tensor(i)["idx"] for i in range(N.n_tensors)]
    live = {}
    for idx in full:
        for i in idx:
            live[i] = live.get(i, 0) + 1
    live = {i: max(c, 2) for i, c in live.items()}
    T = [set(idx) - cut for idx in full]
    used = set()
    flops = 0
    moved = []
    for s, (a, b) in enumerate(path):
        assert 0 <= a < len(T) and 0 <= b < len(T) and a != b, (s, a, b)
        assert a not in used and b not in used, (s, a, b)
        used |= {a, b}
        summed = {i for i in T[a] & T[b] if live[i] == 2}
        r = (T[a] | T[b]) - summed
        for i in T[a] | T[b]:
            live[i] -= (i in T[a]) + (i in T[b]) - (i in r)
        flops += 2 ** len(r) * (2 ** (len(summed) + 1) - 1)
        moved.append(8 * (2 ** len(T[a]) + 2 ** len(T[b]) + 2 ** len(r)))  # operands read, result written
        T.append(r)
    assert len(path) == N.n_tensors - 1
    assert set(range(len(T) - 1)) == used  # every tensor but the root consumed once
    _recount.bytes_per_slice = sum(moved)
    return flops * 2 ** len(sliced), max(len(t) for t in T)


@pytest.mark.parametrize("method", METHODS)
def test_paths_are_valid_and_stats_recount(api, method):
    for name, C, N in _networks(api):
        for target in (0, 3):
            P = api.Plan(N, method=method, seed=5, repeats=4, temperature=0.3, target_log2=target)
            path, sliced = P.path()
            st = P.stats()
            flops, width = _recount(N, path, sliced)
            assert st["n_steps"] == len(path) and st["n_sliced"] == len(sliced)
            assert abs(flops - st["flops"]) <= 1e-9 * flops, (name, flops, st)
            assert width == st["max_log2_width"], (name, width, st)
            if path:  # bytes moved per slice: every step's operands and result (the m q + n q memory term)
                assert abs(2 ** st["log2_bytes_per_slice"] - _recount.bytes_per_slice) <= 1e-9 * _recount.bytes_per_slice
            if target:
                assert width <= target, (name, st)
            Q = api.Plan(N, path=path, sliced=sliced)
            assert Q.stats() == st


def _widens(a, b, live):
    """Indices of the contraction of index sets a and b (an index on both is
    summed unless a third live tensor holds it), and whether it has more
    indices than the larger operand."""
    summed = {i for i in a & b if live[i] == 2}
    r = (a | b) - summed
    return r, len(r) > max(len(a), len(b))


@pytest.mark.parametrize("method", METHODS)
def test_rank_simplification_opens_the_path(api, method):
    """Rank simplification (Sec. 3.2.1): with the option on, the path starts
    with contractions that never widen the network, and when the first
    widening step comes no pair of tensors sharing an index could still be
    contracted without widening (the simplification ran to completion before
    the finder took over).  The path stays a valid SSA path whose FLOP and
    width statistics recount, and it round-trips through the caller-path
    form."""
    simplified = 0
    for name, C, N in _networks(api):
        for target in (0, 3):
            P = api.Plan(N, method=method, seed=5, repeats=4, temperature=0.3, target_log2=target,
                         rank_simplify=True)
            path, sliced = P.path()
            st = P.stats()
            flops, width = _recount(N, path, sliced)
            assert abs(flops - st["flops"]) <= 1e-9 * flops and width == st["max_log2_width"], (name, st)
            assert api.Plan(N, path=path, sliced=sliced).stats() == st
            full = [set(N.tensor(i)["idx"]) for i in range(N.n_tensors)]
            live = {}
            for idx in full:
                for i in idx:
                    live[i] = live.get(i, 0) + 1
            live = {i: max(c, 2) for i, c in live.items()}
            T, alive = list(full), set(range(len(full)))
            for a, b in path:
                r, wide = _widens(T[a], T[b], live)
                if wide:
                    for x in alive:
                        for y in alive:
                            if x < y and T[x] & T[y]:
                                assert _widens(T[x], T[y], live)[1], (name, "unsimplified pair", x, y)
                    break
                simplified += 1
                for i in T[a] | T[b]:
                    live[i] -= (i in T[a]) + (i in T[b]) - (i in r)
                alive -= {a, b}
                alive.add(len(T))
                T.append(r)
    assert simplified > 0


def test_rank_simplification_option_checked(api):
    from paper_2301_05451_gb300 import _abi as A
    N = api.Network(api.Circuit(W.hea6()[0]), "expval", 0)
    h = ctypes.c_void_p()
    bad = A.PlanOpts(A.TDQ_PATH_GREEDY, 0, 0.0, 0, 1, 0, 0, 2)
    assert A.lib().tdq_plan_find(N.h, ctypes.byref(bad), ctypes.byref(h)) == A.TDQ_ERR_ARG


@pytest.mark.parametrize("method", ["random_greedy", "partition"])
def test_slicing_meets_target(api, method):
    C = api.Circuit(W.grid_u3cz(depth=12)[0])
    N = api.Network(C, "amplitude", 0, False, True)
    for target in (24, 20, 16):
        P = api.Plan(N, method=method, seed=1, repeats=4, temperature=0.3, target_log2=target)
        st = P.stats()
        assert st["max_log2_width"] <= target and st["n_sliced"] >= 1, st
        flops, width = _recount(N, *P.path())
        assert abs(flops - st["flops"]) <= 1e-9 * flops and width == st["max_log2_width"]


@pytest.mark.parametrize("method", ["random_greedy", "partition"])
def test_two_phase_slicing_never_above_single_greedy_slicing(api, method):
    """Phase 1 scores each trial tree by its best of many randomised slicings
    (the single greedy slicing among them), phase 2 slices the winner again:
    the result is at most the single-slicing plan over the same trees."""
    C = api.Circuit(W.grid_u3cz(depth=12)[0])
    N = api.Network(C, "amplitude", 0, False, True)
    for target in (22, 18):
        one = api.Plan(N, method=method, seed=3, repeats=6, temperature=0.3, target_log2=target,
                       slice_trials=0, slice_final=0).stats()
        two = api.Plan(N, method=method, seed=3, repeats=6, temperature=0.3, target_log2=target,
                       slice_trials=64, slice_final=256).stats()
        assert two["flops"] <= one["flops"] and two["max_log2_width"] <= target, (one, two)


def test_partition_beats_greedy_on_deep_grids(api):
    for depth, margin in ((8, 10.0), (12, 10.0)):
        C = api.Circuit(W.grid_u3cz(depth=depth)[0])
        N = api.Network(C, "amplitude", 0, False, True)
        g = api.Plan(N, method="greedy").stats()["flops"]
        rg = api.Plan(N, method="random_greedy", seed=1, repeats=16, temperature=0.3).stats()["flops"]
        part = api.Plan(N, method="partition", seed=1, repeats=16).stats()["flops"]
        assert part * margin < rg < g, (depth, part, rg, g)


def test_partition_is_deterministic(api):
    """Trials run on several host threads; the plan depends on the seed only."""
    C = api.Circuit(W.grid_u3cz(rows=5, cols=6, depth=8)[0])
    N = api.Network(C, "amplitude", 0, False, True)
    a = api.Plan(N, method="partition", seed=9, repeats=12, target_log2=12)
    b = api.Plan(N, method="partition", seed=9, repeats=12, target_log2=12)
    assert a.path() == b.path() and a.stats() == b.stats()


def test_plan_find_argument_errors(api):
    from paper_2301_05451_gb300 import _abi as A
    C = api.Circuit(W.hea6()[0])
    N = api.Network(C, "expval", 0)
    L = A.lib()
    h = ctypes.c_void_p()
    for opts in (A.PlanOpts(3, 0, 0.0, 0, 1, 0, 0), A.PlanOpts(A.TDQ_PATH_PARTITION, 0, 0.0, 0, 1, -1, 0),
                 A.PlanOpts(A.TDQ_PATH_PARTITION, 0, 0.0, 0, 1, 0, (1 << 20) + 1),
                 A.PlanOpts(A.TDQ_PATH_PARTITION, 0, 0.0, 41, 1, 0, 0)):
        assert L.tdq_plan_find(N.h, ctypes.byref(opts), ctypes.byref(h)) == A.TDQ_ERR_ARG
    ok = A.PlanOpts(A.TDQ_PATH_PARTITION, 0, 0.0, 4, 2, 8, 8)
    assert L.tdq_plan_find(N.h, ctypes.byref(ok), ctypes.byref(h)) == A.TDQ_OK
    L.tdq_plan_destroy(h)


# ---------------------------------------------------------------- network values

def _leaf_tensor(N, spec, ang, i):
    """Leaf i of the network as a numpy array, from the oracle's gate matrices
    and the structural definitions of each leaf kind."""
    from oracle import gate_matrix
    L = N.tensor(i)
    kind, g, conj, bit = L["kind"], L["gate"], L["conj"], L["bit"]
    M = None
    if g >= 0:
        gate = spec.gates[g]
        M = gate_matrix(gate.name, ang[g][:3])
    if kind == 0:  # |0>
        t = np.array([1, 0], complex)
    elif kind == 3:  # <b|
        t = np.eye(2, dtype=complex)[bit]
    elif kind == 2:  # Z between (bra, ket)
        t = np.diag([1, -1]).astype(complex)
    elif kind == 1 and M.shape[0] == 2:  # (out, in)
        t = M.copy()
    elif kind == 1:  # (oa, ob, ia, ib)
        t = M.reshape(2, 2, 2, 2).copy()
    elif kind == 4:  # (bond, out, in): copy tensor
        t = np.zeros((2, 2, 2), complex)
        t[0, 0, 0] = t[1, 1, 1] = 1
    elif kind == 5:  # (bond, out, in) = block `bond` of the gate, diagonal in its first qubit
        t = np.stack([M[2 * s:2 * s + 2, 2 * s:2 * s + 2] for s in range(2)])
    elif kind == 6 and g < 0:  # the Z observable's diagonal
        t = np.array([1, -1], complex)
    elif kind == 6 and spec.gates[g].name == "Y":  # anti-diagonal reduction: Y[1 - i][i]
        t = np.array([M[1, 0], M[0, 1]])
    elif kind == 6 and M.shape[0] == 2:  # one-qubit diagonal
        t = np.diag(M).copy()
    elif kind == 6:  # two-qubit diagonal (a, b)
        t = np.diag(M).reshape(2, 2).copy()
    elif kind == 7:  # (control, out, in) = block `control` of the CNOT
        t = np.stack([M[2 * c:2 * c + 2, 2 * c:2 * c + 2] for c in range(2)])
    else:
        raise AssertionError(kind)
    assert t.ndim == len(L["idx"]), (kind, t.shape, L["idx"])
    for a in range(t.ndim):  # complemented indices (anti-diagonal reduction)
        if (L["flip"] >> a) & 1:
            t = np.flip(t, axis=a)
    return t.conj() if conj else t, L["idx"]


def _network_value(N, spec, ang):
    import string
    letters = string.ascii_letters
    ops, subs = [], []
    for i in range(N.n_tensors):
        t, idx = _leaf_tensor(N, spec, ang, i)
        assert max(idx) < len(letters)
        ops.append(t)
        subs.append("".join(letters[j] for j in idx))
    return np.einsum(",".join(subs) + "->", *ops, optimize="greedy")


def _small_circuits():
    out = []
    for seed in range(6):
        n = 3 + seed % 2
        spec, params, _ = W.random_circuit(n, 7 + n, 2100 + seed, amplitudes=1,
                                           gates=("H", "X", "Y", "Z", "RX", "RY", "RZ", "U3", "CNOT", "CZ", "RZZ"))
        out.append((spec, W.resolve_angles(spec, params)[0]))
    return out


@pytest.mark.parametrize("hyper", [False, True])
def test_network_values_match_the_oracle(api, orc, hyper):
    """Step (a) and the diagonal reduction of step (b): every network of a
    circuit -- amplitude and expectation, with and without the light cone, the
    split two-qubit gates or the hyperedges -- contracted by numpy's einsum
    from leaves made of the oracle's gate matrices, equals the oracle's state
    vector result."""
    for spec, ang in _small_circuits():
        C = api.Circuit(spec)
        psi = orc.statevector(spec, ang)
        bits = spec.amplitudes[0]
        ref_amp = psi[int("".join(str(b) for b in bits), 2)]
        for split in (False, True):
            N = api.Network(C, "amplitude", 0, False, split, hyper)
            assert abs(_network_value(N, spec, ang) - ref_amp) < 1e-12
        for t, (qs, coeff, grp) in enumerate(spec.terms):
            single = W.CircuitSpec(spec.n_qubits)
            single.gates, single.terms, single.n_groups = spec.gates, [(qs, coeff, 0)], 1
            ref = orc.expvals(single, ang[None])[0, 0]
            for lc in (False, True):
                N = api.Network(C, "expval", t, lc, not hyper, hyper)
                v = coeff * _network_value(N, spec, ang)
                assert abs(v - ref) < 1e-12 and abs(v.imag) < 1e-12, (t, lc, v, ref)


def test_anti_diagonal_reduction(api, orc):
    """X and Y in a hyper network leave no gate tensor: the wire keeps its
    index and later tensors read it complemented (Sec. 3.2.1, structural
    simplification); a Y leaves its phases as a one-index tensor.  Values of
    X / Y-heavy circuits, amplitudes and expectations, ket and bra sides,
    against the oracle; and the reduced network has fewer tensors."""
    for seed in range(4):
        spec, params, _ = W.random_circuit(4, 14, 3300 + seed, amplitudes=2,
                                           gates=("X", "Y", "H", "RY", "RZ", "CNOT", "CZ", "RZZ"))
        for q in range(4):
            spec.add("X" if (q + seed) % 2 else "Y", [q])
        ang = W.resolve_angles(spec, params)[0]
        C = api.Circuit(spec)
        psi = orc.statevector(spec, ang)
        for a, bits in enumerate(spec.amplitudes):
            N = api.Network(C, "amplitude", a, False, False, True)
            ref = psi[int("".join(str(b) for b in bits), 2)]
            assert abs(_network_value(N, spec, ang) - ref) < 1e-12
            plain = api.Network(C, "amplitude", a, False, True, False)
            n_anti = sum(1 for g in spec.gates if g.name in ("X", "Y"))
            n_y = sum(1 for g in spec.gates if g.name == "Y")
            assert N.n_tensors <= plain.n_tensors - (n_anti - n_y)
            assert any(N.tensor(i)["flip"] for i in range(N.n_tensors))
        for t, (qs, coeff, grp) in enumerate(spec.terms):
            single = W.CircuitSpec(spec.n_qubits)
            single.gates, single.terms, single.n_groups = spec.gates, [(qs, coeff, 0)], 1
            ref = orc.expvals(single, ang[None])[0, 0]
            for lc in (False, True):
                N = api.Network(C, "expval", t, lc, False, True)
                v = coeff * _network_value(N, spec, ang)
                assert abs(v - ref) < 1e-12 and abs(v.imag) < 1e-12, (seed, t, lc, v, ref)


def test_hyper_networks_have_hyperedges_and_fewer_indices(api):
    spec = W.grid_brickwork(rows=4, cols=5, layers=6, observed=7)[0]
    C = api.Circuit(spec)
    plain = api.Network(C, "expval", 0, True, True)
    hyp = api.Network(C, "expval", 0, True, False, True)
    holders = {}
    for i in range(hyp.n_tensors):
        for j in hyp.tensor(i)["idx"]:
            holders[j] = holders.get(j, 0) + 1
    assert max(holders.values()) > 2
    assert hyp.n_indices < plain.n_indices
    for method in ("greedy", "partition"):
        a = api.Plan(plain, method=method, seed=1, repeats=8).stats()
        b = api.Plan(hyp, method=method, seed=1, repeats=8).stats()
        assert b["flops"] < a["flops"], (method, a, b)


def test_plan_checkpoint_round_trip(api, tmp_path):
    """A saved plan reloads for the same network with the same path, slices
    and statistics (no new search); another network or a tampered file is
    refused."""
    from paper_2301_05451_gb300 import checkpoint
    C = api.Circuit(W.grid_u3cz(rows=5, cols=5, depth=8)[0])
    N = api.Network(C, "amplitude", 0, False, False, True)
    P = api.Plan(N, method="partition", seed=2, repeats=8, target_log2=10)
    f = tmp_path / "plan.json"
    checkpoint.save_plan(P, str(f))
    Q = checkpoint.load_plan(N, str(f))
    assert Q.path() == P.path() and Q.stats() == P.stats()
    other = api.Network(C, "amplitude", 0, False, True, False)
    with pytest.raises(ValueError):
        checkpoint.load_plan(other, str(f))
    import json
    doc = json.loads(f.read_text())
    doc["stats"]["flops"] *= 2
    f.write_text(json.dumps(doc))
    with pytest.raises(ValueError):
        checkpoint.load_plan(N, str(f))



def test_plan_from_path_refuses_corrupt_paths(api):
    """A caller's path is checked on the host: wrong length, an id used twice,
    an id not yet made, a bad sliced index -- each ERR_ARG, no plan."""
    import ctypes
    from paper_2301_05451_gb300 import _abi as A
    C = api.Circuit(W.hea6()[0])
    N = api.Network(C, "expval", 0)
    path, _ = api.Plan(N).path()
    L = A.lib()
    h = ctypes.c_void_p()

    def call(p, sl=()):
        flat = [x for pair in p for x in pair]
        return L.tdq_plan_from_path(N.h, A.int_array(flat or [0]), len(p), A.int_array(list(sl) or [0]), len(sl),
                                    ctypes.byref(h))

    assert call(path) == A.TDQ_OK
    L.tdq_plan_destroy(h)
    assert call(path[:-1]) == A.TDQ_ERR_ARG
    bad = list(path)
    bad[-1] = (bad[0][0], bad[-1][1])  # a tensor consumed twice
    assert call(bad) == A.TDQ_ERR_ARG
    ahead = list(path)
    ahead[0] = (N.n_tensors + 3, ahead[0][1])  # a result that does not exist yet
    assert call(ahead) == A.TDQ_ERR_ARG
    assert call(path, [N.n_indices]) == A.TDQ_ERR_ARG


@pytest.mark.parametrize("hyper", [False, True])
def test_plan_features_host_only(api, hyper):
    """tdq_plan_features needs no device: one unit for the fused subtree launch
    and one per large step, finite features, a one-hot kernel class per unit,
    log2 of the batch entries (plus the step's hyperedge bits) at least log2 B."""
    import math
    C = api.Circuit(W.grid_u3cz()[0])
    N = api.Network(C, "amplitude", 0, False, not hyper, hyper)
    P = api.Plan(N, method="partition", seed=1, repeats=8, target_log2=0)
    assert P.stats()["max_log2_width"] > 11  # some steps too large for the fused subtree launch
    feats, repeats = P.features(batch=4)
    assert len(feats) >= 2 and repeats == 1
    for f in feats:
        assert all(math.isfinite(x) for x in f)
        assert sum(f[0:6]) == 1.0
        assert f[9] >= math.log2(4) - 1e-6


def test_best_plan_takes_the_cheapest_finder(api):
    for spec, kind, lc in ((W.grid_brickwork()[0], "expval", True), (W.grid_u3cz(depth=10)[0], "amplitude", False)):
        N = api.Network(api.Circuit(spec), kind, 0, lc, False, True)
        best = api.best_plan(N, target_log2=18, seed=2, repeats=4).stats()
        for method in ("greedy", "random_greedy", "partition"):
            for rs in (False, True):
                st = api.Plan(N, method=method, seed=2, temperature=0.3, target_log2=18, repeats=4,
                              rank_simplify=rs).stats()
                assert best["flops"] <= st["flops"], (method, rs, best, st)
