"""Contraction paths and slicing on the host (Sec. 3.2.2-3.2.3), no device
work: every path finder returns a valid SSA path over all tensors, whose
FLOPs p(2q - 1) per step (Eq. 5) and widths -- recomputed here from the
network's index sets -- are the plan's statistics; slicing meets its width
target; the two-phase slicing-aware search never ends above the single
greedy slicing of the same trees; the hypergraph-partition finder beats the
greedy finders on deep grid networks."""
import ctypes

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
    for name, spec, kind, lc, split in [
            ("random6_expval", r6, "expval", False, False),
            ("random6_expval_split_cone", r6, "expval", True, True),
            ("random6_amp", r6, "amplitude", False, True),
            ("grid4x4", W.grid_u3cz(rows=4, cols=4, depth=6)[0], "amplitude", False, True),
            ("disconnected", single, "amplitude", False, False),
            ("two_tensors", bare, "amplitude", False, False)]:
        C = api.Circuit(spec)
        out.append((name, C, api.Network(C, kind, 0, lc, split)))
    return out


def _recount(N, path, sliced):
    """FLOPs over all slices, log2 width: from the index sets, sliced indices removed."""
    cut = set(sliced)
    T = [set(N.tensor(i)["idx"]) - cut for i in range(N.n_tensors)]
    used = set()
    flops = 0
    for s, (a, b) in enumerate(path):
        assert 0 <= a < len(T) and 0 <= b < len(T) and a != b, (s, a, b)
        assert a not in used and b not in used, (s, a, b)
        used |= {a, b}
        shared = len(T[a] & T[b])
        r = T[a] ^ T[b]
        flops += 2 ** len(r) * (2 ** (shared + 1) - 1)
        T.append(r)
    assert len(path) == N.n_tensors - 1
    assert set(range(len(T) - 1)) == used  # every tensor but the root consumed once
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
            if target:
                assert width <= target, (name, st)
            Q = api.Plan(N, path=path, sliced=sliced)
            assert Q.stats() == st


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
