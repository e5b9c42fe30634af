#!/usr/bin/env python
"""Benchmark of the batched value + gradient contraction.

Default workload: the largest value + gradient configuration, the 20-qubit
RY/RZ + CNOT-ladder ansatz (6 layers, 240 parameters, observable
sum_i Z_i Z_i+1) for a batch of 64 parameter sets, expectation value and
adjoint gradient of every row in one tdq_execute.  One step = one such
execute.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload ladder20|qnn12|hea6|ladder20_ps|grid7x7_amp|grid7x7_amp_rg|grid5x10_lightcone|
                              hea6_tree|hea_sv20|multi12|costmodel]

--impl reference times the FP64 CPU oracle (state vector + parameter shift) on
the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "circuit evals/s (value+grad, batched) vs plain form; % roofline at ≤1e-5 err"
UNIT = "circuit evals/s"


def workload(name):
    from paper_2301_05451_gb300 import workloads as W
    if name == "qnn12":
        spec, params, inputs = W.qnn12()
        return dict(spec=spec, params=params[0], inputs=inputs, B=256, grad="adjoint",
                    desc="qnn12: 12 qubits, RY encoding + 4 x (RX RY RZ + CZ chain), 144 params, "
                         "mean<Z_i>, batch 256, value + adjoint gradient")
    if name == "hea6":
        spec, params, _ = W.hea6()
        return dict(spec=spec, params=params, inputs=None, B=1, grad="adjoint",
                    desc="hea6: 6 qubits, 3 x (RY RZ + CNOT ring), <Z_0>, batch 1, value + adjoint gradient")
    if name == "ladder20":
        spec, params, _ = W.ladder20()
        return dict(spec=spec, params=params, inputs=None, B=64, grad="adjoint",
                    desc="ladder20: 20 qubits, 6 x (RY RZ + CNOT ladder), 240 params, sum Z_iZ_i+1, "
                         "batch 64 parameter sets, value + adjoint gradient")
    if name == "ladder20_ps":
        spec, params, _ = W.ladder20(batch=1)
        return dict(spec=spec, params=params, inputs=None, B=1, grad="param_shift",
                    desc="ladder20 parameter shift: 1 sample, 480 shifted circuits + 1 in one batch")
    if name in ("grid7x7_amp", "grid7x7_amp_rg"):
        spec, params, _ = W.grid_u3cz()
        if name == "grid7x7_amp":
            tree = dict(output="amplitude", hyper=True, method="partition", seed=1, repeats=256, target=14)
            how = ("the hypergraph-partition path (256 trials) of the diagonally reduced network (CZ wires as "
                   "hyperedges), two-phase slicing to 2^14 entries")
        else:
            tree = dict(output="amplitude", split=True, method="random_greedy", seed=1, repeats=16, target=17)
            how = "a random-greedy path of the split network (16 trials), sliced to 2^17 entries"
        return dict(spec=spec, params=params, inputs=None, B=1, grad="none", tree=tree, unit="amplitudes/s",
                    desc="%s: 49 qubits, 8 cycles of U3 + CZ, <0|U|0> along %s, slices batched, FP64 slice sum"
                         % (name, how))
    if name == "grid5x10_lightcone":
        spec, params, _ = W.grid_brickwork()
        return dict(spec=spec, params=params, inputs=None, B=1, grad="none", tree=dict(
            output="expval", lightcone=True, method="greedy"), unit="circuit evals/s",
            desc="grid5x10_lightcone: 50 qubits, 4 brickwork layers of RZZ + RX, <Z_25> on its light cone, "
                 "greedy path")
    if name == "hea_sv20":
        spec, params, _ = W.hea_sv()
        return dict(spec=spec, params=params, inputs=None, B=params.shape[0], grad="none", output="probs",
                    init="neel", unit="states/s",
                    desc="hea_sv20: state-vector mode, 20 qubits, 3 x (RY RZ + CNOT ring), 120 params, "
                         "16 parameter sets from the Neel state |0101...>; output: the 2^20 probabilities of "
                         "every row")
    if name == "multi12":
        r = np.random.default_rng(4000)
        specs, plist = [], []
        for i in range(12):  # uneven qubit counts, depths and batches
            n, layers, rows = int(r.integers(6, 13)), int(r.integers(2, 7)), int(r.choice([8, 16, 32, 64]))
            spec, p, _ = W.ladder20(seed=4000 + i, batch=rows, n=n, layers=layers)
            specs.append(spec)
            plist.append(p)
        return dict(spec=specs[0], params=plist[0], inputs=None, B=sum(p.shape[0] for p in plist), grad="adjoint",
                    multi=dict(specs=specs, params=plist),
                    desc="multi12: 12 circuits of 6-12 qubits and 2-6 layers of RY RZ + CNOT ladder, 8-64 "
                         "parameter sets each (%d rows), value + adjoint gradient, one persistent launch" % (
                             sum(p.shape[0] for p in plist)))
    if name == "hea6_tree":
        spec, params, _ = W.hea6()
        return dict(spec=spec, params=params, inputs=None, B=1, grad="none", tree=dict(
            output="expval", method="greedy"), unit="circuit evals/s",
            desc="hea6_tree: 6 qubits, <Z_0> along the greedy path, batch 1, one fused launch")
    raise SystemExit("unknown workload " + name)


def dist_env():
    from paper_2301_05451_gb300 import replicas
    return replicas.env()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to the system's temporary directory; the bench
        # line carries their summary
        self.path = os.path.join(os.environ.get("TDQ_CLOCKS_DIR", tempfile.gettempdir()),
                                 "clocks_bench_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def recorded_traffic(workload_name, kernel, launch=None):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, only
    while the sources that determine that kernel (the record's file list, else
    every library source) are the ones the capture was taken of."""
    from paper_2301_05451_gb300 import build
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(workload_name)
    except (OSError, ValueError):
        return None
    if not rec or not rec.get("kernel", "").startswith(kernel):
        return None
    files = rec.get("source_files")
    current = build.files_digest(files) if files else build._digest()
    if rec.get("source_digest") != current:
        return None
    if rec.get("launch") is not None and launch is not None and rec["launch"] != launch:
        return None  # the capture is of another launch configuration
    return rec["dram_bytes_per_launch"]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def neel_state(n):
    """|0101...> as complex64 [2^n] (qubit 0 = most significant bit)."""
    v = np.zeros(1 << n, np.complex64)
    v[int("01" * (n // 2) + "0" * (n % 2), 2)] = 1
    return v


def oracle_rows_per_s(wl, budget_s=10.0, max_rows=None, nthreads=None):
    """Oracle rows of the workload per second, on a sample bounded by budget_s:
    value + parameter-shift gradient, or (state-vector workloads) the
    probabilities.  A gradient row is 1 + 2 A state-vector evaluations (A =
    the row's parameterised angles); the sample runs the value and the shifted
    evaluations in chunks of angles and stops between chunks once budget_s has
    passed, so a partly done row counts by the evaluations it finished.
    Returns (rows/s, rows done, seconds, threads)."""
    import oracle
    from paper_2301_05451_gb300 import workloads as W
    spec, params, inputs, B = wl["spec"], wl["params"], wl["inputs"], wl["B"]
    params2 = params if params.ndim == 2 else params[None, :]
    init = neel_state(spec.n_qubits).astype(np.complex128) if wl.get("init") == "neel" else None
    multi = wl.get("multi")
    flat = None if multi is None else [(sp, p) for sp, pl in zip(multi["specs"], multi["params"]) for p in pl]
    threads = nthreads or oracle.max_threads()
    t0 = time.perf_counter()
    rows, b = 0.0, 0
    while True:
        sp = spec
        if flat is not None:  # every circuit's rows in turn
            sp, prow = flat[b % len(flat)]
        else:
            prow = params2[b % B] if params2.shape[0] > 1 else params2[0]
        x = None if inputs is None else inputs[b % B]
        ang = W.resolve_angles(sp, prow[None, :], None if x is None else x[None, :], batch=1)
        if wl.get("output") in ("state", "probs"):
            oracle.probabilities(sp, ang[0], init=init)
            rows += 1
        else:
            which = [(g, i) for g, gate in enumerate(sp.gates) for i in range(len(gate.angles))
                     if gate.angles[i][0] != "c"]
            per_row = 1 + 2 * len(which)
            oracle.expvals(sp, ang, nthreads=threads)
            done = 1
            chunk = max(1, threads // 2)  # 2 x chunk shifted evaluations: one round of the threads
            for c0 in range(0, len(which), chunk):
                if time.perf_counter() - t0 >= budget_s:
                    break
                oracle.angle_grads_param_shift(sp, ang[0], which=which[c0:c0 + chunk], nthreads=threads)
                done += 2 * len(which[c0:c0 + chunk])
            rows += done / per_row
        b += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_rows and rows >= max_rows):
            break
    return rows / el, rows, el, threads


def oracle_tree_units_per_s(wl, budget_s=10.0, nthreads=None):
    """The oracle on a tree workload (values only), on a sample bounded by
    budget_s: expectations by the state vector (on the observable's light cone
    when the workload uses it), amplitudes by the oracle's loop-nest
    contraction in its linear order (all host threads; it takes no thread
    count).  Returns (units/s, units, seconds, threads, what)."""
    import oracle
    from paper_2301_05451_gb300 import workloads as W
    spec, params, tree = wl["spec"], wl["params"], wl["tree"]
    ang = W.resolve_angles(spec, params)
    t0 = time.perf_counter()
    units = 0
    while True:
        if tree["output"] == "amplitude":
            oracle.tn_amplitude(spec, ang[0], order="linear")
            what, threads = "FP64 loop-nest contraction of the amplitude network, linear order", oracle.max_threads()
        else:
            z = list(spec.terms[0][0])
            if tree.get("lightcone"):
                red, kept, _ = oracle.lightcone(spec, z)
                oracle.expvals(red, ang[:, kept, :], nthreads=nthreads)
                what = "FP64 state vector on the observable's light cone"
            else:
                oracle.expvals(spec, ang, nthreads=nthreads)
                what = "FP64 state vector"
            threads = nthreads or oracle.max_threads()
        units += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return units / el, units, el, threads, what


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    # each step: a bounded sample of rows of the same workload
    for _ in range(args.warmup):
        oracle_rows_per_s(wl, budget_s=0.0)
    times, rows_tot = [], 0
    for _ in range(args.steps):
        rps, rows, el, cores = oracle_rows_per_s(wl, budget_s=2.0)
        times.append(el)
        rows_tot += rows
    value = rows_tot / sum(times)
    sample = ("%.3f rows of the workload over %d steps of about 2 s (value + parameter-shift gradient per row, "
              "a row being 1 + 2 x angles state-vector evaluations; a partly done row counts by its "
              "evaluations)" % (rows_tot, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl["desc"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def plain_form(wl, max_rows=4):
    """The plain form of the same value + gradient on the same GPU: for each
    row and each observable term, the term's expectation network contracted
    along the greedy FLOP path with one launch per pairwise step, and its
    gradient by the reverse tree, also one launch per step (batch 1, rows
    looped, no fusion, no slicing batch).  Returns rows/s over `max_rows` rows."""
    import torch
    from paper_2301_05451_gb300 import api
    spec = wl["spec"]
    C = api.Circuit(spec)
    execs = []
    for t in range(len(spec.terms)):
        N = api.Network(C, "expval", t)
        execs.append(api.TreeExec(api.Plan(N, method="greedy"), 1, plain=True, grad="adjoint"))
    params = np.asarray(wl["params"], np.float32)
    inputs = wl["inputs"]
    rows = min(max_rows, wl["B"])
    dev_p = [torch.as_tensor(params if params.ndim == 1 else params[b]).cuda() for b in range(rows)]
    dev_x = [None if inputs is None else torch.as_tensor(inputs[b:b + 1]).cuda() for b in range(rows)]
    outs = [E.alloc_outputs() for E in execs]
    for E, (v, g) in zip(execs, outs):  # warm-up
        E.run(dev_p[0], dev_x[0], values=v, grads=g)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    launches = 0
    for b in range(rows):
        for E, (v, g) in zip(execs, outs):
            E.run(dev_p[b], dev_x[b], values=v, grads=g)
            launches += E.launches()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    return rows / el, rows, launches // rows


def plain_tree_form(N, device, budget_s=3.0, max_runs=50):
    """The plain form of a tree workload on the same GPU: the workload's
    network along the greedy FLOP path (sliced to 2^24 entries where wider),
    batch 1, one launch per pairwise step, no fused subtrees, no concurrent
    steps, no graph replay.  Returns (units/s, runs, launches per run)."""
    import torch
    from paper_2301_05451_gb300 import api
    P = api.Plan(N, method="greedy")
    if P.stats()["max_log2_width"] > 24:
        P = api.Plan(N, method="greedy", target_log2=24)
    E = api.TreeExec(P, 1, device=device.index, plain=True)
    spec = N.circuit.spec
    p = torch.rand(max(spec.n_params, 1), device=device) * (2 * np.pi)
    v, _ = E.alloc_outputs()
    E.run(p, values=v)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    runs = 0
    while runs < max_runs and time.perf_counter() - t0 < budget_s:
        E.run(p, values=v)
        runs += 1
        torch.cuda.synchronize()
    return runs / (time.perf_counter() - t0), runs, E.launches()


def unbatched_form(wl, device, max_rows=16):
    """The same compiled kernels called once per row (batch 1, rows looped,
    L2 not flushed): what batching the rows into one launch gains, apart
    from fusion.  Returns rows/s over max_rows rows."""
    import torch
    from paper_2301_05451_gb300 import api
    spec = wl["spec"]
    E1 = api.Exec(api.Circuit(spec), 1, output=wl.get("output", "expval"), grad=wl["grad"], device=device.index)
    if wl.get("init") == "neel":
        E1.set_initial_state(torch.as_tensor(neel_state(spec.n_qubits)).to(device))
    params = np.asarray(wl["params"], np.float32)
    inputs = wl["inputs"]
    rows = min(max_rows, wl["B"])
    dev_p = [torch.as_tensor(params if params.ndim == 1 else params[b]).to(device) for b in range(rows)]
    dev_x = [None if inputs is None else torch.as_tensor(inputs[b:b + 1]).to(device) for b in range(rows)]
    v, g = E1.alloc_outputs()
    for _ in range(2):
        E1.run(dev_p[0], dev_x[0], values=v, grads=g)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for b in range(rows):
        E1.run(dev_p[b], dev_x[b], values=v, grads=g)
    e1.record(st)
    torch.cuda.synchronize()
    return rows / (e0.elapsed_time(e1) / 1000.0), rows, E1.launches()


def run_costmodel(args):
    """Learned path cost model: train on ~20k per-launch timings of random
    20-50 qubit grid brickwork circuits, rank 64 candidates of 200 held-out
    circuits (every launch unit of every candidate in one inference launch),
    measure the learned and the FLOP-greedy choices (and all 64 candidates of
    20 circuits for the regret against the best)."""
    import torch
    from paper_2301_05451_gb300 import build
    build.build()
    from paper_2301_05451_gb300 import costmodel as cm
    t0 = time.perf_counter()
    X, t = cm.collect(args.cm_train_circuits, plans_per_circuit=8, seed=100, reps=2)
    t_collect = time.perf_counter() - t0
    M = cm.CostModel(12, 64, seed=11)
    t0 = time.perf_counter()
    losses = M.fit(X, t, epochs=2000, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    plan_lists = []
    t0 = time.perf_counter()
    for c in range(args.cm_heldout):
        spec, _, _ = cm.training_circuit(50000 + c)
        _, _, plans = cm.candidates(spec, 64, 50000 + c)
        plan_lists.append(plans)
    t_cand = time.perf_counter() - t0
    t0 = time.perf_counter()
    pred = cm.rank(M, plan_lists)
    t_rank = time.perf_counter() - t0
    ratios, regrets = [], []
    for ci, (plans, pr) in enumerate(zip(plan_lists, pred)):
        il, iflop = int(np.argmin(pr)), cm.flops_choice(plans)
        tl = cm.measure(plans[il], reps=3)[0]
        tf = tl if iflop == il else cm.measure(plans[iflop], reps=3)[0]
        ratios.append(tf / tl)
        if ci < args.cm_full_measure:
            meas = [cm.measure(P, reps=3)[0] for P in plans]
            regrets.append(tl / min(meas) - 1.0)
    gm = float(np.exp(np.mean(np.log(ratios))))
    line = {"metric": "learned path ranking: geomean measured speedup of the chosen plan over the greedy FLOP choice",
            "value": gm, "unit": "x", "n_gpus": 1, "steps": args.cm_heldout, "warmup": 0,
            "ms_per_step": 1000.0 * t_rank / max(1, args.cm_heldout), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "costmodel: MLP 12-64-64-1 on %d launch timings of %d random grid brickwork "
                                   "circuits (20-50 qubits); %d held-out circuits x 64 candidates" % (
                                       len(t), args.cm_train_circuits, args.cm_heldout)},
            "train_rows": int(len(t)), "train_loss_first_last": [float(losses[0]), float(losses[-1])],
            "rank_time_s": t_rank, "candidate_search_s": t_cand, "collect_s": t_collect, "train_s": t_train,
            "regret_vs_best_mean": float(np.mean(regrets)) if regrets else None,
            "regret_vs_best_circuits": len(regrets),
            "speedup_vs_flops_min_max": [float(min(ratios)), float(max(ratios))]}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ladder20")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain", action="store_true", help="tree workloads: one launch per pairwise step")
    ap.add_argument("--autotune", action="store_true",
                    help="sweep and multi-circuit workloads: pick the launch configuration by timing candidates")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-form comparison")
    ap.add_argument("--rank-simplify", action="store_true",
                    help="tree workloads: rank simplification before the path search")
    ap.add_argument("--target-log2", type=int, default=None,
                    help="tree workloads: slice to at most 2^N entries per tensor (default: the workload's)")
    ap.add_argument("--interpret", action="store_true",
                    help="state sweep: generic kernels instead of kernels specialised to the circuit")
    ap.add_argument("--subtree-log2", type=int, default=0,
                    help="tree workloads: steps whose tensors all have at most 2^N entries run inside subtree CTAs "
                         "(0 = the library default)")
    ap.add_argument("--tc-min-log2", type=int, default=0,
                    help="tree workloads: steps below 2^N complex multiply-adds stay off the tensor cores "
                         "(0 = the library default)")
    ap.add_argument("--fwd-bits", type=int, default=0, help="state sweep: register bits per forward pass (0 = default: 2 whole-state, 4 tiled)")
    ap.add_argument("--rev-bits", type=int, default=0, help="state sweep: register bits per reverse pass (0 = default: 2 whole-state, 4 tiled)")
    ap.add_argument("--cm-train-circuits", type=int, default=400)
    ap.add_argument("--cm-heldout", type=int, default=200)
    ap.add_argument("--cm-full-measure", type=int, default=20)
    args = ap.parse_args()
    if args.workload == "costmodel":
        return run_costmodel(args)
    wl = workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, wl)

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2301_05451_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if dist is not None:
        dist.barrier()
    from paper_2301_05451_gb300 import api

    spec, B = wl["spec"], wl["B"]
    C = api.Circuit(spec)
    tree = wl.get("tree")
    multi = wl.get("multi")
    Pl = None
    if tree is not None:
        N = api.Network(C, tree["output"], 0, tree.get("lightcone", False), tree.get("split", False),
                        tree.get("hyper", False))
        rs = bool(tree.get("rank_simplify", False)) or args.rank_simplify
        if args.target_log2 is not None:
            tree["target"] = args.target_log2
        Pl = api.Plan(N, method=tree.get("method", "greedy"), seed=tree.get("seed", 0), temperature=0.3,
                      target_log2=tree.get("target", 0), repeats=tree.get("repeats", 1), rank_simplify=rs)
        pst = Pl.stats()
        wl["plan"] = {"method": tree.get("method", "greedy"), "hyper": bool(tree.get("hyper", False)),
                      "rank_simplify": rs,
                      "flops": pst["flops"], "n_sliced": pst["n_sliced"],
                      "max_log2_width": pst["max_log2_width"], "n_steps": pst["n_steps"]}

    def build_exec(autotune):
        if multi is not None:
            return api.MultiExec([api.Circuit(s) for s in multi["specs"]], [p.shape[0] for p in multi["params"]],
                                 grad=wl["grad"], device=local, autotune=autotune)
        if tree is not None:
            te = api.TreeExec(Pl, B, device=local, plain=args.plain, subtree_log2=args.subtree_log2,
                              tc_min_log2=args.tc_min_log2)
            if world > 1:  # the plan's slices shared out over the ranks, one FP64 all-reduce
                from paper_2301_05451_gb300 import shard
                return shard.ShardedTreeExec(te, 1 << Pl.stats()["n_sliced"], dist)
            return te
        ex = api.Exec(C, B, output=wl.get("output", "expval"), grad=wl["grad"], device=local,
                      interpret=args.interpret, fwd_reg_bits=args.fwd_bits, rev_reg_bits=args.rev_bits,
                      autotune=autotune, record_timings=True)
        if wl.get("init") == "neel":
            ex.set_initial_state(torch.as_tensor(neel_state(spec.n_qubits)).to(torch.device("cuda", local)))
        return ex

    E = build_exec(args.autotune)
    dev = torch.device("cuda", local)
    if multi is not None:
        params = E.pack(multi["params"])
    else:
        params = torch.as_tensor(wl["params"], dtype=torch.float32).to(dev).contiguous()
    inputs = None if wl["inputs"] is None else torch.as_tensor(wl["inputs"]).to(dev).contiguous()
    values, grads = E.alloc_outputs()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    for _ in range(max(args.warmup, 3)):
        E.run(params, inputs, values=values, grads=grads)
    torch.cuda.synchronize()
    E.status()
    launches_per_step = E.launches()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    # tiled sweeps: the library's events around every tile-pass launch of each
    # timed step (read after the step; the step itself is timed by its own events)
    tiled = tree is None and multi is None and E.work()[2] == 1
    unit_ms = []
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            E.run(params, inputs, values=values, grads=grads)
            ends[i].record(stream)
            if tiled:
                unit_ms.append(E.timings())
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    E.status()
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    from paper_2301_05451_gb300 import replicas
    t_ms = replicas.max_over_ranks(sum(per), dist, dev)
    # replicas: every rank runs the whole workload (weak scaling); a sliced
    # tree plan on several ranks: the ranks share one workload's slices
    # (strong scaling), so the job completes B units per step
    strong = tree is not None and world > 1
    rows_total = B * args.steps * (1 if strong else world)
    value = rows_total / (t_ms / 1000.0)

    # end to end through the public API, one stream, nothing overlapped: every
    # step copies its inputs from pinned host memory, executes, and reads its
    # results (values and gradients) back to pinned host memory; each step is
    # timed by its own events and L2 is flushed between steps, outside them,
    # as in the device-timed loop.
    hp = params.cpu().pin_memory()
    hx = None if inputs is None else inputs.cpu().pin_memory()
    dp, dx = torch.empty_like(params), (None if inputs is None else torch.empty_like(inputs))
    hv = torch.empty(values.shape, dtype=values.dtype).pin_memory()
    hg = None if grads is None else torch.empty(grads.shape, dtype=grads.dtype).pin_memory()
    for _ in range(2):  # warm the copies (and any graph capture of the new pointers)
        E.run(dp, dx, values=values, grads=grads)
    torch.cuda.synchronize()
    es = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        es[i][0].record(stream)
        dp.copy_(hp, non_blocking=True)
        if hx is not None:
            dx.copy_(hx, non_blocking=True)
        E.run(dp, dx, values=values, grads=grads)
        hv.copy_(values, non_blocking=True)
        if hg is not None:
            hg.copy_(grads, non_blocking=True)
        es[i][1].record(stream)
    torch.cuda.synchronize()
    E.status()
    e2e_ms = replicas.max_over_ranks(sum(a.elapsed_time(b) for a, b in es), dist, dev)
    h2d = hp.numel() * 4 + (0 if hx is None else hx.numel() * 4)
    d2h = hv.numel() * 8 + (0 if hg is None else hg.numel() * 4)

    flops_row, bytes_row, kclass = E.work()
    peaks, src = measured_peaks()
    dur_s = statistics.mean(per) / 1000.0
    if kclass in (2, 3, 4):  # whole state in shared memory / tree steps: FP32 ALU bound
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = sm_count * 128 * 2 * mhz * 1e6 / 1e12
        ach = flops_row * B / dur_s / 1e12
        kern = ("k2_sweep_smem" if args.interpret else "tdq_k2_specialised") if kclass == 2 else "tree step kernels"
        if multi is not None:
            kern = "tdq_k2_multi"
        roof = {"bound": "alu", "kernel": kern, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": recorded_traffic(args.workload, kern, E.config() if tree is None else None),
                "peak_note": "FP32 SIMT %d SMs x 128 lanes x 2 flop x %.0f MHz (%s max clock)" % (
                    sm_count, mhz, src)}
    else:  # HBM-resident tiles: FP32 arithmetic and the HBM traffic model, the larger time floor binds
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = peaks.get("sm_max_mhz", 2070.0)
        alu_peak = sm_count * 128 * 2 * mhz * 1e6 / 1e12
        hbm_peak = peaks.get("hbm_gbs", 6800.0)
        ach_f = flops_row * B / dur_s / 1e12
        ach_b = bytes_row * B / dur_s / 1e9
        ach_f_step, ach_b_step = ach_f / alu_peak, ach_b / hbm_peak
        kern = "k1 tiled passes (whole step)" if args.interpret else "tdq_k1f_* / tdq_k1r_* (whole step)"
        alu = {"bound": "alu", "achieved": ach_f, "peak": alu_peak, "unit": "TFLOP/s", "frac": ach_f / alu_peak,
               "peak_note": "FP32 SIMT %d SMs x 128 lanes x 2 flop x %.0f MHz (%s max clock)" % (sm_count, mhz, src)}
        hbm = {"bound": "hbm", "achieved": ach_b, "peak": hbm_peak, "unit": "GB/s", "frac": ach_b / hbm_peak,
               "peak_note": "%s copy bandwidth" % src}
        first, second = (alu, hbm) if alu["frac"] >= hbm["frac"] else (hbm, alu)
        roof = dict(first, kernel=kern, traffic=None,
                    arithmetic_intensity_flop_per_byte=flops_row / max(bytes_row, 1.0),
                    ridge_flop_per_byte=alu_peak * 1e3 / hbm_peak, other=second)
        if unit_ms:
            # the dominant kernel family by live device time: forward tile
            # passes, the fused last pass, or the reverse tile passes
            work = E.launch_work()
            t_unit = np.mean(np.asarray(unit_ms), axis=0)  # ms per launch, over the timed steps
            names = {0: "tdq_k1f_* (forward tile passes)", 1: "tdq_k1f_<last> (last pass: observable + reverse)",
                     2: "tdq_k1r_* (reverse tile passes)"}
            share = {k: float(sum(t for t, w in zip(t_unit, work) if w[2] == k)) for k in (0, 1, 2)}
            dom = max(share, key=share.get)
            fl = sum(w[0] for w in work if w[2] == dom)
            by = sum(w[1] for w in work if w[2] == dom)
            tt = share[dom] / 1000.0
            launches = sum(1 for w in work if w[2] == dom)
            ach_f, ach_b = fl / tt / 1e12, by / tt / 1e9
            alu = dict(alu, achieved=ach_f, frac=ach_f / alu_peak)
            hbm = dict(hbm, achieved=ach_b, frac=ach_b / hbm_peak)
            first, second = (alu, hbm) if alu["frac"] >= hbm["frac"] else (hbm, alu)
            by_launch = by / max(launches, 1)
            roof = dict(first, kernel=names[dom],
                        traffic=None if args.interpret else recorded_traffic(args.workload, names[dom], E.config()),
                        algorithmic_bytes_per_launch=by_launch, launches_per_step=launches,
                        kernel_ms_per_step=share[dom], kernel_share_of_step=share[dom] / statistics.mean(per),
                        arithmetic_intensity_flop_per_byte=fl / max(by, 1.0),
                        ridge_flop_per_byte=alu_peak * 1e3 / hbm_peak, other=second,
                        per_kind_ms_per_step={names[k]: share[k] for k in share},
                        whole_step={"alu_frac": ach_f_step, "hbm_frac": ach_b_step})

    plain = None
    if rank == 0 and tree is None and multi is None and wl["grad"] == "adjoint" and not args.no_plain:
        pv, prows, plaunch = plain_form(wl)
        plain = {"value": pv, "unit": UNIT, "rows": prows, "launches_per_row": plaunch,
                 "form": "per observable term: greedy FLOP path, one launch per pairwise step forward and "
                         "per reverse step, batch 1, rows looped", "speedup": value / pv}
    if rank == 0 and tree is not None and not args.no_plain and not args.plain:
        pv, pruns, plaunch = plain_tree_form(N, dev)
        plain = {"value": pv, "unit": wl.get("unit", UNIT), "runs": pruns, "launches_per_run": plaunch,
                 "form": "greedy FLOP path of the same network (sliced to 2^24 where wider), batch 1, one launch "
                         "per pairwise step, no fused subtrees, no concurrent steps, no graph", "speedup": value / pv}
    unbatched = None
    if rank == 0 and tree is None and multi is None and B > 1 and not args.no_plain:
        ub, urows, ulaunch = unbatched_form(wl, dev)
        unbatched = {"value": ub, "unit": wl.get("unit", UNIT), "rows": urows, "launches_per_row": ulaunch,
                     "form": "the same kernels, batch 1, rows looped (one execute per row)",
                     "batched_speedup": value / ub}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and tree is not None:
        ups, units, el, cores, what = oracle_tree_units_per_s(wl, budget_s=10.0)
        cpu = {"value": ups, "unit": wl.get("unit", UNIT), "cores": cores, "kind": "oracle",
               "sample": "%d evaluations of the same workload in %.1f s (%s)" % (units, el, what)}
        if wl["tree"]["output"] != "amplitude":
            ups1, units1, el1, _, _ = oracle_tree_units_per_s(wl, budget_s=5.0, nthreads=1)
            cpu["single_thread"] = {"value": ups1, "cores": 1,
                                    "sample": "%d evaluations in %.1f s on one thread" % (units1, el1)}
    if rank == 0 and not args.no_cpu_baseline and tree is None:
        rps, rows, el, cores = oracle_rows_per_s(wl, budget_s=10.0)
        rps1, rows1, el1, _ = oracle_rows_per_s(wl, budget_s=5.0, nthreads=1)
        what = ("FP64 state vector from the initial state, probabilities" if wl.get("output") in ("state", "probs")
                else "FP64 state vector + parameter shift, OpenMP over shifted evaluations; a row is 1 + 2 x angles "
                     "state-vector evaluations, a partly done row counts by its evaluations")
        cpu = {"value": rps, "unit": wl.get("unit", UNIT), "cores": cores, "kind": "oracle",
               "sample": "%.3f rows of the same workload in %.1f s (%s)" % (rows, el, what),
               "single_thread": {"value": rps1, "cores": 1,
                                 "sample": "%.4f rows in %.1f s on one thread" % (rows1, el1)}}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": wl.get("unit", UNIT), "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                "scaling": "strong" if strong else "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": wl["desc"], "batch": B, "n_qubits": spec.n_qubits,
                           "gates": len(spec.gates), "params": spec.n_params,
                           "l2": "flushed between steps (256 MiB write)",
                           "parallelism": ("slices sharded over ranks, one FP64 all-reduce" if strong else
                                           "replicas" if world > 1 else "single"), **(
                               {"plan": wl["plan"]} if "plan" in wl else {}), **(
                               {"subtree_log2": args.subtree_log2, "tc_min_log2": args.tc_min_log2}
                               if tree is not None and (args.subtree_log2 or args.tc_min_log2) else {}), **(
                               {"launch": E.config(), "autotune": bool(args.autotune)} if tree is None else {})},
                "e2e": {"value": rows_total / (e2e_ms / 1000.0), "unit": wl.get("unit", UNIT),
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "streams": 1,
                        "l2": "flushed between steps, outside the timed region"},
                "gpu_launches": launches_per_step * args.steps,
                "roofline": roof, "cpu_baseline": cpu, "plain_form": plain, "unbatched": unbatched,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
