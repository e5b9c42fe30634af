"""Learned path cost model: rank candidate contraction plans by predicted GB300
time instead of FLOPs.

The paper ranks contraction orders by FLOPs p(2q-1) (Sec. 3.2.2, Eq. 5).  Here a
3-layer perceptron (K8, hand-written CUDA in ``csrc/mlp.cu``) is trained on the
engine's own per-launch timings (K9, ``tdq_exec_timings``) against the launch
features of a plan (``tdq_plan_features``: kernel class, sizes, batch, FLOPs,
bytes), predicts the log time of every launch of a candidate plan, and the
candidate with the least predicted total wins.  The candidate with the fewest
FLOPs is the fallback and the reference for regret.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _abi as A
from . import api
from . import workloads as W

N_FEATURES = 12


def _vp(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class CostModel:
    """The MLP on the GPU (tdq_costmodel_*), with the feature standardisation
    fitted on its training rows."""

    def __init__(self, n_features=N_FEATURES, hidden=64, seed=0, device=0):
        h = ctypes.c_void_p()
        A.call("tdq_costmodel_create", n_features, hidden, ctypes.c_uint64(seed), device, ctypes.byref(h))
        self.h = h
        self.F, self.H = n_features, hidden
        self.mean = np.zeros(n_features, np.float32)
        self.std = np.ones(n_features, np.float32)
        n = ctypes.c_int()
        A.call("tdq_costmodel_params", h, None, ctypes.byref(n), 0)
        self.n_params = n.value

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value and A._lib is not None:
            A.lib().tdq_costmodel_destroy(h)
            self.h = None

    # packed parameters <-> host
    def get_params(self):
        buf = (ctypes.c_float * self.n_params)()
        A.call("tdq_costmodel_params", self.h, buf, None, 0)
        return np.frombuffer(buf, dtype=np.float32).copy()

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        A.call("tdq_costmodel_params", self.h, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), None, 1)

    def unpack(self, flat):
        F, H = self.F, self.H
        o = 0
        W1 = flat[o:o + H * F].reshape(H, F); o += H * F
        b1 = flat[o:o + H]; o += H
        W2 = flat[o:o + H * H].reshape(H, H); o += H * H
        b2 = flat[o:o + H]; o += H
        W3 = flat[o:o + H].reshape(1, H); o += H
        b3 = flat[o:o + 1]
        return W1, b1, W2, b2, W3, b3

    def _norm(self, X):
        return torch.as_tensor((np.asarray(X, np.float32) - self.mean) / self.std).cuda().contiguous()

    def loss_grad(self, Xd, td):
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        g = torch.zeros(self.n_params, dtype=torch.float32, device="cuda")
        A.call("tdq_costmodel_loss_grad", self.h, _vp(Xd), _vp(td), Xd.shape[0], _vp(loss), _vp(g), _stream())
        return loss, g

    def adam_step(self, lr):
        A.call("tdq_costmodel_adam_step", self.h, ctypes.c_float(lr), _stream())

    def fit(self, X, t, epochs=800, lr=3e-3):
        X = np.asarray(X, np.float32)
        self.mean = X.mean(0)
        self.std = X.std(0) + 1e-3
        Xd = self._norm(X)
        td = torch.as_tensor(np.asarray(t, np.float32)).cuda().contiguous()
        losses = torch.zeros(epochs, dtype=torch.float32, device="cuda")
        A.call("tdq_costmodel_train", self.h, _vp(Xd), _vp(td), Xd.shape[0], epochs, ctypes.c_float(lr),
               _vp(losses), _stream())
        return losses.cpu().numpy()

    def predict(self, X):
        Xd = self._norm(X)
        y = torch.empty(Xd.shape[0], dtype=torch.float32, device="cuda")
        A.call("tdq_costmodel_predict", self.h, _vp(Xd), Xd.shape[0], _vp(y), _stream())
        return y.cpu().numpy()


# ---------------------------------------------------------------- circuits and plans
def training_circuit(seed):
    """A random grid brickwork circuit of 20..50 qubits (U3 layers, CZ on edge
    class d mod 4), depth 4..8, amplitude <0|U|0>."""
    r = np.random.default_rng(seed)
    while True:
        rows, cols = int(r.integers(4, 8)), int(r.integers(4, 11))
        if 20 <= rows * cols <= 50:
            break
    depth = int(r.integers(4, 9))
    return W.grid_u3cz(seed=seed, rows=rows, cols=cols, depth=depth)


def candidates(spec, n, seed, split=True):
    """n candidate plans: greedy, random-greedy at several temperatures and
    (every fourth) single-trial hypergraph-partition trees, each with a
    slicing target drawn near the greedy width."""
    C = api.Circuit(spec)
    N = api.Network(C, "amplitude", 0, False, split)
    r = np.random.default_rng(seed)
    out = []
    base = api.Plan(N, method="greedy")
    width = base.stats()["max_log2_width"]
    cap = 24  # every candidate is sliced to at most 2^24 entries per tensor
    if width > cap:
        base = api.Plan(N, method="greedy", target_log2=cap)
    for i in range(n):
        if i == 0:
            P = base
        else:
            tgt = 0 if r.random() < 0.4 else int(max(8, width - r.integers(0, 5)))
            temp = float(r.choice([0.05, 0.2, 0.5, 1.0]))
            if i % 4 == 3:
                kw = dict(method="partition", seed=int(seed * 1000 + i), slice_trials=8, slice_final=0)
            else:
                kw = dict(method="random_greedy", seed=int(seed * 1000 + i), temperature=temp)
            P = api.Plan(N, target_log2=min(tgt, cap) if tgt else 0, **kw)
            if P.stats()["max_log2_width"] > cap:
                P = api.Plan(N, target_log2=cap, **kw)
        out.append(P)
    return C, N, out


def measure(plan, reps=5, warmup=2, record=False):
    """Median device time (ms) of tdq_execute for the plan; with record also
    the per-unit timings of the last run."""
    E = api.TreeExec(plan, 1, record_timings=record)
    spec = plan.network.circuit.spec
    p = torch.rand(max(spec.n_params, 1), device="cuda") * (2 * math.pi)
    values, _ = E.alloc_outputs()
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        E.run(p, values=values)
    times = []
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(st)
        E.run(p, values=values)
        e.record(st)
        torch.cuda.synchronize()
        times.append(s.elapsed_time(e))
    units = E.timings() if record else None
    return float(np.median(times)), units


def collect(n_circuits, plans_per_circuit=4, seed=0, reps=3):
    """Training rows: (features of each launch unit, log time in us)."""
    X, t = [], []
    for c in range(n_circuits):
        spec, _, _ = training_circuit(seed + c)
        _, _, plans = candidates(spec, plans_per_circuit, seed + c)
        for P in plans:
            feats, rep = P.features()
            per_unit = []
            for _ in range(reps):
                _, units = measure(P, reps=1, warmup=1, record=True)
                per_unit.append(units)
            med = np.median(np.asarray(per_unit), axis=0)
            for f, ms in zip(feats, med):
                X.append(f)
                t.append(math.log(max(ms, 1e-4) * 1000.0))
    return np.asarray(X, np.float32), np.asarray(t, np.float32)


def rank(model, plan_lists):
    """Predicted time (ms) of every candidate of every circuit, all launch
    units of all candidates in one batched inference launch."""
    rows, owner, reps = [], [], []
    for ci, plans in enumerate(plan_lists):
        for pi, P in enumerate(plans):
            feats, rep = P.features()
            rows.extend(feats)
            owner.extend([(ci, pi)] * len(feats))
            reps.append(((ci, pi), rep))
    y = model.predict(np.asarray(rows, np.float32))
    pred = {}
    for (key, v) in zip(owner, y):
        pred[key] = pred.get(key, 0.0) + math.exp(float(v)) / 1000.0
    for key, rep in reps:
        pred[key] *= rep
    return [[pred[(ci, pi)] for pi in range(len(plans))] for ci, plans in enumerate(plan_lists)]


def flops_choice(plans):
    return int(np.argmin([P.stats()["flops"] for P in plans]))
