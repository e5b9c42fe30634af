"""Python surface over the C ABI: circuit construction, compilation and
execution on torch-owned device memory.  Marshalling only; every step of the
contraction runs in the library's CUDA kernels."""
from __future__ import annotations

import ctypes

import torch

from . import _abi as A


class Circuit:
    """A circuit handle built through tdq_circuit_* from a CircuitSpec-like
    object (``n_qubits``, ``gates`` of ``name/qubits/angles``, ``terms``,
    ``amplitudes``)."""

    def __init__(self, spec):
        h = ctypes.c_void_p()
        A.call("tdq_circuit_create", spec.n_qubits, ctypes.byref(h))
        self.h = h
        self.spec = spec
        for g in spec.gates:
            src, fixed = [], []
            for a in g.angles:
                if a[0] == "p":
                    src.append(int(a[1])); fixed.append(0.0)
                elif a[0] == "x":
                    src.append(A.TDQ_INPUT(int(a[1]))); fixed.append(0.0)
                else:
                    src.append(A.TDQ_FIXED); fixed.append(float(a[1]))
            A.call("tdq_circuit_gate", self.h, A.GATES[g.name], A.int_array(g.qubits),
                   len(g.qubits), A.int_array(src), A.double_array(fixed))
        for qs, coeff, group in spec.terms:
            A.call("tdq_circuit_observable", self.h, A.int_array(qs), len(qs), float(coeff),
                   int(group))
        for bits in spec.amplitudes:
            arr = (ctypes.c_uint8 * spec.n_qubits)(*bits)
            A.call("tdq_circuit_amplitude", self.h, arr)
        vals = [ctypes.c_int() for _ in range(6)]
        A.call("tdq_circuit_info", self.h, *[ctypes.byref(v) for v in vals])
        (self.n_gates, self.n_params, self.n_inputs, self.n_groups, self.n_terms,
         self.n_amplitudes) = [v.value for v in vals]

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value and A._lib is not None:
            A.lib().tdq_circuit_destroy(h)
            self.h = None

    def specialised_source(self, grad="adjoint", tile_qubits=0):
        """CUDA source of the kernels specialised to this circuit
        (tdq_sweep_source): whole-state (tile_qubits = 0) or tiled."""
        g = {"none": A.TDQ_GRAD_NONE, "adjoint": A.TDQ_GRAD_ADJOINT}[grad]
        n = ctypes.c_size_t()
        A.call("tdq_sweep_source", self.h, g, int(tile_qubits), None, 0, ctypes.byref(n))
        buf = ctypes.create_string_buffer(n.value)
        A.call("tdq_sweep_source", self.h, g, int(tile_qubits), buf, n.value, ctypes.byref(n))
        return buf.value.decode()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class Exec:
    """A compiled contraction (tdq_compile_sweep) bound to a device."""

    def __init__(self, circuit: Circuit, batch, output="expval", grad="none", device=0,
                 max_smem_qubits=0, tile_qubits=0, interpret=False, fwd_reg_bits=0, rev_reg_bits=0, autotune=False,
                 record_timings=False):
        self.circuit = circuit
        self.batch = int(batch)
        self.output = {"expval": A.TDQ_OUT_EXPVAL, "amplitude": A.TDQ_OUT_AMPLITUDE,
                       "state": A.TDQ_OUT_STATE, "probs": A.TDQ_OUT_PROBS}[output]
        self.grad = {"none": A.TDQ_GRAD_NONE, "adjoint": A.TDQ_GRAD_ADJOINT,
                     "param_shift": A.TDQ_GRAD_PARAM_SHIFT}[grad]
        self._init = None
        self.device = torch.device("cuda", device)
        opts = A.CompileOpts(self.batch, self.output, self.grad, device, max_smem_qubits, tile_qubits, 0, 0,
                             int(bool(record_timings)), int(bool(interpret)), int(fwd_reg_bits), int(rev_reg_bits))
        opts.autotune = int(bool(autotune))
        h = ctypes.c_void_p()
        A.call("tdq_compile_sweep", circuit.h, ctypes.byref(opts), ctypes.byref(h))
        self.h = h
        c = circuit
        dim = 1 << c.spec.n_qubits
        self.n_out = {A.TDQ_OUT_EXPVAL: c.n_groups, A.TDQ_OUT_AMPLITUDE: 2 * c.n_amplitudes,
                      A.TDQ_OUT_STATE: 2 * dim, A.TDQ_OUT_PROBS: dim}[self.output]

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value and A._lib is not None:
            A.lib().tdq_exec_destroy(h)
            self.h = None

    def alloc_outputs(self):
        B, dev = self.batch, self.device
        values = torch.empty((B, self.n_out), dtype=torch.float64, device=dev)
        grads = None
        if self.grad != A.TDQ_GRAD_NONE:
            grads = torch.empty((B, max(self.circuit.n_params, 1)), dtype=torch.float32, device=dev)
        return values, grads

    def run(self, params, inputs=None, grad_weights=None, values=None, grads=None, stream=None):
        """Enqueue one execution.  params: float32 [B, P] or [P] (shared);
        inputs: float32 [B, F]; grad_weights: float64 [B, n_groups]."""
        if values is None:
            values, g2 = self.alloc_outputs()
            grads = grads if grads is not None else g2
        P = self.circuit.n_params
        stride = 0
        if params is not None:
            assert params.dtype == torch.float32 and params.is_cuda and params.is_contiguous()
            stride = 0 if params.dim() == 1 else params.shape[1]
        if inputs is not None:
            assert inputs.dtype == torch.float32 and inputs.is_cuda and inputs.is_contiguous()
        st = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        A.call("tdq_execute", self.h, _ptr(params), ctypes.c_int64(stride), _ptr(inputs),
               _ptr(values), _ptr(grad_weights), _ptr(grads), ctypes.c_void_p(st))
        return values, grads

    def status(self):
        A.call("tdq_exec_status", self.h)

    def set_initial_state(self, psi0):
        """Start every later run from psi0 (complex64 [2^n] shared by all rows, or
        [B, 2^n]) instead of |0...0>; None restores |0...0>.  The tensor is kept
        referenced here, as the library reads it at every run."""
        if psi0 is None:
            A.call("tdq_exec_set_initial_state", self.h, None, ctypes.c_int64(0))
            self._init = None
            return
        assert psi0.dtype == torch.complex64 and psi0.is_cuda and psi0.is_contiguous()
        dim = 1 << self.circuit.spec.n_qubits
        assert psi0.shape[-1] == dim
        stride = 0 if psi0.dim() == 1 else dim
        A.call("tdq_exec_set_initial_state", self.h, _ptr(psi0), ctypes.c_int64(stride))
        self._init = psi0

    def launches(self):
        return A.lib().tdq_exec_launches(self.h)

    def work(self):
        f, b, k = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        A.call("tdq_exec_work", self.h, ctypes.byref(f), ctypes.byref(b), ctypes.byref(k))
        return f.value, b.value, k.value

    def timings(self):
        """Device time (ms) of every tile-pass launch of the last run (tiled
        sweeps compiled with record_timings; tdq_exec_timings)."""
        n = ctypes.c_int()
        A.call("tdq_exec_timings", self.h, None, 0, ctypes.byref(n))
        buf = (ctypes.c_float * max(n.value, 1))()
        A.call("tdq_exec_timings", self.h, buf, n.value, ctypes.byref(n))
        return list(buf[:n.value])

    def launch_work(self):
        """Per tile-pass launch: (algorithmic FLOPs, modelled HBM bytes, kind
        0 forward / 1 fused last / 2 reverse) -- tdq_exec_launch_work."""
        n = ctypes.c_int()
        A.call("tdq_exec_launch_work", self.h, None, None, None, 0, ctypes.byref(n))
        f, b, k = (ctypes.c_double * n.value)(), (ctypes.c_double * n.value)(), (ctypes.c_int * n.value)()
        A.call("tdq_exec_launch_work", self.h, f, b, k, n.value, ctypes.byref(n))
        return list(zip(f[:], b[:], k[:]))

    def config(self):
        """Launch configuration (tdq_exec_config): threads, register bits, tile bits."""
        c = (ctypes.c_int * 4)()
        A.call("tdq_exec_config", self.h, c)
        return {"threads": c[0], "fwd_reg_bits": c[1], "rev_reg_bits": c[2], "tile_qubits": c[3]}


class CircuitFunction(torch.autograd.Function):
    """Expectation values of a compiled circuit as a differentiable torch op
    (the custom autograd function of Sec. 4.3).  Forward runs the value-only
    exec; backward runs the adjoint exec with the incoming gradient as the
    weights of the output groups (a vector-Jacobian product)."""

    @staticmethod
    def forward(ctx, params, inputs, fwd_exec, bwd_exec):
        values, _ = fwd_exec.run(params.contiguous(), inputs)
        ctx.save_for_backward(params, inputs if inputs is not None else torch.empty(0))
        ctx.has_inputs = inputs is not None
        ctx.bwd = bwd_exec
        return values

    @staticmethod
    def backward(ctx, grad_out):
        params, inputs = ctx.saved_tensors
        inputs = inputs if ctx.has_inputs else None
        _, grads = ctx.bwd.run(params.contiguous(), inputs,
                               grad_weights=grad_out.to(torch.float64).contiguous())
        g = grads[:, :params.shape[-1]]
        if params.dim() == 1:
            g = g.sum(0)
        return g.to(params.dtype), None, None, None


class QuantumLayer(torch.nn.Module):
    """Compiled circuit as an nn.Module with trainable parameters (shared by
    the batch) and per-sample input features (the quantum layer of Sec. 5.3.2)."""

    def __init__(self, spec, batch, init=None, device=0):
        super().__init__()
        self.circuit = Circuit(spec)
        self.fwd = Exec(self.circuit, batch, "expval", "none", device)
        self.bwd = Exec(self.circuit, batch, "expval", "adjoint", device)
        p = torch.zeros(self.circuit.n_params) if init is None else torch.as_tensor(init).reshape(-1)
        self.weight = torch.nn.Parameter(p.to(torch.float32).to(torch.device("cuda", device)))

    def forward(self, inputs=None):
        return CircuitFunction.apply(self.weight, inputs, self.fwd, self.bwd)


class Network:
    """Tensor network of one output of a circuit (tdq_network_build)."""

    def __init__(self, circuit: Circuit, output="expval", index=0, lightcone=False, split_2q=False, hyper=False):
        self.circuit = circuit
        self.output = {"expval": A.TDQ_OUT_EXPVAL, "amplitude": A.TDQ_OUT_AMPLITUDE}[output]
        h = ctypes.c_void_p()
        A.call("tdq_network_build", circuit.h,
               ctypes.byref(A.NetOpts(self.output, int(index), int(bool(lightcone)), int(bool(split_2q)),
                                      int(bool(hyper)))),
               ctypes.byref(h))
        self.h = h
        v = [ctypes.c_int() for _ in range(4)]
        A.call("tdq_network_info", h, *[ctypes.byref(x) for x in v])
        self.n_tensors, self.n_indices, self.n_qubits, self.n_gates = [x.value for x in v]

    def tensor(self, i):
        v = [ctypes.c_int() for _ in range(5)]
        idx = (ctypes.c_int * 8)()
        A.call("tdq_network_tensor", self.h, i, *[ctypes.byref(x) for x in v], idx)
        kind, gate, conj, bit, rank = [x.value for x in v]
        flip = ctypes.c_int()
        A.call("tdq_network_tensor_flips", self.h, i, ctypes.byref(flip))
        return dict(kind=kind, gate=gate, conj=conj, bit=bit, idx=list(idx[:rank]), flip=flip.value)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value and A._lib is not None:
            A.lib().tdq_network_destroy(h)
            self.h = None


class Plan:
    """Contraction path + sliced indices (tdq_plan_find / tdq_plan_from_path).

    method: "greedy", "random_greedy" or "partition" (recursive hypergraph
    bipartition).  slice_trials / slice_final: the two phases of the
    slicing-aware search (randomised slicings per trial tree, then on the
    winning tree); None means 128 / 1024 for "partition" and 0 / 0 (the single
    greedy slicing) otherwise.  rank_simplify: contract the pairs that do not
    widen the network first (Sec. 3.2.1), then search the tensors left."""

    def __init__(self, network: Network, method="greedy", seed=0, temperature=1.0, target_log2=0,
                 repeats=1, path=None, sliced=(), slice_trials=None, slice_final=None, rank_simplify=False):
        self.network = network
        h = ctypes.c_void_p()
        if path is not None:
            flat = [int(x) for pair in path for x in pair]
            A.call("tdq_plan_from_path", network.h, A.int_array(flat), len(path),
                   A.int_array(list(sliced)), len(sliced), ctypes.byref(h))
        else:
            m = {"greedy": A.TDQ_PATH_GREEDY, "random_greedy": A.TDQ_PATH_RANDOM_GREEDY,
                 "partition": A.TDQ_PATH_PARTITION}[method]
            part = m == A.TDQ_PATH_PARTITION
            st = (128 if part else 0) if slice_trials is None else int(slice_trials)
            sf = (1024 if part else 0) if slice_final is None else int(slice_final)
            A.call("tdq_plan_find", network.h,
                   ctypes.byref(A.PlanOpts(m, int(seed), float(temperature), int(target_log2), int(repeats), st, sf,
                                           int(bool(rank_simplify)))),
                   ctypes.byref(h))
        self.h = h

    def stats(self):
        st = A.Stats()
        A.call("tdq_plan_stats", self.h, ctypes.byref(st))
        return {f: getattr(st, f) for f, _ in A.Stats._fields_}

    N_FEATURES = 12

    def features(self, batch=1, workspace_bytes=0):
        """(features [units][12] as a list of rows, repeats) of the compiled plan."""
        n, rep = ctypes.c_int(), ctypes.c_int()
        A.call("tdq_plan_features", self.h, int(batch), ctypes.c_int64(workspace_bytes), None, 0,
               ctypes.byref(n), ctypes.byref(rep))
        buf = (ctypes.c_float * (max(n.value, 1) * 12))()
        A.call("tdq_plan_features", self.h, int(batch), ctypes.c_int64(workspace_bytes), buf, n.value,
               ctypes.byref(n), ctypes.byref(rep))
        return [list(buf[12 * i:12 * i + 12]) for i in range(n.value)], rep.value

    def path(self):
        st = self.stats()
        pairs = (ctypes.c_int * max(2 * st["n_steps"], 1))()
        sl = (ctypes.c_int * max(st["n_sliced"], 1))()
        A.call("tdq_plan_path", self.h, pairs, sl)
        return [(pairs[2 * i], pairs[2 * i + 1]) for i in range(st["n_steps"])], list(sl[:st["n_sliced"]])

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value and A._lib is not None:
            A.lib().tdq_plan_destroy(h)
            self.h = None


def best_plan(network: Network, target_log2=0, seed=0, repeats=16):
    """The plan with the fewest FLOPs over all slices (ties: fewer sliced
    indices) among the greedy, random-greedy and hypergraph-partition finders
    (Sec. 3.2.2), each with and without rank simplification (Sec. 3.2.1),
    with the same slicing target: greedy is often best on small light-cone
    networks, partition on deep ones, and the simplification helps some
    networks and not others."""
    cands = []
    for rs in (False, True):
        cands += [Plan(network, method="greedy", seed=seed, target_log2=target_log2, rank_simplify=rs),
                  Plan(network, method="random_greedy", seed=seed, temperature=0.3, target_log2=target_log2,
                       repeats=repeats, rank_simplify=rs),
                  Plan(network, method="partition", seed=seed, target_log2=target_log2, repeats=repeats,
                       rank_simplify=rs)]
    return min(cands, key=lambda p: (p.stats()["flops"], p.stats()["n_sliced"]))


class MultiExec:
    """Many circuits in one persistent launch (tdq_compile_multi): circuit c
    runs batches[c] rows; buffers are packed by circuit (see layout()).
    Expectation outputs; grad "none", "adjoint" or "param_shift"."""

    def __init__(self, circuits, batches, grad="none", device=0, autotune=False, fwd_reg_bits=0, rev_reg_bits=0):
        self.circuits = list(circuits)
        self.batches = [int(b) for b in batches]
        assert len(self.circuits) == len(self.batches) and self.circuits
        self.grad = {"none": A.TDQ_GRAD_NONE, "adjoint": A.TDQ_GRAD_ADJOINT,
                     "param_shift": A.TDQ_GRAD_PARAM_SHIFT}[grad]
        self.device = torch.device("cuda", device)
        opts = A.CompileOpts(1, A.TDQ_OUT_EXPVAL, self.grad, device, 0, 0, 0, 0, 0, 0, int(fwd_reg_bits),
                             int(rev_reg_bits))
        opts.autotune = int(bool(autotune))
        hs = (ctypes.c_void_p * len(self.circuits))(*[c.h.value for c in self.circuits])
        h = ctypes.c_void_p()
        A.call("tdq_compile_multi", hs, A.int_array(self.batches), len(self.circuits), ctypes.byref(opts),
               ctypes.byref(h))
        self.h = h
        self.offsets = [self._layout(c) for c in range(len(self.circuits))]
        cfg = (ctypes.c_int * 4)()
        A.call("tdq_multi_layout", self.h, 0, None, None, None, cfg)
        self.launch = {"threads": cfg[0], "fwd_reg_bits": cfg[1], "rev_reg_bits": cfg[2], "ctas": cfg[3]}
        last = len(self.circuits) - 1
        lc, lb = self.circuits[last], self.batches[last]
        self.n_params_total = self.offsets[last]["params"] + lb * lc.n_params
        self.n_inputs_total = self.offsets[last]["inputs"] + lb * lc.n_inputs
        self.n_values_total = self.offsets[last]["values"] + lb * lc.n_groups

    def _layout(self, c):
        p, x, v = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        A.call("tdq_multi_layout", self.h, int(c), ctypes.byref(p), ctypes.byref(x), ctypes.byref(v), None)
        return {"params": p.value, "inputs": x.value, "values": v.value}

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value and A._lib is not None:
            A.lib().tdq_exec_destroy(h)
            self.h = None

    def pack(self, per_circuit, what="params"):
        """Concatenate per-circuit float32 rows ([batch_c][width_c]) into one device tensor."""
        return torch.cat([torch.as_tensor(x, dtype=torch.float32).reshape(-1) for x in per_circuit]).to(
            self.device).contiguous()

    def unpack(self, packed, what="values"):
        """Split a packed values ([..][n_groups_c]) or grads ([..][P_c]) tensor per circuit."""
        out = []
        for c, (C, B) in enumerate(zip(self.circuits, self.batches)):
            w = C.n_groups if what == "values" else C.n_params
            o = self.offsets[c]["values" if what == "values" else "params"]
            out.append(packed[o:o + B * w].reshape(B, w))
        return out

    def alloc_outputs(self):
        values = torch.empty(max(self.n_values_total, 1), dtype=torch.float64, device=self.device)
        grads = None
        if self.grad != A.TDQ_GRAD_NONE:
            grads = torch.empty(max(self.n_params_total, 1), dtype=torch.float32, device=self.device)
        return values, grads

    def run(self, params, inputs=None, grad_weights=None, values=None, grads=None, stream=None):
        """Enqueue one launch over every circuit: params / inputs packed float32,
        grad_weights packed float64 like the values."""
        if values is None:
            values, g2 = self.alloc_outputs()
            grads = grads if grads is not None else g2
        for t in (params, inputs):
            if t is not None:
                assert t.dtype == torch.float32 and t.is_cuda and t.is_contiguous()
        st = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        A.call("tdq_execute", self.h, _ptr(params), ctypes.c_int64(0), _ptr(inputs), _ptr(values),
               _ptr(grad_weights), _ptr(grads), ctypes.c_void_p(st))
        return values, grads

    def status(self):
        A.call("tdq_exec_status", self.h)

    def launches(self):
        return A.lib().tdq_exec_launches(self.h)

    def work(self):
        f, b, k = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        A.call("tdq_exec_work", self.h, ctypes.byref(f), ctypes.byref(b), ctypes.byref(k))
        return f.value, b.value, k.value

    def config(self):
        """Launch configuration: threads per CTA, register bits, persistent CTAs."""
        return dict(self.launch)


class TreeExec(Exec):
    """A compiled tensor-network plan (tdq_plan_compile): values only."""

    def __init__(self, plan: Plan, batch, device=0, plain=False, workspace_bytes=0, record_timings=False,
                 grad="none", subtree_log2=0, tc_min_log2=0):
        self.plan = plan
        self.circuit = plan.network.circuit
        self.batch = int(batch)
        self.output = plan.network.output
        self.grad = {"none": A.TDQ_GRAD_NONE, "adjoint": A.TDQ_GRAD_ADJOINT}[grad]
        self.device = torch.device("cuda", device)
        opts = A.CompileOpts(self.batch, self.output, self.grad, device, 0, 0, int(bool(plain)),
                             int(workspace_bytes), int(bool(record_timings)), 0, 0, 0)
        opts.subtree_log2 = int(subtree_log2)
        opts.tc_min_log2 = int(tc_min_log2)
        h = ctypes.c_void_p()
        A.call("tdq_plan_compile", plan.h, ctypes.byref(opts), ctypes.byref(h))
        self.h = h
        self.n_out = 1 if self.output == A.TDQ_OUT_EXPVAL else 2

    def config(self):
        """Reverse-tree mode (0 none, 1 fused, 2 values kept, 3 recomputed), recompute
        regions, slices per launch, workspace entries per batch entry."""
        c = (ctypes.c_int * 4)()
        A.call("tdq_exec_config", self.h, c)
        return {"reverse": c[0], "regions": c[1], "chunk": c[2], "workspace_entries": c[3]}

    def set_slice_range(self, first, count):
        """Contract only slices [first, first + count) from the next run on
        (tdq_exec_set_slice_range): the outputs are then partial sums."""
        A.call("tdq_exec_set_slice_range", self.h, ctypes.c_int64(int(first)), ctypes.c_int64(int(count)))

    def timings(self):
        n = ctypes.c_int()
        A.call("tdq_exec_timings", self.h, None, 0, ctypes.byref(n))
        buf = (ctypes.c_float * max(n.value, 1))()
        A.call("tdq_exec_timings", self.h, buf, n.value, ctypes.byref(n))
        return list(buf[:n.value])
