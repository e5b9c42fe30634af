"""FP64 CPU oracle for the circuit tensor-network hot path.

TEST INFRASTRUCTURE ONLY: imported by the tests, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline leg; never by the product package, which
shares no code with it.  The arithmetic lives in ``tdq_oracle.c`` (plain loop
code, double precision); this module marshals circuit descriptions (duck-typed:
``n_qubits``, ``gates`` with ``name/qubits/angles``, ``terms``, ``n_groups``,
``amplitudes``) into it, and adds the three pieces that are clearer in Python:

* the light cone of an observable: the gates in the backward causal cone of the
  measured qubits; every other gate meets its own conjugate in
  ``<0|U^dagger O U|0>`` and cancels (U U^dagger = 1, Sec. 3.2.1 network);
* central finite differences (Sec. 4.2, Eq. 10, second line, made central);
* the FP64 multilayer perceptron used to check the learned cost model.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tdq_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

KIND = {"H": 0, "X": 1, "Y": 2, "Z": 3, "RX": 4, "RY": 5, "RZ": 6, "U3": 7,
        "CNOT": 8, "CZ": 9, "RZZ": 10,
        # projectors |0><0| and |1><1| on one wire: fixing that wire's index to
        # one value, i.e. one slice of it (Sec. 3.2.3); not unitary
        "P0": 11, "P1": 12}

_lib = None


def build(force=False):
    """Compile tdq_oracle.c with gcc (OpenMP) into liboracle.so beside it."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                           "-Wall", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C")
        ci, cl = ctypes.c_int, ctypes.c_int64
        L.oracle_gate_matrix.argtypes = [ci, f64p, f64p]
        L.oracle_sv_state.argtypes = [ci, ci, i32p, i32p, i32p, f64p, f64p]
        vp = ctypes.c_void_p  # an initial state (float64 pairs) or NULL
        L.oracle_sv_state_from.argtypes = [ci, ci, i32p, i32p, i32p, f64p, vp, f64p]
        L.oracle_expval_from.argtypes = [ci, ci, i32p, i32p, i32p, ci, f64p, vp, cl, ci, i64p, f64p, i32p,
                                         ci, f64p, ci]
        L.oracle_param_shift_from.argtypes = [ci, ci, i32p, i32p, i32p, f64p, vp, ci, i32p, i32p, ci,
                                              i64p, f64p, i32p, ci, f64p, f64p, ci]
        L.oracle_expval.argtypes = [ci, ci, i32p, i32p, i32p, ci, f64p, ci, i64p, f64p, i32p,
                                    ci, f64p, ci]
        L.oracle_amplitude.argtypes = [ci, ci, i32p, i32p, i32p, ci, f64p, ci, u8p, f64p, ci]
        L.oracle_param_shift.argtypes = [ci, ci, i32p, i32p, i32p, f64p, ci, i32p, i32p, ci,
                                         i64p, f64p, i32p, ci, f64p, f64p, ci]
        L.oracle_tn_amplitude.argtypes = [ci, ci, i32p, i32p, i32p, f64p, u8p, f64p, cl,
                                          ctypes.POINTER(ctypes.c_int), ci]
        L.oracle_tn_expval.argtypes = [ci, ci, i32p, i32p, i32p, f64p, cl, f64p, cl,
                                       ctypes.POINTER(ctypes.c_int), ci]
        L.oracle_max_threads.restype = ci
        _lib = L
    return _lib


def max_threads():
    return int(lib().oracle_max_threads())


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with code %d" % (what, rc))


def _gate_arrays(circuit):
    G = len(circuit.gates)
    kind = np.zeros(G, np.int32)
    q0 = np.zeros(G, np.int32)
    q1 = np.full(G, -1, np.int32)
    for g, gate in enumerate(circuit.gates):
        kind[g] = KIND[gate.name]
        q0[g] = gate.qubits[0]
        if len(gate.qubits) > 1:
            q1[g] = gate.qubits[1]
    return G, kind, q0, q1


def _term_arrays(circuit):
    T = len(circuit.terms)
    zmask = np.zeros(max(T, 1), np.int64)
    coeff = np.zeros(max(T, 1), np.float64)
    group = np.zeros(max(T, 1), np.int32)
    for t, (qs, c, g) in enumerate(circuit.terms):
        m = 0
        for q in qs:
            m ^= 1 << q
        zmask[t], coeff[t], group[t] = m, c, g
    return T, zmask, coeff, group


def gate_matrix(name, angles=()):
    a = np.zeros(3, np.float64)
    a[:len(angles)] = angles
    out = np.zeros(32, np.float64)
    d = lib().oracle_gate_matrix(KIND[name], a, out)
    if d < 0:
        raise ValueError(name)
    return (out[0:2 * d * d:2] + 1j * out[1:2 * d * d:2]).reshape(d, d)


def _vp(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _init_pairs(init, n, rows=None):
    """Initial state(s) as contiguous (re, im) float64 pairs: [2^n] shared by
    every row, or [rows][2^n]; None stays None (|0...0>)."""
    if init is None:
        return None, 0
    a = np.asarray(init, np.complex128)
    if a.ndim == 1:
        assert a.shape[0] == 1 << n
        return np.ascontiguousarray(np.stack([a.real, a.imag], -1)), 0
    assert a.shape[-1] == 1 << n and (rows is None or a.shape[0] == rows)
    return np.ascontiguousarray(np.stack([a.real, a.imag], -1)), 1 << n


def statevector(circuit, angles_row, init=None):
    """|psi> = U|psi0> as complex128 [2^n] (qubit 0 = most significant bit);
    psi0 = init ([2^n] complex), default |0...0>."""
    n = circuit.n_qubits
    G, kind, q0, q1 = _gate_arrays(circuit)
    ang = np.ascontiguousarray(np.asarray(angles_row, np.float64).reshape(G, 3))
    out = np.zeros(2 << n, np.float64)
    if init is None:
        _check(lib().oracle_sv_state(n, G, kind, q0, q1, ang, out), "sv_state")
    else:
        p0, _ = _init_pairs(init, n)
        _check(lib().oracle_sv_state_from(n, G, kind, q0, q1, ang, _vp(p0), out), "sv_state")
    return out[0::2] + 1j * out[1::2]


def probabilities(circuit, angles_row, init=None):
    """|<x|U|psi0>|^2 for every basis state x, [2^n] float64."""
    return np.abs(statevector(circuit, angles_row, init)) ** 2


def expvals(circuit, angles, nthreads=None, init=None):
    """Grouped expectation values [B][n_groups] for angles [B][G][3], from
    |0...0> or from init ([2^n] shared, or [B][2^n])."""
    n = circuit.n_qubits
    G, kind, q0, q1 = _gate_arrays(circuit)
    T, zmask, coeff, group = _term_arrays(circuit)
    ang = np.ascontiguousarray(np.asarray(angles, np.float64).reshape(-1, G, 3))
    B = ang.shape[0]
    out = np.zeros((B, max(circuit.n_groups, 1)), np.float64)
    if init is None:
        _check(lib().oracle_expval(n, G, kind, q0, q1, B, ang, T, zmask, coeff, group,
                                   max(circuit.n_groups, 1), out, nthreads or max_threads()),
               "expval")
    else:
        p0, stride = _init_pairs(init, n, B)
        _check(lib().oracle_expval_from(n, G, kind, q0, q1, B, ang, _vp(p0), stride, T, zmask, coeff, group,
                                        max(circuit.n_groups, 1), out, nthreads or max_threads()),
               "expval")
    return out


def amplitudes(circuit, angles, nthreads=None):
    """Amplitudes <x_a|U|0> [B][A] (complex128) for angles [B][G][3]."""
    n = circuit.n_qubits
    G, kind, q0, q1 = _gate_arrays(circuit)
    ang = np.ascontiguousarray(np.asarray(angles, np.float64).reshape(-1, G, 3))
    B = ang.shape[0]
    bits = np.ascontiguousarray(np.asarray(circuit.amplitudes, np.uint8).reshape(-1, n))
    A = bits.shape[0]
    out = np.zeros((B, A, 2), np.float64)
    _check(lib().oracle_amplitude(n, G, kind, q0, q1, B, ang, A, bits, out,
                                  nthreads or max_threads()), "amplitude")
    return out[..., 0] + 1j * out[..., 1]


def angle_grads_param_shift(circuit, angles_row, weights=None, which=None, nthreads=None, init=None):
    """dF/d(angle) by the parameter-shift rule for F = sum_g weights[g] f_g,
    from |0...0> or the initial state init ([2^n]).  Returns [G][3] (zeros
    for angles not requested)."""
    n = circuit.n_qubits
    G, kind, q0, q1 = _gate_arrays(circuit)
    T, zmask, coeff, group = _term_arrays(circuit)
    ng = max(circuit.n_groups, 1)
    w = np.ones(ng, np.float64) if weights is None else np.asarray(weights, np.float64).reshape(ng)
    if which is None:
        which = [(g, i) for g, gate in enumerate(circuit.gates) for i in range(len(gate.angles))
                 if gate.angles[i][0] != "c"]
    wg = np.asarray([p[0] for p in which], np.int32)
    wa = np.asarray([p[1] for p in which], np.int32)
    ang = np.ascontiguousarray(np.asarray(angles_row, np.float64).reshape(G, 3))
    out = np.zeros(max(len(which), 1), np.float64)
    if len(which):
        p0, _ = _init_pairs(init, n)
        _check(lib().oracle_param_shift_from(n, G, kind, q0, q1, ang, _vp(p0), len(which), wg, wa, T, zmask,
                                             coeff, group, ng, np.ascontiguousarray(w), out,
                                             nthreads or max_threads()), "param_shift")
    res = np.zeros((G, 3), np.float64)
    for j, (g, i) in enumerate(which):
        res[g, i] = out[j]
    return res


def param_grads_from_angle_grads(circuit, angle_grads, n_params):
    """Chain rule from angle derivatives to parameter columns: every angle fed
    by ("p", j) adds its derivative to column j."""
    out = np.zeros(n_params, np.float64)
    for g, gate in enumerate(circuit.gates):
        for i, src in enumerate(gate.angles):
            if src[0] == "p":
                out[src[1]] += angle_grads[g, i]
    return out


def _angles_from(circuit, params_row, inputs_row):
    G = len(circuit.gates)
    a = np.zeros((G, 3), np.float64)
    for g, gate in enumerate(circuit.gates):
        for i, src in enumerate(gate.angles):
            if src[0] == "p":
                a[g, i] = params_row[src[1]]
            elif src[0] == "x":
                a[g, i] = inputs_row[src[1]]
            else:
                a[g, i] = src[1]
    return a


def param_grads_param_shift(circuit, params_row, inputs_row=None, weights=None, nthreads=None, init=None):
    """dF/dparams for one row via parameter shift on every parameterised angle."""
    params_row = np.asarray(params_row, np.float64)
    ag = angle_grads_param_shift(circuit, _angles_from(circuit, params_row, inputs_row),
                                 weights, nthreads=nthreads, init=init)
    return param_grads_from_angle_grads(circuit, ag, params_row.shape[0])


def param_grads_finite_difference(circuit, params_row, inputs_row=None, weights=None, h=1e-5,
                                  nthreads=None, init=None):
    """Central difference [F(p + h e_j) - F(p - h e_j)] / 2h in FP64."""
    params_row = np.asarray(params_row, np.float64)
    P = params_row.shape[0]
    ng = max(circuit.n_groups, 1)
    w = np.ones(ng) if weights is None else np.asarray(weights, np.float64).reshape(ng)
    rows = []
    for j in range(P):
        for sgn in (1.0, -1.0):
            p = params_row.copy()
            p[j] += sgn * h
            rows.append(_angles_from(circuit, p, inputs_row))
    f = expvals(circuit, np.stack(rows), nthreads, init=init) @ w
    return (f[0::2] - f[1::2]) / (2 * h)


class _Sliced:
    """The circuit with projectors P0 / P1 inserted (duck-typed like the
    circuit descriptions this module takes)."""

    def __init__(self, circuit, gates):
        self.n_qubits = circuit.n_qubits
        self.gates = gates
        self.terms = getattr(circuit, "terms", [])
        self.n_groups = getattr(circuit, "n_groups", 0)
        self.amplitudes = getattr(circuit, "amplitudes", [])


def sliced_amplitudes(circuit, angles_row, cuts, value, method="sv", nthreads=None):
    """Amplitudes <x_a|U|0> [A] of one slice (Sec. 3.2.3): the wires listed
    in cuts -- (qubit q, g), the wire of q right after gate g, g = -1 for
    its input wire -- each fixed to one value, bit i of `value` for cut i.
    Fixing a wire's index to v is a projector |v><v| on that wire; as
    sum_v |v><v| = 1, the slices of any set of cuts sum to the amplitude.
    angles_row [G][3] of the uncut circuit.  method "sv": the state vector;
    "tn": the loop-nest contraction in its linear order (the projectors are
    rank-2 tensors of the network like any one-qubit gate)."""
    from types import SimpleNamespace
    G = len(circuit.gates)
    ang = np.asarray(angles_row, np.float64).reshape(G, 3)
    at = {}
    for i, (q, g) in enumerate(cuts):
        at.setdefault(int(g), []).append((int(q), (int(value) >> i) & 1))
    gates, rows = [], []
    for q, v in at.get(-1, []):
        gates.append(SimpleNamespace(name="P%d" % v, qubits=(q,), angles=()))
        rows.append(np.zeros(3))
    for g in range(G):
        gates.append(circuit.gates[g])
        rows.append(ang[g])
        for q, v in at.get(g, []):
            gates.append(SimpleNamespace(name="P%d" % v, qubits=(q,), angles=()))
            rows.append(np.zeros(3))
    cut = _Sliced(circuit, gates)
    if method == "tn":
        return np.asarray([tn_amplitude(cut, np.asarray(rows), bits=b, order="linear")[0]
                           for b in circuit.amplitudes])
    return amplitudes(cut, np.asarray(rows)[None], nthreads=nthreads)[0]


def tn_amplitude(circuit, angles_row, bits=None, max_elems=1 << 28, order="greedy"):
    """<x|U|0> by contracting the amplitude network pairwise (loop nests).
    order "greedy": smallest result first; "linear": split block-diagonal
    two-qubit gates and fold tensors in (qubit, time) order.
    Returns (complex value, largest intermediate rank)."""
    n = circuit.n_qubits
    G, kind, q0, q1 = _gate_arrays(circuit)
    ang = np.ascontiguousarray(np.asarray(angles_row, np.float64).reshape(G, 3))
    b = np.ascontiguousarray(np.asarray(bits if bits is not None else circuit.amplitudes[0],
                                        np.uint8).reshape(n))
    out = np.zeros(2, np.float64)
    peak = ctypes.c_int(0)
    _check(lib().oracle_tn_amplitude(n, G, kind, q0, q1, ang, b, out, max_elems,
                                     ctypes.byref(peak), int(order == "linear")),
           "tn_amplitude")
    return complex(out[0], out[1]), peak.value


def tn_expval(circuit, angles_row, zqubits, max_elems=1 << 28, order="greedy"):
    """<0|U^dagger Z_zqubits U|0> by contracting ket, observable and conjugate
    bra networks pairwise.  Returns (complex value, largest intermediate rank)."""
    n = circuit.n_qubits
    G, kind, q0, q1 = _gate_arrays(circuit)
    ang = np.ascontiguousarray(np.asarray(angles_row, np.float64).reshape(G, 3))
    m = 0
    for q in zqubits:
        m ^= 1 << q
    out = np.zeros(2, np.float64)
    peak = ctypes.c_int(0)
    _check(lib().oracle_tn_expval(n, G, kind, q0, q1, ang, m, out, max_elems,
                                  ctypes.byref(peak), int(order == "linear")), "tn_expval")
    return complex(out[0], out[1]), peak.value


class _Gate:
    def __init__(self, name, qubits, angles):
        self.name, self.qubits, self.angles = name, tuple(qubits), tuple(angles)


class _Circuit:
    def __init__(self, n):
        self.n_qubits, self.gates, self.terms, self.n_groups, self.amplitudes = n, [], [], 0, []


def lightcone(circuit, zqubits):
    """Reduce <0|U^dagger Z U|0> to the backward causal cone of `zqubits`.

    Walk the gates from last to first keeping a gate iff it touches a qubit
    already in the cone (then all its qubits join).  Returns (reduced circuit
    with qubits renumbered in increasing order, kept gate indices, qubit map).
    """
    cone = set(zqubits)
    kept = []
    for g in range(len(circuit.gates) - 1, -1, -1):
        qs = circuit.gates[g].qubits
        if cone.intersection(qs):
            kept.append(g)
            cone.update(qs)
    kept.reverse()
    qmap = {q: i for i, q in enumerate(sorted(cone))}
    red = _Circuit(len(qmap))
    for g in kept:
        gate = circuit.gates[g]
        red.gates.append(_Gate(gate.name, [qmap[q] for q in gate.qubits], gate.angles))
    red.terms = [(tuple(qmap[q] for q in zqubits), 1.0, 0)]
    red.n_groups = 1
    return red, kept, qmap


# ------------------------------------------------------------------ FP64 MLP
def mlp_forward(params, X):
    """3-layer perceptron y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 in FP64.
    params = (W1 [H,F], b1 [H], W2 [H,H], b2 [H], W3 [1,H], b3 [1])."""
    W1, b1, W2, b2, W3, b3 = [np.asarray(p, np.float64) for p in params]
    X = np.asarray(X, np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + b3
    return y[:, 0], (X, z1, h1, z2, h2)


def mlp_loss_and_grads(params, X, t):
    """Mean squared error L = mean_i (y_i - t_i)^2 and dL/d(each parameter)."""
    W1, b1, W2, b2, W3, b3 = [np.asarray(p, np.float64) for p in params]
    y, (X, z1, h1, z2, h2) = mlp_forward(params, X)
    N = X.shape[0]
    r = y - np.asarray(t, np.float64)
    loss = float(np.mean(r * r))
    dy = (2.0 / N) * r[:, None]
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dh2 = dy @ W3
    dz2 = dh2 * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    return loss, (gW1, gb1, gW2, gb2, gW3, gb3)


def adam_step(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, Algorithm 1) in FP64; returns new lists."""
    out_p, out_m, out_v = [], [], []
    for p, g, mm, vv in zip(params, grads, m, v):
        mm = b1 * mm + (1 - b1) * g
        vv = b2 * vv + (1 - b2) * g * g
        mh = mm / (1 - b1 ** t)
        vh = vv / (1 - b2 ** t)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(mm)
        out_v.append(vv)
    return out_p, out_m, out_v
