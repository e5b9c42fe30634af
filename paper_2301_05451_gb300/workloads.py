"""Seeded synthetic circuits and inputs shared by the CUDA path and the oracle.

This module holds circuit *structure* (which gate acts on which qubits, which
parameter or input feeds which angle) and seeded random numbers only; it holds
none of the method's arithmetic (no gate matrices, no contraction).  Both the
CUDA path and the FP64 oracle receive what it returns.

Angle sources: ``("p", j)`` is parameter column j, ``("x", j)`` is input
feature j (angle encoding, Sec. 5.3, Eq. 11), ``("c", v)`` is the constant v.

The workloads follow the circuit families of the configurations: a 6-qubit
hardware-efficient ansatz, a 12-qubit angle-encoded QNN classifier, a 20-qubit
RY/RZ + CNOT-ladder ansatz, a 5x10 grid brickwork of RZZ + RX for a light-cone
expectation, a 7x7 grid of random U3 + CZ cycles for an amplitude, and random
brickwork circuits for the learned cost model.  Seeds are ``1000 + index``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ONE_QUBIT = ("H", "X", "Y", "Z", "RX", "RY", "RZ", "U3")
TWO_QUBIT = ("CNOT", "CZ", "RZZ")
N_ANGLES = {"H": 0, "X": 0, "Y": 0, "Z": 0, "RX": 1, "RY": 1, "RZ": 1, "U3": 3,
            "CNOT": 0, "CZ": 0, "RZZ": 1}


@dataclass
class Gate:
    name: str
    qubits: tuple
    angles: tuple = ()


@dataclass
class CircuitSpec:
    """A parameterised circuit with Z-product observables and/or amplitudes."""
    n_qubits: int
    gates: list = field(default_factory=list)
    # observable terms: (qubits carrying Z, coefficient, output group)
    terms: list = field(default_factory=list)
    n_groups: int = 0
    # amplitude bitstrings <x|U|0>, x[q] = value of qubit q
    amplitudes: list = field(default_factory=list)
    n_params: int = 0
    n_inputs: int = 0

    def add(self, name, qubits, *angles):
        assert name in N_ANGLES, name
        assert len(angles) == N_ANGLES[name], (name, angles)
        q = tuple(int(v) for v in qubits)
        assert len(q) == (2 if name in TWO_QUBIT else 1)
        self.gates.append(Gate(name, q, tuple(angles)))
        for a in angles:
            if a[0] == "p":
                self.n_params = max(self.n_params, a[1] + 1)
            elif a[0] == "x":
                self.n_inputs = max(self.n_inputs, a[1] + 1)

    def z(self, qubits, coeff=1.0, group=0):
        self.terms.append((tuple(int(q) for q in qubits), float(coeff), int(group)))
        self.n_groups = max(self.n_groups, group + 1)

    def amplitude(self, bits):
        bits = tuple(int(b) for b in bits)
        assert len(bits) == self.n_qubits
        self.amplitudes.append(bits)


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- C1
def hea6(seed=1000, n=6, layers=3):
    """6-qubit hardware-efficient ansatz: per layer RY(theta) RZ(phi) on every
    qubit, then a CNOT ring q -> q+1 mod n; observable <Z_0>; batch 1.
    Parameter column of (layer l, qubit q, k in {theta, phi}) is 2(l n + q) + k."""
    c = CircuitSpec(n)
    for l in range(layers):
        for q in range(n):
            c.add("RY", [q], ("p", 2 * (l * n + q)))
            c.add("RZ", [q], ("p", 2 * (l * n + q) + 1))
        for q in range(n):
            c.add("CNOT", [q, (q + 1) % n])
    c.z([0])
    params = _rng(seed).uniform(0, 2 * math.pi, size=(1, c.n_params))
    return c, params.astype(np.float32), None


def hea_sv(seed=1005, n=20, layers=3, batch=16):
    """State-vector mode workload (Sec. 3.1; the hardware-efficient ansatz of
    the multiple-qubit-rotation experiment, Sec. 6.1): per layer RY RZ on every
    qubit and a CNOT ring q -> q+1 mod n, no observable -- the output is the
    state or its probabilities.  batch parameter sets ~ U[0, 2 pi); the bench
    starts it from the Neel state |0101...> as the initial state."""
    c = CircuitSpec(n)
    for l in range(layers):
        for q in range(n):
            c.add("RY", [q], ("p", 2 * (l * n + q)))
            c.add("RZ", [q], ("p", 2 * (l * n + q) + 1))
        for q in range(n):
            c.add("CNOT", [q, (q + 1) % n])
    params = _rng(seed).uniform(0, 2 * math.pi, size=(batch, c.n_params))
    return c, params.astype(np.float32), None


# ---------------------------------------------------------------- C2
def qnn12(seed=1001, batch=256, n=12, layers=4):
    """12-qubit QNN classifier: RY(x_q) angle encoding, then per layer RX, RY,
    RZ on every qubit and a CZ chain (q, q+1); observable mean_i <Z_i>.
    Parameters (shared by the batch) ~ N(0, 0.1): column 3(l n + q) + k."""
    c = CircuitSpec(n)
    for q in range(n):
        c.add("RY", [q], ("x", q))
    for l in range(layers):
        for q in range(n):
            base = 3 * (l * n + q)
            c.add("RX", [q], ("p", base))
            c.add("RY", [q], ("p", base + 1))
            c.add("RZ", [q], ("p", base + 2))
        for q in range(n - 1):
            c.add("CZ", [q, q + 1])
    for q in range(n):
        c.z([q], 1.0 / n)
    r = _rng(seed)
    params = r.normal(0.0, 0.1, size=(1, c.n_params))
    inputs = r.uniform(0.0, math.pi, size=(batch, n))
    return c, params.astype(np.float32), inputs.astype(np.float32)


# ---------------------------------------------------------------- C3
def ladder20(seed=1002, batch=64, n=20, layers=6):
    """20-qubit ansatz: per layer RY, RZ on every qubit, then CNOT(q -> q+1)
    for q = 0..n-2 in order; observable sum_{i=0}^{n-2} Z_i Z_{i+1}; `batch`
    independent parameter sets ~ U[0, 2 pi)."""
    c = CircuitSpec(n)
    for l in range(layers):
        for q in range(n):
            c.add("RY", [q], ("p", 2 * (l * n + q)))
            c.add("RZ", [q], ("p", 2 * (l * n + q) + 1))
        for q in range(n - 1):
            c.add("CNOT", [q, q + 1])
    for i in range(n - 1):
        c.z([i, i + 1])
    params = _rng(seed).uniform(0, 2 * math.pi, size=(batch, c.n_params))
    return c, params.astype(np.float32), None


# ---------------------------------------------------------------- C4a / C4b
def grid_edges(rows, cols):
    """Edge classes of a rows x cols grid, qubit q = cols*r + c:
    A horizontal (c even), B horizontal (c odd), C vertical (r even),
    D vertical (r odd)."""
    A, B, C, D = [], [], [], []
    for r in range(rows):
        for cc in range(cols - 1):
            (A if cc % 2 == 0 else B).append((cols * r + cc, cols * r + cc + 1))
    for r in range(rows - 1):
        for cc in range(cols):
            (C if r % 2 == 0 else D).append((cols * r + cc, cols * (r + 1) + cc))
    return [A, B, C, D]


def grid_brickwork(seed=1003, rows=5, cols=10, layers=4, observed=25):
    """Brickwork on a grid: layer l applies RZZ(theta) on edge class l mod 4,
    then RX(theta) on every qubit; one parameter per gate ~ U[0, 2 pi);
    observable <Z_observed>."""
    n = rows * cols
    c = CircuitSpec(n)
    classes = grid_edges(rows, cols)
    p = 0
    for l in range(layers):
        for (a, b) in classes[l % 4]:
            c.add("RZZ", [a, b], ("p", p)); p += 1
        for q in range(n):
            c.add("RX", [q], ("p", p)); p += 1
    c.z([observed])
    params = _rng(seed).uniform(0, 2 * math.pi, size=(1, c.n_params))
    return c, params.astype(np.float32), None


def grid_u3cz(seed=1004, rows=7, cols=7, depth=8, bits=None):
    """Random circuit on a grid: cycle d applies U3(theta, phi, lambda) on every
    qubit then CZ on edge class d mod 4; no final U3 layer.  Output: the
    amplitude <x|U|0> (x = 0...0 unless given).  Angles ~ U[0, 2 pi)."""
    n = rows * cols
    c = CircuitSpec(n)
    classes = grid_edges(rows, cols)
    p = 0
    for d in range(depth):
        for q in range(n):
            c.add("U3", [q], ("p", p), ("p", p + 1), ("p", p + 2)); p += 3
        for (a, b) in classes[d % 4]:
            c.add("CZ", [a, b])
    c.amplitude(bits if bits is not None else [0] * n)
    params = _rng(seed).uniform(0, 2 * math.pi, size=(1, c.n_params))
    return c, params.astype(np.float32), None


def grid_u3cz_mirror(seed=1005, rows=7, cols=7, depth=4):
    """U followed by U^dagger for a random U3/CZ grid circuit of `depth` cycles:
    the amplitude <0|U^dagger U|0> is exactly 1.  The inverse half reuses the
    structure in reverse with inverted angles supplied as parameters:
    U3(t, f, l)^dagger = U3(-t, -l, -f), CZ^dagger = CZ."""
    n = rows * cols
    c = CircuitSpec(n)
    classes = grid_edges(rows, cols)
    r = _rng(seed)
    fwd = []
    p = 0
    vals = []
    for d in range(depth):
        for q in range(n):
            ang = r.uniform(0, 2 * math.pi, size=3)
            c.add("U3", [q], ("p", p), ("p", p + 1), ("p", p + 2)); p += 3
            vals.extend(ang)
            fwd.append(("U3", q, ang))
        for (a, b) in classes[d % 4]:
            c.add("CZ", [a, b])
            fwd.append(("CZ", (a, b), None))
    for item in reversed(fwd):
        if item[0] == "CZ":
            c.add("CZ", list(item[1]))
        else:
            t, f, l = item[2]
            c.add("U3", [item[1]], ("p", p), ("p", p + 1), ("p", p + 2)); p += 3
            vals.extend([-t, -l, -f])
    c.amplitude([0] * n)
    params = np.asarray(vals, dtype=np.float64)[None, :]
    return c, params.astype(np.float32), None


# ---------------------------------------------------------------- tests / C5
def random_circuit(n, n_gates, seed, gates=("H", "X", "RX", "RY", "RZ", "U3", "CNOT", "CZ", "RZZ"),
                   batch=1, observables=True, amplitudes=0):
    """Random circuit over `gates`; every angle its own parameter ~ U[0, 2 pi).
    Observables: Z on each qubit (group per qubit) and one ZZ term."""
    r = _rng(seed)
    c = CircuitSpec(n)
    p = 0
    names = [g for g in gates if (g not in TWO_QUBIT or n >= 2)]
    for _ in range(n_gates):
        name = names[r.integers(len(names))]
        if name in TWO_QUBIT:
            a, b = r.choice(n, size=2, replace=False)
            qs = [a, b]
        else:
            qs = [r.integers(n)]
        k = N_ANGLES[name]
        c.add(name, qs, *[("p", p + i) for i in range(k)])
        p += k
    if observables:
        for q in range(n):
            c.z([q], 1.0, q)
        if n >= 2:
            c.z([0, n - 1], 0.5, n)
    for _ in range(amplitudes):
        c.amplitude(r.integers(0, 2, size=n))
    params = r.uniform(0, 2 * math.pi, size=(batch, max(c.n_params, 1)))
    return c, params.astype(np.float32), None


def random_circuit_tied(n, n_gates, n_params, seed, batch=1):
    """Random circuit whose angles draw from a pool of n_params parameters, so
    that several gates, and the angles of one gate, share a parameter (the
    gradient of a parameter is then the sum over every angle it feeds).
    Observables: Z on each qubit (group per qubit)."""
    r = _rng(seed)
    c = CircuitSpec(n)
    names = ["RX", "RY", "RZ", "U3", "RZZ", "CNOT", "CZ", "H"] if n >= 2 else ["RX", "RY", "RZ", "U3", "H"]
    for _ in range(n_gates):
        name = names[r.integers(len(names))]
        qs = list(r.choice(n, size=2, replace=False)) if name in TWO_QUBIT else [r.integers(n)]
        c.add(name, qs, *[("p", int(r.integers(n_params))) for _ in range(N_ANGLES[name])])
    for q in range(n):
        c.z([q], 1.0, q)
    c.n_params = n_params
    params = r.uniform(0, 2 * math.pi, size=(batch, n_params))
    return c, params.astype(np.float32), None


def brickwork(n, depth, seed, two_qubit="CZ"):
    """1-D brickwork of U3 layers and alternating even/odd entangler layers,
    used for the learned cost model's training and held-out circuits."""
    r = _rng(seed)
    c = CircuitSpec(n)
    p = 0
    for d in range(depth):
        for q in range(n):
            c.add("U3", [q], ("p", p), ("p", p + 1), ("p", p + 2)); p += 3
        for q in range(d % 2, n - 1, 2):
            c.add(two_qubit, [q, q + 1], *([("p", p)] if two_qubit == "RZZ" else []))
            if two_qubit == "RZZ":
                p += 1
    c.amplitude([0] * n)
    params = r.uniform(0, 2 * math.pi, size=(1, c.n_params))
    return c, params.astype(np.float32), None


def resolve_angles(circuit, params, inputs=None, batch=None):
    """Angle table [B][G][3] (float64): every gate's angles with sources read
    from params [B or 1][P] and inputs [B][F].  Pure indexing, no arithmetic."""
    params = np.asarray(params, dtype=np.float64)
    if params.ndim == 1:
        params = params[None, :]
    B = batch or max(params.shape[0], 1 if inputs is None else np.asarray(inputs).shape[0])
    out = np.zeros((B, len(circuit.gates), 3), dtype=np.float64)
    for g, gate in enumerate(circuit.gates):
        for i, src in enumerate(gate.angles):
            if src[0] == "p":
                out[:, g, i] = params[:, src[1]] if params.shape[0] == B else params[0, src[1]]
            elif src[0] == "x":
                out[:, g, i] = np.asarray(inputs, dtype=np.float64)[:, src[1]]
            else:
                out[:, g, i] = src[1]
    return out
