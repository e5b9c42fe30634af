"""Pins for the FP64 oracle: closed forms, textbook identities, brute force and
independent cross-checks (state vector vs. loop-nest contraction), so that a
dropped term, a wrong sign, a transposed operand or a wrong qubit order in the
oracle fails here.  CPU only."""
import cmath
import json
import math
import os

import numpy as np
import pytest

from paper_2301_05451_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _spec_from_json(d):
    c = W.CircuitSpec(d["n_qubits"])
    for name, qs, angles in d["gates"]:
        c.add(name, qs, *[tuple(a) for a in angles])
    return c


# ------------------------------------------------------------------ gates
def test_printed_ry_and_cnot_tensors(orc):
    """RY and CNOT as printed with the worked example of Sec. 3.2.1."""
    for t in (0.0, 0.4, 2.0, -1.3):
        c, s = math.cos(t / 2), math.sin(t / 2)
        np.testing.assert_allclose(orc.gate_matrix("RY", [t]), [[c, -s], [s, c]], atol=1e-15)
    M = orc.gate_matrix("CNOT")
    # E[e,f,c,d] = M[2e+f][2c+d]; blocks over the control pair (e, c)
    E = M.reshape(2, 2, 2, 2).transpose(0, 2, 1, 3)  # [e][c][f][d]
    np.testing.assert_array_equal(E[0, 0], np.eye(2))
    np.testing.assert_array_equal(E[1, 1], [[0, 1], [1, 0]])
    np.testing.assert_array_equal(E[0, 1], np.zeros((2, 2)))
    np.testing.assert_array_equal(E[1, 0], np.zeros((2, 2)))


def test_gates_unitary(orc):
    r = np.random.default_rng(0)
    for name in ("H", "X", "Y", "Z", "RX", "RY", "RZ", "U3", "CNOT", "CZ", "RZZ"):
        a = r.uniform(-7, 7, size=W.N_ANGLES[name])
        M = orc.gate_matrix(name, a)
        np.testing.assert_allclose(M @ M.conj().T, np.eye(M.shape[0]), atol=1e-14)


def test_gate_identities(orc):
    """Textbook relations that tie the conventions together."""
    X, Y, Z, H = (orc.gate_matrix(g) for g in "XYZH")
    I2 = np.eye(2)
    np.testing.assert_allclose(X @ Y, 1j * Z, atol=1e-15)
    np.testing.assert_allclose(H @ Z @ H, X, atol=1e-15)
    for t in (0.3, 1.7, -2.9):
        # exp(-i t P / 2) = cos(t/2) I - i sin(t/2) P
        for name, P in (("RX", X), ("RY", Y), ("RZ", Z)):
            np.testing.assert_allclose(orc.gate_matrix(name, [t]),
                                       math.cos(t / 2) * I2 - 1j * math.sin(t / 2) * P, atol=1e-15)
        np.testing.assert_allclose(orc.gate_matrix("U3", [t, 0, 0]), orc.gate_matrix("RY", [t]),
                                   atol=1e-15)
        np.testing.assert_allclose(orc.gate_matrix("U3", [t, -math.pi / 2, math.pi / 2]),
                                   orc.gate_matrix("RX", [t]), atol=1e-15)
        np.testing.assert_allclose(orc.gate_matrix("U3", [0, 0, t]),
                                   cmath.exp(1j * t / 2) * orc.gate_matrix("RZ", [t]), atol=1e-15)
        # U3(t, f, l) = e^{i(f+l)/2} RZ(f) RY(t) RZ(l)
        f, l = 0.7 * t, -1.1 * t
        np.testing.assert_allclose(
            orc.gate_matrix("U3", [t, f, l]),
            cmath.exp(0.5j * (f + l)) * orc.gate_matrix("RZ", [f]) @ orc.gate_matrix("RY", [t])
            @ orc.gate_matrix("RZ", [l]), atol=1e-14)
        # RZZ(t) = CNOT (I x RZ(t)) CNOT
        C = orc.gate_matrix("CNOT")
        np.testing.assert_allclose(orc.gate_matrix("RZZ", [t]),
                                   C @ np.kron(I2, orc.gate_matrix("RZ", [t])) @ C, atol=1e-15)
    # CZ = (I x H) CNOT (I x H)
    np.testing.assert_allclose(orc.gate_matrix("CZ"),
                               np.kron(I2, H) @ orc.gate_matrix("CNOT") @ np.kron(I2, H), atol=1e-15)


# ------------------------------------------------------------------ closed forms
def test_worked_example_closed_form(orc):
    """Sec. 3.2.1: X(q0), RY(theta)(q1), CNOT(0,1); <I x Z> = sin^2 - cos^2."""
    d = json.load(open(os.path.join(GOLDEN, "worked_example_sec321.json")))
    c = _spec_from_json(d["circuit"])
    c.z(d["circuit"]["observable_z"])
    for t in d["thetas"]:
        want = math.sin(t / 2) ** 2 - math.cos(t / 2) ** 2
        a = W.resolve_angles(c, np.array([[t]]))
        assert abs(orc.expvals(c, a)[0, 0] - want) < 1e-14
        for order in ("greedy", "linear"):
            v, _ = orc.tn_expval(c, a[0], [1], order=order)
            assert abs(v - want) < 1e-14


def test_single_qubit_rotations(orc):
    for t in (0.0, 0.5, 2.0, 4.4):
        for name in ("RX", "RY"):
            c = W.CircuitSpec(1)
            c.add(name, [0], ("p", 0))
            c.z([0])
            c.amplitude([1])
            a = W.resolve_angles(c, np.array([[t]]))
            assert abs(orc.expvals(c, a)[0, 0] - math.cos(t)) < 1e-14
            want1 = (-1j if name == "RX" else 1.0) * math.sin(t / 2)
            assert abs(orc.amplitudes(c, a)[0, 0] - want1) < 1e-14
        c = W.CircuitSpec(1)
        c.add("RZ", [0], ("p", 0))
        c.amplitude([0])
        a = W.resolve_angles(c, np.array([[t]]))
        assert abs(orc.amplitudes(c, a)[0, 0] - cmath.exp(-0.5j * t)) < 1e-14


def test_qubit_zero_is_most_significant(orc):
    """Sec. 5.1.1: the zeroth qubit is written on the left."""
    c = W.CircuitSpec(3)
    c.add("X", [0])
    psi = orc.statevector(c, np.zeros((1, 3)))
    assert abs(psi[4] - 1) < 1e-15 and np.sum(np.abs(psi) ** 2) == pytest.approx(1)
    c = W.CircuitSpec(3)
    c.add("X", [0])
    c.add("CNOT", [0, 2])   # control 0, target 2 -> |101>
    psi = orc.statevector(c, np.zeros((2, 3)))
    assert abs(psi[5] - 1) < 1e-15


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_ghz_amplitudes(orc, n):
    c = W.CircuitSpec(n)
    c.add("H", [0])
    for q in range(n - 1):
        c.add("CNOT", [q, q + 1])
    c.amplitude([0] * n)
    c.amplitude([1] * n)
    c.amplitude([1] + [0] * (n - 1))
    a = W.resolve_angles(c, np.zeros((1, 1)))
    amp = orc.amplitudes(c, a)[0]
    np.testing.assert_allclose(amp, [2 ** -0.5, 2 ** -0.5, 0], atol=1e-15)
    for bits, want in zip(c.amplitudes, [2 ** -0.5, 2 ** -0.5, 0]):
        for order in ("greedy", "linear"):
            v, _ = orc.tn_amplitude(c, a[0], bits, order=order)
            assert abs(v - want) < 1e-14


def test_mirror_circuit_amplitude_is_one(orc):
    c, p, _ = W.grid_u3cz_mirror(rows=3, cols=4, depth=4)
    a = W.resolve_angles(c, p)
    assert abs(orc.amplitudes(c, a)[0, 0] - 1) < 1e-12
    for order in ("greedy", "linear"):
        v, _ = orc.tn_amplitude(c, a[0], order=order)
        assert abs(v - 1) < 1e-12


def test_mirror_7x7_tn_linear(orc):
    """The full 7x7 structure (4 forward + 4 inverse cycles) through the
    loop-nest contractor: exactly 1."""
    c, p, _ = W.grid_u3cz_mirror(rows=7, cols=7, depth=4)
    v, peak = orc.tn_amplitude(c, W.resolve_angles(c, p)[0], order="linear", max_elems=1 << 24)
    assert abs(v - 1) < 1e-10 and peak <= 22


# ------------------------------------------------------------------ cross-checks
@pytest.mark.parametrize("seed", range(6))
def test_statevector_vs_loop_nest_contraction(orc, seed):
    """Two independent codes: full-amplitude propagation and pairwise loop nests."""
    n = 3 + seed % 5
    c, p, _ = W.random_circuit(n, 40, seed, amplitudes=3)
    a = W.resolve_angles(c, p)
    amps = orc.amplitudes(c, a)[0]
    for bits, want in zip(c.amplitudes, amps):
        v, _ = orc.tn_amplitude(c, a[0], bits)
        assert abs(v - want) < 1e-13
        v, _ = orc.tn_amplitude(c, a[0], bits, order="linear")
        assert abs(v - want) < 1e-13
    ev = orc.expvals(c, a)[0]
    for (qs, coeff, g) in c.terms:
        v, _ = orc.tn_expval(c, a[0], qs)
        assert abs(v.imag) < 1e-13
        assert abs(coeff * v.real - ev[g]) < 1e-13


def test_grid_amplitude_statevector_vs_contraction(orc):
    c, p, _ = W.grid_u3cz(rows=4, cols=5, depth=8, seed=7)
    a = W.resolve_angles(c, p)
    v, _ = orc.tn_amplitude(c, a[0], order="linear")
    assert abs(v - orc.amplitudes(c, a)[0, 0]) < 1e-14


def test_expectation_brute_force(orc):
    """<psi|Z_i Z_j|psi> against an explicit diagonal operator on the state."""
    c, p, _ = W.random_circuit(5, 30, 11)
    a = W.resolve_angles(c, p)
    psi = orc.statevector(c, a[0])
    ev = orc.expvals(c, a)[0]
    for (qs, coeff, g) in c.terms:
        diag = np.ones(32)
        for x in range(32):
            for q in qs:
                if (x >> (4 - q)) & 1:
                    diag[x] *= -1
        assert abs(coeff * np.vdot(psi, diag * psi).real - ev[g]) < 1e-14


def test_batch_rows_independent(orc):
    c, p, x = W.qnn12(batch=5)
    a = W.resolve_angles(c, p, x)
    full = orc.expvals(c, a)
    for b in range(5):
        np.testing.assert_allclose(orc.expvals(c, a[b:b + 1])[0], full[b], atol=0, rtol=0)


# ------------------------------------------------------------------ gradients
def test_param_shift_closed_form(orc):
    """d<Z>/dt for RY(t)|0> is -sin t."""
    c = W.CircuitSpec(1)
    c.add("RY", [0], ("p", 0))
    c.z([0])
    for t in (0.2, 1.0, 3.0):
        g = orc.param_grads_param_shift(c, np.array([t]))
        assert abs(g[0] + math.sin(t)) < 1e-14


@pytest.mark.parametrize("seed", range(3))
def test_param_shift_equals_finite_difference(orc, seed):
    c, p, _ = W.random_circuit(4, 25, 100 + seed)
    w = np.linspace(0.5, 1.5, c.n_groups)
    ps = orc.param_grads_param_shift(c, p[0].astype(np.float64), weights=w)
    fd = orc.param_grads_finite_difference(c, p[0].astype(np.float64), weights=w)
    np.testing.assert_allclose(ps, fd, atol=1e-7)


def test_param_shift_shared_parameter(orc):
    """A parameter feeding two gates: the shift rule summed over occurrences."""
    c = W.CircuitSpec(2)
    c.add("RX", [0], ("p", 0))
    c.add("CNOT", [0, 1])
    c.add("RY", [1], ("p", 0))
    c.z([1])
    for t in (0.3, 1.9):
        ps = orc.param_grads_param_shift(c, np.array([t]))
        fd = orc.param_grads_finite_difference(c, np.array([t]))
        assert abs(ps[0] - fd[0]) < 1e-8


@pytest.mark.parametrize("n", [3, 7])
def test_param_shift_tied_random_circuits(orc, n):
    """The tied-parameter circuits of the GPU parity test (a pool of
    parameters feeding many gates, U3 angles included): the shift rule summed
    over every angle a parameter feeds equals the FP64 central difference."""
    c, p, _ = W.random_circuit_tied(n, 12 * n, max(2, n - 2), 600 + n, batch=3)
    assert c.n_params < sum(len(g.angles) for g in c.gates)  # parameters are shared
    for row in (0, 2):
        ps = orc.param_grads_param_shift(c, p[row].astype(np.float64))
        fd = orc.param_grads_finite_difference(c, p[row].astype(np.float64))
        np.testing.assert_allclose(ps, fd, atol=1e-7)
        assert np.abs(ps).max() > 1e-2  # not a trivially zero gradient


# ------------------------------------------------------------------ light cone
def test_lightcone_preserves_expectation(orc):
    c, p, _ = W.grid_brickwork(rows=3, cols=4, layers=4, observed=5)
    a = W.resolve_angles(c, p)
    full = orc.expvals(c, a)[0, 0]
    red, kept, qmap = orc.lightcone(c, [5])
    assert len(kept) < len(c.gates)
    ra = a[:, kept, :]
    assert abs(orc.expvals(red, ra)[0, 0] - full) < 1e-13


def test_lightcone_5x10_size(orc):
    c, p, _ = W.grid_brickwork()
    red, kept, qmap = orc.lightcone(c, [25])
    assert red.n_qubits == 16 and len(kept) == 30


# ------------------------------------------------------------------ MLP
def test_mlp_gradients_vs_finite_difference(orc):
    r = np.random.default_rng(3)
    F, H, N = 5, 7, 11
    params = [r.normal(size=(H, F)), r.normal(size=H), r.normal(size=(H, H)), r.normal(size=H),
              r.normal(size=(1, H)), r.normal(size=1)]
    X = r.normal(size=(N, F))
    t = r.normal(size=N)
    loss, grads = orc.mlp_loss_and_grads(params, X, t)
    h = 1e-6
    for k, P in enumerate(params):
        it = np.nditer(P, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            pp = [q.copy() for q in params]
            pm = [q.copy() for q in params]
            pp[k][idx] += h
            pm[k][idx] -= h
            fd = (orc.mlp_loss_and_grads(pp, X, t)[0] - orc.mlp_loss_and_grads(pm, X, t)[0]) / (2 * h)
            assert abs(fd - grads[k][idx]) < 1e-6 * max(1, abs(fd))


def test_mlp_forward_by_hand(orc):
    W1 = np.array([[1.0, -1.0]]); b1 = np.array([0.5])
    W2 = np.array([[2.0]]); b2 = np.array([-1.0])
    W3 = np.array([[3.0]]); b3 = np.array([0.25])
    y, _ = orc.mlp_forward((W1, b1, W2, b2, W3, b3), np.array([[2.0, 1.0], [0.0, 3.0]]))
    # row 0: z1 = 1.5 -> h1 = 1.5 -> z2 = 2 -> y = 6.25; row 1: z1 = -2.5 -> 0 -> -1 -> 0 -> 0.25
    np.testing.assert_allclose(y, [6.25, 0.25])


def test_adam_first_step(orc):
    """Bias correction makes the first Adam step lr * g / (|g| + eps)."""
    p = [np.array([1.0, -2.0])]
    g = [np.array([0.5, -4.0])]
    newp, m, v = orc.adam_step(p, g, [np.zeros(2)], [np.zeros(2)], 1, lr=0.1)
    np.testing.assert_allclose(newp[0], [1.0 - 0.1, -2.0 + 0.1], atol=1e-7)


# ------------------------------------------------- initial states (Sec. 3.1)
def _random_state(r, n):
    v = r.normal(size=1 << n) + 1j * r.normal(size=1 << n)
    return v / np.linalg.norm(v)


def test_initial_basis_state_equals_prepended_x_gates(orc):
    """U|x> from an initial state equals U X^{bits of x} |0...0> built from X
    gates (a different code path), with qubit 0 the most significant bit."""
    n = 5
    spec, params, _ = W.random_circuit(n, 40, 71)
    ang = W.resolve_angles(spec, params)[0]
    for x in (0, 1, 6, 19, 31):
        c = W.CircuitSpec(n)
        for q in range(n):
            if (x >> (n - 1 - q)) & 1:
                c.add("X", [q])
        for g in spec.gates:
            c.add(g.name, g.qubits, *g.angles)
        ref = orc.statevector(c, W.resolve_angles(c, params)[0])
        got = orc.statevector(spec, ang, init=np.eye(1 << n)[x])
        np.testing.assert_allclose(got, ref, atol=1e-13)
    np.testing.assert_allclose(orc.statevector(spec, ang, init=np.eye(1 << n)[0]), orc.statevector(spec, ang),
                               atol=1e-15)


def test_initial_state_linearity_and_norm(orc):
    """U (a psi1 + b psi2) = a U psi1 + b U psi2; the norm is preserved."""
    r = np.random.default_rng(72)
    n = 6
    spec, params, _ = W.random_circuit(n, 50, 73)
    ang = W.resolve_angles(spec, params)[0]
    p1, p2 = _random_state(r, n), _random_state(r, n)
    a, b = 0.3 - 1.1j, 0.8 + 0.25j
    lhs = orc.statevector(spec, ang, init=a * p1 + b * p2)
    rhs = a * orc.statevector(spec, ang, init=p1) + b * orc.statevector(spec, ang, init=p2)
    np.testing.assert_allclose(lhs, rhs, atol=1e-13)
    assert abs(np.linalg.norm(orc.statevector(spec, ang, init=p1)) - 1) < 1e-13
    pr = orc.probabilities(spec, ang, init=p1)
    assert abs(pr.sum() - 1) < 1e-13 and pr.min() >= 0


def test_initial_state_expvals_and_gradients(orc):
    """Grouped expectations from an initial state equal the diagonal sums over
    U psi0 by brute force; the shift rule from psi0 equals central differences."""
    r = np.random.default_rng(74)
    n = 5
    spec, params, _ = W.random_circuit(n, 30, 75, batch=3)
    ang = W.resolve_angles(spec, params)
    init = np.stack([_random_state(r, n) for _ in range(3)])
    got = orc.expvals(spec, ang, init=init)
    for b in range(3):
        psi = orc.statevector(spec, ang[b], init=init[b])
        for g in range(spec.n_groups):
            ref = 0.0
            for qs, coeff, grp in spec.terms:
                if grp != g:
                    continue
                sign = np.array([(-1) ** sum((x >> (n - 1 - q)) & 1 for q in qs) for x in range(1 << n)])
                ref += coeff * float(np.sum(sign * np.abs(psi) ** 2))
            assert abs(got[b, g] - ref) < 1e-12
    # one shared state for every row
    shared = orc.expvals(spec, ang, init=init[1])
    np.testing.assert_allclose(shared[1], got[1], atol=1e-14)
    w = r.normal(size=spec.n_groups)
    ps = orc.param_grads_param_shift(spec, params[0].astype(np.float64), weights=w, init=init[0])
    fd = orc.param_grads_finite_difference(spec, params[0].astype(np.float64), weights=w, init=init[0])
    np.testing.assert_allclose(ps, fd, atol=1e-7)


def test_slice_projectors_pinned(orc):
    """Fixing a wire to one value is the projector |v><v| (Sec. 3.2.3): the
    matrices, a closed form, and the slicing identity (the slices of any cut
    set sum to the amplitude) by both the state vector and the loop-nest
    contraction."""
    np.testing.assert_array_equal(orc.gate_matrix("P0"), np.diag([1, 0]))
    np.testing.assert_array_equal(orc.gate_matrix("P1"), np.diag([0, 1]))
    # one qubit, RY(t)|0>, cut after the gate: <0|P0 RY|0> = cos t/2,
    # <0|P1 RY|0> = 0, <1|P1 RY|0> = sin t/2
    t = 0.7
    c = W.CircuitSpec(1)
    c.add("RY", [0], ("p", 0))
    c.amplitude([0])
    c.amplitude([1])
    ang = W.resolve_angles(c, np.array([[t]], np.float32))[0]
    a0 = orc.sliced_amplitudes(c, ang, [(0, 0)], 0)
    a1 = orc.sliced_amplitudes(c, ang, [(0, 0)], 1)
    tt = float(np.float32(t))
    np.testing.assert_allclose(a0, [np.cos(tt / 2), 0], atol=1e-15)
    np.testing.assert_allclose(a1, [0, np.sin(tt / 2)], atol=1e-15)
    # the identity on a 3x3 grid circuit, three cuts (one on an input wire)
    g, p, _ = W.grid_u3cz(seed=7, rows=3, cols=3, depth=4)
    angr = W.resolve_angles(g, p)[0]
    whole = orc.amplitudes(g, angr[None])[0, 0]
    cuts = [(4, 20), (0, -1), (8, 30)]
    for method in ("sv", "tn"):
        parts = [orc.sliced_amplitudes(g, angr, cuts, s, method=method)[0] for s in range(8)]
        assert abs(sum(parts) - whole) < 1e-12
        assert abs(parts[2]) < 1e-15 and abs(parts[3]) < 1e-15  # input wire of qubit 0 is |0>: value 1 gives 0


def test_adam_later_steps_pinned(orc):
    """Adam beyond its first step (Kingma and Ba, Algorithm 1): with a
    constant gradient g the bias-corrected moments are exactly g and g^2 at
    every step, so each update is lr g / (|g| + eps); with g1 then g2 the
    second step's corrected moments are the (1 - b)-weighted means of the
    two gradients, worked out by hand."""
    g = np.array([0.3, -2.0, 5e-3])
    p = [np.array([1.0, 2.0, -1.0])]
    m, v = [np.zeros(3)], [np.zeros(3)]
    lr, b1, b2, eps = 0.05, 0.9, 0.999, 1e-8
    cur = p
    for t in range(1, 8):
        cur, m, v = orc.adam_step(cur, [g], m, v, t, lr=lr, b1=b1, b2=b2, eps=eps)
        np.testing.assert_allclose(cur[0], p[0] - t * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-13)
    g1, g2 = np.array([1.0, -0.5]), np.array([-0.25, 2.0])
    q = [np.array([0.0, 0.0])]
    q1, m1, v1 = orc.adam_step(q, [g1], [np.zeros(2)], [np.zeros(2)], 1, lr=lr, b1=b1, b2=b2, eps=eps)
    q2, _, _ = orc.adam_step(q1, [g2], m1, v1, 2, lr=lr, b1=b1, b2=b2, eps=eps)
    mh = (b1 * (1 - b1) * g1 + (1 - b1) * g2) / (1 - b1 ** 2)
    vh = (b2 * (1 - b2) * g1 ** 2 + (1 - b2) * g2 ** 2) / (1 - b2 ** 2)
    step1 = lr * g1 / (np.abs(g1) + eps)
    np.testing.assert_allclose(q2[0], -step1 - lr * mh / (np.sqrt(vh) + eps), rtol=0, atol=1e-13)
