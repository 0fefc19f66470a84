"""Pins of the FP64 oracle against facts fixed outside it.

Each test checks the oracle against something it does not compute itself:
matrix exponentials and projector constructions of the gates, a dense
Kronecker-product brute force, closed-form states (Hadamard layer, GHZ, the
DFT column produced by the QFT circuit), unit norm and the U.U^dagger round
trip.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import sim
from synth import circuits as C

I2 = np.eye(2)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
P0 = np.array([[1, 0], [0, 0]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)


def k2(a_q1, a_q0):
    """4x4 operator with index b = b0 + 2*b1: a_q0 on bit 0, a_q1 on bit 1."""
    return np.kron(a_q1, a_q0)


RNG = np.random.default_rng(1234)


@pytest.mark.parametrize("t", [0.0, 0.37, 2.1, 5.9])
def test_single_qubit_matrices(t):
    assert np.allclose(sim.gate_matrix(C.H), (PX + PZ) / math.sqrt(2), atol=1e-15)
    assert np.allclose(sim.gate_matrix(C.X), PX, atol=0)
    assert np.allclose(sim.gate_matrix(C.RX, [t]), expm(-0.5j * t * PX), atol=1e-14)
    assert np.allclose(sim.gate_matrix(C.RZ, [t]), expm(-0.5j * t * PZ), atol=1e-14)


def test_u3_decomposition():
    # U3(t,p,l) = e^{i(p+l)/2} RZ(p) RY(t) RZ(l)
    for _ in range(10):
        t, p, l = RNG.uniform(0, 2 * math.pi, 3)
        ref = np.exp(0.5j * (p + l)) * expm(-0.5j * p * PZ) @ expm(-0.5j * t * PY) @ expm(-0.5j * l * PZ)
        assert np.allclose(sim.gate_matrix(C.U3, [t, p, l]), ref, atol=1e-14)
    assert np.allclose(sim.gate_matrix(C.U3, [math.pi / 2, 0, math.pi]), sim.gate_matrix(C.H), atol=1e-15)
    assert np.allclose(sim.gate_matrix(C.U3, [math.pi, 0, math.pi]), PX, atol=1e-15)


def test_two_qubit_matrices():
    t = 1.234
    cx = k2(I2, P0) + k2(PX, P1)  # control on q0 (bit 0), X on q1 (bit 1)
    assert np.allclose(sim.gate_matrix(C.CX), cx, atol=0)
    assert np.allclose(sim.gate_matrix(C.CZ), k2(I2, P0) + k2(PZ, P1), atol=0)
    assert np.allclose(sim.gate_matrix(C.CP, [t]), k2(I2, I2) + (np.exp(1j * t) - 1) * k2(P1, P1), atol=1e-15)
    assert np.allclose(sim.gate_matrix(C.CP, [math.pi]), sim.gate_matrix(C.CZ), atol=1e-15)
    sw = 0.5 * (k2(I2, I2) + k2(PX, PX) + k2(PY, PY) + k2(PZ, PZ))
    assert np.allclose(sim.gate_matrix(C.SWAP), sw, atol=1e-15)
    assert np.allclose(sim.gate_matrix(C.RXX, [t]), expm(-0.5j * t * k2(PX, PX)), atol=1e-14)
    # SWAP = CX(a,b) CX(b,a) CX(a,b): built from the oracle's CX with swapped roles
    cx_rev = k2(P0, I2) + k2(P1, PX)
    assert np.allclose(cx @ cx_rev @ cx, sim.gate_matrix(C.SWAP), atol=0)


def test_all_gates_unitary():
    for t in range(10):
        m = sim.gate_matrix(t, RNG.uniform(0, 2 * math.pi, 3))
        assert np.allclose(m @ m.conj().T, np.eye(m.shape[0]), atol=1e-14)


# ---- dense brute force -------------------------------------------------------

def embed(n, ops):
    """Kronecker product over n qubits, ops = {qubit: 2x2}; qubit n-1 leftmost."""
    out = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        out = np.kron(out, ops.get(q, I2))
    return out


def full_operator(n, g):
    t = int(g["type"])
    m = sim.gate_matrix(t, [g["p0"], g["p1"], g["p2"]])
    if C.NQ[t] == 1:
        return embed(n, {int(g["q0"]): m})
    q0, q1 = int(g["q0"]), int(g["q1"])
    out = np.zeros((1 << n, 1 << n), dtype=complex)
    for r in range(4):
        for c in range(4):
            if m[r, c] == 0:
                continue
            e0 = np.zeros((2, 2)); e0[r & 1, c & 1] = 1
            e1 = np.zeros((2, 2)); e1[r >> 1, c >> 1] = 1
            out += m[r, c] * embed(n, {q0: e0, q1: e1})
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_dense(seed):
    n = 6
    g = C.concat(C.mixed_circuit(n, 60, seed), C.entangling_circuit(n, 2, seed))
    u = np.eye(1 << n, dtype=complex)
    for gi in g:
        u = full_operator(n, gi) @ u
    psi0 = np.array([1, 1j]) @ np.random.default_rng(seed).normal(size=(2, 1 << n))
    psi0 /= np.linalg.norm(psi0)
    assert np.allclose(sim.apply(n, g, psi0), u @ psi0, atol=1e-13)
    assert np.allclose(sim.apply(n, g), u[:, 0], atol=1e-13)


def test_brute_force_every_pair_order():
    # every ordered qubit pair, asymmetric gates, so swapped roles fail
    n = 4
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            g = C.make_gates([(C.U3, a, None, 0.3, 1.1, 2.2), (C.U3, b, None, 1.7, 0.4, 0.9),
                              (C.CX, a, b), (C.CP, a, b, 0.77), (C.RXX, a, b, 1.3),
                              (C.SWAP, a, b), (C.RX, b, None, 0.5)])
            u = np.eye(1 << n, dtype=complex)
            for gi in g:
                u = full_operator(n, gi) @ u
            assert np.allclose(sim.apply(n, g), u[:, 0], atol=1e-14)


# ---- closed forms -------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 5, 12])
def test_hadamard_layer_uniform(n):
    psi = sim.apply(n, C.hadamard_layer(n))
    assert np.allclose(psi, 2 ** (-n / 2), atol=1e-14)


@pytest.mark.parametrize("n", [2, 7, 16])
def test_ghz(n):
    psi = sim.apply(n, C.ghz(n))
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert np.allclose(psi, ref, atol=1e-14)


@pytest.mark.parametrize("n,x", [(3, 5), (6, 1), (10, 777), (14, 12345)])
def test_qft_is_dft(n, x):
    N = 1 << n
    psi = sim.apply(n, C.concat(C.basis_prep(n, x), C.qft(n)))
    y = np.arange(N)
    ref = np.exp(2j * np.pi * x * y / N) / math.sqrt(N)
    assert np.allclose(psi, ref, atol=1e-12)
    # the same column from numpy's FFT (unnormalised inverse DFT)
    e = np.zeros(N, dtype=complex); e[x] = 1
    assert np.allclose(psi, np.fft.ifft(e) * math.sqrt(N), atol=1e-12)


@pytest.mark.parametrize("gen", ["layered", "mixed", "entangling"])
def test_unit_norm_and_round_trip(gen):
    n = 12
    g = {"layered": C.layered_u3_cz(n, 6, 3), "mixed": C.mixed_circuit(n, 400, 3),
         "entangling": C.entangling_circuit(n, 4, 3)}[gen]
    psi = sim.apply(n, g)
    assert abs(sim.norm2(psi) - 1) < 1e-12
    back = sim.apply(n, C.adjoint(g), psi)
    assert abs(abs(back[0]) - 1) < 1e-12
    assert np.max(np.abs(back[1:])) < 1e-12


def test_kernel_unitary_matches_embedding():
    n = 5
    g = C.mixed_circuit(n, 30, 9)
    qubits = [3, 0, 4, 1, 2]  # a permuted qubit list: index bit j <- qubit qubits[j]
    u = sim.kernel_unitary(g, qubits)
    assert np.allclose(u @ u.conj().T, np.eye(32), atol=1e-13)
    full = np.eye(1 << n, dtype=complex)
    for gi in g:
        full = full_operator(n, gi) @ full
    # permute: local index l has bit j = bit qubits[j] of the global index
    perm = np.array([sum(((l >> j) & 1) << qubits[j] for j in range(n)) for l in range(32)])
    assert np.allclose(u, full[np.ix_(perm, perm)], atol=1e-13)


def test_bad_gate_rejected():
    with pytest.raises(ValueError):
        sim.apply(3, C.make_gates([(C.CX, 1, 1)]))
    with pytest.raises(ValueError):
        sim.apply(3, C.make_gates([(C.H, 5)]))


def _golden_pairs():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "eq1_pair_indices.txt")
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, body = line.split(":")
        n, q = (int(x) for x in head.split())
        pairs = [tuple(int(x) for x in p.split()) for p in body.split(";")]
        yield n, q, pairs


def test_one_qubit_gate_follows_eq1_pair_indices():
    # the oracle updates exactly the pairs Eq. 1 names, with u00 acting on
    # the lower index of each pair (fixture: tests/golden/eq1_pair_indices.txt)
    import numpy as np
    from oracle import sim
    from synth import circuits as C
    cases = list(_golden_pairs())
    assert len(cases) == 5
    for n, q, pairs in cases:
        assert len(pairs) == 2 ** (n - 1)
        rng = np.random.default_rng(10 * n + q)
        psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
        g = C.make_gates([(C.U3, q, None, 0.7, 1.1, -0.4)])
        u = sim.gate_matrix(C.U3, (0.7, 1.1, -0.4))
        out = sim.apply(n, g, psi.copy())
        expect = psi.copy()
        for a, b in pairs:
            expect[a] = u[0, 0] * psi[a] + u[0, 1] * psi[b]
            expect[b] = u[1, 0] * psi[a] + u[1, 1] * psi[b]
        assert np.allclose(out, expect, atol=1e-14)
