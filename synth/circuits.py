"""Seeded synthetic circuit generators (input data only).

This module is shared by the FP64 oracle (``oracle/``), the tests and the
benchmark.  It draws gate sequences and nothing else: it holds no gate
matrices and applies nothing to a state, so it carries none of the
simulator's arithmetic.

Gate records use the layout of ``qs_gate`` in ``include/qsim.h``::

    int32 type, int32 nq, int32 q0, int32 q1, float64 p0, p1, p2   (40 bytes)

Type codes (the input encoding, shared by every consumer):

    H=0 X=1 RX=2 RZ=3 U3=4 CX=5 CZ=6 CP=7 SWAP=8 RXX=9

Qubit q is bit q of the amplitude index (little-endian, Eq. 1 of the paper).
For CX, q0 is the control and q1 the target.  Angles are drawn from
U[0, 2*pi).

Workloads (the paper's benchmark circuits, MQT Bench / NWQBench, Table 1, are
not available; these seeded circuits stand in for them with matching qubit
counts and gate counts):

* ``layered_u3_cz``  -- every layer: U3 on each qubit, then CZ on a uniformly
  random perfect matching (20 qubits x 20 layers = 600 gates; 35 qubits x 30
  layers for the host-staged case).
* ``mixed_circuit``  -- exactly ``ngates`` gates, type uniform over
  {H, X, RX, RZ, CX, CZ, CP, SWAP}; first qubit uniform, partner at distance
  1 + Geom(0.3) with a uniform sign, redrawn when out of range
  (28 or 30 qubits, 5000 gates).
* ``entangling_circuit`` -- every layer: U3 on each qubit, then a random
  perfect matching whose pairs each get CP(t1) then RXX(t2)
  (32 qubits x 40 layers = 2560 gates; also at 28 and 30 qubits).
* ``random_subcircuit`` -- the cost-model training distribution: an active
  set of 1..max_active qubits out of 30 (10 by default; the cost-model
  generator asks for up to 13, and up to 6 for fused samples), 1..64 gates
  acting inside it, of the mixed set or of a given gate set (the generator
  alternates the mixed set and all ten types).
"""
from __future__ import annotations

import math

import numpy as np

H, X, RX, RZ, U3, CX, CZ, CP, SWAP, RXX = range(10)
NAMES = ["H", "X", "RX", "RZ", "U3", "CX", "CZ", "CP", "SWAP", "RXX"]
NQ = [1, 1, 1, 1, 1, 2, 2, 2, 2, 2]
NPARAM = [0, 0, 1, 1, 3, 0, 0, 1, 0, 1]
MIXED_SET = [H, X, RX, RZ, CX, CZ, CP, SWAP]
ALL_TYPES = list(range(10))

GATE_DTYPE = np.dtype(
    {
        "names": ["type", "nq", "q0", "q1", "p0", "p1", "p2"],
        "formats": ["<i4", "<i4", "<i4", "<i4", "<f8", "<f8", "<f8"],
        "offsets": [0, 4, 8, 12, 16, 24, 32],
        "itemsize": 40,
    }
)

TWO_PI = 2.0 * math.pi


def make_gates(items) -> np.ndarray:
    """Build a record array from (type, q0, q1, p0, p1, p2) tuples."""
    items = list(items)
    out = np.zeros(len(items), dtype=GATE_DTYPE)
    for i, it in enumerate(items):
        t = int(it[0])
        q0 = int(it[1])
        q1 = int(it[2]) if len(it) > 2 and it[2] is not None else -1
        ps = list(it[3:6]) + [0.0] * (3 - len(it[3:6]))
        out[i] = (t, NQ[t], q0, q1 if NQ[t] == 2 else -1, ps[0], ps[1], ps[2])
    return out


def _angles(rng, k):
    return rng.uniform(0.0, TWO_PI, size=k)


def random_matching(rng: np.random.Generator, n: int) -> list[tuple[int, int]]:
    """Uniform random perfect matching: Fisher-Yates shuffle, pair neighbours."""
    perm = list(range(n))
    for i in range(n - 1, 0, -1):
        j = int(rng.integers(0, i + 1))
        perm[i], perm[j] = perm[j], perm[i]
    return [(perm[2 * i], perm[2 * i + 1]) for i in range(n // 2)]


def layered_u3_cz(n: int = 20, layers: int = 20, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    items = []
    for _ in range(layers):
        for q in range(n):
            t, p, l = _angles(rng, 3)
            items.append((U3, q, None, t, p, l))
        for a, b in random_matching(rng, n):
            items.append((CZ, a, b))
    return make_gates(items)


def _partner(rng, n, q, p_geom=0.3):
    while True:
        d = int(rng.geometric(p_geom))  # support {1, 2, ...} = 1 + Geom on {0, 1, ...}
        s = 1 if rng.integers(0, 2) else -1
        r = q + s * d
        if 0 <= r < n:
            return r


def mixed_circuit(n: int = 28, ngates: int = 5000, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    items = []
    for _ in range(ngates):
        t = MIXED_SET[int(rng.integers(0, len(MIXED_SET)))]
        q = int(rng.integers(0, n))
        if NQ[t] == 2:
            r = _partner(rng, n, q)
            th = float(_angles(rng, 1)[0]) if t == CP else 0.0
            items.append((t, q, r, th))
        else:
            th = float(_angles(rng, 1)[0]) if t in (RX, RZ) else 0.0
            items.append((t, q, None, th))
    return make_gates(items)


def entangling_circuit(n: int = 32, layers: int = 40, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    items = []
    for _ in range(layers):
        for q in range(n):
            t, p, l = _angles(rng, 3)
            items.append((U3, q, None, t, p, l))
        for a, b in random_matching(rng, n):
            t1, t2 = _angles(rng, 2)
            items.append((CP, a, b, t1))
            items.append((RXX, a, b, t2))
    return make_gates(items)


def random_subcircuit(n: int = 30, seed: int = 0, max_active: int = 10,
                      max_gates: int = 64, gate_set=None):
    """One cost-model sample: (gates, sorted active qubit list).  Gate types
    are drawn uniformly from `gate_set` (default: the mixed-circuit set)."""
    rng = np.random.default_rng(seed)
    na = int(rng.integers(1, max_active + 1))
    act = sorted(int(x) for x in rng.choice(n, size=na, replace=False))
    ng = int(rng.integers(1, max_gates + 1))
    pool = MIXED_SET if gate_set is None else list(gate_set)
    types = pool if na >= 2 else [t for t in pool if NQ[t] == 1]
    items = []
    for _ in range(ng):
        t = types[int(rng.integers(0, len(types)))]
        th = [float(x) for x in _angles(rng, NPARAM[t])] if NPARAM[t] else []
        if NQ[t] == 2:
            a, b = rng.choice(na, size=2, replace=False)
            items.append((t, act[int(a)], act[int(b)], *th))
        else:
            q = act[int(rng.integers(0, na))]
            items.append((t, q, None, *th))
    return make_gates(items), act


# ---- closed-form circuits used as oracle pins ---------------------------

def hadamard_layer(n: int) -> np.ndarray:
    return make_gates((H, q) for q in range(n))


def ghz(n: int) -> np.ndarray:
    return make_gates([(H, 0)] + [(CX, q, q + 1) for q in range(n - 1)])


def basis_prep(n: int, x: int) -> np.ndarray:
    """X on every set bit of x: maps |0...0> to |x>."""
    return make_gates((X, q) for q in range(n) if (x >> q) & 1)


def qft(n: int) -> np.ndarray:
    """Textbook QFT on little-endian qubits (qubit n-1 most significant):
    H on each qubit from the top down, each followed by controlled phases
    pi/2^d from the lower qubits, then the qubit-order reversal."""
    items = []
    for j in range(n - 1, -1, -1):
        items.append((H, j))
        for k in range(j - 1, -1, -1):
            items.append((CP, k, j, math.pi / float(2 ** (j - k))))
    for i in range(n // 2):
        items.append((SWAP, i, n - 1 - i))
    return make_gates(items)


def adjoint(gates: np.ndarray) -> np.ndarray:
    """The inverse circuit: reversed order, each gate replaced by its inverse
    (self-inverse gates unchanged, rotation angles negated, and
    U3(t, p, l)^-1 = U3(-t, -l, -p))."""
    out = gates[::-1].copy()
    for g in out:
        t = int(g["type"])
        if t in (RX, RZ, CP, RXX):
            g["p0"] = -g["p0"]
        elif t == U3:
            th, ph, la = float(g["p0"]), float(g["p1"]), float(g["p2"])
            g["p0"], g["p1"], g["p2"] = -th, -la, -ph
    return out


def concat(*parts: np.ndarray) -> np.ndarray:
    return np.concatenate([p.astype(GATE_DTYPE) for p in parts])


def describe(gates: np.ndarray) -> str:
    counts = {}
    for t in gates["type"]:
        counts[NAMES[int(t)]] = counts.get(NAMES[int(t)], 0) + 1
    return ", ".join(f"{k}:{v}" for k, v in sorted(counts.items()))
