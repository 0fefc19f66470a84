"""The staging ILP of Sec. 4 (Eq. 2 and its constraints, Alg. 2), written out
as a binary program for ``scipy.optimize.milp`` -- test infrastructure only:
the library's stager is checked against it, nothing in the library calls it.

One GPU holds every stage, so there are no global qubits (G = 0): the
global-qubit variables B and their update indicators T are identically zero
and drop out, and the objective is the number of qubits that become local
from one stage to the next.  Variables, all binary:

* ``A[q, k]`` -- logical qubit q is local in stage k (0 <= k < s);
* ``F[g, k]`` -- gate g is finished by the end of stage k;
* ``S[q, k]`` -- qubit q becomes local from stage k to stage k + 1.

Constraints (the paper's, with G = 0): S[q, k] >= A[q, k+1] - A[q, k];
F[g, k] <= F[g, k+1]; F[g, k] <= F[g, k-1] + A[q, k] for every non-insular
qubit q of g (F[g, -1] = 0); F[g1, k] >= F[g2, k] for every pair of gates
adjacent on a qubit (g1 first); F[g, s-1] = 1; sum_q A[q, k] = L.
``fixed_local`` adds A[q, k] = 1 for the given qubits, the restriction the
library's stager places on the lowest qubits (not part of the paper's ILP).

:func:`stage` is Alg. 2: the smallest s whose program is feasible, and an
optimal assignment for it.  :func:`brute_force` finds the fewest stages and
the least cost at that count by trying every sequence of local sets, each
stage taking every gate it can -- the pin for tiny circuits.
"""
from __future__ import annotations

import itertools

import numpy as np

from oracle.plan import gate_qubits, noninsular_qubits


def adjacent_pairs(gates):
    """E: (earlier, later) for gates that touch a qubit one after the other."""
    last, pairs = {}, set()
    for j in range(len(gates)):
        for q in gate_qubits(gates[j]):
            if q in last:
                pairs.add((last[q], j))
            last[q] = j
    return sorted(pairs)


def solve(gates, n, L, s, fixed_local=()):
    """The program for exactly s stages.  Returns None when infeasible, else
    (cost, local sets, stage of each gate)."""
    from scipy.optimize import Bounds, LinearConstraint, milp
    from scipy.sparse import lil_matrix

    ng = len(gates)
    nA, nF, nS = n * s, ng * s, n * max(s - 1, 0)
    nv = nA + nF + nS
    iA = lambda q, k: q * s + k  # noqa: E731
    iF = lambda g, k: nA + g * s + k  # noqa: E731
    iS = lambda q, k: nA + nF + q * (s - 1) + k  # noqa: E731
    rows, lo, hi = [], [], []

    def add(coefs, lb, ub):
        rows.append(coefs)
        lo.append(lb)
        hi.append(ub)

    for q in range(n):
        for k in range(s - 1):
            add({iA(q, k + 1): 1, iA(q, k): -1, iS(q, k): -1}, -np.inf, 0)
    for g in range(ng):
        for k in range(s - 1):
            add({iF(g, k): 1, iF(g, k + 1): -1}, -np.inf, 0)
        for q in noninsular_qubits(gates[g]):
            for k in range(s):
                c = {iF(g, k): 1, iA(q, k): -1}
                if k > 0:
                    c[iF(g, k - 1)] = -1
                add(c, -np.inf, 0)
        add({iF(g, s - 1): 1}, 1, 1)
    for g1, g2 in adjacent_pairs(gates):
        for k in range(s):
            add({iF(g2, k): 1, iF(g1, k): -1}, -np.inf, 0)
    for k in range(s):
        add({iA(q, k): 1 for q in range(n)}, L, L)
        for q in fixed_local:
            add({iA(q, k): 1}, 1, 1)
    M = lil_matrix((len(rows), nv))
    for r, coefs in enumerate(rows):
        for v, c in coefs.items():
            M[r, v] = c
    cost = np.zeros(nv)
    cost[nA + nF:] = 1.0
    res = milp(cost, constraints=LinearConstraint(M.tocsr(), lo, hi), integrality=np.ones(nv),
               bounds=Bounds(0, 1))
    if res.status != 0:
        return None
    x = np.round(res.x).astype(int)
    local = [frozenset(q for q in range(n) if x[iA(q, k)]) for k in range(s)]
    stage_of = [min(k for k in range(s) if x[iF(g, k)]) for g in range(ng)]
    return int(round(res.fun)), local, stage_of


def stage(gates, n, L, fixed_local=(), s_max=16):
    """Alg. 2: s = 1, 2, ... until the program is feasible.  Returns
    (s, cost, stages) with stages a list of (local set, gate ids in circuit
    order)."""
    for s in range(1, s_max + 1):
        r = solve(gates, n, L, s, fixed_local)
        if r is not None:
            cost, local, stage_of = r
            stages = [(local[k], [g for g in range(len(gates)) if stage_of[g] == k]) for k in range(s)]
            return s, cost, stages
    raise ValueError(f"no staging within {s_max} stages")


def take(gates, done, S):
    """Every gate a stage with local set S can finish after the gates in
    `done`: in circuit order, a gate is taken when its non-insular qubits are
    local and no earlier unfinished gate it follows on a qubit was left."""
    blocked, out = set(), set(done)
    for g in range(len(gates)):
        if g in done:
            continue
        q = gate_qubits(gates[g])
        if q & blocked or not noninsular_qubits(gates[g]) <= S:
            blocked |= q
        else:
            out.add(g)
    return frozenset(out)


def brute_force(gates, n, L, fixed_local=(), s_max=6):
    """(fewest stages, least objective at that count), over every sequence
    of local sets (tiny n only)."""
    fixed = frozenset(fixed_local)
    sets = [frozenset(c) for c in itertools.combinations(range(n), L) if fixed <= frozenset(c)]
    everything = frozenset(range(len(gates)))
    # layer k: (done set, local set of stage k) -> least cost so far
    layer = {}
    for S in sets:
        key = (take(gates, frozenset(), S), S)
        layer[key] = 0
    for s in range(1, s_max + 1):
        best = [c for (d, _), c in layer.items() if d == everything]
        if best:
            return s, min(best)
        nxt = {}
        for (d, S0), c in layer.items():
            for S in sets:
                key = (take(gates, d, S), S)
                v = c + len(S - S0)
                if nxt.get(key, v + 1) > v:
                    nxt[key] = v
        layer = nxt
    raise ValueError(f"no staging within {s_max} stages")
