"""Kernelization checks in plain Python -- test infrastructure only.

* :func:`check_plan` -- a plan (a sequence of kernels, each an ordered list of
  gate ids) is valid when every gate appears exactly once and the
  concatenated order is topologically equivalent to the circuit (Theorem 2):
  two gates that share a qubit keep their circuit order unless that qubit is
  insular for both (Definition 2: diagonal-in-the-qubit gates and control
  qubits; two gates that are both diagonal in every shared qubit commute).
* :func:`kernel_cost` -- the analytic cost of one kernel ("Cost Function in
  Kernelize"): a fusion kernel costs ``fuse_cost[|Qubits(K)|]``; a
  shared-memory kernel costs ``alpha + sum(gate_cost[type(g)])`` and its
  active set is the union of its gates' non-insular qubits plus the forced
  low qubits (footnote of that section); each kernel takes the cheaper
  feasible type.
* :func:`brute_force_contiguous` -- the optimum of Problem 1 over all
  2^(|C|-1) contiguous segmentations.
* :func:`brute_force_any_order` -- the optimum over all topologically
  equivalent orders and all segmentations of them (tiny circuits).
* :func:`extensible_by_definition` -- Definition 4 evaluated literally.
* :func:`check_stages` -- a staged plan (Sec. 4): every stage has exactly L
  local qubits, every gate of a stage has all its non-insular qubits local,
  every kernel stays inside its stage's local qubits, and the concatenated
  kernels form a valid plan of the whole circuit.
"""
from __future__ import annotations

from synth.circuits import NQ, RZ, CX, CZ, CP

INF = float("inf")


def gate_qubits(g) -> frozenset:
    t = int(g["type"])
    return frozenset([int(g["q0"])] if NQ[t] == 1 else [int(g["q0"]), int(g["q1"])])


def noninsular_qubits(g) -> frozenset:
    """Qubits that a gate touches neither diagonally nor as a control."""
    t = int(g["type"])
    if t in (RZ, CZ, CP):
        return frozenset()
    if t == CX:
        return frozenset([int(g["q1"])])
    return gate_qubits(g)


def insular_qubits(g) -> frozenset:
    return gate_qubits(g) - noninsular_qubits(g)


def must_precede(g1, g2) -> bool:
    """True when g1 (earlier in the circuit) and g2 do not commute."""
    shared = gate_qubits(g1) & gate_qubits(g2)
    return any(q in noninsular_qubits(g1) or q in noninsular_qubits(g2) for q in shared)


def check_plan(gates, kernels) -> None:
    """Raises AssertionError unless ``kernels`` is a valid plan of ``gates``."""
    order = [int(i) for k in kernels for i in k]
    assert sorted(order) == list(range(len(gates))), "every gate exactly once"
    pos = {g: p for p, g in enumerate(order)}
    last = {}  # qubit -> list of earlier gate ids on it
    for j in range(len(gates)):
        for q in gate_qubits(gates[j]):
            for i in last.get(q, []):
                if must_precede(gates[i], gates[j]):
                    assert pos[i] < pos[j], f"gate {i} must precede gate {j}"
            last.setdefault(q, []).append(j)


def check_stages(gates, stages, L) -> None:
    """``stages``: list of (local qubit set, [(kernel type, kernel qubit set,
    gate ids), ...]).  Kernel type 0 is shared-memory (its qubit set is the
    active set), 1 is fused (its qubit set is the fused targets)."""
    flat = []
    for local, kernels in stages:
        local = frozenset(local)
        assert len(local) == L, "a stage holds exactly L local qubits"
        for ktype, kq, ids in kernels:
            assert frozenset(kq) <= local, "kernel qubits are local"
            for i in ids:
                assert noninsular_qubits(gates[i]) <= local, f"gate {i}: non-insular qubit not local"
                if ktype == 1:
                    assert gate_qubits(gates[i]) <= frozenset(kq), f"gate {i} outside its fused kernel"
            flat.append(list(ids))
    check_plan(gates, flat)


class CostModel:
    def __init__(self, alpha, gate_cost, fuse_cost, shm_max, forced_low, fuse_kmax):
        self.alpha = float(alpha)
        self.gate_cost = list(gate_cost)  # indexed by gate type
        self.fuse_cost = list(fuse_cost)  # indexed by qubit count (entry 0 unused)
        self.shm_max = int(shm_max)
        self.forced_low = int(forced_low)
        self.fuse_kmax = int(fuse_kmax)

    def fusion(self, gates, ids):
        q = frozenset().union(*(gate_qubits(gates[i]) for i in ids))
        if len(q) > self.fuse_kmax:
            return INF
        return self.fuse_cost[len(q)]

    def shm(self, gates, ids):
        a = frozenset(range(self.forced_low)).union(*(noninsular_qubits(gates[i]) for i in ids))
        if len(a) > self.shm_max:
            return INF
        return self.alpha + sum(self.gate_cost[int(gates[i]["type"])] for i in ids)

    def kernel_cost(self, gates, ids):
        return min(self.fusion(gates, ids), self.shm(gates, ids))


def plan_cost(model: CostModel, gates, kernels) -> float:
    return sum(model.kernel_cost(gates, k) for k in kernels)


def brute_force_contiguous(model: CostModel, gates) -> float:
    """min over all segmentations of 0..L-1 into contiguous kernels."""
    L = len(gates)
    if L == 0:
        return 0.0
    best = INF
    for cuts in range(1 << (L - 1)):
        total, start = 0.0, 0
        for i in range(L):
            if i == L - 1 or (cuts >> i) & 1:
                total += model.kernel_cost(gates, list(range(start, i + 1)))
                start = i + 1
                if total >= best:
                    break
        best = min(best, total)
    return best


def topological_orders(gates):
    L = len(gates)
    preds = [set(i for i in range(j) if must_precede(gates[i], gates[j])) for j in range(L)]
    done, out, cur = set(), [], []

    def rec():
        if len(cur) == L:
            out.append(list(cur))
            return
        for j in range(L):
            if j not in done and preds[j] <= done:
                done.add(j); cur.append(j)
                rec()
                cur.pop(); done.discard(j)

    rec()
    return out


def brute_force_any_order(model: CostModel, gates) -> float:
    """min over every topologically equivalent order and every segmentation."""
    best = INF
    for order in topological_orders(gates):
        L = len(order)
        for cuts in range(1 << max(L - 1, 0)):
            total, start = 0.0, 0
            for i in range(L):
                if i == L - 1 or (cuts >> i) & 1:
                    total += model.kernel_cost(gates, order[start:i + 1])
                    start = i + 1
                    if total >= best:
                        break
            best = min(best, total)
    return best


def extensible_by_definition(gates, kernel_ids, i, nqubits) -> frozenset:
    """Definition 4: the qubits q for which adding a gate on q to the kernel
    K (its gates among C[0..i-1] are ``kernel_ids``) at position i keeps
    weak convexity and monotonicity."""
    K = set(kernel_ids)
    out = set()
    for q in range(nqubits):
        ok = True
        # weak convexity: no j1 < j2 < i, C[j1] in K, C[j2] not in K, q in both
        for j2 in range(i):
            if j2 in K or q not in gate_qubits(gates[j2]):
                continue
            if any(j1 < j2 and q in gate_qubits(gates[j1]) for j1 in K):
                ok = False
                break
        if ok:
            # monotonicity: C[j] not in K, j < i, shares a qubit with K|j  =>  q in Qubits(K|j)
            for j in range(i):
                if j in K:
                    continue
                kj = [g for g in K if g < j]
                qk = frozenset().union(*(gate_qubits(gates[g]) for g in kj)) if kj else frozenset()
                if gate_qubits(gates[j]) & qk and q not in qk:
                    ok = False
                    break
        if ok:
            out.add(q)
    return frozenset(out)
