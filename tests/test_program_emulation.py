"""CPU check of the shared-memory program compiler (phase scheduling, known
bits, gate fusion into 2x2 and 4x4 blocks, global-phase folding): every
kernel's register-phased program, executed by a plain numpy emulator of its
op semantics (tests/program_emulator.py), must reproduce the FP64 oracle.
No GPU is involved; the GPU parity tests run the same programs on the
device."""
import numpy as np
import pytest

from oracle import sim
from synth import circuits as C
from tests.program_emulator import run_plan

Q = pytest.importorskip("paper_2408_09055_gb300.qsim")


def _random_state(n, seed):
    rng = np.random.default_rng(seed)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return psi / np.linalg.norm(psi)


CIRCUITS = {
    "mixed": lambda n, s: C.mixed_circuit(n, 250, s),
    "entangling": lambda n, s: C.entangling_circuit(n, 4, s),
    "layered": lambda n, s: C.layered_u3_cz(n, 5, s),
    "qft": lambda n, s: C.qft(n),
}


@pytest.mark.parametrize("kind", list(CIRCUITS))
@pytest.mark.parametrize("algo,smax", [(2, 10), (3, 12), (3, 14), (1, 11)])
@pytest.mark.parametrize("n", [12, 14])
def test_programs_reproduce_the_oracle(kind, algo, smax, n):
    g = CIRCUITS[kind](n, n + smax)
    plan = Q.Plan(n, g, algo=algo, fuse_kmax=0, shm_max_active=smax, shm_variant=2)
    psi0 = _random_state(n, 3 * n + smax)
    got = run_plan(plan, n, psi0.copy())
    ref = sim.apply(n, g, psi0.copy())
    fid = abs(np.vdot(ref, got)) ** 2 / (np.vdot(got, got).real * np.vdot(ref, ref).real)
    assert fid >= 1 - 1e-6, fid
    assert np.max(np.abs(got - ref)) <= 1e-5


def test_fusion_produces_dense_two_slot_blocks():
    # the entangling circuit's CP/RXX pairs with their one-qubit gates become
    # PK_G2 ops; the emulator above checks their values
    n = 14
    g = C.entangling_circuit(n, 6, 1)
    plan = Q.Plan(n, g, fuse_kmax=0, shm_max_active=12, shm_variant=2)
    g2 = 0
    for k in range(plan.stats().num_kernels):
        words, _, _, _ = plan.kernel_program(k)
        pc = 0
        sizes = {0: 0, 1: 9, 2: 5, 3: 5, 4: 9, 5: 1, 6: 1, 7: 1, 8: 5, 9: 3, 10: 9, 11: 9, 12: 3, 13: 9,
                 14: 1, 15: 3, 16: 3, 18: 33}
        while True:
            op = int(words[pc]) & 0xFF
            if op == 0:
                break
            if op == 18:
                g2 += 1
            pc += (1 + 5 + ((int(words[pc]) >> 8) & 0xFF)) if op == 17 else sizes[op]
    assert g2 > 0


@pytest.mark.parametrize("n,L,kind", [(14, 12, "mixed"), (16, 12, "entangling"), (15, 13, "layered"),
                                      (14, 12, "qft")])
def test_staged_programs_reproduce_the_oracle(n, L, kind):
    # a stage's programs address its chunk view: positions 0..L-1 are the
    # local qubits in ascending order, L..n-1 the regional ones; running them
    # on the whole permuted state covers every chunk (the regional bits are
    # the batch bits above L)
    from tests.program_emulator import run_kernel
    g = CIRCUITS[kind](n, 7 * n + L)
    plan = Q.Plan(n, g, fuse_kmax=0, local_qubits=L, shm_max_active=min(12, L), shm_variant=2)
    assert plan.stats().num_stages > 1
    psi = _random_state(n, n + L)
    ref = sim.apply(n, g, psi.copy())
    idx = np.arange(1 << n)
    for si in range(plan.stats().num_stages):
        st = plan.stage(si)
        local = [q for q in range(n) if (st["local_mask"] >> q) & 1]
        order = local + [q for q in range(n) if not (st["local_mask"] >> q) & 1]
        # view index v has bit p = logical qubit order[p]
        logical = np.zeros_like(idx)
        for p, q in enumerate(order):
            logical |= ((idx >> p) & 1) << q
        view = psi[logical]
        for k in range(st["first_kernel"], st["first_kernel"] + st["num_kernels"]):
            words, m, act, R = plan.kernel_program(k)
            assert max(act) < L  # every kernel stays inside the chunk
            run_kernel(view, n, words, m, act, R)
        psi[logical] = view
    fid = abs(np.vdot(ref, psi)) ** 2 / (np.vdot(psi, psi).real * np.vdot(ref, ref).real)
    assert fid >= 1 - 1e-6, fid
    assert np.max(np.abs(psi - ref)) <= 1e-5


def _apply_unitary(psi, n, qubits, u):
    # psi[.. index bit qubits[j] ..] <- sum over the target bits of u[r, c]
    # (index bit j of r and c = qubits[j]); plain gather / matmul / scatter
    k = len(qubits)
    sub = np.zeros(1 << k, dtype=np.int64)
    for j, q in enumerate(qubits):
        sub |= ((np.arange(1 << k) >> j) & 1) << q
    rest = [q for q in range(n) if q not in qubits]
    base = np.zeros(1 << (n - k), dtype=np.int64)
    for j, q in enumerate(rest):
        base |= ((np.arange(1 << (n - k)) >> j) & 1) << q
    idx = base[:, None] | sub[None, :]
    psi[idx] = psi[idx] @ u.T


def _run_mixed(plan, n, psi, kernels, qubit_pos):
    from tests.program_emulator import run_kernel
    for k in kernels:
        d = plan.kernel(k)
        if d.type == Q.QS_KERNEL_FUSED:
            qubits = [qubit_pos[q] for q in range(n) if (d.qubit_mask >> q) & 1]
            _apply_unitary(psi, n, qubits, plan.fused_matrix(k))
        else:
            words, m, act, R = plan.kernel_program(k)
            run_kernel(psi, n, words, m, act, R)


@pytest.mark.parametrize("kind", list(CIRCUITS))
@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("n,L", [(14, 0), (16, 0), (14, 12), (16, 12)])
def test_mixed_plans_reproduce_the_oracle(kind, precision, n, L):
    # fusion made cheap enough that the planner mixes fused and shared-memory
    # kernels: the fused kernels' FP64 unitaries (widened to six targets for
    # the tensor-core precisions) and the programs, applied in plan order,
    # must reproduce the oracle; staged plans run on the stage's chunk view
    g = CIRCUITS[kind](n, 5 * n + L + precision)
    cost = Q.default_cost_table()
    for k in range(16):
        cost.fuse_cost[k] *= 0.3
    kw = dict(precision=precision, shm_max_active=12, shm_variant=2, cost=cost)
    if L:
        kw["local_qubits"] = L
    plan = Q.Plan(n, g, **kw)
    psi = _random_state(n, 11 * n + L + precision)
    ref = sim.apply(n, g, psi.copy())
    s = plan.stats()
    if not L:
        _run_mixed(plan, n, psi, range(s.num_kernels), list(range(n)))
    else:
        idx = np.arange(1 << n)
        for si in range(s.num_stages):
            st = plan.stage(si)
            local = [q for q in range(n) if (st["local_mask"] >> q) & 1]
            order = local + [q for q in range(n) if not (st["local_mask"] >> q) & 1]
            logical = np.zeros_like(idx)
            for p, q in enumerate(order):
                logical |= ((idx >> p) & 1) << q
            pos = {q: p for p, q in enumerate(order)}
            view = psi[logical]
            ks = range(st["first_kernel"], st["first_kernel"] + st["num_kernels"])
            for k in ks:
                d = plan.kernel(k)
                assert d.qubit_mask & ~st["local_mask"] == 0  # inside the chunk
            _run_mixed(plan, n, view, ks, pos)
            psi[logical] = view
    if precision:
        for k in range(s.num_kernels):
            d = plan.kernel(k)
            if d.type == Q.QS_KERNEL_FUSED:
                assert d.nqubits >= min(6, n) and plan.fused_matrix(k).shape == (1 << d.nqubits,) * 2
    fid = abs(np.vdot(ref, psi)) ** 2 / (np.vdot(psi, psi).real * np.vdot(ref, ref).real)
    assert fid >= 1 - 1e-6, fid
    assert np.max(np.abs(psi - ref)) <= 1e-5


def _stress_circuit(style, m, rng):
    import itertools
    items = []
    if style == "allpairs":  # every pair of the active set, dense and diagonal
        for a, b in itertools.combinations(range(m), 2):
            items += [(C.CX, a, b), (C.U3, a, None, 0.3, 0.2, 0.1), (C.CP, b, a, 0.7)]
    elif style == "swaps":  # register permutations across every phase
        for _ in range(300):
            a, b = rng.choice(m, size=2, replace=False)
            items += [(C.SWAP, int(a), int(b)), (C.H, int(rng.integers(0, m)), None)]
    else:  # the forced low qubits only: one long in-phase fusion run
        for _ in range(300):
            a, b = rng.choice(4, size=2, replace=False)
            items.append((int(rng.choice([C.CX, C.CZ, C.RXX, C.SWAP])), int(a), int(b), 0.5))
    return C.make_gates(items)


@pytest.mark.parametrize("style", ["allpairs", "swaps", "lowonly"])
@pytest.mark.parametrize("m", [10, 14])
def test_programs_under_stress(style, m):
    # long runs of two-qubit gates over a full active set stress the phase
    # scheduler and the in-phase fusion; the emulated programs must still
    # reproduce the oracle
    from tests.program_emulator import run_any_plan
    rng = np.random.default_rng(m)
    n = m + 1
    g = _stress_circuit(style, m, rng)
    for algo in (2, 3):
        p = Q.Plan(n, g, algo=algo, shm_max_active=m, fuse_kmax=0, shm_variant=2)
        psi0 = _random_state(n, 7 * m + algo)
        got = run_any_plan(p, n, psi0.copy())
        assert got is not None
        assert np.max(np.abs(got - sim.apply(n, g, psi0.copy()))) <= 1e-5
