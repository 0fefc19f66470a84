"""Planner checks on the CPU against oracle/plan.py (no GPU needed).

* every plan is valid (Theorem 2): each gate once, non-commuting pairs in
  circuit order -- checked by the library and independently by the oracle;
* OrderedKernelize (Alg. 5) reaches the brute-force optimum over all
  contiguous segmentations (Problem 1);
* Kernelize (Alg. 3) without pruning or gate attachment costs no more than
  OrderedKernelize (Theorem 6), and no less than the optimum over every
  topologically equivalent order;
* reported plan costs match the oracle's cost of the returned kernels.
"""
import numpy as np
import pytest

from oracle import plan as OP
from oracle import sim
from synth import circuits as C

Q = pytest.importorskip("paper_2408_09055_gb300.qsim")

ORDERED, KERNELIZE = 2, 3


def model_from(opts, table):
    return OP.CostModel(table.alpha, list(table.gate_cost), list(table.fuse_cost),
                        opts.shm_max_active, opts.forced_low, opts.fuse_kmax)


def circuits(seed):
    return [(8, C.mixed_circuit(8, 60, seed)), (10, C.entangling_circuit(10, 3, seed)),
            (12, C.layered_u3_cz(12, 4, seed)), (9, C.mixed_circuit(9, 120, seed + 7))]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("algo", [0, 1, ORDERED, KERNELIZE])
def test_every_plan_is_valid(seed, algo):
    for n, g in circuits(seed):
        for attach in (0, 1):
            for fk in (0, 4):
                p = Q.Plan(n, g, algo=algo, attach_single=attach, shm_variant=1, fuse_kmax=fk,
                           shm_max_active=6, prune_T=16 + 100 * seed)
                assert p.validate() == 0
                OP.check_plan(g, p.kernels())


def test_plan_validation_rejects_a_corrupted_plan():
    g = C.mixed_circuit(6, 20, 1)
    p = Q.Plan(6, g, algo=ORDERED, shm_variant=1, fuse_kmax=4, shm_max_active=6)
    ks = p.kernels()
    flat = [i for k in ks for i in k]
    bad = list(reversed(flat))
    with pytest.raises(AssertionError):
        OP.check_plan(g, [bad])
    assert p.validate(C.mixed_circuit(6, 20, 2)) != 0  # a different circuit


@pytest.mark.parametrize("seed", range(8))
def test_ordered_kernelize_is_optimal_over_contiguous_segmentations(seed):
    rng = np.random.default_rng(seed)
    n = 6
    g = C.mixed_circuit(n, 11, seed)
    table = Q.default_cost_table()
    table.alpha = float(rng.uniform(50, 150))
    for t in range(10):
        table.gate_cost[t] = float(rng.uniform(1, 30))
    for k in range(16):
        table.fuse_cost[k] = float(40 + 12 * k * k + rng.uniform(0, 5))
    opts = Q.default_opts(algo=ORDERED, shm_max_active=5, forced_low=2, fuse_kmax=4, fuse_kmin=1,
                          shm_variant=1, cost=table)
    p = Q.Plan(n, g, opts)
    m = model_from(opts, table)
    best = OP.brute_force_contiguous(m, g)
    assert abs(p.stats().cost - best) < 1e-6
    assert abs(OP.plan_cost(m, g, p.kernels()) - best) < 1e-6


@pytest.mark.parametrize("seed", range(10))
def test_kernelize_no_worse_than_ordered(seed):
    for n, g in [(8, C.mixed_circuit(8, 12, seed)), (6, C.entangling_circuit(6, 1, seed)),
                 (6, C.layered_u3_cz(6, 2, seed))]:
        for fk in (0, 4):
            o = Q.Plan(n, g, algo=ORDERED, fuse_kmax=fk, shm_max_active=6, shm_variant=1)
            k = Q.Plan(n, g, algo=KERNELIZE, fuse_kmax=fk, shm_max_active=6, shm_variant=1,
                       prune_T=0, attach_single=0)
            assert k.stats().cost <= o.stats().cost + 1e-9


@pytest.mark.parametrize("seed", range(6))
def test_kernelize_bounded_by_optimum_over_all_orders(seed):
    n = 5
    g = C.mixed_circuit(n, 7, seed)
    table = Q.default_cost_table()
    opts = Q.default_opts(algo=KERNELIZE, shm_max_active=5, forced_low=2, fuse_kmax=3, fuse_kmin=1,
                          prune_T=0, attach_single=0, shm_variant=1, cost=table)
    p = Q.Plan(n, g, opts)
    m = model_from(opts, table)
    opt = OP.brute_force_any_order(m, g)
    got = OP.plan_cost(m, g, p.kernels())
    assert opt <= got + 1e-9
    assert got <= p.stats().cost + 1e-9  # each kernel at its cheaper type


def test_kernelize_beats_ordered_on_the_benchmark_circuit():
    g = C.mixed_circuit(30, 5000, 100)
    o = Q.Plan(30, g, algo=ORDERED, fuse_kmax=0, shm_max_active=13, shm_variant=1).stats()
    k = Q.Plan(30, g, algo=KERNELIZE, fuse_kmax=0, shm_max_active=13, shm_variant=1).stats()
    assert k.num_kernels < o.num_kernels and k.cost < o.cost


def test_greedy_respects_its_width():
    g = C.entangling_circuit(12, 3, 0)
    p = Q.Plan(12, g, algo=1, fuse_kmax=5, shm_variant=1)
    for k in range(p.stats().num_kernels):
        ids = p.kernel_gates(k)
        qs = set()
        for i in ids:
            qs |= OP.gate_qubits(g[i])
        assert len(qs) <= 5


def test_plan_fused_matrix_matches_oracle():
    n = 8
    g = C.entangling_circuit(n, 2, 4)
    cost = Q.default_cost_table()
    for k in range(16):
        cost.fuse_cost[k] = 1.0
    plan = Q.Plan(n, g, algo=ORDERED, fuse_kmax=5, cost=cost, shm_variant=1)
    found = 0
    for k in range(plan.stats().num_kernels):
        d = plan.kernel(k)
        if d.type != Q.QS_KERNEL_FUSED:
            continue
        qubits = [q for q in range(n) if (d.qubit_mask >> q) & 1]
        u_ref = sim.kernel_unitary(g[plan.kernel_gates(k)], qubits)
        assert np.allclose(plan.fused_matrix(k), u_ref, atol=1e-12)
        found += 1
    assert found > 0


@pytest.mark.parametrize("precision", [0, 2])
def test_plan_fused_matrices_are_unitary(precision):
    # every fused kernel's FP64 product is unitary to 1e-12, widened kernels
    # (six targets for the tensor-core precisions) included
    n = 14
    cost = Q.default_cost_table()
    for k in range(16):
        cost.fuse_cost[k] = 1.0
    for g in (C.entangling_circuit(n, 3, 5), C.mixed_circuit(n, 200, 6), C.qft(n)):
        plan = Q.Plan(n, g, algo=ORDERED, fuse_kmax=6, cost=cost, precision=precision, shm_variant=1)
        for k in range(plan.stats().num_kernels):
            if plan.kernel(k).type != Q.QS_KERNEL_FUSED:
                continue
            u = plan.fused_matrix(k)
            assert np.max(np.abs(u @ u.conj().T - np.eye(len(u)))) <= 1e-12


def test_invalid_inputs_are_rejected():
    g = C.make_gates([(C.CX, 0, 1)])
    with pytest.raises(Q.QsError):
        Q.Plan(1, g)  # qubit 1 out of range
    with pytest.raises(Q.QsError):
        Q.Plan(4, g, shm_max_active=20)
    with pytest.raises(Q.QsError):
        Q.Plan(4, g, fuse_kmax=9)


@pytest.mark.parametrize("n", [14, 20, 34])
def test_lone_qubit_gates_do_not_overfill_a_unit(n):
    # a Hadamard on every qubit, then CX gates on a few: the other qubits'
    # Hadamards are only adjacent to single-qubit gates, so they attach to
    # the closest multi-qubit gate (App. A.2) -- but not past what a kernel
    # can hold; such a qubit's gates then form a unit of their own
    g = C.make_gates([(C.H, q) for q in range(n)] + [(C.CX, n - 1, 5), (C.CX, n - 2, 2), (C.H, 5)])
    for smax, kmax in ((12, 0), (10, 4), (14, 6)):
        plan = Q.Plan(n, g, algo=KERNELIZE, shm_max_active=smax, fuse_kmax=kmax, shm_variant=1)
        assert plan.validate() == 0
        OP.check_plan(g, plan.kernels())
    if n == 14:
        from tests.program_emulator import run_plan
        plan = Q.Plan(n, g, algo=KERNELIZE, shm_max_active=12, fuse_kmax=0, shm_variant=2)
        got = run_plan(plan, n, sim.zero_state(n))
        ref = sim.apply(n, g)
        assert np.max(np.abs(got - ref)) <= 1e-5
