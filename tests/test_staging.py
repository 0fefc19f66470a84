"""Staged plans (Alg. 1's Partition, Sec. 4) on the CPU: the stager's
invariants checked by oracle/plan.check_stages, and the staged execution
order applied gate by gate with the FP64 oracle equals the circuit."""
import numpy as np
import pytest

from oracle import plan as OP
from oracle import sim
from synth import circuits as C

Q = pytest.importorskip("paper_2408_09055_gb300.qsim")

KERNELIZE, ORDERED = 3, 2


def stages_of(p):
    out = []
    for st in p.stages():
        local = [q for q in range(64) if (st["local_mask"] >> q) & 1]
        ks = []
        for k in range(st["first_kernel"], st["first_kernel"] + st["num_kernels"]):
            d = p.kernel(k)
            kq = [q for q in range(64) if (d.qubit_mask >> q) & 1]
            ks.append((d.type, kq, p.kernel_gates(k)))
            assert d.stage == len(out)
        out.append((local, ks))
    return out


CASES = [
    (16, 12, lambda s: C.mixed_circuit(16, 400, s)),
    (18, 13, lambda s: C.entangling_circuit(18, 6, s)),
    (20, 16, lambda s: C.mixed_circuit(20, 600, s)),
    (15, 12, lambda s: C.qft(15)),
    (14, 12, lambda s: C.layered_u3_cz(14, 8, s)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("algo", [ORDERED, KERNELIZE])
def test_staged_plan_invariants(case, algo):
    n, L, make = CASES[case]
    g = make(case)
    p = Q.Plan(n, g, algo=algo, local_qubits=L, shm_max_active=min(12, L), fuse_kmax=4, shm_variant=2)
    assert p.validate() == 0
    st = p.stats()
    assert st.num_stages == len(p.stages()) >= 1
    assert sum(s["num_gates"] for s in p.stages()) == len(g)
    assert sum(s["num_kernels"] for s in p.stages()) == st.num_kernels
    OP.check_stages(g, stages_of(p), L)


def test_staged_execution_order_is_the_circuit():
    n, L = 14, 12
    g = C.mixed_circuit(n, 300, 5)
    p = Q.Plan(n, g, local_qubits=L, shm_max_active=12, fuse_kmax=4, shm_variant=2)
    assert p.stats().num_stages > 1
    order = [i for k in p.kernels() for i in k]
    assert order != list(range(len(g)))  # the stager moved gates
    a = sim.apply(n, g)
    b = sim.apply(n, g[order])
    assert np.max(np.abs(a - b)) < 1e-12


def test_a_gate_on_regional_qubits_only_through_insular_qubits():
    # CZ / CP / RZ are insular in every qubit: they never force a qubit local
    n, L = 14, 12
    g = C.make_gates([(C.H, 13), (C.H, 12), (C.CZ, 12, 13), (C.CP, 13, 0, 0.3), (C.RZ, 12, None, 0.2),
                      (C.H, 0)])
    p = Q.Plan(n, g, local_qubits=L, shm_max_active=12, fuse_kmax=4, shm_variant=2)
    OP.check_stages(g, stages_of(p), L)


def test_stage_count_is_one_when_every_qubit_fits():
    n = 16
    g = C.mixed_circuit(n, 200, 3)
    p = Q.Plan(n, g, local_qubits=n, shm_variant=2)
    assert p.stats().num_stages == 1 and p.stage(0)["local_mask"] == (1 << n) - 1


@pytest.mark.parametrize("L,kw", [(11, {}), (12, {"shm_max_active": 13}), (12, {"forced_low": 11})])
def test_staged_options_are_checked(L, kw):
    with pytest.raises(Q.QsError):
        Q.Plan(16, C.mixed_circuit(16, 50, 0), local_qubits=L, **kw)


def test_ghz_needs_a_stage_per_new_high_target():
    # a CX chain walks its target up the register: with L local qubits,
    # (n - L) qubits stay regional and at least one restage is needed
    n, L = 16, 12
    g = C.ghz(n)
    p = Q.Plan(n, g, local_qubits=L, shm_max_active=12, shm_variant=2)
    OP.check_stages(g, stages_of(p), L)
    assert p.stats().num_stages >= 2


def test_staged_plan_has_no_resident_form():
    # qs_run_plan and timers are refused before any device work
    n = 16
    p = Q.Plan(n, C.mixed_circuit(n, 80, 2), local_qubits=12, shm_max_active=12, shm_variant=2)
    st = Q.State(n, 1 << 20)  # an aligned address the library never touches here
    with pytest.raises(Q.QsError) as e:
        st.run(p)
    assert e.value.status == -3
    with pytest.raises(Q.QsError):
        Q.Timer(p, 1)


def test_host_run_rejects_bad_arguments_before_device_work():
    # a misaligned or missing host state is refused before any CUDA call
    n = 14
    p = Q.Plan(n, C.mixed_circuit(n, 40, 3), local_qubits=12, shm_max_active=12, shm_variant=2)
    with pytest.raises(Q.QsError) as e:
        p.run_host(0)
    assert e.value.status == -1
    with pytest.raises(Q.QsError) as e:
        p.run_host(1 << 20 | 8)  # not 16-byte aligned
    assert e.value.status == -1
    assert Q._lib.qs_run_plan_host(None, None, None, 0, None) == -1


def test_staged_empty_circuit():
    n = 16
    p = Q.Plan(n, C.make_gates([]), local_qubits=12, shm_max_active=12, shm_variant=2)
    assert p.validate(C.make_gates([])) == 0
    assert p.stats().num_kernels == 0
    p.run_host(1 << 20)  # nothing to apply: returns before any device work


def _sparse_circuit(rng, n, ng):
    # all ten gate types, two-qubit gates only among a random subset of the
    # qubits: regional insular qubits (CZ, CP partners, CX controls) and lone
    # qubits both appear
    from synth.circuits import NPARAM, NQ
    pool = sorted(rng.choice(n, size=int(rng.integers(2, n)), replace=False).tolist())
    items = []
    for _ in range(ng):
        t = int(rng.integers(0, 10))
        th = list(rng.uniform(0, 6.28, size=NPARAM[t]))
        if NQ[t] == 2:
            a, b = rng.choice(pool, size=2, replace=False)
            items.append((t, int(a), int(b), *th))
        else:
            items.append((t, int(rng.integers(0, n)), None, *th))
    return C.make_gates(items)


@pytest.mark.parametrize("algo", [1, 2, 3])
def test_every_planner_stages_sparse_circuits(algo):
    # each planner keeps its kernels on the stage's local positions, also
    # when fused packing meets a regional insular qubit (the greedy packer
    # once grew a fused kernel onto one and then fit no kernel type)
    # (|A| <= 6 with four forced low qubits leaves two free active qubits:
    # there a fused kernel on a regional qubit fits no shared-memory kernel)
    rng = np.random.default_rng(7)
    for it in range(40):
        n = int(rng.integers(13, 17))
        L = int(rng.integers(12, n))
        g = _sparse_circuit(rng, n, int(rng.integers(20, 100)))
        p = Q.Plan(n, g, algo=algo, local_qubits=L, shm_max_active=6, fuse_kmax=6 if it % 2 else 4,
                   forced_low=4, shm_variant=1)
        assert p.validate() == 0
        OP.check_stages(g, stages_of(p), L)


@pytest.mark.parametrize("stager", [0, 1])
def test_many_regional_qubits_use_the_grown_local_set(stager):
    # with seven or more regional qubits the choices of local set exceed what
    # the stager enumerates; it grows one in circuit order instead, and the
    # exact search claims nothing
    rng = np.random.default_rng(3)
    for it in range(10):
        n = int(rng.integers(19, 23))
        L = int(rng.integers(12, n - 6))
        g = _sparse_circuit(rng, n, int(rng.integers(20, 200))) if it % 2 else C.mixed_circuit(n, 300, it)
        p = Q.Plan(n, g, local_qubits=L, shm_max_active=min(12, L), fuse_kmax=4, shm_variant=1, stager=stager)
        assert p.validate() == 0 and p.stats().staging_optimal == 0
        OP.check_stages(g, stages_of(p), L)
