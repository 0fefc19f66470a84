"""The staging ILP of Sec. 4 (oracle/stage_ilp.py), pinned by exhaustive
search and closed forms on tiny circuits, and the library's stager measured
against it: the stager may not use fewer stages than the ILP's optimum (that
would mean a broken ILP or a stage that breaks a dependency), and on these
seeded circuits it reaches that optimum."""
import numpy as np
import pytest

from oracle import plan as OP
from synth import circuits as C

pytest.importorskip("scipy.optimize")
SI = pytest.importorskip("oracle.stage_ilp")


def _check_ilp_staging(g, n, L, stages):
    # every stage: L local qubits, each gate's non-insular qubits local, and
    # the concatenation keeps every non-commuting pair in circuit order
    OP.check_stages(g, [(loc, [(0, OP.noninsular_qubits(g[i]), [i]) for i in ids]) for loc, ids in stages], L)


@pytest.mark.parametrize("seed", range(10))
def test_ilp_matches_exhaustive_search(seed):
    n, L = (6, 3) if seed % 2 else (7, 4)
    g = C.mixed_circuit(n, 12 + 2 * seed, seed)
    s, cost, stages = SI.stage(g, n, L)
    assert (s, cost) == SI.brute_force(g, n, L)
    _check_ilp_staging(g, n, L, stages)


def test_ilp_with_fixed_local_qubits_matches_exhaustive_search():
    for seed in range(4):
        g = C.mixed_circuit(7, 18, 40 + seed)
        s, cost, stages = SI.stage(g, 7, 4, fixed_local=(0, 1))
        assert (s, cost) == SI.brute_force(g, 7, 4, fixed_local=(0, 1))
        assert all({0, 1} <= set(loc) for loc, _ in stages)


def test_ilp_closed_forms():
    # a Hadamard on every qubit in turn: ceil(n / L) stages, and every qubit
    # outside the first stage becomes local exactly once (n - L)
    for n, L in ((6, 3), (6, 2), (5, 2), (7, 3)):
        s, cost, _ = SI.stage(C.hadamard_layer(n), n, L)
        assert (s, cost) == (-(-n // L), n - L)
    # diagonal gates have no non-insular qubit: one stage whatever L is
    g = C.make_gates([(C.CZ, 0, 5), (C.RZ, 3, None, 0.4), (C.CP, 1, 4, 0.2), (C.CZ, 2, 3)])
    assert SI.stage(g, 6, 1)[:2] == (1, 0)
    # CX needs only its target local: a fan-out from one control fits L = 1
    # only one target at a time
    g = C.make_gates([(C.CX, 0, t) for t in range(1, 5)])
    s, cost, stages = SI.stage(g, 5, 1)
    assert (s, cost) == (4, 3)
    assert [sorted(loc) for loc, _ in stages] == [[1], [2], [3], [4]]


def test_ilp_enforces_dependencies():
    # X(0), then CX(0 -> 1), then X(0): with L = 1 the middle gate needs
    # qubit 1 local, the others qubit 0, and no reordering is allowed
    g = C.make_gates([(C.X, 0), (C.CX, 0, 1), (C.X, 0)])
    s, _, stages = SI.stage(g, 2, 1)
    assert s == 3 and [ids for _, ids in stages] == [[0], [1], [2]]


Q = pytest.importorskip("paper_2408_09055_gb300.qsim")


def _library_stages(n, L, g):
    p = Q.Plan(n, g, local_qubits=L, shm_max_active=12, fuse_kmax=0, shm_variant=1)
    masks = [p.stage(k)["local_mask"] for k in range(p.stats().num_stages)]
    return len(masks), sum(bin(masks[k] & ~masks[k - 1]).count("1") for k in range(1, len(masks)))


CASES = [("mixed", 14, 12, 120, 0), ("mixed", 14, 12, 120, 2), ("mixed", 16, 12, 120, 3), ("mixed", 15, 13, 180, 4),
         ("layered", 16, 12, 3, 1), ("entangling", 16, 12, 2, 2), ("qft", 16, 12, 0, 0), ("mixed", 17, 14, 200, 5)]


@pytest.mark.parametrize("kind,n,L,size,seed", CASES)
def test_library_stager_reaches_the_ilp_stage_count(kind, n, L, size, seed):
    g = {"mixed": lambda: C.mixed_circuit(n, size, seed), "layered": lambda: C.layered_u3_cz(n, size, seed),
         "entangling": lambda: C.entangling_circuit(n, size, seed), "qft": lambda: C.qft(n)}[kind]()
    ours, our_cost = _library_stages(n, L, g)
    # the stager keeps the L - 8 lowest qubits local (long host runs)
    s, cost, _ = SI.stage(g, n, L, fixed_local=range(max(0, L - 8)))
    assert ours == s
    assert our_cost >= cost  # the ILP's objective is optimal for that count


def _make(kind, n, size, seed):
    return {"mixed": lambda: C.mixed_circuit(n, size, seed), "layered": lambda: C.layered_u3_cz(n, size, seed),
            "entangling": lambda: C.entangling_circuit(n, size, seed), "qft": lambda: C.qft(n)}[kind]()


@pytest.mark.parametrize("kind,n,L,size,seed", CASES)
def test_exact_stager_equals_the_ilp(kind, n, L, size, seed):
    # Theorem 1: the fewest stages, and at that count the ILP's objective;
    # the exact stager proves both within its default budget here
    g = _make(kind, n, size, seed)
    p = Q.Plan(n, g, local_qubits=L, shm_max_active=12, fuse_kmax=0, shm_variant=1, stager=Q.QS_STAGER_EXACT)
    st = p.stats()
    assert st.staging_optimal == 2  # both the count and the objective proven
    s, cost, _ = SI.stage(g, n, L, fixed_local=range(max(0, L - 8)))
    assert (st.num_stages, st.staging_cost) == (s, cost)
    assert p.validate() == 0
    masks = [p.stage(k)["local_mask"] for k in range(st.num_stages)]
    assert all(m & ((1 << (L - 8)) - 1) == (1 << (L - 8)) - 1 for m in masks)


def test_exact_stager_out_of_budget_keeps_the_beam_staging():
    g = C.mixed_circuit(16, 120, 3)
    beam = Q.Plan(16, g, local_qubits=12, shm_max_active=12, fuse_kmax=0, shm_variant=1)
    cut = Q.Plan(16, g, local_qubits=12, shm_max_active=12, fuse_kmax=0, shm_variant=1,
                 stager=Q.QS_STAGER_EXACT, stager_budget=1)
    assert cut.stats().staging_optimal == 0 and beam.stats().staging_optimal == 0
    assert [s["local_mask"] for s in cut.stages()] == [s["local_mask"] for s in beam.stages()]
    assert cut.stats().staging_cost == beam.stats().staging_cost


def test_staging_cost_counts_new_local_qubits():
    g = C.mixed_circuit(16, 200, 9)
    p = Q.Plan(16, g, local_qubits=12, shm_max_active=12, fuse_kmax=0, shm_variant=1)
    m = [s["local_mask"] for s in p.stages()]
    assert p.stats().staging_cost == sum(bin(m[k] & ~m[k - 1]).count("1") for k in range(1, len(m)))
    # unstaged plans have no boundary
    assert Q.Plan(16, g, shm_variant=1).stats().staging_cost == 0


def test_unknown_stager_is_rejected():
    with pytest.raises(Q.QsError) as e:
        Q.Plan(16, C.mixed_circuit(16, 50, 1), local_qubits=12, shm_max_active=12, stager=7)
    assert e.value.status == Q.QS_EINVAL


def test_exact_stager_claims_on_random_sparse_circuits():
    # whatever the exact stager claims proven must be the ILP's optimum; on
    # these sparse circuits (all gate types, lone and regional insular
    # qubits) it proves both the count and the objective
    from tests.test_staging import _sparse_circuit
    rng = np.random.default_rng(99)
    proven = 0
    for _ in range(20):
        n = int(rng.integers(13, 17))
        L = int(rng.integers(12, n))
        g = _sparse_circuit(rng, n, int(rng.integers(20, 120)))
        p = Q.Plan(n, g, local_qubits=L, shm_max_active=12, fuse_kmax=0, shm_variant=1, stager=Q.QS_STAGER_EXACT)
        st = p.stats()
        s, cost, _ = SI.stage(g, n, L, fixed_local=range(max(0, L - 8)), s_max=16)
        assert st.num_stages >= s
        if st.staging_optimal >= 1:
            assert st.num_stages == s
        if st.staging_optimal == 2:
            assert st.staging_cost == cost
            proven += 1
    assert proven >= 15
