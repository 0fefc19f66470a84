"""Anti-diagonal insular gates in staging (App. A.2, Definition 2).

With qs_plan_opts.insular_x an X gate on a regional qubit is executed as a
relabelling of the stage's chunks: the stage's later controls and diagonal
factors on that qubit are conjugated (the control flip of App. A.2), and each
stored chunk is written back to the host chunk with the flipped bits.  Here
every stage's programs (and fused unitaries) run on the state permuted into
the stage's chunk view, the view is written back through the frame, and the
result must equal the FP64 oracle's; the plans pass Theorem 2's check with X
insular.  No GPU is needed.
"""
import numpy as np
import pytest

from oracle import sim
from synth import circuits as C

Q = pytest.importorskip("paper_2408_09055_gb300.qsim")


def _random_state(n, seed):
    rng = np.random.default_rng(seed)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return psi / np.linalg.norm(psi)


def _apply_unitary(psi, n, qubits, u):
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


def _emulate_staged(plan, n, psi):
    from tests.program_emulator import run_kernel
    idx = np.arange(1 << n)
    frames = 0
    for si in range(plan.stats().num_stages):
        st = plan.stage(si)
        frame, flips = plan.stage_frame(si)
        assert frame & st["local_mask"] == 0  # only regional qubits are relabelled
        frames += frame != 0
        local = [q for q in range(n) if (st["local_mask"] >> q) & 1]
        order = local + [q for q in range(n) if not (st["local_mask"] >> q) & 1]
        pos = {q: p for p, q in enumerate(order)}
        logical = np.zeros_like(idx)
        for p, q in enumerate(order):
            logical |= ((idx >> p) & 1) << q
        view = psi[logical]
        for k in range(st["first_kernel"], st["first_kernel"] + st["num_kernels"]):
            d = plan.kernel(k)
            assert d.qubit_mask & ~st["local_mask"] == 0
            if d.type == Q.QS_KERNEL_FUSED:
                qubits = [pos[q] for q in range(n) if (d.qubit_mask >> q) & 1]
                _apply_unitary(view, n, qubits, plan.fused_matrix(k))
            else:
                words, m, act, R = plan.kernel_program(k)
                run_kernel(view, n, words, m, act, R)
        psi[logical ^ frame] = view  # stored chunk c -> logical chunk c ^ frame
    return frames


def _rule_circuit(n, L, seed):
    """Dense gates on the low L qubits, then X on the two regional qubits
    followed by every insular use of them (controls, CZ, CP, RZ, both
    flipped together), then dense gates that make them local later."""
    rng = np.random.default_rng(seed)
    a, b = n - 1, n - 2
    items = [(C.H, q, None, 0, 0, 0) for q in range(L)]
    items += [(C.X, a, None, 0, 0, 0), (C.CZ, a, 2, 0, 0, 0), (C.CP, 5, a, rng.uniform(0, 6.28), 0, 0),
              (C.CX, a, 3, 0, 0, 0), (C.RZ, a, None, rng.uniform(0, 6.28), 0, 0),
              (C.X, b, None, 0, 0, 0), (C.CZ, a, b, 0, 0, 0), (C.CP, b, a, rng.uniform(0, 6.28), 0, 0),
              (C.CX, b, 7, 0, 0, 0), (C.RZ, b, None, rng.uniform(0, 6.28), 0, 0),
              (C.X, a, None, 0, 0, 0), (C.CP, a, 1, rng.uniform(0, 6.28), 0, 0)]
    items += [(C.U3, q, None, *rng.uniform(0, 6.28, 3)) for q in range(L)]
    items += [(C.H, a, None, 0, 0, 0), (C.H, b, None, 0, 0, 0), (C.CX, a, 0, 0, 0, 0), (C.CZ, b, 4, 0, 0, 0)]
    return C.make_gates(items)


@pytest.mark.parametrize("fuse", [0, 6])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_every_conjugation_rule_reproduces_the_oracle(seed, fuse):
    n, L = 14, 12
    g = _rule_circuit(n, L, seed)
    kw = dict(local_qubits=L, shm_max_active=12, shm_variant=2, insular_x=Q.QS_INSULAR_X_STAGED,
              fuse_kmax=fuse)
    if fuse:
        cost = Q.default_cost_table()
        for k in range(16):
            cost.fuse_cost[k] *= 0.3
        kw["cost"] = cost
    plan = Q.Plan(n, g, **kw)
    assert plan.validate(g) == 0
    psi = _random_state(n, seed)
    ref = sim.apply(n, g, psi.copy())
    frames = _emulate_staged(plan, n, psi)
    assert frames >= 1  # the X gates on the regional qubits became relabellings
    fid = abs(np.vdot(ref, psi)) ** 2 / (np.vdot(psi, psi).real * np.vdot(ref, ref).real)
    assert fid >= 1 - 1e-6, fid
    assert np.max(np.abs(psi - ref)) <= 1e-5


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("kind,n,L", [("mixed", 14, 12), ("mixed", 16, 12), ("mixed", 16, 13),
                                      ("layered", 15, 12)])
def test_staged_mixed_circuits_with_insular_x(kind, n, L, mode):
    g = C.mixed_circuit(n, 400, 3 * n + L) if kind == "mixed" else C.layered_u3_cz(n, 6, n + L)
    if kind == "layered":  # X layers between the U3/CZ layers
        extra = C.make_gates([(C.X, q, None, 0, 0, 0) for q in range(0, n, 2)])
        g = C.concat(g[: len(g) // 2], extra, g[len(g) // 2:], extra)
    plan = Q.Plan(n, g, local_qubits=L, shm_max_active=12, shm_variant=2, insular_x=mode)
    assert plan.validate(g) == 0
    psi = _random_state(n, 5 * n + L)
    ref = sim.apply(n, g, psi.copy())
    _emulate_staged(plan, n, psi)
    fid = abs(np.vdot(ref, psi)) ** 2 / (np.vdot(psi, psi).real * np.vdot(ref, ref).real)
    assert fid >= 1 - 1e-6, fid
    assert np.max(np.abs(psi - ref)) <= 1e-5


def test_insular_x_never_needs_more_stages_on_mixed_circuits():
    # X no longer forces its qubit local, so a stage admits at least the
    # gates it did; on these circuits that saves stages or ties
    for seed, (n, L) in enumerate([(20, 14), (22, 16), (24, 16), (24, 18)]):
        g = C.mixed_circuit(n, 1500, 40 + seed)
        a = Q.Plan(n, g, local_qubits=L, shm_max_active=12, fuse_kmax=0, shm_variant=2).stats().num_stages
        b = Q.Plan(n, g, local_qubits=L, shm_max_active=12, fuse_kmax=0, shm_variant=2,
                   insular_x=Q.QS_INSULAR_X_STAGED).stats().num_stages
        assert b <= a, (n, L, a, b)


def test_frame_export_on_unstaged_and_bad_stage():
    g = C.mixed_circuit(12, 50, 1)
    plan = Q.Plan(12, g)
    assert plan.stage_frame(0) == (0, [])
    with pytest.raises(Q.QsError):
        plan.stage_frame(1)


def _random_all_types(n, count, seed):
    rng = np.random.default_rng(seed)
    items = []
    for _ in range(count):
        t = int(rng.integers(0, 10))
        a = int(rng.integers(0, n))
        if t >= C.CX:
            b = int(rng.integers(0, n - 1))
            b += b >= a
            items.append((t, a, b, *rng.uniform(0, 6.28, 3)))
        else:
            items.append((t, a, None, *rng.uniform(0, 6.28, 3)))
        if rng.uniform() < 0.3:  # plenty of X gates
            items.append((C.X, int(rng.integers(0, n)), None, 0, 0, 0))
    return C.make_gates(items)


@pytest.mark.parametrize("seed", range(12))
def test_pauli_frame_rewrite_is_the_same_circuit(seed):
    # every X moves to the end through the frame; the rewritten circuit must
    # give the oracle's state exactly (global phase included)
    n = 6 + seed % 4
    g = _random_all_types(n, 120, seed)
    r = Q.qs_insular_x_rewrite(n, g)
    a = sim.apply(n, g)
    b = sim.apply(n, r)
    assert np.max(np.abs(a - b)) < 1e-12
    # no X before the final frame layer (and the phase fix on qubit 0)
    types = list(r["type"])
    first_x = types.index(C.X) if C.X in types else len(types)
    assert all(t in (C.X, C.RZ, C.U3) for t in types[first_x:])
    assert sum(1 for t in types[:first_x] if t == C.X) == 0


@pytest.mark.parametrize("seed", range(4))
def test_pauli_frame_closed_forms(seed):
    # X H = H Z: an X then H leaves a Z frame; H X H = Z exactly
    n = 3
    g = C.make_gates([(C.H, 0, None, 0, 0, 0), (C.X, 0, None, 0, 0, 0), (C.H, 0, None, 0, 0, 0)])
    r = Q.qs_insular_x_rewrite(n, g)
    assert C.X not in list(r["type"][:2])
    assert np.max(np.abs(sim.apply(n, g) - sim.apply(n, r))) < 1e-14
    # an X on a CX control followed by the CX: the frame spreads to the target
    g = C.make_gates([(C.X, 1, None, 0, 0, 0), (C.CX, 1, 2, 0, 0, 0), (C.RZ, 2, None, 0.7, 0, 0)])
    r = Q.qs_insular_x_rewrite(n, g)
    assert list(r["type"][:2]) == [C.CX, C.RZ] and r["p0"][1] == -0.7
    assert np.max(np.abs(sim.apply(n, g) - sim.apply(n, r))) < 1e-14


@pytest.mark.parametrize("kind", ["mixed", "entangling", "all"])
def test_insular_x_plans_reproduce_the_oracle(kind):
    from tests.program_emulator import run_kernel
    n = 14
    g = {"mixed": lambda: C.mixed_circuit(n, 500, 5), "entangling": lambda: C.entangling_circuit(n, 4, 6),
         "all": lambda: _random_all_types(n, 300, 7)}[kind]()
    cost = Q.default_cost_table()
    for k in range(16):
        cost.fuse_cost[k] *= 0.3
    plan = Q.Plan(n, g, shm_max_active=12, shm_variant=2, insular_x=Q.QS_INSULAR_X_REWRITE, cost=cost)
    assert plan.validate(g) == 0
    psi = _random_state(n, 3)
    ref = sim.apply(n, g, psi.copy())
    for k in range(plan.stats().num_kernels):
        d = plan.kernel(k)
        if d.type == Q.QS_KERNEL_FUSED:
            _apply_unitary(psi, n, [q for q in range(n) if (d.qubit_mask >> q) & 1], plan.fused_matrix(k))
        else:
            words, m, act, R = plan.kernel_program(k)
            run_kernel(psi, n, words, m, act, R)
    assert np.max(np.abs(psi - ref)) <= 1e-5
    fid = abs(np.vdot(ref, psi)) ** 2 / (np.vdot(psi, psi).real * np.vdot(ref, ref).real)
    assert fid >= 1 - 1e-6
