"""GPU parity of staged execution (Alg. 1's Execute with the state in host
memory, qs_run_plan_host): the host state after every stage's chunks have
been through the GPU, against the FP64 oracle element by element."""
import numpy as np
import pytest

from oracle import sim
from synth import circuits as C
from tests.gpu_util import assert_close_state, fidelity, need_gpu, run_plan_on_gpu, torch

pytestmark = pytest.mark.gpu


def pinned_state(n, psi0=None):
    h = torch.zeros(2 << n, dtype=torch.float32).pin_memory()
    v = h.numpy().view(np.complex64)
    if psi0 is None:
        v[0] = 1.0
    else:
        v[:] = psi0.astype(np.complex64)
    return h, v


def run_host(plan, n, psi0=None, nbuf=None):
    h, v = pinned_state(n, psi0)
    dev = None
    s = torch.cuda.current_stream()
    if nbuf is None:
        plan.run_host(h.data_ptr(), stream=s.cuda_stream)
    else:
        L = plan.opts.local_qubits if 0 < plan.opts.local_qubits < n else n
        dev = torch.empty(nbuf << (L + 1), dtype=torch.float32, device="cuda")
        plan.run_host(h.data_ptr(), dev.data_ptr(), dev.numel() * 4, stream=s.cuda_stream)
    s.synchronize()
    return v.copy()


def random_state(n, seed):
    rng = np.random.default_rng(seed)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi /= np.linalg.norm(psi)
    return psi.astype(np.complex64).astype(np.complex128)


CASES = {
    "mixed": (20, 16, lambda: C.mixed_circuit(20, 600, 3), {}),
    "entangling-fused": (19, 14, lambda: C.entangling_circuit(19, 5, 4), {"fuse_kmax": 5}),
    "layered": (18, 12, lambda: C.layered_u3_cz(18, 8, 5), {"shm_max_active": 12}),
    "qft": (17, 13, lambda: C.qft(17), {"shm_max_active": 12}),
}


@pytest.mark.parametrize("nbuf", [None, 1, 2, 3, 4])
@pytest.mark.parametrize("case", list(CASES))
def test_staged_plans_match_oracle(case, nbuf):
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n, L, make, kw = CASES[case]
    g = make()
    plan = Q.Plan(n, g, local_qubits=L, **kw)
    assert plan.validate() == 0 and plan.stats().num_stages > 1
    got = run_host(plan, n, nbuf=nbuf)
    assert_close_state(got, sim.apply(n, g))


def test_exact_stager_plan_matches_oracle():
    # the exact stager's local sets through the same chunked executor
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n, L = 16, 12
    g = C.mixed_circuit(n, 120, 3)
    plan = Q.Plan(n, g, local_qubits=L, shm_max_active=12, stager=Q.QS_STAGER_EXACT)
    st = plan.stats()
    assert st.staging_optimal >= 1 and st.num_stages > 1 and plan.validate() == 0
    psi0 = random_state(n, 17)
    got = run_host(plan, n, psi0, nbuf=2)
    assert_close_state(got, sim.apply(n, g, psi0.copy()))


@pytest.mark.parametrize("variant,nbuf", [(1, 2), (2, 3), (3, 4), (3, 1)])
def test_staged_random_initial_state(variant, nbuf):
    # every amplitude nonzero: a chunk gathered or scattered to the wrong
    # host run shows up element by element
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n, L = 18, 13
    g = C.mixed_circuit(n, 500, 8)
    psi0 = random_state(n, 9)
    plan = Q.Plan(n, g, local_qubits=L, shm_max_active=12, shm_variant=variant)
    assert plan.stats().num_stages > 3
    got = run_host(plan, n, psi0, nbuf=nbuf)
    assert_close_state(got, sim.apply(n, g, psi0.copy()))


def test_staged_tensor_core_fused_kernels():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n, L = 18, 14
    g = C.entangling_circuit(n, 4, 12)
    cost = Q.default_cost_table()
    for k in range(16):
        cost.fuse_cost[k] = 1.0  # every feasible fusion is cheaper than a shared-memory kernel
    plan = Q.Plan(n, g, algo=2, fuse_kmax=6, precision=Q.QS_PREC_TF32X3, cost=cost, local_qubits=L)
    st = plan.stats()
    assert st.num_fused > 0 and st.num_stages > 1
    got = run_host(plan, n, nbuf=3)
    assert_close_state(got, sim.apply(n, g))


def test_unstaged_plan_through_host_path_equals_resident_run():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 16
    g = C.mixed_circuit(n, 300, 13)
    plan = Q.Plan(n, g)
    got = run_host(plan, n)
    res, _, _ = run_plan_on_gpu(n, plan)
    assert np.array_equal(got, res)  # same kernels on the same data
    assert_close_state(got, sim.apply(n, g))


def test_pageable_host_state_is_rejected():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 14
    plan = Q.Plan(n, C.mixed_circuit(n, 50, 1), local_qubits=12, shm_max_active=12)
    h = np.zeros(2 << n, dtype=np.float32)
    with pytest.raises(Q.QsError):
        plan.run_host(h.ctypes.data)
    dev = torch.empty(1 << 10, dtype=torch.float32, device="cuda")  # smaller than one chunk
    hp, _ = pinned_state(n)
    with pytest.raises(Q.QsError):
        plan.run_host(hp.data_ptr(), dev.data_ptr(), dev.numel() * 4)


def test_staged_30_qubits_circuit_then_adjoint_returns_to_zero():
    # a 30-qubit state (8 GiB, 16 chunks of 2^26) staged through host memory;
    # C followed by its adjoint is the identity, a property at any size
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n, L = 30, 26
    g = C.mixed_circuit(n, 400, 21)
    full = C.concat(g, C.adjoint(g))
    plan = Q.Plan(n, full, local_qubits=L)
    assert plan.stats().num_stages > 1
    got = run_host(plan, n, nbuf=2)
    ref = np.zeros(1 << n, dtype=np.complex64)
    ref[0] = 1.0
    f = fidelity(ref, got)
    assert f >= 1 - 1e-6, f
    assert float(np.max(np.abs(got[1:]))) <= 1e-5


def test_many_small_chunks_and_stages():
    # 2^8 chunks per stage: the chunk-level waits between stages, the buffer
    # rotation across stages and the unit split of copy-ins at every boundary
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n, L = 20, 12
    g = C.mixed_circuit(n, 300, 31)
    psi0 = random_state(n, 32)
    plan = Q.Plan(n, g, local_qubits=L, shm_max_active=12)
    assert plan.stats().num_stages > 5
    got = run_host(plan, n, psi0, nbuf=3)
    assert_close_state(got, sim.apply(n, g, psi0.copy()))


def test_host_timer_timeline_is_ordered():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n, L = 18, 14
    g = C.mixed_circuit(n, 300, 41)
    plan = Q.Plan(n, g, local_qubits=L)
    h, v = pinned_state(n)
    dev = torch.empty(3 << (L + 1), dtype=torch.float32, device="cuda")
    tm = Q.HostTimer(plan)
    s = torch.cuda.current_stream()
    tm.run(h.data_ptr(), dev.data_ptr(), dev.numel() * 4, stream=s.cuda_stream)
    s.synchronize()
    T = tm.read()
    assert T.shape == (plan.stats().num_stages, 1 << (n - L), 4)
    assert np.all(T >= 0) and np.all(np.diff(T, axis=2) >= 0)
    assert_close_state(v.copy(), sim.apply(n, g))


def test_alloc_state_starts_at_zero_and_runs_a_plan():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 15
    g = C.mixed_circuit(n, 200, 51)
    s = torch.cuda.current_stream().cuda_stream
    st = Q.State.alloc(n, s)
    v = st.read(stream=s)
    assert v[0] == 1 and np.count_nonzero(v) == 1
    st.run(Q.Plan(n, g), s)
    assert_close_state(st.read(stream=s), sim.apply(n, g))


def _insular_x_rule_circuit(n, L, seed):
    # dense gates keep the low L qubits local; X gates on the two highest
    # (regional) qubits, then every insular use of them: controls, CZ, CP,
    # RZ, both flipped together; later dense gates make them local
    rng = np.random.default_rng(seed)
    a, b = n - 1, n - 2
    items = [(C.H, q, None, 0, 0, 0) for q in range(L)]
    items += [(C.X, a, None, 0, 0, 0), (C.CZ, a, 2, 0, 0, 0), (C.CP, 5, a, rng.uniform(0, 6.28), 0, 0),
              (C.CX, a, 3, 0, 0, 0), (C.RZ, a, None, rng.uniform(0, 6.28), 0, 0),
              (C.X, b, None, 0, 0, 0), (C.CZ, a, b, 0, 0, 0), (C.CP, b, a, rng.uniform(0, 6.28), 0, 0),
              (C.CX, b, 7, 0, 0, 0), (C.RZ, b, None, rng.uniform(0, 6.28), 0, 0)]
    items += [(C.U3, q, None, *rng.uniform(0, 6.28, 3)) for q in range(L)]
    items += [(C.H, a, None, 0, 0, 0), (C.H, b, None, 0, 0, 0), (C.CX, a, 0, 0, 0, 0), (C.CZ, b, 4, 0, 0, 0)]
    return C.make_gates(items)


@pytest.mark.parametrize("nbuf", [None, 2, 3, 4])
@pytest.mark.parametrize("case", ["rules", "mixed"])
def test_insular_x_stages_match_oracle(case, nbuf):
    # X gates on regional qubits run as chunk relabellings (App. A.2): chunks
    # are written back in pairs to their partners' host chunks
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    if case == "rules":
        n, L = 17, 12
        g = _insular_x_rule_circuit(n, L, nbuf or 0)
    else:
        n, L = 19, 14
        g = C.mixed_circuit(n, 900, 11)
    plan = Q.Plan(n, g, local_qubits=L, insular_x=Q.QS_INSULAR_X_STAGED, shm_max_active=12)
    frames = [plan.stage_frame(i)[0] for i in range(plan.stats().num_stages)]
    assert any(frames)
    psi0 = random_state(n, 3 + (nbuf or 0))
    got = run_host(plan, n, psi0, nbuf)
    assert_close_state(got, sim.apply(n, g, psi0.copy()))


def test_insular_x_stages_need_two_chunk_buffers():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n, L = 17, 12
    g = _insular_x_rule_circuit(n, L, 0)
    plan = Q.Plan(n, g, local_qubits=L, insular_x=Q.QS_INSULAR_X_STAGED, shm_max_active=12)
    with pytest.raises(Q.QsError) as ei:
        run_host(plan, n, None, 1)
    assert ei.value.status == Q.QS_EINVAL
