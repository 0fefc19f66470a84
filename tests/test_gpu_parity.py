"""GPU parity: plans executed by libqsim's CUDA kernels against the FP64
oracle, element by element (fidelity >= 1 - 1e-6, max-abs <= 1e-5)."""
import numpy as np
import pytest

from oracle import sim
from synth import circuits as C
from tests.gpu_util import assert_close_state, need_gpu, run_plan_on_gpu, torch

pytestmark = pytest.mark.gpu

ALGOS = {"per_gate": 0, "greedy": 1, "ordered": 2, "kernelize": 3}


def gen(kind, n, seed):
    if kind == "layered":
        return C.layered_u3_cz(n, 6, seed)
    if kind == "mixed":
        return C.mixed_circuit(n, 400, seed)
    return C.entangling_circuit(n, 4, seed)


@pytest.mark.parametrize("kind", ["layered", "mixed", "entangling"])
@pytest.mark.parametrize("algo", list(ALGOS))
@pytest.mark.parametrize("n", [12, 17])
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_shm_plans_match_oracle(kind, algo, n, variant):
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    g = gen(kind, n, n)
    plan = Q.Plan(n, g, algo=ALGOS[algo], fuse_kmax=0, shm_variant=variant)
    assert plan.validate() == 0
    st = plan.stats()
    assert st.num_phased == (st.num_shm if variant >= 2 else 0)
    assert st.num_jit == (st.num_shm if variant == 3 else 0)
    got, _, _ = run_plan_on_gpu(n, plan)
    assert_close_state(got, sim.apply(n, g))


@pytest.mark.parametrize("kmax", [3, 5, 6, 7])
def test_fused_fp32_plans_match_oracle(kmax):
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 16
    g = C.entangling_circuit(n, 4, 11)
    cost = Q.default_cost_table()
    for k in range(16):
        cost.fuse_cost[k] = 1.0  # make every feasible fusion cheaper than shm
    plan = Q.Plan(n, g, algo=2, fuse_kmax=kmax, fuse_kmin=kmax, cost=cost, precision=Q.QS_PREC_FP32)
    st = plan.stats()
    assert st.num_fused > 0
    got, _, _ = run_plan_on_gpu(n, plan)
    assert_close_state(got, sim.apply(n, g))


@pytest.mark.parametrize("m", [10, 11, 12, 13, 14])
@pytest.mark.parametrize("variant", [2, 3])
def test_phased_kernel_every_tile_size(m, variant):
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 18
    g = C.concat(C.mixed_circuit(n, 700, m), C.entangling_circuit(n, 3, m))
    plan = Q.Plan(n, g, algo=2, fuse_kmax=0, shm_max_active=m, shm_variant=variant)
    st = plan.stats()
    assert st.num_phased == st.num_shm and st.num_exchanges > 0
    rng = np.random.default_rng(m)
    psi0 = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n))
    psi0 = (psi0 / np.linalg.norm(psi0)).astype(np.complex64).astype(np.complex128)
    got, _, _ = run_plan_on_gpu(n, plan, psi0)
    assert_close_state(got, sim.apply(n, g, psi0))


def test_random_input_state_and_mixed_kernel_types():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 15
    rng = np.random.default_rng(5)
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi0 /= np.linalg.norm(psi0)
    psi0 = psi0.astype(np.complex64).astype(np.complex128)
    g = C.mixed_circuit(n, 600, 5)
    plan = Q.Plan(n, g, algo=2, fuse_kmax=5)
    got, _, _ = run_plan_on_gpu(n, plan, psi0)
    assert_close_state(got, sim.apply(n, g, psi0))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 9])
def test_tiny_states(n):
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    g = C.mixed_circuit(n, 50, n) if n >= 2 else C.make_gates([(C.H, 0), (C.RZ, 0, None, 0.3), (C.U3, 0, None, 1, 2, 3)])
    for algo in (0, 2):
        plan = Q.Plan(n, g, algo=algo, fuse_kmax=min(n, 4))
        got, _, _ = run_plan_on_gpu(n, plan)
        assert_close_state(got, sim.apply(n, g))


def test_empty_circuit_is_identity():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 10
    plan = Q.Plan(n, C.make_gates([]))
    assert plan.stats().num_kernels == 0
    got, _, _ = run_plan_on_gpu(n, plan)
    ref = np.zeros(1 << n, dtype=complex); ref[0] = 1
    assert np.array_equal(got, ref.astype(np.complex64))


def test_lone_qubit_gates_plan_and_run():
    # Hadamards on qubits no multi-qubit gate touches form units of their own
    # when attaching them would overfill a kernel
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 16
    g = C.make_gates([(C.H, q) for q in range(n)] + [(C.CX, n - 1, 5), (C.CX, n - 2, 2), (C.H, 5)])
    for variant in (1, 2, 3):
        plan = Q.Plan(n, g, shm_max_active=12, fuse_kmax=0, shm_variant=variant)
        got, _, _ = run_plan_on_gpu(n, plan)
        assert_close_state(got, sim.apply(n, g))


def test_closed_forms_on_gpu():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 20
    plan = Q.Plan(n, C.ghz(n))
    got, _, _ = run_plan_on_gpu(n, plan)
    ref = np.zeros(1 << n, dtype=complex); ref[0] = ref[-1] = 2 ** -0.5
    assert_close_state(got, ref)
    x = 0xABCDE
    g = C.concat(C.basis_prep(n, x), C.qft(n))
    got, _, _ = run_plan_on_gpu(n, Q.Plan(n, g))
    y = np.arange(1 << n)
    assert_close_state(got, np.exp(2j * np.pi * x * y / (1 << n)) / 2 ** (n / 2))


def test_norm_and_compare_reductions():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 18
    g = C.layered_u3_cz(n, 4, 2)
    plan = Q.Plan(n, g)
    got, st, _ = run_plan_on_gpu(n, plan)
    ref = sim.apply(n, g)
    assert abs(st.norm2() - np.sum(np.abs(got.astype(np.complex128)) ** 2)) < 1e-9
    assert abs(st.norm2() - 1) < 1e-5
    ref_dev = torch.from_numpy(ref.view(np.float64)).cuda()
    fid, mx = st.compare_c128(ref_dev.data_ptr())
    exp = abs(np.vdot(ref, got.astype(np.complex128))) ** 2 / np.sum(np.abs(got.astype(np.complex128)) ** 2)
    assert abs(fid - exp) < 1e-12
    assert abs(mx - np.max(np.abs(ref - got))) < 1e-7


@pytest.mark.parametrize("kind", ["random", "identity", "reverse", "rotate"])
@pytest.mark.parametrize("n", [6, 10, 14, 21])
def test_remap_permutes_bits(n, kind):
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    rng = np.random.default_rng(n)
    perm = {"random": rng.permutation(n), "identity": np.arange(n), "reverse": np.arange(n)[::-1],
            "rotate": (np.arange(n) + 7) % n}[kind]
    x = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(np.complex64)
    src = torch.from_numpy(x.view(np.float32)).cuda()
    dst = torch.empty_like(src)
    Q.qs_remap(src.data_ptr(), dst.data_ptr(), n, perm, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    out = dst.cpu().numpy().view(np.complex64)
    i = np.arange(1 << n)
    j = np.zeros_like(i)
    for b in range(n):
        j |= ((i >> b) & 1) << int(perm[b])
    ref = np.empty_like(x); ref[j] = x
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("k", [1, 2, 4, 5, 6, 7])
def test_apply_fused_matches_kernel_unitary(k):
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 16
    rng = np.random.default_rng(k)
    targets = [int(t) for t in rng.permutation(n)[:k]]
    sub = C.mixed_circuit(k, 40, k) if k >= 2 else C.make_gates([(C.U3, 0, None, 0.4, 0.5, 0.6)])
    u = sim.kernel_unitary(sub, list(range(k)))
    # the same gates placed on `targets` of the n-qubit state
    g = sub.copy()
    g["q0"] = [targets[q] for q in sub["q0"]]
    g["q1"] = [targets[q] if q >= 0 else -1 for q in sub["q1"]]
    psi0 = sim.apply(n, C.hadamard_layer(n))
    psi0 = sim.apply(n, C.mixed_circuit(n, 60, 3), psi0)
    ref = sim.apply(n, g, psi0)
    buf = torch.from_numpy(psi0.astype(np.complex64).view(np.float32)).cuda()
    Q.qs_apply_fused(buf.data_ptr(), n, targets, u, Q.QS_PREC_FP32, torch.cuda.current_stream().cuda_stream)
    got = buf.cpu().numpy().view(np.complex64)
    assert_close_state(got, ref)


@pytest.mark.parametrize("plan_kind", ["A", "F-TF32X3"])
def test_full_size_bench_circuit_then_adjoint(plan_kind):
    # the bench's workload and launch configuration at full size (30 qubits,
    # 8 GiB): the 5000-gate mixed circuit followed by its adjoint must return
    # to |0...0>, a property that holds at any size
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 30
    g = C.mixed_circuit(n, 5000, 100)
    full = C.concat(g, C.adjoint(g))
    if plan_kind == "A":
        plan = Q.Plan(n, full, algo=3, fuse_kmax=0, shm_max_active=12)
    else:
        cost = Q.default_cost_table()
        for k in range(16):
            cost.fuse_cost[k] = 1.0
        part = g[:600]  # fused kernels on the mixed circuit are many: a prefix keeps it short
        full = C.concat(part, C.adjoint(part))
        plan = Q.Plan(n, full, algo=3, fuse_kmax=6, fuse_kmin=6, precision=Q.QS_PREC_TF32X3, cost=cost)
    s = torch.cuda.current_stream().cuda_stream
    st = Q.State.alloc(n, s)
    st.run(plan, s)
    norm = st.norm2(s)  # FP64 reduction on the device
    got = st.read(stream=s)
    f = abs(complex(got[0])) ** 2 / norm
    assert f >= 1 - 1e-6, f
    got[0] = 0
    assert float(np.max(np.abs(got))) <= 1e-5
