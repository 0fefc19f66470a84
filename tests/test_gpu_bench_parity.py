"""Element-wise parity of the benchmark's plans at 26 qubits, and a resident
33-qubit round trip.

The benchmark runs its circuit generators at 30 qubits, where the FP64
oracle cannot run in test time.  At 26 qubits (a 512 MiB complex64 state,
larger than L2) the same generators, seeds and planner options produce the
same kinds of kernels at high batch bits -- shared-memory kernels with
|A| <= 12, fused 3xTF32 tensor-core kernels of the learned plan, every
kernel fused -- and the oracle computes the exact state in about a minute
on 16 host cores.  Every amplitude is compared (fidelity >= 1 - 1e-6,
max-abs <= 1e-5 against complex128).

At 33 qubits (64 GiB resident) the kernels take their 64-bit-offset forms
and the shared-memory kernels touching qubit 32 the generic tile kernel; the
oracle cannot hold that state, so the circuit followed by its adjoint must
return to |0...0> (Theorem 2 makes the plan's result the circuit's).
"""
import numpy as np
import pytest

from oracle import sim
from synth import circuits as C
from tests.gpu_util import assert_close_state, need_gpu, run_plan_on_gpu, torch

pytestmark = pytest.mark.gpu

N = 26
SHM_MAX = 12  # the benchmark's active-set cap


def _gates(workload):
    if workload == "mixed":
        return C.mixed_circuit(N, 5000, 100)
    return C.entangling_circuit(N, 40, 100)


_REF = {}


def _reference(workload):
    if workload not in _REF:
        _REF[workload] = sim.apply(N, _gates(workload))
    return _REF[workload]


def _plan(Q, gates, which, n=N):
    # "-x": planned as the Pauli-frame rewrite (insular X), as the bench does
    ix = 1 if which.endswith("-x") else 0
    which = which[:-2] if ix else which
    if which == "A":  # analytic-cost Kernelize, shared-memory kernels, FP32
        return Q.Plan(n, gates, algo=Q.QS_ALGO_KERNELIZE, fuse_kmax=0, shm_max_active=SHM_MAX, insular_x=ix)
    if which == "B":  # learned-cost Kernelize, fused kernels in 3xTF32
        from paper_2408_09055_gb300 import costmodel as CM
        net, _ = CM.load()
        opts = Q.default_opts(algo=Q.QS_ALGO_KERNELIZE, precision=Q.QS_PREC_TF32X3,
                              shm_max_active=SHM_MAX, fuse_kmax=6, mlp=net, insular_x=ix)
        plan = Q.Plan(n, gates, opts)
        plan._net = net
        return plan
    prec = {"F-FP32": Q.QS_PREC_FP32, "F-TF32X3": Q.QS_PREC_TF32X3}[which]
    cost = Q.default_cost_table()
    for k in range(16):
        cost.fuse_cost[k] = 1.0
    return Q.Plan(n, gates, algo=Q.QS_ALGO_KERNELIZE, fuse_kmax=6, fuse_kmin=6, precision=prec, cost=cost)


@pytest.mark.parametrize("which", ["A", "B", "F-TF32X3", "A-x", "B-x"])
@pytest.mark.parametrize("workload", ["mixed", "entangling"])
def test_bench_plans_match_oracle_elementwise_at_26_qubits(workload, which):
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    gates = _gates(workload)
    plan = _plan(Q, gates, which)
    st = plan.stats()
    assert plan.validate(gates) == 0
    if which == "F-TF32X3":
        assert st.num_fused == st.num_kernels > 0
    got, _, _ = run_plan_on_gpu(N, plan)
    assert_close_state(got, _reference(workload))


@pytest.mark.parametrize("which", ["A", "F-TF32X3"])
def test_resident_33_qubit_circuit_then_adjoint(which):
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 33
    if torch.cuda.mem_get_info()[0] < (8 << n) + (4 << 30):
        pytest.skip("needs 68 GiB of free device memory")
    g = C.mixed_circuit(n, 1500 if which == "A" else 400, 100)
    full = C.concat(g, C.adjoint(g))
    plan = _plan(Q, full, which, n=n)
    if which == "A":
        # kernels on qubit 32 exceed the register-phased forms' 32-bit offsets
        assert any(plan.kernel(k).qubit_mask >> 32 for k in range(plan.stats().num_kernels))
    s = torch.cuda.current_stream().cuda_stream
    st = Q.State.alloc(n, s)
    try:
        counts0 = Q.qs_debug_tc_launch_counts()
        st.run(plan, s)
        norm = st.norm2(s)
        head = st.read(0, 1 << 20, stream=s)
        tail = st.read((1 << n) - (1 << 20), 1 << 20, stream=s)
        if which != "A":
            assert Q.qs_debug_tc_launch_counts()["wide"] > counts0["wide"]
    finally:
        del st
    assert abs(norm - 1.0) < 1e-4
    f = abs(complex(head[0])) ** 2 / norm
    assert f >= 1 - 1e-6, f
    head[0] = 0
    assert float(np.max(np.abs(head))) <= 1e-5
    assert float(np.max(np.abs(tail))) <= 1e-5
