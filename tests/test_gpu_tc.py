"""Tensor-core fused kernels (tcgen05, TF32 and 3xTF32) against the FP64
oracle.  3xTF32 must meet the FP32 accuracy target; one TF32 product is
measurably less accurate, which is what the split recovers."""
import numpy as np
import pytest

from oracle import sim
from synth import circuits as C
from tests.gpu_util import assert_close_state, fidelity, need_gpu, run_plan_on_gpu, torch

pytestmark = pytest.mark.gpu


def _apply(n, targets, u, precision, psi0):
    from paper_2408_09055_gb300 import qsim as Q
    buf = torch.from_numpy(psi0.astype(np.complex64).view(np.float32).copy()).cuda()
    Q.qs_apply_fused(buf.data_ptr(), n, targets, u, precision, torch.cuda.current_stream().cuda_stream)
    return buf.cpu().numpy().view(np.complex64).astype(np.complex128)


def _case(n, k, seed, high=False):
    rng = np.random.default_rng(seed)
    # high: targets among qubits >= 6, so a tile's columns are the 64 lowest
    # qubits (contiguous rows: the bulk-staged load path)
    pool = np.arange(6, n) if high else np.arange(n)
    targets = [int(t) for t in rng.permutation(pool)[:k]]
    sub = C.entangling_circuit(k, 3, seed) if k >= 2 else C.make_gates([(C.U3, 0, None, 0.4, 0.5, 0.6)])
    u = sim.kernel_unitary(sub, list(range(k)))
    g = sub.copy()
    g["q0"] = [targets[q] for q in sub["q0"]]
    g["q1"] = [targets[q] if q >= 0 else -1 for q in sub["q1"]]
    psi0 = sim.apply(n, C.hadamard_layer(n))
    psi0 = sim.apply(n, C.mixed_circuit(n, 80, seed), psi0)
    return targets, u, psi0, sim.apply(n, g, psi0)


@pytest.mark.parametrize("k", [6, 4, 1])
@pytest.mark.parametrize("n", [11, 12, 16])
def test_tf32x3_meets_fp32_accuracy(n, k):
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    targets, u, psi0, ref = _case(n, k, 10 * n + k)
    got = _apply(n, targets, u, Q.QS_PREC_TF32X3, psi0)
    assert_close_state(got, ref)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("n", [12, 13, 18])
def test_contiguous_tile_rows_bulk_path(n, precision):
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    targets, u, psi0, ref = _case(n, 6, 7 * n + precision, high=True)
    got = _apply(n, targets, u, precision, psi0)
    if precision == Q.QS_PREC_TF32X3:
        assert_close_state(got, ref)
    else:
        assert fidelity(ref, got) > 1 - 1e-4


@pytest.mark.parametrize("n", [12, 17])
def test_tf32_single_product_is_less_accurate(n):
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    targets, u, psi0, ref = _case(n, 6, n)
    e1 = np.max(np.abs(_apply(n, targets, u, Q.QS_PREC_TF32, psi0) - ref))
    e3 = np.max(np.abs(_apply(n, targets, u, Q.QS_PREC_TF32X3, psi0) - ref))
    scale = np.max(np.abs(ref))
    assert e1 / scale < 5e-3          # TF32: 10-bit mantissa products
    assert e3 < e1 / 20               # the split recovers most of the lost bits
    assert fidelity(ref, _apply(n, targets, u, Q.QS_PREC_TF32, psi0)) > 1 - 1e-4


@pytest.mark.parametrize("precision", [1, 2])
def test_tensor_core_plans_match_oracle(precision):
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 14
    g = C.entangling_circuit(n, 3, 21)
    cost = Q.default_cost_table()
    for k in range(16):
        cost.fuse_cost[k] = 1.0  # every feasible fusion is cheaper than a shared-memory kernel
    plan = Q.Plan(n, g, algo=2, fuse_kmax=6, precision=precision, cost=cost)
    st = plan.stats()
    assert st.num_fused > 0
    got, _, _ = run_plan_on_gpu(n, plan)
    ref = sim.apply(n, g)
    if precision == Q.QS_PREC_TF32X3:
        assert_close_state(got, ref)
    else:
        assert fidelity(ref, got) > 1 - 1e-3
