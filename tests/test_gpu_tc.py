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


def _case_high(n, seed):
    """Five or six targets at qubit >= 18 and none below 6: every tile row is
    64 contiguous amplitudes in its own 2 MiB page (the bulk-copy path)."""
    rng = np.random.default_rng(seed)
    hi = [int(t) for t in rng.permutation(np.arange(18, n))[:6]]
    lo = [int(t) for t in rng.permutation(np.arange(6, 18))[:6 - len(hi)]]
    targets = [int(t) for t in rng.permutation(hi + lo)]
    sub = C.entangling_circuit(6, 3, seed)
    u = sim.kernel_unitary(sub, list(range(6)))
    g = sub.copy()
    g["q0"] = [targets[q] for q in sub["q0"]]
    g["q1"] = [targets[q] if q >= 0 else -1 for q in sub["q1"]]
    psi0 = sim.apply(n, C.hadamard_layer(n))
    psi0 = sim.apply(n, C.mixed_circuit(n, 40, seed), psi0)
    return targets, u, psi0, sim.apply(n, g, psi0)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("n", [12, 13, 18])
def test_contiguous_tile_rows_register_path(n, precision):
    # columns are the 64 lowest qubits, but fewer than five targets sit at
    # qubit 18 or above: the register-gather path
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    targets, u, psi0, ref = _case(n, 6, 7 * n + precision, high=True)
    before = Q.qs_debug_tc_launch_counts()
    got = _apply(n, targets, u, precision, psi0)
    after = Q.qs_debug_tc_launch_counts()
    assert after["register"] == before["register"] + 1 and after["bulk"] == before["bulk"]
    if precision == Q.QS_PREC_TF32X3:
        assert_close_state(got, ref)
    else:
        assert fidelity(ref, got) > 1 - 1e-4


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("n", [23, 24])
def test_bulk_row_copy_path_matches_oracle(n, precision):
    # five (n = 23) or six (n = 24) targets at qubit >= 18: the loader warp
    # moves each tile row with cp.async.bulk into the raw ring
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    targets, u, psi0, ref = _case_high(n, 5 * n + precision)
    assert sum(t >= 18 for t in targets) >= 5 and min(targets) >= 6
    before = Q.qs_debug_tc_launch_counts()
    got = _apply(n, targets, u, precision, psi0)
    after = Q.qs_debug_tc_launch_counts()
    assert after["bulk"] == before["bulk"] + 1, (before, after)
    if precision == Q.QS_PREC_TF32X3:
        assert_close_state(got, ref)
    else:
        assert fidelity(ref, got) > 1 - 1e-4


def _batch_indices(n, targets, bases):
    """Indices of the 64 amplitudes of each sampled batch (row j of the
    unitary = target bits j), for batch values `bases` of the other bits."""
    off = np.zeros(64, dtype=np.int64)
    for j, t in enumerate(targets):
        off |= ((np.arange(64) >> j) & 1) << t
    return bases[:, None] | off[None, :]


@pytest.mark.parametrize("precision", [2, 0])
def test_64bit_offsets_at_33_qubits_on_sampled_batches(precision):
    # a 64 GiB resident state: the fused kernels address it with 64-bit
    # offsets.  The oracle cannot hold 2^33 amplitudes, so 512 sampled
    # batches (64 amplitudes each, every target combination) are checked
    # against the oracle's application of the same gates to that batch.
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 33
    if torch.cuda.mem_get_info()[0] < (8 << n) + (4 << 30):
        pytest.skip("needs 68 GiB of free device memory")
    rng = np.random.default_rng(33 + precision)
    targets = [32, 3, 25, 31, 12, 20]
    sub = C.entangling_circuit(6, 3, 5 + precision)
    u = sim.kernel_unitary(sub, list(range(6)))
    buf = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1234)
    buf.normal_(generator=gen)
    tmask = sum(1 << t for t in targets)
    bases = rng.integers(0, 1 << n, size=512, dtype=np.int64) & ~tmask
    bases[0], bases[1] = 0, ((1 << n) - 1) & ~tmask  # the first and last batches
    idx = torch.from_numpy(_batch_indices(n, targets, bases).reshape(-1)).cuda()
    view = buf.view(-1, 2)
    before = view[idx].double().cpu().numpy()
    before = (before[:, 0] + 1j * before[:, 1]).reshape(-1, 64)
    counts0 = Q.qs_debug_tc_launch_counts()
    Q.qs_apply_fused(buf.data_ptr(), n, targets, u.astype(np.complex64), precision,
                     torch.cuda.current_stream().cuda_stream)
    if precision != Q.QS_PREC_FP32:
        assert Q.qs_debug_tc_launch_counts()["wide"] == counts0["wide"] + 1
    after = view[idx].double().cpu().numpy()
    after = (after[:, 0] + 1j * after[:, 1]).reshape(-1, 64)
    for b in range(len(bases)):
        ref = sim.apply(6, sub, before[b] / np.linalg.norm(before[b]))
        assert_close_state(after[b] / np.linalg.norm(before[b]), ref)


def test_expired_tensor_core_wait_reaches_the_caller():
    # every tensor-core launch first waits (20 ms at most) on a barrier
    # nothing signals, then gives up: nothing reaches the tensor pipe, the
    # state is left as it was and the next synchronising call returns
    # QS_ETIMEDOUT -- for qs_apply_fused, and for qs_run_plan through
    # qs_read_amplitudes and qs_sync.  The context stays usable.
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 14
    g = C.entangling_circuit(n, 2, 8)
    cost = Q.default_cost_table()
    for k in range(16):
        cost.fuse_cost[k] = 1.0
    plan = Q.Plan(n, g, algo=2, fuse_kmax=6, precision=Q.QS_PREC_TF32X3, cost=cost)
    assert plan.stats().num_fused > 0
    s = torch.cuda.current_stream().cuda_stream
    st = Q.State.alloc(n, s)
    buf = torch.zeros(2 << n, dtype=torch.float32, device="cuda")
    buf[0] = 1.0
    try:
        Q.qs_debug_tc_stall(20000)
        with pytest.raises(Q.QsError) as ei:
            Q.qs_apply_fused(buf.data_ptr(), n, list(range(6)), np.eye(64, dtype=np.complex64),
                             Q.QS_PREC_TF32X3, s)
        assert ei.value.status == Q.QS_ETIMEDOUT
        st.run(plan, s)  # asynchronous: no error yet
        with pytest.raises(Q.QsError) as ei:
            st.read(stream=s)
        assert ei.value.status == Q.QS_ETIMEDOUT
        st.set_zero(s)
        st.run(plan, s)
        with pytest.raises(Q.QsError) as ei:
            Q.qs_sync(s)
        assert ei.value.status == Q.QS_ETIMEDOUT
        Q.qs_sync(s)  # reported once: the flag is cleared
    finally:
        Q.qs_debug_tc_stall(0)
    got = buf.cpu().numpy().view(np.complex64)
    assert got[0] == 1 and not np.any(got[1:])  # the stalled launch changed nothing
    st.set_zero(s)
    st.run(plan, s)
    assert_close_state(st.read(stream=s), sim.apply(n, g))


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
