"""The allocation-free entry point qs_apply_fused_static against
qs_apply_fused, which allocates its matrix staging buffer per call.

Some callers cannot allocate device memory while they apply a gate (all of it
already belongs to another allocator or budget, or an allocation's
synchronisation is not acceptable at that point); the static entry point
serves them from a fixed device array.  This file is collected last so that
a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from oracle import sim
from synth import circuits as C
from tests.gpu_util import assert_close_state, need_gpu, torch

pytestmark = pytest.mark.gpu


def _random_state(n, seed):
    rng = np.random.default_rng(seed)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return (psi / np.linalg.norm(psi)).astype(np.complex64)


def _unitary(k, seed):
    g = C.mixed_circuit(k, 30, seed) if k >= 2 else C.make_gates([(C.U3, 0, None, 0.3, 0.2, 0.1)])
    return sim.kernel_unitary(g, list(range(k))).astype(np.complex64)


def test_static_entry_point_matches_allocating_one_twice_in_a_row():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 16
    psi0 = _random_state(n, 7)
    a = torch.from_numpy(psi0.view(np.float32).copy()).cuda()
    b = torch.from_numpy(psi0.view(np.float32).copy()).cuda()
    s = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(3)
    for call, k in enumerate((7, 5)):  # two calls in a row, different sizes
        targets = [int(t) for t in rng.permutation(n)[:k]]
        u = _unitary(k, 10 + call)
        Q.qs_apply_fused(a.data_ptr(), n, targets, u, Q.QS_PREC_FP32, s)
        Q.qs_apply_fused_static(b.data_ptr(), n, targets, u, Q.QS_PREC_FP32, s)
        got_a = a.cpu().numpy().view(np.complex64)
        got_b = b.cpu().numpy().view(np.complex64)
        assert_close_state(got_b, got_a.astype(np.complex128))


def test_static_entry_point_rejects_too_wide_unitary():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 10
    buf = torch.zeros(2 << n, dtype=torch.float32, device="cuda")
    u = np.eye(1 << 8, dtype=np.complex64)
    with pytest.raises(Q.QsError) as ei:
        Q.qs_apply_fused_static(buf.data_ptr(), n, list(range(8)), u, Q.QS_PREC_FP32,
                                torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == Q.QS_EINVAL
