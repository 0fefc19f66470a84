"""The allocation-free entry point qs_apply_fused_static against
qs_apply_fused, which allocates its staging buffer on every call.

Some callers cannot allocate device memory while they apply a gate: all of
it already belongs to another allocator or budget, or an allocation's
synchronisation and failure modes are not acceptable at that point.  The
static entry point serves them from one fixed device array.  These tests
check that it gives the allocating entry point's results in every precision
(FP32 matrix; TF32 and 3xTF32 weights prepared on the host, k < 6 widened),
on calls in a row whose matrices differ (so stale array contents would
show), and that after its first call on a device it takes nothing from the
device's memory pool or free memory.  This file is collected last so that a
failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

from oracle import sim
from synth import circuits as C
from tests.gpu_util import assert_close_state, fidelity, need_gpu, torch

pytestmark = pytest.mark.gpu

# driver API memory-pool attributes (cuda.h, CUmemPool_attribute)
CU_MEMPOOL_ATTR_USED_MEM_CURRENT = 7
CU_MEMPOOL_ATTR_USED_MEM_HIGH = 8


def _random_state(n, seed):
    rng = np.random.default_rng(seed)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return psi / np.linalg.norm(psi)


def _gates_and_unitary(n, k, targets, seed):
    sub = C.mixed_circuit(k, 30, seed) if k >= 2 else C.make_gates([(C.U3, 0, None, 0.3, 0.2, 0.1)])
    u = sim.kernel_unitary(sub, list(range(k)))
    g = sub.copy()
    g["q0"] = [targets[q] for q in sub["q0"]]
    g["q1"] = [targets[q] if q >= 0 else -1 for q in sub["q1"]]
    return g, u.astype(np.complex64)


def _widths(precision):
    from paper_2408_09055_gb300 import qsim as Q
    # FP32: the widest matrix the array holds, then a narrower one; tensor
    # cores: the kernel's own width, then one that is widened to it
    return (7, 5) if precision == Q.QS_PREC_FP32 else (6, 4)


def _check_precision(precision, got, ref):
    from paper_2408_09055_gb300 import qsim as Q
    if precision == Q.QS_PREC_TF32:  # one TF32 product: 10-bit mantissas
        assert fidelity(ref, got) > 1 - 1e-4
    else:
        assert_close_state(got, ref)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_static_entry_point_matches_allocating_one_twice_in_a_row(precision):
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 16
    psi = _random_state(n, 7 + precision)
    a = torch.from_numpy(psi.astype(np.complex64).view(np.float32).copy()).cuda()
    b = torch.from_numpy(psi.astype(np.complex64).view(np.float32).copy()).cuda()
    s = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(3 + precision)
    for call, k in enumerate(_widths(precision)):  # two calls in a row, different matrices
        targets = [int(t) for t in rng.permutation(n)[:k]]
        g, u = _gates_and_unitary(n, k, targets, 10 + call)
        Q.qs_apply_fused(a.data_ptr(), n, targets, u, precision, s)
        Q.qs_apply_fused_static(b.data_ptr(), n, targets, u, precision, s)
        got_a = a.cpu().numpy().view(np.complex64).astype(np.complex128)
        got_b = b.cpu().numpy().view(np.complex64).astype(np.complex128)
        # the same kernel on the same staged data: the allocating entry
        # point's result, within the FP32 bar
        assert_close_state(got_b, got_a)
        psi = sim.apply(n, g, psi)  # FP64 reference of both calls so far
        _check_precision(precision, got_b, psi)


def _pool_and_driver():
    cu = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int()
    assert cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetMemPool(ctypes.byref(pool), dev) == 0
    return cu, pool


def _pool_attr(cu, pool, attr):
    v = ctypes.c_uint64()
    assert cu.cuMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
    return v.value


def _reset_pool_high(cu, pool):
    z = ctypes.c_uint64(0)
    assert cu.cuMemPoolSetAttribute(pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, ctypes.byref(z)) == 0


def test_static_entry_point_takes_no_device_memory():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 16
    buf = torch.from_numpy(_random_state(n, 5).astype(np.complex64).view(np.float32).copy()).cuda()
    s = torch.cuda.current_stream().cuda_stream
    targets = [3, 9, 1, 14, 6, 11]
    _, u = _gates_and_unitary(n, 6, targets, 4)
    for p in (Q.QS_PREC_FP32, Q.QS_PREC_TF32, Q.QS_PREC_TF32X3):  # first calls: set-up, module loads
        Q.qs_apply_fused_static(buf.data_ptr(), n, targets, u, p, s)
    torch.cuda.synchronize()
    cu, pool = _pool_and_driver()
    _reset_pool_high(cu, pool)
    used0 = _pool_attr(cu, pool, CU_MEMPOOL_ATTR_USED_MEM_CURRENT)
    free0 = torch.cuda.mem_get_info()[0]
    for p in (Q.QS_PREC_FP32, Q.QS_PREC_TF32, Q.QS_PREC_TF32X3, Q.QS_PREC_TF32X3):
        Q.qs_apply_fused_static(buf.data_ptr(), n, targets, u, p, s)
    torch.cuda.synchronize()
    assert _pool_attr(cu, pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH) <= used0
    assert torch.cuda.mem_get_info()[0] == free0
    # the probe does see the allocating entry point's stream-ordered buffer
    Q.qs_apply_fused(buf.data_ptr(), n, targets, u, Q.QS_PREC_TF32X3, s)
    assert _pool_attr(cu, pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH) >= used0 + 128 * 1024


def test_static_entry_point_rejects_what_it_cannot_hold():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    s = torch.cuda.current_stream().cuda_stream
    n = 12
    buf = torch.zeros(2 << n, dtype=torch.float32, device="cuda")
    buf[0] = 1.0
    with pytest.raises(Q.QsError) as ei:  # 2^8 x 2^8 exceeds the array
        Q.qs_apply_fused_static(buf.data_ptr(), n, list(range(8)), np.eye(1 << 8, dtype=np.complex64),
                                Q.QS_PREC_FP32, s)
    assert ei.value.status == Q.QS_EINVAL
    with pytest.raises(Q.QsError) as ei:  # the tensor-core kernel is 6 targets wide
        Q.qs_apply_fused_static(buf.data_ptr(), n, list(range(7)), np.eye(1 << 7, dtype=np.complex64),
                                Q.QS_PREC_TF32X3, s)
    assert ei.value.status == Q.QS_EUNSUPPORTED
    small = torch.zeros(2 << 10, dtype=torch.float32, device="cuda")
    with pytest.raises(Q.QsError) as ei:  # fewer than 32 columns per tile
        Q.qs_apply_fused_static(small.data_ptr(), 10, [0, 1], np.eye(4, dtype=np.complex64),
                                Q.QS_PREC_TF32, s)
    assert ei.value.status == Q.QS_EUNSUPPORTED
    # nothing was applied: the state is still |0...0>
    got = buf.cpu().numpy().view(np.complex64)
    assert got[0] == 1 and not np.any(got[1:])
