"""The C ABI's documented argument errors, checked on the CPU: every call
below is refused before the library touches a GPU (device addresses here are
only compared and never dereferenced)."""
import ctypes

import numpy as np
import pytest

from synth import circuits as C

Q = pytest.importorskip("paper_2408_09055_gb300.qsim")
L = Q.lib
EINVAL, EUNSUP = Q.QS_EINVAL, Q.QS_EUNSUPPORTED
FAKE = 0x7F0000000000  # a 256-B aligned address that is never dereferenced


def _i32(v):
    a = (ctypes.c_int32 * len(v))(*v)
    return ctypes.cast(a, ctypes.POINTER(ctypes.c_int32)), a


def test_status_strings_cover_every_code():
    for code in (Q.QS_OK, EINVAL, Q.QS_ENOMEM, EUNSUP, Q.QS_ETIMEDOUT, Q.QS_ECUDA, Q.QS_EPLAN):
        assert L.qs_strerror(code)
    assert L.qs_strerror(12345)  # unknown codes still give a string


def test_state_view_needs_no_device_work():
    h = ctypes.c_void_p()
    assert L.qs_state_create(10, None, None) == EINVAL
    for n in (0, 35):
        assert L.qs_state_create(n, ctypes.c_void_p(FAKE), ctypes.byref(h)) == EINVAL
    assert L.qs_state_create(10, ctypes.c_void_p(FAKE + 8), ctypes.byref(h)) == EINVAL  # misaligned
    assert L.qs_state_create(10, ctypes.c_void_p(FAKE), ctypes.byref(h)) == Q.QS_OK
    assert L.qs_state_device_ptr(h) == FAKE
    # amplitude ranges are checked before any copy
    buf = np.zeros(16, dtype=np.float32)
    fp = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    assert L.qs_read_amplitudes(h, 0, 4, None, None) == EINVAL
    assert L.qs_read_amplitudes(h, 1020, 8, fp, None) == EINVAL
    assert L.qs_write_amplitudes(h, 1025, 1, fp, None) == EINVAL
    assert L.qs_read_amplitudes(h, 1024, 0, fp, None) == Q.QS_OK  # empty range
    assert L.qs_state_norm2(h, None, None) == EINVAL
    assert L.qs_state_compare_c128(h, None, None, None, None) == EINVAL
    # a plan of another width is refused
    p = Q.Plan(12, C.mixed_circuit(12, 20, 1), shm_variant=1)
    assert L.qs_run_plan(p.h, h, None) == EINVAL
    assert L.qs_run_plan(None, h, None) == EINVAL
    L.qs_state_free(h)  # a view: nothing to free on the device


def test_remap_arguments():
    perm, _keep = _i32([1, 0, 2])
    assert L.qs_remap(None, ctypes.c_void_p(FAKE), 3, perm, None) == EINVAL
    assert L.qs_remap(ctypes.c_void_p(FAKE), ctypes.c_void_p(FAKE + 4096), 3, None, None) == EINVAL
    for n in (0, 35):
        assert L.qs_remap(ctypes.c_void_p(FAKE), ctypes.c_void_p(FAKE + (1 << 40)), n, perm, None) == EINVAL
    for bad in ([0, 0, 2], [0, 1, 3], [-1, 1, 2]):  # not a permutation of 0..n-1
        pb, _k = _i32(bad)
        assert L.qs_remap(ctypes.c_void_p(FAKE), ctypes.c_void_p(FAKE + 4096), 3, pb, None) == EINVAL
    # the two buffers (2^3 complex64 = 64 B) may not overlap
    assert L.qs_remap(ctypes.c_void_p(FAKE), ctypes.c_void_p(FAKE + 32), 3, perm, None) == EINVAL


@pytest.mark.parametrize("entry", ["qs_apply_fused", "qs_apply_fused_static"])
def test_fused_apply_arguments(entry):
    f = getattr(L, entry)
    u = np.zeros(2 * 64 * 64, dtype=np.float32)
    up = u.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    st = ctypes.c_void_p(FAKE)
    t2, _a = _i32([0, 1])
    assert f(None, 12, t2, 2, up, 0, None) == EINVAL
    assert f(st, 12, None, 2, up, 0, None) == EINVAL
    assert f(st, 12, t2, 2, None, 0, None) == EINVAL
    assert f(st, 12, t2, 0, up, 0, None) == EINVAL  # k < 1
    assert f(st, 1, t2, 2, up, 0, None) == EINVAL   # n < k
    assert f(st, 35, t2, 2, up, 0, None) == EINVAL  # n > 34
    assert f(st, 12, t2, 2, up, 3, None) == EINVAL  # unknown precision
    for bad in ([0, 0], [0, 12], [-1, 1]):
        tb, _k = _i32(bad)
        assert f(st, 12, tb, 2, up, 0, None) == EINVAL
    t9, _b = _i32(list(range(9)))
    assert f(st, 12, t9, 9, up, 0, None) == EINVAL  # wider than any fused kernel


def test_tensor_core_apply_limits():
    u = np.zeros(2 * 128 * 128, dtype=np.float32)
    up = u.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    t7, _a = _i32(list(range(7)))
    t2, _b = _i32([0, 1])
    assert L.qs_apply_fused(ctypes.c_void_p(FAKE), 14, t7, 7, up, Q.QS_PREC_TF32X3, None) == EUNSUP
    assert L.qs_apply_fused(ctypes.c_void_p(FAKE), 10, t2, 2, up, Q.QS_PREC_TF32, None) == EUNSUP


def test_plan_accessors_reject_bad_indices():
    n = 14
    cost = Q.default_cost_table()
    for k in range(16):
        cost.fuse_cost[k] *= 0.5  # fused and shared-memory kernels both appear
    p = Q.Plan(n, C.mixed_circuit(n, 250, 1), shm_max_active=12, cost=cost, shm_variant=2)
    st = p.stats()
    nk = st.num_kernels
    d = Q.qs_kernel_desc()
    assert L.qs_plan_kernel(p.h, nk, ctypes.byref(d)) == EINVAL
    assert L.qs_plan_kernel(None, 0, ctypes.byref(d)) == EINVAL
    assert L.qs_plan_kernel_gates(p.h, nk, None, 0) == EINVAL
    cnt = L.qs_plan_kernel_gates(p.h, 0, None, 0)
    assert cnt > 0
    if cnt > 1:
        ids, _k = _i32([0] * (cnt - 1))
        assert L.qs_plan_kernel_gates(p.h, 0, ids, cnt - 1) == EINVAL  # buffer too small
    types = [p.kernel(k).type for k in range(nk)]
    assert Q.QS_KERNEL_FUSED in types and Q.QS_KERNEL_SHM in types
    shm, fused = types.index(Q.QS_KERNEL_SHM), types.index(Q.QS_KERNEL_FUSED)
    out = np.zeros(2 << 14, dtype=np.float64)
    dp = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.qs_plan_fused_matrix(p.h, shm, dp, out.size) == EINVAL      # not a fused kernel
    assert L.qs_plan_fused_matrix(p.h, fused, dp, 1) == EINVAL           # buffer too small
    assert L.qs_plan_kernel_program(p.h, fused, None, 0, None) == EINVAL  # no program
    assert L.qs_plan_kernel_program(p.h, shm, None, 0, None) > 0
    assert L.qs_plan_kernel_source(p.h, fused, None, 0) == EINVAL
    a, b, c_, d_ = ctypes.c_uint64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    assert L.qs_plan_stage(p.h, 1, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c_), ctypes.byref(d_)) == EINVAL
    assert L.qs_plan_stage(p.h, -1, None, None, None, None) == EINVAL
    assert L.qs_plan_stage(p.h, 0, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c_), ctypes.byref(d_)) == 0
    assert a.value == (1 << n) - 1 and b.value == 250 and d_.value == nk
    assert L.qs_plan_stats_get(None, ctypes.byref(st)) == EINVAL


def test_timers_refuse_before_device_work():
    h = ctypes.c_void_p()
    p = Q.Plan(12, C.mixed_circuit(12, 20, 1), shm_variant=1)
    assert L.qs_timer_create(p.h, 0, ctypes.byref(h)) == EINVAL
    assert L.qs_timer_create(None, 1, ctypes.byref(h)) == EINVAL
    staged = Q.Plan(16, C.mixed_circuit(16, 100, 2), local_qubits=12, shm_max_active=12, shm_variant=1)
    assert L.qs_timer_create(staged.h, 1, ctypes.byref(h)) == EUNSUP  # staged plans: the host timer
    assert L.qs_run_plan(staged.h, ctypes.c_void_p(FAKE), None) == EUNSUP
    assert L.qs_host_timer_create(None, ctypes.byref(h)) == EINVAL
    # more stage x chunk records than a host timer holds
    wide = Q.Plan(30, C.mixed_circuit(30, 50, 3), local_qubits=12, shm_max_active=12, shm_variant=1)
    assert L.qs_host_timer_create(wide.h, ctypes.byref(h)) == EINVAL


def test_network_handles_are_checked():
    assert L.qs_mlp_num_params(None) == EINVAL
    f, hdn = ctypes.c_int32(), ctypes.c_int32()
    assert L.qs_mlp_shape(None, ctypes.byref(f), ctypes.byref(hdn)) == EINVAL
    assert L.qs_mlp_get_params(None, None, 0) == EINVAL
    assert L.qs_mlp_set_params(None, None, 0) == EINVAL
    out = ctypes.c_void_p()
    for feats, hidden in ((0, 16), (44, 0), (5000, 16), (44, 2048)):
        assert L.qs_mlp_create(feats, hidden, 0, ctypes.byref(out)) == EINVAL
    assert L.qs_mlp_create(44, 16, 0, None) == EINVAL
    assert L.qs_mlp_forward(None, None, 1, None, 1, None) == EINVAL
    assert L.qs_mlp_gradient(None, None, None, 1, None, None, None) == EINVAL


def test_planning_failures_say_why():
    g = C.make_gates([(C.H, 0), (C.CX, 5, 6), (C.H, 2)])
    with pytest.raises(Q.QsError) as e:
        Q.Plan(8, g, shm_max_active=2, forced_low=2, fuse_kmax=0, shm_variant=1)
    assert e.value.status == Q.QS_EPLAN
    msg = L.qs_last_error().decode()
    assert msg.startswith("gate 1 (CX) fits no kernel") and "3 active qubits > shm_max_active 2" in msg
    assert "fits no kernel" in str(e.value)
    with pytest.raises(Q.QsError) as e:
        Q.Plan(8, g, precision=Q.QS_PREC_TF32X3, fuse_kmax=6)
    assert e.value.status == EUNSUP and "n >= 11" in str(e.value)
    # a success clears it
    Q.Plan(8, g, shm_variant=1)
    assert L.qs_last_error() == b""


def test_new_entry_points_refuse_bad_arguments_on_the_host():
    # test-only stall limit out of range; launch counters with no room
    assert L.qs_debug_tc_stall(-1) == Q.QS_EINVAL
    assert L.qs_debug_tc_stall(10_000_001) == Q.QS_EINVAL
    assert L.qs_debug_tc_stall(0) == Q.QS_OK
    assert L.qs_debug_tc_launch_counts(None, 4) == Q.QS_EINVAL
    out = (ctypes.c_uint64 * 1)()
    assert L.qs_debug_tc_launch_counts(out, 1) == 4  # four load paths, one written
    # expectile outside (0, 1) and a null network
    assert L.qs_mlp_set_expectile(None, 0.5) == Q.QS_EINVAL
    # the insular-X rewrite: a malformed gate, and an output buffer too small
    cnt = ctypes.c_uint64()
    bad = C.make_gates([(C.CX, 0, 0, 0, 0, 0)])  # both qubits the same
    assert L.qs_insular_x_rewrite(4, Q._gates_array(bad).ctypes.data_as(ctypes.c_void_p), 1, None, 0,
                                    ctypes.byref(cnt)) == Q.QS_EINVAL
    g = Q._gates_array(C.mixed_circuit(6, 40, 2))
    assert L.qs_insular_x_rewrite(6, g.ctypes.data_as(ctypes.c_void_p), len(g), None, 0, ctypes.byref(cnt)) == 0
    small = np.zeros(max(1, cnt.value - 1), dtype=g.dtype)
    assert L.qs_insular_x_rewrite(6, g.ctypes.data_as(ctypes.c_void_p), len(g),
                                    small.ctypes.data_as(ctypes.c_void_p), len(small), ctypes.byref(cnt)) == Q.QS_EINVAL
    # insular_x outside its bit mask; a staged plan's frame export with no room
    with pytest.raises(Q.QsError) as ei:
        Q.Plan(6, C.mixed_circuit(6, 20, 3), insular_x=4)
    assert ei.value.status == Q.QS_EINVAL
    n, loc = 14, 12
    items = [(C.H, q, None, 0, 0, 0) for q in range(loc)] + [(C.X, 13, None, 0, 0, 0), (C.X, 12, None, 0, 0, 0)]
    plan = Q.Plan(n, C.make_gates(items), local_qubits=loc, shm_max_active=12, insular_x=Q.QS_INSULAR_X_STAGED)
    frame, flips = plan.stage_frame(0)
    assert frame == (1 << 12) | (1 << 13) and sorted(flips) == [loc, loc + 1]
    fr, k = ctypes.c_uint64(), ctypes.c_int64()
    one = (ctypes.c_int32 * 1)()
    assert L.qs_plan_stage_frame(plan.h, 0, ctypes.byref(fr), one, 1, ctypes.byref(k)) == Q.QS_EINVAL
