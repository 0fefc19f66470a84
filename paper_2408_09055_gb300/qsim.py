"""ctypes binding of libqsim (include/qsim.h): argument marshalling only.

Every function here calls the C entry point of the same name; all compute
runs in the library's CUDA kernels.  Importing this module loads the
in-tree ``libqsim.so`` and raises if it is missing -- there is no fallback
path.  PyTorch is used by callers only for device memory and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqsim.so")

QS_OK, QS_EINVAL, QS_ENOMEM, QS_EUNSUPPORTED, QS_ETIMEDOUT, QS_ECUDA, QS_EPLAN = 0, -1, -2, -3, -4, -5, -6
QS_ALGO_PER_GATE, QS_ALGO_GREEDY, QS_ALGO_ORDERED, QS_ALGO_KERNELIZE = 0, 1, 2, 3
QS_COST_ANALYTIC, QS_COST_LEARNED = 0, 1
QS_PREC_FP32, QS_PREC_TF32, QS_PREC_TF32X3 = 0, 1, 2
QS_KERNEL_SHM, QS_KERNEL_FUSED = 0, 1
QS_STAGER_BEAM, QS_STAGER_EXACT = 0, 1
QS_MLP_FEATURES = 44
NUM_GATE_TYPES = 10


class QsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {_lib.qs_strerror(status).decode()} ({status})"
        cuda = _lib.qs_last_cuda_error().decode()
        if status == QS_ECUDA and cuda:
            msg += f" [{cuda}]"
        detail = _lib.qs_last_error().decode() if where == "qs_plan_circuit" else ""
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


QS_INSULAR_X_REWRITE, QS_INSULAR_X_STAGED = 1, 2


class qs_gate(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("nq", ctypes.c_int32), ("q", ctypes.c_int32 * 2),
                ("p", ctypes.c_double * 3)]


class qs_cost_table(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("gate_cost", ctypes.c_double * NUM_GATE_TYPES),
                ("fuse_cost", ctypes.c_double * 16)]


class qs_plan_opts(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("cost_kind", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("shm_max_active", ctypes.c_int32),
                ("forced_low", ctypes.c_int32), ("fuse_kmin", ctypes.c_int32),
                ("fuse_kmax", ctypes.c_int32), ("prune_T", ctypes.c_int32),
                ("attach_single", ctypes.c_int32), ("local_qubits", ctypes.c_int32),
                ("shm_variant", ctypes.c_int32),
                ("cost", ctypes.POINTER(qs_cost_table)), ("mlp", ctypes.c_void_p),
                ("stager_budget", ctypes.c_int64), ("stager", ctypes.c_int32),
                ("insular_x", ctypes.c_int32)]


class qs_plan_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("num_stages", ctypes.c_int32),
                ("num_gates", ctypes.c_uint64), ("num_kernels", ctypes.c_uint64),
                ("num_shm", ctypes.c_uint64), ("num_fused", ctypes.c_uint64),
                ("cost", ctypes.c_double), ("planner_ms", ctypes.c_double),
                ("dp_states", ctypes.c_uint64), ("num_phased", ctypes.c_uint64),
                ("num_exchanges", ctypes.c_uint64), ("num_jit", ctypes.c_uint64),
                ("jit_ms", ctypes.c_double), ("staging_cost", ctypes.c_int32),
                ("staging_optimal", ctypes.c_int32)]


class qs_kernel_desc(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("stage", ctypes.c_int32), ("nqubits", ctypes.c_int32),
                ("num_gates", ctypes.c_int32), ("qubit_mask", ctypes.c_uint64),
                ("cost", ctypes.c_double)]


assert ctypes.sizeof(qs_gate) == 40


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libqsim.so is not built ({LIB_PATH}); run paper_2408_09055_gb300/build.py")
    L = ctypes.CDLL(LIB_PATH)
    vp, u64, i32, i64 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64
    dp = ctypes.POINTER(ctypes.c_double)
    fp = ctypes.POINTER(ctypes.c_float)
    ip = ctypes.POINTER(ctypes.c_int32)
    sigs = {
        "qs_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "qs_last_cuda_error": ([], ctypes.c_char_p),
        "qs_last_error": ([], ctypes.c_char_p),
        "qs_plan_opts_default": ([ctypes.POINTER(qs_plan_opts)], None),
        "qs_cost_table_default": ([ctypes.POINTER(qs_cost_table)], None),
        "qs_plan_circuit": ([i32, vp, u64, ctypes.POINTER(qs_plan_opts), ctypes.POINTER(vp)], ctypes.c_int),
        "qs_plan_free": ([vp], None),
        "qs_plan_stats_get": ([vp, ctypes.POINTER(qs_plan_stats)], ctypes.c_int),
        "qs_plan_kernel": ([vp, u64, ctypes.POINTER(qs_kernel_desc)], ctypes.c_int),
        "qs_plan_kernel_gates": ([vp, u64, ip, u64], i64),
        "qs_plan_fused_matrix": ([vp, u64, dp, u64], ctypes.c_int),
        "qs_plan_validate": ([vp, vp, u64], ctypes.c_int),
        "qs_insular_x_rewrite": ([i32, vp, u64, vp, u64, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "qs_plan_kernel_source": ([vp, u64, ctypes.c_char_p, u64], i64),
        "qs_plan_kernel_program": ([vp, u64, ctypes.POINTER(ctypes.c_uint32), u64, ip], i64),
        "qs_state_create": ([i32, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "qs_alloc_state": ([i32, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "qs_state_free": ([vp], None),
        "qs_state_device_ptr": ([vp], vp),
        "qs_state_set_zero": ([vp, vp], ctypes.c_int),
        "qs_run_plan": ([vp, vp, vp], ctypes.c_int),
        "qs_run_plan_host": ([vp, vp, vp, u64, vp], ctypes.c_int),
        "qs_host_timer_create": ([vp, ctypes.POINTER(vp)], ctypes.c_int),
        "qs_run_plan_host_timed": ([vp, vp, vp, u64, vp, vp], ctypes.c_int),
        "qs_host_timer_read": ([vp, dp, u64, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "qs_host_timer_free": ([vp], None),
        "qs_plan_stage_frame": ([vp, i32, ctypes.POINTER(ctypes.c_uint64), ip, i64, ctypes.POINTER(ctypes.c_int64)],
                                ctypes.c_int),
        "qs_plan_stage": ([vp, i32, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int64), ip, ip],
                          ctypes.c_int),
        "qs_timer_create": ([vp, u64, ctypes.POINTER(vp)], ctypes.c_int),
        "qs_run_plan_timed": ([vp, vp, vp, vp], ctypes.c_int),
        "qs_timer_read": ([vp, dp, u64, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "qs_timer_free": ([vp], None),
        "qs_read_amplitudes": ([vp, u64, u64, fp, vp], ctypes.c_int),
        "qs_write_amplitudes": ([vp, u64, u64, fp, vp], ctypes.c_int),
        "qs_state_norm2": ([vp, dp, vp], ctypes.c_int),
        "qs_state_compare_c128": ([vp, vp, dp, dp, vp], ctypes.c_int),
        "qs_remap": ([vp, vp, i32, ip, vp], ctypes.c_int),
        "qs_apply_fused": ([vp, i32, ip, i32, fp, i32, vp], ctypes.c_int),
        "qs_apply_fused_static": ([vp, i32, ip, i32, fp, i32, vp], ctypes.c_int),
        "qs_sync": ([vp], ctypes.c_int),
        "qs_debug_tc_stall": ([i64], ctypes.c_int),
        "qs_debug_tc_launch_counts": ([ctypes.POINTER(ctypes.c_uint64), i32], i32),
        "qs_mlp_create": ([i32, i32, u64, ctypes.POINTER(vp)], ctypes.c_int),
        "qs_mlp_free": ([vp], None),
        "qs_mlp_num_params": ([vp], i64),
        "qs_mlp_shape": ([vp, ip, ip], ctypes.c_int),
        "qs_mlp_get_params": ([vp, fp, u64], ctypes.c_int),
        "qs_mlp_set_params": ([vp, fp, u64], ctypes.c_int),
        "qs_mlp_gradient": ([vp, vp, vp, i32, fp, fp, vp], ctypes.c_int),
        "qs_mlp_set_expectile": ([vp, ctypes.c_float], ctypes.c_int),
        "qs_mlp_train_step": ([vp, vp, vp, i32, ctypes.c_float, fp, vp], ctypes.c_int),
        "qs_mlp_forward": ([vp, vp, i32, vp, i32, vp], ctypes.c_int),
        "qs_kernel_features": ([i32, vp, u64, i32, u64, fp], ctypes.c_int),
    }
    for name, (args, res) in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


_lib = _load()
lib = _lib


def check(status: int, where: str) -> int:
    if status < 0:
        raise QsError(int(status), where)
    return status


def _gates_array(gates) -> np.ndarray:
    """Accepts a record array with fields type, nq, q0, q1, p0, p1, p2
    (the 40-byte ``qs_gate`` layout) and returns a contiguous copy."""
    g = np.ascontiguousarray(gates)
    if g.dtype.itemsize != 40:
        raise ValueError("gate records must use the 40-byte qs_gate layout")
    return g


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream", stream))


def default_opts(**kw) -> qs_plan_opts:
    o = qs_plan_opts()
    _lib.qs_plan_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k in ("cost", "mlp"):
            continue
        setattr(o, k, v)
    if kw.get("cost") is not None:
        o.cost = ctypes.pointer(kw["cost"])
    if kw.get("mlp") is not None:
        o.mlp = kw["mlp"].h.value
        o.cost_kind = QS_COST_LEARNED
    # the options hold raw pointers: keep their owners alive with them
    o._owners = (kw.get("cost"), kw.get("mlp"))
    return o


def default_cost_table() -> qs_cost_table:
    t = qs_cost_table()
    _lib.qs_cost_table_default(ctypes.byref(t))
    return t


class Plan:
    """Owns a ``qs_plan*`` (qs_plan_circuit / qs_plan_free)."""

    def __init__(self, n: int, gates, opts: qs_plan_opts | None = None, **kw):
        g = _gates_array(gates)
        self._gates = g
        self.opts = opts if opts is not None else default_opts(**kw)
        h = ctypes.c_void_p()
        check(_lib.qs_plan_circuit(int(n), g.ctypes.data_as(ctypes.c_void_p), len(g),
                                   ctypes.byref(self.opts), ctypes.byref(h)), "qs_plan_circuit")
        self.h = h
        self.n = n

    def __del__(self):
        if getattr(self, "h", None):
            _lib.qs_plan_free(self.h)
            self.h = None

    def stats(self) -> qs_plan_stats:
        s = qs_plan_stats()
        check(_lib.qs_plan_stats_get(self.h, ctypes.byref(s)), "qs_plan_stats_get")
        return s

    def kernel(self, k: int) -> qs_kernel_desc:
        d = qs_kernel_desc()
        check(_lib.qs_plan_kernel(self.h, k, ctypes.byref(d)), "qs_plan_kernel")
        return d

    def kernel_gates(self, k: int) -> list[int]:
        cnt = check(_lib.qs_plan_kernel_gates(self.h, k, None, 0), "qs_plan_kernel_gates")
        buf = (ctypes.c_int32 * max(cnt, 1))()
        check(_lib.qs_plan_kernel_gates(self.h, k, buf, cnt), "qs_plan_kernel_gates")
        return list(buf[:cnt])

    def kernels(self) -> list[list[int]]:
        return [self.kernel_gates(k) for k in range(self.stats().num_kernels)]

    def fused_matrix(self, k: int) -> np.ndarray:
        d = self.kernel(k)
        dim = 1 << d.nqubits
        out = np.zeros(2 * dim * dim, dtype=np.float64)
        check(_lib.qs_plan_fused_matrix(self.h, k, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        out.size), "qs_plan_fused_matrix")
        return out.view(np.complex128).reshape(dim, dim)

    def kernel_source(self, k: int) -> str:
        n = check(_lib.qs_plan_kernel_source(self.h, k, None, 0), "qs_plan_kernel_source")
        buf = ctypes.create_string_buffer(n + 1)
        check(_lib.qs_plan_kernel_source(self.h, k, buf, n + 1), "qs_plan_kernel_source")
        return buf.value.decode()

    def kernel_program(self, k: int):
        """(words, m, active qubits, load-phase slot bits) of shared-memory
        kernel k's register-phased program (qs_plan_kernel_program)."""
        cnt = check(_lib.qs_plan_kernel_program(self.h, k, None, 0, None), "qs_plan_kernel_program")
        words = np.zeros(max(cnt, 1), dtype=np.uint32)
        layout = (ctypes.c_int32 * 20)()
        check(_lib.qs_plan_kernel_program(self.h, k, words.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                          words.size, layout), "qs_plan_kernel_program")
        m = int(layout[0])
        return words[:cnt], m, [int(x) for x in layout[1:1 + m]], [int(x) for x in layout[15:20]]

    def validate(self, gates=None) -> int:
        g = self._gates if gates is None else _gates_array(gates)
        return _lib.qs_plan_validate(self.h, g.ctypes.data_as(ctypes.c_void_p), len(g))

    def stage(self, i: int) -> dict:
        """qs_plan_stage: local qubit mask, gate count and kernel range."""
        mask, ng = ctypes.c_uint64(), ctypes.c_int64()
        first, cnt = ctypes.c_int32(), ctypes.c_int32()
        check(_lib.qs_plan_stage(self.h, int(i), ctypes.byref(mask), ctypes.byref(ng), ctypes.byref(first),
                                 ctypes.byref(cnt)), "qs_plan_stage")
        return {"local_mask": int(mask.value), "num_gates": int(ng.value),
                "first_kernel": int(first.value), "num_kernels": int(cnt.value)}

    def stage_frame(self, i: int) -> tuple[int, list[int]]:
        """qs_plan_stage_frame: (flipped regional qubits as a mask, circuit
        indices of the X gates the stage executes as a relabelling)."""
        fr, cnt = ctypes.c_uint64(), ctypes.c_int64()
        check(_lib.qs_plan_stage_frame(self.h, int(i), ctypes.byref(fr), None, 0, ctypes.byref(cnt)),
              "qs_plan_stage_frame")
        ids = (ctypes.c_int32 * max(1, cnt.value))()
        check(_lib.qs_plan_stage_frame(self.h, int(i), ctypes.byref(fr), ids, cnt.value, ctypes.byref(cnt)),
              "qs_plan_stage_frame")
        return int(fr.value), [int(ids[k]) for k in range(cnt.value)]

    def stages(self) -> list[dict]:
        return [self.stage(i) for i in range(self.stats().num_stages)]

    def run_host(self, host_ptr: int, device_buffer: int = 0, buffer_bytes: int = 0, stream=None):
        """qs_run_plan_host: applies the plan to a page-locked host state
        (2^n complex64) chunk by chunk; asynchronous on `stream`."""
        check(_lib.qs_run_plan_host(self.h, ctypes.c_void_p(host_ptr), ctypes.c_void_p(device_buffer or None),
                                    int(buffer_bytes), _stream_ptr(stream)), "qs_run_plan_host")


class Timer:
    """Per-kernel CUDA-event timer (qs_timer_*)."""

    def __init__(self, plan: Plan, max_runs: int):
        h = ctypes.c_void_p()
        check(_lib.qs_timer_create(plan.h, int(max_runs), ctypes.byref(h)), "qs_timer_create")
        self.h = h
        self.plan = plan

    def __del__(self):
        if getattr(self, "h", None):
            _lib.qs_timer_free(self.h)
            self.h = None

    def read(self):
        nk = self.plan.stats().num_kernels
        out = np.zeros(max(nk, 1), dtype=np.float64)
        runs = ctypes.c_uint64()
        check(_lib.qs_timer_read(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.size,
                                 ctypes.byref(runs)), "qs_timer_read")
        return out[:nk], int(runs.value)


class HostTimer:
    """Per-chunk timeline of a staged host run (qs_host_timer_*)."""

    def __init__(self, plan: Plan):
        h = ctypes.c_void_p()
        check(_lib.qs_host_timer_create(plan.h, ctypes.byref(h)), "qs_host_timer_create")
        self.h = h
        self.plan = plan

    def __del__(self):
        if getattr(self, "h", None):
            _lib.qs_host_timer_free(self.h)
            self.h = None

    def run(self, host_ptr: int, device_buffer: int = 0, buffer_bytes: int = 0, stream=None):
        check(_lib.qs_run_plan_host_timed(self.plan.h, ctypes.c_void_p(host_ptr),
                                          ctypes.c_void_p(device_buffer or None), int(buffer_bytes), self.h,
                                          _stream_ptr(stream)), "qs_run_plan_host_timed")

    def read(self) -> np.ndarray:
        """Array [stages, chunks, 4] of ms since the call began: copy-in
        start, kernels start, copy-out start, copy-out end."""
        st = self.plan.stats()
        nrec = ctypes.c_uint64()
        L = self.plan.opts.local_qubits if 0 < self.plan.opts.local_qubits < self.plan.n else self.plan.n
        cap = st.num_stages << (self.plan.n - L)
        out = np.zeros(4 * cap, dtype=np.float64)
        check(_lib.qs_host_timer_read(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.size,
                                      ctypes.byref(nrec)), "qs_host_timer_read")
        return out.reshape(st.num_stages, -1, 4)


class State:
    """Owns a ``qs_state*``; ``device_ptr`` (e.g. a torch tensor's data_ptr)
    makes it a view of caller memory."""

    @classmethod
    def alloc(cls, n: int, stream=None) -> "State":
        """qs_alloc_state: a library-owned state initialised to |0...0>."""
        self = cls.__new__(cls)
        h = ctypes.c_void_p()
        check(_lib.qs_alloc_state(int(n), _stream_ptr(stream), ctypes.byref(h)), "qs_alloc_state")
        self.h = h
        self.n = n
        return self

    def __init__(self, n: int, device_ptr: int | None = None):
        h = ctypes.c_void_p()
        check(_lib.qs_state_create(int(n), device_ptr, ctypes.byref(h)), "qs_state_create")
        self.h = h
        self.n = n

    def __del__(self):
        if getattr(self, "h", None):
            _lib.qs_state_free(self.h)
            self.h = None

    @property
    def device_ptr(self) -> int:
        return _lib.qs_state_device_ptr(self.h)

    def set_zero(self, stream=None):
        check(_lib.qs_state_set_zero(self.h, _stream_ptr(stream)), "qs_state_set_zero")

    def run(self, plan: Plan, stream=None):
        check(_lib.qs_run_plan(plan.h, self.h, _stream_ptr(stream)), "qs_run_plan")

    def run_timed(self, plan: Plan, timer: Timer, stream=None):
        check(_lib.qs_run_plan_timed(plan.h, self.h, timer.h, _stream_ptr(stream)), "qs_run_plan_timed")

    def read(self, first: int = 0, count: int | None = None, out: np.ndarray | None = None,
             stream=None) -> np.ndarray:
        count = (1 << self.n) - first if count is None else count
        if out is None:
            out = np.empty(count, dtype=np.complex64)
        f = out.view(np.float32)
        check(_lib.qs_read_amplitudes(self.h, first, count, f.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                      _stream_ptr(stream)), "qs_read_amplitudes")
        return out

    def write(self, amps: np.ndarray, first: int = 0, stream=None):
        a = np.ascontiguousarray(amps, dtype=np.complex64)
        check(_lib.qs_write_amplitudes(self.h, first, a.size,
                                       a.view(np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                       _stream_ptr(stream)), "qs_write_amplitudes")

    def norm2(self, stream=None) -> float:
        v = ctypes.c_double()
        check(_lib.qs_state_norm2(self.h, ctypes.byref(v), _stream_ptr(stream)), "qs_state_norm2")
        return v.value

    def compare_c128(self, ref_device_ptr: int, stream=None) -> tuple[float, float]:
        f, m = ctypes.c_double(), ctypes.c_double()
        check(_lib.qs_state_compare_c128(self.h, ref_device_ptr, ctypes.byref(f), ctypes.byref(m),
                                         _stream_ptr(stream)), "qs_state_compare_c128")
        return f.value, m.value


def qs_remap(in_ptr: int, out_ptr: int, n: int, perm, stream=None):
    p = (ctypes.c_int32 * n)(*[int(x) for x in perm])
    check(_lib.qs_remap(in_ptr, out_ptr, n, p, _stream_ptr(stream)), "qs_remap")


def qs_apply_fused(state_ptr: int, n: int, targets, u: np.ndarray, precision: int, stream=None):
    t = (ctypes.c_int32 * len(targets))(*[int(x) for x in targets])
    uu = np.ascontiguousarray(u, dtype=np.complex64)
    check(_lib.qs_apply_fused(state_ptr, n, t, len(targets),
                              uu.view(np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                              precision, _stream_ptr(stream)), "qs_apply_fused")


def qs_apply_fused_static(state_ptr: int, n: int, targets, u: np.ndarray, precision: int, stream=None):
    """Allocation-free form of qs_apply_fused (k <= 7, shared static staging buffer)."""
    t = (ctypes.c_int32 * len(targets))(*[int(x) for x in targets])
    uu = np.ascontiguousarray(u, dtype=np.complex64)
    check(_lib.qs_apply_fused_static(state_ptr, n, t, len(targets),
                                     uu.view(np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                     precision, _stream_ptr(stream)), "qs_apply_fused_static")


def qs_insular_x_rewrite(n: int, gates) -> np.ndarray:
    """The Pauli-frame rewrite an insular-X plan executes (gate array)."""
    g = _gates_array(gates)
    cnt = ctypes.c_uint64()
    check(_lib.qs_insular_x_rewrite(int(n), g.ctypes.data_as(ctypes.c_void_p), len(g), None, 0,
                                    ctypes.byref(cnt)), "qs_insular_x_rewrite")
    out = np.zeros(cnt.value, dtype=g.dtype)
    check(_lib.qs_insular_x_rewrite(int(n), g.ctypes.data_as(ctypes.c_void_p), len(g),
                                    out.ctypes.data_as(ctypes.c_void_p), len(out), ctypes.byref(cnt)),
          "qs_insular_x_rewrite")
    return out


def qs_sync(stream=None):
    """Synchronises the stream; raises QsError (QS_ETIMEDOUT, QS_ECUDA) for
    errors of the work queued on it."""
    check(_lib.qs_sync(_stream_ptr(stream)), "qs_sync")


def qs_debug_tc_stall(limit_us: int):
    """Test-only: later tensor-core launches give up after limit_us on a
    barrier nothing signals (0: off)."""
    check(_lib.qs_debug_tc_stall(int(limit_us)), "qs_debug_tc_stall")


def qs_debug_tc_launch_counts() -> dict:
    """Tensor-core fused launches so far, per load path (test-only)."""
    out = (ctypes.c_uint64 * 4)()
    nv = _lib.qs_debug_tc_launch_counts(out, 4)
    if nv < 0:
        check(nv, "qs_debug_tc_launch_counts")
    return {"register": int(out[0]), "bulk": int(out[1]), "wide": int(out[2]), "cpasync": int(out[3])}


def _fp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Mlp:
    """Owns a ``qs_mlp*`` (learned kernel-cost model, device parameters)."""

    def __init__(self, features: int = QS_MLP_FEATURES, hidden: int = 128, seed: int = 0):
        h = ctypes.c_void_p()
        check(_lib.qs_mlp_create(int(features), int(hidden), int(seed), ctypes.byref(h)), "qs_mlp_create")
        self.h = h
        self.features, self.hidden = features, hidden

    def __del__(self):
        if getattr(self, "h", None):
            _lib.qs_mlp_free(self.h)
            self.h = None

    @property
    def num_params(self) -> int:
        return int(_lib.qs_mlp_num_params(self.h))

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params, dtype=np.float32)
        check(_lib.qs_mlp_get_params(self.h, _fp(out), out.size), "qs_mlp_get_params")
        return out

    def set_params(self, theta) -> None:
        t = np.ascontiguousarray(theta, dtype=np.float32)
        check(_lib.qs_mlp_set_params(self.h, _fp(t), t.size), "qs_mlp_set_params")

    def gradient(self, x_ptr: int, t_ptr: int, batch: int, stream=None):
        g = np.empty(self.num_params, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        check(_lib.qs_mlp_gradient(self.h, x_ptr, t_ptr, int(batch), _fp(g), _fp(loss), _stream_ptr(stream)),
              "qs_mlp_gradient")
        return float(loss[0]), g

    def set_expectile(self, tau: float) -> None:
        check(_lib.qs_mlp_set_expectile(self.h, float(tau)), "qs_mlp_set_expectile")

    def train_step(self, x_ptr: int, t_ptr: int, batch: int, lr: float, stream=None) -> float:
        loss = np.zeros(1, dtype=np.float32)
        check(_lib.qs_mlp_train_step(self.h, x_ptr, t_ptr, int(batch), float(lr), _fp(loss),
                                     _stream_ptr(stream)), "qs_mlp_train_step")
        return float(loss[0])

    def forward(self, x_ptr: int, batch: int, y_ptr: int, bf16: bool, stream=None) -> None:
        check(_lib.qs_mlp_forward(self.h, x_ptr, int(batch), y_ptr, 1 if bf16 else 0, _stream_ptr(stream)),
              "qs_mlp_forward")


def qs_kernel_features(n: int, gates, kernel_type: int, qubit_mask: int) -> np.ndarray:
    g = _gates_array(gates)
    out = np.zeros(QS_MLP_FEATURES, dtype=np.float32)
    check(_lib.qs_kernel_features(int(n), g.ctypes.data_as(ctypes.c_void_p), len(g), int(kernel_type),
                                  int(qubit_mask), _fp(out)), "qs_kernel_features")
    return out
