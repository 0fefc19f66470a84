"""ctypes wrapper of ``oracle/oracle.c`` (test infrastructure only).

The C file is compiled with plain gcc (-O2, OpenMP, no fast-math) into
``oracle/liboracle.so`` by :func:`build`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            L.or_gate_matrix.argtypes = [ctypes.c_int, dp, dp]
            L.or_apply_gate.argtypes = [ctypes.c_int, dp, ctypes.c_void_p]
            L.or_apply_circuit.argtypes = [ctypes.c_int, dp, ctypes.c_void_p, ctypes.c_int64]
            L.or_zero_state.argtypes = [ctypes.c_int, dp]
            L.or_norm2.argtypes = [ctypes.c_int, dp]
            L.or_norm2.restype = ctypes.c_double
            L.or_kernel_unitary.argtypes = [ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.POINTER(ctypes.c_int32), ctypes.c_int, dp]
            L.or_threads.restype = ctypes.c_int
            L.or_set_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _gates(gates: np.ndarray) -> np.ndarray:
    from synth.circuits import GATE_DTYPE
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    return g


def gate_matrix(gtype: int, params=(0.0, 0.0, 0.0)) -> np.ndarray:
    p = np.zeros(3, dtype=np.float64)
    p[: len(params)] = params
    dim = 4 if gtype >= 5 else 2
    m = np.zeros(2 * dim * dim, dtype=np.float64)
    rc = lib().or_gate_matrix(int(gtype), _dp(p), _dp(m))
    if rc != 0:
        raise ValueError(f"bad gate type {gtype}")
    return m.view(np.complex128).reshape(dim, dim)


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def apply(n: int, gates: np.ndarray, psi: np.ndarray | None = None) -> np.ndarray:
    """Applies ``gates`` in order to ``psi`` (a copy; default |0...0>)."""
    out = zero_state(n) if psi is None else np.array(psi, dtype=np.complex128, copy=True)
    if out.shape != (1 << n,):
        raise ValueError("state length must be 2^n")
    g = _gates(gates)
    f = out.view(np.float64)
    rc = lib().or_apply_circuit(int(n), _dp(f), g.ctypes.data_as(ctypes.c_void_p), int(len(g)))
    if rc != 0:
        raise ValueError(f"invalid gate at index {-1 - rc}")
    return out


def norm2(psi: np.ndarray) -> float:
    n = int(np.log2(psi.size))
    return float(lib().or_norm2(n, _dp(np.ascontiguousarray(psi).view(np.float64))))


def kernel_unitary(gates: np.ndarray, qubits) -> np.ndarray:
    """2^k x 2^k unitary of ``gates`` on ``qubits`` (qubits[j] -> index bit j)."""
    q = np.asarray(qubits, dtype=np.int32)
    k = len(q)
    u = np.zeros(2 * (1 << k) * (1 << k), dtype=np.float64)
    g = _gates(gates)
    rc = lib().or_kernel_unitary(g.ctypes.data_as(ctypes.c_void_p), int(len(g)),
                                 q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), k, _dp(u))
    if rc != 0:
        raise ValueError("gate outside the kernel's qubits")
    return u.view(np.complex128).reshape(1 << k, 1 << k)


def threads() -> int:
    return int(lib().or_threads())


def set_threads(t: int) -> None:
    lib().or_set_threads(int(t))
