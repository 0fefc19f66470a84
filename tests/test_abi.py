"""The C-ABI library loads on the CPU and exports every entry point that
include/qsim.h declares (no compute calls: no GPU is needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "qsim.h")).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    names = re.findall(r"\b(qs_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["qs_plan_circuit", "qs_state_create", "qs_run_plan", "qs_read_amplitudes",
                 "qs_write_amplitudes", "qs_state_norm2", "qs_remap", "qs_apply_fused",
                 "qs_plan_validate", "qs_strerror"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2408_09055_gb300 import qsim as Q
    lib = ctypes.CDLL(Q.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_defaults_without_gpu():
    from paper_2408_09055_gb300 import qsim as Q
    assert Q.lib.qs_strerror(Q.QS_EINVAL) == b"invalid argument"
    o = Q.default_opts()
    assert o.shm_max_active == 13 and o.forced_low == 4 and o.prune_T == 500 and o.algo == Q.QS_ALGO_KERNELIZE
