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


def test_binding_structs_match_the_header_layout():
    import shutil
    import tempfile
    build = os.path.join(ROOT, "paper_2408_09055_gb300", "_build")
    os.makedirs(build, exist_ok=True)
    scratch = tempfile.mkdtemp(prefix="layout-", dir=build)
    try:
        _check_layout(scratch)
    finally:
        shutil.rmtree(scratch, ignore_errors=True)


def _check_layout(scratch):
    # sizeof and every field offset of the header's structs, from a C
    # compiler, against the ctypes mirrors in the binding
    import shutil
    import subprocess
    from paper_2408_09055_gb300 import qsim as Q
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [Q.qs_gate, Q.qs_cost_table, Q.qs_plan_opts, Q.qs_plan_stats, Q.qs_kernel_desc]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "qsim.h"', "int main(void) {"]
    for S in structs:
        name = S.__name__
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f in S._fields_:
            lines.append(f'  printf("{name}.{f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = os.path.join(scratch, "layout.c")
    with open(src, "w") as f:
        f.write("\n".join(lines) + "\n")
    exe = os.path.join(scratch, "layout")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([exe], check=True, capture_output=True,
                                                              text=True).stdout.splitlines())
    for S in structs:
        assert int(got[S.__name__]) == ctypes.sizeof(S), S.__name__
        for f in S._fields_:
            assert int(got[f"{S.__name__}.{f[0]}"]) == getattr(S, f[0]).offset, f"{S.__name__}.{f[0]}"
    # every field the header declares is mirrored: C size = ctypes size above,
    # and the default options fill the stager fields
    o = Q.default_opts()
    assert o.stager == Q.QS_STAGER_BEAM and o.stager_budget == 0
