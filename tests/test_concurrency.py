"""Plans built from several threads at once (ctypes releases the GIL for the
call) equal the plans built one at a time: the planner, the stager and the
specialised-kernel compiler and its on-disk cache share no unguarded state."""
import os
import shutil
import tempfile
import threading

import pytest

from synth import circuits as C

Q = pytest.importorskip("paper_2408_09055_gb300.qsim")


def _fingerprint(p):
    out = []
    for k in range(p.stats().num_kernels):
        d = p.kernel(k)
        out.append((d.type, d.qubit_mask, d.cost, tuple(p.kernel_gates(k))))
    return out, [s["local_mask"] for s in p.stages()] if p.stats().num_stages > 1 else []


CASES = [
    (16, C.mixed_circuit(16, 300, 1), {}),
    (16, C.entangling_circuit(16, 4, 2), {"fuse_kmax": 5}),
    (18, C.mixed_circuit(18, 200, 3), {"local_qubits": 14, "stager": 1}),
    (15, C.qft(15), {"shm_variant": 3}),
]


def test_concurrent_planning_is_deterministic(monkeypatch):
    build = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2408_09055_gb300",
                         "_build")
    os.makedirs(build, exist_ok=True)
    scratch = tempfile.mkdtemp(prefix="jit-concurrency-", dir=build)
    try:
        _run(scratch, monkeypatch)
    finally:
        shutil.rmtree(scratch, ignore_errors=True)


def _run(scratch, monkeypatch):
    monkeypatch.setenv("QSIM_JIT_CACHE", os.path.join(scratch, "jit1"))
    want = [_fingerprint(Q.Plan(n, g, shm_max_active=12, **kw)) for n, g, kw in CASES]
    monkeypatch.setenv("QSIM_JIT_CACHE", os.path.join(scratch, "jit2"))  # cold: the threads fill it together
    got, errors = {}, []

    def work(t):
        try:
            for r in range(3):
                i = (t + r) % len(CASES)
                n, g, kw = CASES[i]
                got[(t, r)] = (i, _fingerprint(Q.Plan(n, g, shm_max_active=12, **kw)))
        except Exception as e:  # reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=work, args=(t,)) for t in range(6)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    assert len(got) == 18
    for i, fp in got.values():
        assert fp == want[i]


_FINGERPRINT = '''
import hashlib, sys
sys.path.insert(0, sys.argv[1])
from synth import circuits as C
from paper_2408_09055_gb300 import qsim as Q
h = hashlib.sha256()
for n, g, kw in ((24, C.mixed_circuit(24, 800, 5), {}), (18, C.mixed_circuit(18, 200, 2), {"local_qubits": 14, "stager": 1})):
    p = Q.Plan(n, g, shm_max_active=12, shm_variant=1, **kw)
    for k in range(p.stats().num_kernels):
        d = p.kernel(k)
        h.update(repr((d.type, d.qubit_mask, d.cost, list(p.kernel_gates(k)))).encode())
    h.update(repr([s["local_mask"] for s in p.stages()]).encode())
print(h.hexdigest())
'''


def test_plans_are_the_same_in_another_process():
    # nothing in planning depends on addresses (which differ between
    # processes): a fresh interpreter builds the same plans
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    runs = [subprocess.run([sys.executable, "-c", _FINGERPRINT, root], check=True, capture_output=True,
                           text=True).stdout.strip() for _ in range(2)]
    import contextlib
    import io
    here = io.StringIO()
    saved = sys.argv
    try:
        sys.argv = ["fingerprint", root]
        with contextlib.redirect_stdout(here):
            exec(_FINGERPRINT, {"__name__": "fingerprint"})
    finally:
        sys.argv = saved
    assert runs[0] == runs[1] == here.getvalue().strip() and len(runs[0]) == 64
