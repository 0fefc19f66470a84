"""CPU check of the plan-specialised kernels' generated CUDA source
(csrc/jit.cpp): every shared-memory kernel of a plan is compiled as C++ for
the host with tests/jit_host_shim.hpp and run with one host thread per CUDA
thread, and the state after the whole plan must match the FP64 oracle
within FP32 rounding.  This covers the code generator itself -- renames,
dropped unit terms, the 2x2/4x4 products, deferred row factors, exchanges
and known-bit branches -- on random input states, without a GPU; the GPU
parity tests run the same source compiled by NVRTC."""
import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from oracle import sim
from synth import circuits as C

Q = pytest.importorskip("paper_2408_09055_gb300.qsim")
CXX = shutil.which("g++")
SHIM = os.path.join(os.path.dirname(__file__), "jit_host_shim.hpp")
pytestmark = pytest.mark.skipif(CXX is None, reason="needs g++")


def _random_state(n, seed):
    rng = np.random.default_rng(seed)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return psi / np.linalg.norm(psi)


def _build(plan, tmp_path, tag):
    """One shared library holding every kernel of the plan, each with a
    host entry run_<k>(psi, nb, hi, nthr).  A staged plan names its kernels
    by their index within the stage, so every kernel is renamed hk<k>."""
    nk = plan.stats().num_kernels
    parts = [f'#include "{SHIM}"\n']
    for k in range(nk):
        src = re.sub(r"\bqsk\d+", f"hk{k}", plan.kernel_source(k))
        parts.append(src)
        parts.append(f'extern "C" void run_{k}(float* psi, unsigned long long nb, unsigned long long hi, '
                     f"unsigned nthr) {{ host_launch(hk{k}, psi, nb, hi, nthr); }}\n")
    cpp = tmp_path / f"{tag}.cpp"
    so = tmp_path / f"{tag}.so"
    cpp.write_text("".join(parts))
    subprocess.run([CXX, "-std=c++20", "-O1", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(so), str(cpp),
                    "-lpthread"], check=True, capture_output=True)
    return ctypes.CDLL(str(so))


def _run_host(plan, n, psi, lib):
    st = psi.astype(np.complex64).view(np.float32).copy()
    for k in range(plan.stats().num_kernels):
        m = plan.kernel(k).nqubits
        f = getattr(lib, f"run_{k}")
        f.argtypes = [ctypes.c_void_p, ctypes.c_ulonglong, ctypes.c_ulonglong, ctypes.c_uint]
        f(st.ctypes.data, 1 << (n - m), 0, 1 << (m - 5))
    return st.view(np.complex64).astype(np.complex128)


CASES = [
    ("entangling", 12, lambda n: C.entangling_circuit(n, 6, 11), 10),
    ("entangling", 13, lambda n: C.entangling_circuit(n, 5, 12), 12),
    ("mixed", 13, lambda n: C.mixed_circuit(n, 300, 13), 12),
    ("mixed", 14, lambda n: C.mixed_circuit(n, 300, 14), 11),
    ("layered", 12, lambda n: C.layered_u3_cz(n, 6, 15), 10),
    ("qft", 12, lambda n: C.qft(n), 12),
]


# every case with the default deferral (factors known at generation time),
# three with runtime-conditioned diagonals deferred too, two without
PARAMS = ([c + ("1",) for c in CASES] + [CASES[0] + ("2",), CASES[2] + ("2",), CASES[5] + ("2",)]
          + [CASES[1] + ("0",), CASES[3] + ("0",)])


# and two whose store phase also keeps local bits 2 and 3 on lanes
# (QSIM_STORE_SECTORS=0: a store-only exchange when they are register bits)
PARAMS += [CASES[1] + ("1w",), CASES[3] + ("1w",)]


@pytest.mark.parametrize("kind,n,make,smax,defer", PARAMS, ids=[f"{c[0]}-{c[1]}-defer{c[4]}" for c in PARAMS])
def test_generated_source_matches_the_oracle(kind, n, make, smax, defer, tmp_path, monkeypatch):
    if defer.endswith("w"):
        monkeypatch.setenv("QSIM_STORE_SECTORS", "0")
        defer = defer[:-1]
    monkeypatch.setenv("QSIM_JIT_DEFER", defer)
    g = make(n)
    plan = Q.Plan(n, g, algo=Q.QS_ALGO_KERNELIZE, fuse_kmax=0, shm_max_active=smax, precision=Q.QS_PREC_FP32)
    for k in range(plan.stats().num_kernels):
        assert plan.kernel(k).type == Q.QS_KERNEL_SHM
    lib = _build(plan, tmp_path, f"{kind}{n}_{defer}")
    psi0 = _random_state(n, 7 * n + smax)
    got = _run_host(plan, n, psi0, lib)
    ref = sim.apply(n, g, psi0.copy())
    err = np.max(np.abs(got - ref))
    fid = abs(np.vdot(ref, got)) ** 2 / (np.vdot(got, got).real * np.vdot(ref, ref).real)
    # FP32 rounding over a few hundred gates on amplitudes of size 2^(-n/2)
    assert err < 2e-5 * 2.0 ** (-n / 2) * max(1, len(g)) ** 0.5, err
    assert 1 - fid < 1e-9


def test_deferred_factors_remove_multiplies():
    """The deferred-factor generator writes fewer floating-point multiplies
    for the dense entangling circuit (its U3, RXX and CP gates) than the
    plain one; the count is of fmaf and products in the source."""
    n = 13
    g = C.entangling_circuit(n, 5, 12)
    counts = {}
    for defer in ("1", "0"):
        os.environ["QSIM_JIT_DEFER"] = defer
        try:
            plan = Q.Plan(n, g, algo=Q.QS_ALGO_KERNELIZE, fuse_kmax=0, shm_max_active=12)
            src = "".join(plan.kernel_source(k) for k in range(plan.stats().num_kernels))
        finally:
            del os.environ["QSIM_JIT_DEFER"]
        counts[defer] = src.count("fmaf(") + src.count("f*r") + src.count("f*x")
    assert counts["1"] < 0.85 * counts["0"], counts


def test_staged_plan_sources_match_the_oracle(tmp_path):
    """A staged plan's kernels run chunk by chunk as the host-staging loop
    runs them: each stage sees the state with its local qubits first (in
    ascending order) and its regional qubits above them, every chunk of 2^L
    amplitudes is one launch view, and the chunk's regional bits reach the
    kernel as hi = chunk << L (the known-bit values of regional controls and
    phases)."""
    n, L = 15, 12
    g = C.mixed_circuit(n, 250, 21)
    plan = Q.Plan(n, g, algo=Q.QS_ALGO_KERNELIZE, fuse_kmax=0, shm_max_active=10, local_qubits=L,
                  precision=Q.QS_PREC_FP32)
    stats = plan.stats()
    assert stats.num_stages >= 2
    lib = _build(plan, tmp_path, "staged")
    psi0 = _random_state(n, 99)
    st = psi0.astype(np.complex64)
    idx = np.arange(1 << n)
    regional_controls = 0
    for si in range(stats.num_stages):
        sd = plan.stage(si)
        local = [q for q in range(n) if (sd["local_mask"] >> q) & 1]
        order = local + [q for q in range(n) if not (sd["local_mask"] >> q) & 1]
        logical = np.zeros_like(idx)
        for p_, q in enumerate(order):
            logical |= ((idx >> p_) & 1) << q
        view = st[logical].view(np.float32).copy()
        for k in range(sd["first_kernel"], sd["first_kernel"] + sd["num_kernels"]):
            m = plan.kernel(k).nqubits
            regional_controls += sum(int(b) >= L for b in re.findall(r"\(base \| hi\) >> (\d+)", plan.kernel_source(k)))
            f = getattr(lib, f"run_{k}")
            f.argtypes = [ctypes.c_void_p, ctypes.c_ulonglong, ctypes.c_ulonglong, ctypes.c_uint]
            for c in range(1 << (n - L)):
                chunk = view[2 * (c << L):2 * ((c + 1) << L)]
                f(chunk.ctypes.data, 1 << (L - m), c << L, 1 << (m - 5))
        st[logical] = view.view(np.complex64)
    ref = sim.apply(n, g, psi0.copy())
    got = st.astype(np.complex128)
    assert regional_controls > 0  # some kernel reads a regional bit (one of the chunk's hi bits)
    err = np.max(np.abs(got - ref))
    assert err < 2e-5 * 2.0 ** (-n / 2) * len(g) ** 0.5, err
