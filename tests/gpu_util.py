"""Helpers shared by the GPU tests: run a plan through the C ABI on a device
state and compare with the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

FID_TOL = 1e-6   # fidelity >= 1 - 1e-6 against FP64 in FP32
MAXABS_TOL = 1e-5


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run_plan_on_gpu(n, plan, psi0=None):
    from paper_2408_09055_gb300 import qsim as Q
    buf = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    st = Q.State(n, buf.data_ptr())
    stream = torch.cuda.current_stream().cuda_stream
    if psi0 is None:
        st.set_zero(stream)
    else:
        st.write(psi0.astype(np.complex64), stream=stream)
    st.run(plan, stream)
    out = st.read(stream=stream)
    return out, st, buf


def fidelity(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)


def assert_close_state(got, ref, fid_tol=FID_TOL, maxabs_tol=MAXABS_TOL):
    f = fidelity(ref, got)
    m = float(np.max(np.abs(np.asarray(ref) - np.asarray(got, dtype=np.complex128))))
    assert f >= 1 - fid_tol, f"fidelity {f}"
    assert m <= maxabs_tol, f"max-abs {m}"
    return f, m
