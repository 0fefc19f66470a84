import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# specialised kernels compiled by the tests stay in the build folder
os.environ.setdefault("QSIM_JIT_CACHE", os.path.join(ROOT, "paper_2408_09055_gb300", "_build", "jit-cache"))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
