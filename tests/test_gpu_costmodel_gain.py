"""What the trained cost network gains over the cost model without it.

The committed network (trained on kernels timed on GB300, BF16 inference in
the library's kernels) and the analytic cost ("Cost Function in Kernelize":
alpha + the sum of per-gate costs for a shared-memory kernel, a constant
per width for a fused kernel) both predict the run time of the same
held-out timed kernels.  The analytic form is given its best chance: its
constants are least-squares fitted on the other timed kernels."""
import os

import numpy as np
import pytest

from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _analytic_design(X):
    fused = X[:, 41] > 0.5
    counts = np.rint(X[:, 30:40] * 16.0)
    return np.column_stack([~fused, fused, counts * (~fused)[:, None]]).astype(np.float64)


def test_learned_cost_beats_the_analytic_cost_on_held_out_kernels():
    need_gpu()
    from paper_2408_09055_gb300 import costmodel as CM
    path = os.path.splitext(CM.MODEL_PATH)[0] + "_data.npz"
    d = np.load(path)
    X, y, test = d["X"], d["y"], d["test_idx"]
    rest = np.setdiff1d(np.arange(len(y)), test)
    t = np.exp(y.astype(np.float64))
    net, _ = CM.load()
    learned = np.exp(CM.predict(net, X[test]).astype(np.float64))
    M = _analytic_design(X)
    coef, *_ = np.linalg.lstsq(M[rest], t[rest], rcond=None)
    analytic = M[test] @ coef
    e_learned = float(np.mean(np.abs(learned / t[test] - 1)))
    e_analytic = float(np.mean(np.abs(analytic / t[test] - 1)))
    assert len(test) > 500
    assert e_learned < 0.12, e_learned
    assert e_learned < 0.75 * e_analytic, (e_learned, e_analytic)
