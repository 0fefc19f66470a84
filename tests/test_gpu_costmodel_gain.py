"""What the trained cost network gains over the cost model without it.

The committed network (trained on kernels timed on GB300, BF16 inference in
the library's kernels) and the analytic cost ("Cost Function in Kernelize":
alpha + the sum of per-gate costs for a shared-memory kernel, a constant
per width for a fused kernel) both predict the run time of the same
held-out timed kernels: once with the library's built-in analytic table
(the cost the analytic plans use) and once with the analytic form given its
best chance, its constants least-squares fitted on the other timed
kernels."""
import os

import numpy as np
import pytest

from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

# the learned plan may be this much slower than the analytic plan on the
# held-out seeds (the committed network, trained on 49896 timed kernels,
# measured a gain of 1.012 on seeds 101-109: 0.989 to 1.037 per seed)
GAIN_FLOOR = 0.99


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
    t = np.exp(y.astype(np.float64))
    # kernels whose gates cancel (H.H, X.X, SWAP.SWAP) compile to no code and
    # time as launch overhead (about 6 us); no feature can tell them apart
    # from kernels that move the state, and one of them alone would add
    # ~0.09 to a mean relative error, so they are left out of the comparison
    work = t > 50.0
    test = test[work[test]]
    rest = np.setdiff1d(np.arange(len(y)), test)
    rest = rest[work[rest]]
    net, _ = CM.load()
    learned = np.exp(CM.predict(net, X[test]).astype(np.float64))
    M = _analytic_design(X)
    coef, *_ = np.linalg.lstsq(M[rest], t[rest], rcond=None)
    fitted = M[test] @ coef
    from paper_2408_09055_gb300 import qsim as Q
    tab = Q.default_cost_table()
    per_type = np.array([tab.gate_cost[k] for k in range(10)])
    table = np.where(X[test, 41] > 0.5, tab.fuse_cost[6], tab.alpha + np.rint(X[test, 30:40] * 16.0) @ per_type)
    err = lambda p: float(np.mean(np.abs(p / t[test] - 1)))
    e_learned, e_fitted, e_table = err(learned), err(fitted), err(table)
    assert len(test) > 500
    assert e_learned < 0.12, e_learned
    assert e_learned < 0.9 * e_fitted, (e_learned, e_fitted)
    assert e_learned < 0.5 * e_table, (e_learned, e_table)


def test_learned_plan_against_analytic_plan_on_held_out_seeds():
    # the plan-level comparison of the cost model (config 3's evaluation at
    # 26 qubits): held-out seeds 101-109 of the 5000-gate mixed circuit, Kernelize
    # with the analytic table and with the committed network under the same
    # options, each plan timed on the GPU.  The measured gain is reported;
    # the learned plan must stay within GAIN_FLOOR of the analytic one.
    need_gpu()
    from paper_2408_09055_gb300 import costmodel as CM
    net, meta = CM.load()
    r = CM.plan_gain(net, seeds=range(101, 110), n=26, reps=3)
    print(f"learned-plan gain over the analytic plan: {r['gain']:.4f} "
          f"(analytic {r['analytic_ms']}, learned {r['learned_ms']})")
    assert all(k > 0 for k in r["learned_kernels"])
    assert r["gain"] >= GAIN_FLOOR, r
