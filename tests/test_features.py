"""Kernel features for the learned cost model (CPU)."""
import numpy as np
import pytest

from synth import circuits as C

Q = pytest.importorskip("paper_2408_09055_gb300.qsim")


def test_feature_vector_layout():
    g = C.make_gates([(C.H, 3), (C.CX, 3, 5), (C.CP, 5, 7, 0.4), (C.RZ, 9, None, 0.1), (C.H, 3)])
    mask = (1 << 3) | (1 << 5) | 0xF
    f = Q.qs_kernel_features(30, g, Q.QS_KERNEL_SHM, mask)
    assert f.shape == (Q.QS_MLP_FEATURES,)
    assert list(np.nonzero(f[:30])[0]) == [0, 1, 2, 3, 5]
    assert f[30 + C.H] == 2 / 16 and f[30 + C.CX] == 1 / 16 and f[30 + C.CP] == 1 / 16
    assert f[30 + C.RZ] == 1 / 16
    assert f[40] == 3 / 16          # CX (insular control), CP, RZ
    assert f[41] == 0.0 and f[42] == 5 / 16 and f[43] == 5 / 64
    f2 = Q.qs_kernel_features(30, g, Q.QS_KERNEL_FUSED, mask)
    assert f2[41] == 1.0
