"""The learned cost model's CUDA kernels against the FP64 oracle
(oracle/mlp.py), BF16 inference against FP32, and learned-cost planning."""
import numpy as np
import pytest

from oracle import mlp as OM
from oracle import plan as OP
from oracle import sim
from synth import circuits as C
from tests.gpu_util import assert_close_state, need_gpu, run_plan_on_gpu, torch

pytestmark = pytest.mark.gpu
F = 44


def _data(B, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    x = (rng.uniform(0, 1, size=(B, F)) * scale).astype(np.float32)
    t = rng.normal(2.0, 1.0, size=B).astype(np.float32)
    return x, t


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("H", [16, 128])
def test_gradient_and_forward_match_oracle(H):
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    net = Q.Mlp(F, H, seed=3)
    theta = net.get_params().astype(np.float64)
    x, t = _data(300, H)
    xd, td = _dev(x), _dev(t)
    loss, g = net.gradient(xd.data_ptr(), td.data_ptr(), len(t))
    ref_loss, ref_g = OM.gradient(theta, x.astype(np.float64), t.astype(np.float64), F, H)
    assert abs(loss - ref_loss) <= 1e-4 * max(1.0, ref_loss)
    assert np.linalg.norm(g - ref_g) <= 1e-4 * np.linalg.norm(ref_g)
    # every parameter's gradient: FP32 batch sums of 300 products against
    # FP64, relative 1e-3 with a floor at 1e-5 of the largest entry (entries
    # that cancel to near zero carry only the rounding of their terms)
    np.testing.assert_allclose(g, ref_g, rtol=1e-3, atol=1e-5 * float(np.max(np.abs(ref_g))))
    y = torch.empty(len(t), dtype=torch.float32, device="cuda")
    net.forward(xd.data_ptr(), len(t), y.data_ptr(), bf16=False)
    ref_y, _ = OM.forward(theta, x.astype(np.float64), F, H)
    assert np.max(np.abs(y.cpu().numpy() - ref_y)) <= 1e-4 * max(1.0, np.max(np.abs(ref_y)))


def test_expectile_gradient_matches_oracle():
    # the pessimistic loss (weight 2 tau on underestimates) on the GPU
    # against the FP64 network, element by element
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    H, tau = 64, 0.8
    net = Q.Mlp(F, H, seed=7)
    net.set_expectile(tau)
    theta = net.get_params().astype(np.float64)
    x, t = _data(257, 11)
    xd, td = _dev(x), _dev(t)  # kept alive through the call
    loss, g = net.gradient(xd.data_ptr(), td.data_ptr(), len(t))
    ref_loss, ref_g = OM.gradient(theta, x.astype(np.float64), t.astype(np.float64), F, H, tau=tau)
    assert abs(loss - ref_loss) <= 1e-4 * max(1.0, ref_loss)
    np.testing.assert_allclose(g, ref_g, rtol=1e-3, atol=1e-5 * float(np.max(np.abs(ref_g))))
    with pytest.raises(Q.QsError):
        net.set_expectile(1.0)


def test_merged_ensemble_is_the_mean_of_its_networks():
    # the block-diagonal merge is exact: its FP32 forward equals the mean of
    # the member networks' forwards
    need_gpu()
    from paper_2408_09055_gb300 import costmodel as CM
    from paper_2408_09055_gb300 import qsim as Q
    nets = [Q.Mlp(F, 32, seed=s) for s in (1, 2, 3)]
    merged = CM.merge_ensemble(nets)
    x, _ = _data(200, 13)
    xd = _dev(x)
    ys = []
    for net in nets + [merged]:
        y = torch.empty(200, dtype=torch.float32, device="cuda")
        net.forward(xd.data_ptr(), 200, y.data_ptr(), bf16=False)
        ys.append(y.cpu().numpy().astype(np.float64))
    mean = np.mean(ys[:3], axis=0)
    assert np.max(np.abs(ys[3] - mean)) <= 1e-5 * max(1.0, float(np.max(np.abs(mean))))


def _bf16(a):
    """Round-to-nearest-even to bfloat16, kept in float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_inference_matches_its_definition_and_fp32():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    H = 128
    net = Q.Mlp(F, H, seed=5)
    x, _ = _data(512, 9)
    xd = _dev(x)
    y32 = torch.empty(512, dtype=torch.float32, device="cuda")
    y16 = torch.empty(512, dtype=torch.float32, device="cuda")
    net.forward(xd.data_ptr(), 512, y32.data_ptr(), bf16=False)
    net.forward(xd.data_ptr(), 512, y16.data_ptr(), bf16=True)
    a, b = y32.cpu().numpy(), y16.cpu().numpy()
    # the definition: inputs, weights and hidden activations rounded to
    # BF16, every product accumulated in FP32 (here FP64)
    p = OM.unpack(net.get_params().astype(np.float64), F, H)
    h1 = _bf16(np.maximum(_bf16(x) @ _bf16(p["W1"]) + _bf16(p["b1"]), 0))
    h2 = _bf16(np.maximum(h1 @ _bf16(p["W2"]) + _bf16(p["b2"]), 0))
    emu = h2 @ _bf16(p["W3"]) + _bf16(p["b3"])[0]
    # FP32 accumulation can flip a hidden activation to the neighbouring BF16
    # value (one unit in 2^8); the output moves by far less than that
    d = np.abs(b - emu) / (np.abs(emu) + 1.0)
    assert np.max(d) < 2e-3 and np.mean(d) < 1e-4
    gap = np.abs(a - b) / (np.abs(a) + 1.0)
    assert np.mean(gap) < 5e-3 and np.max(gap) < 3e-2


def test_train_step_is_one_adam_step():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    H = 32
    net = Q.Mlp(F, H, seed=11)
    theta = net.get_params().astype(np.float64)
    x, t = _data(128, 4)
    xd, td = _dev(x), _dev(t)
    # Adam applied to the library's own gradient (the gradient itself is
    # checked against backprop above): near-zero components would otherwise
    # step by +-lr on rounding noise
    _, g = net.gradient(xd.data_ptr(), td.data_ptr(), 128)
    opt = OM.Adam(theta.size, lr=1e-3)
    ref = opt.step(theta, g.astype(np.float64))
    net.train_step(xd.data_ptr(), td.data_ptr(), 128, 1e-3)
    got = net.get_params()
    assert np.allclose(got, ref, atol=2e-7, rtol=0)
    # a second step with the second gradient
    theta2 = got.astype(np.float64)
    _, g2 = net.gradient(xd.data_ptr(), td.data_ptr(), 128)
    ref2 = opt.step(theta2, g2.astype(np.float64))
    net.train_step(xd.data_ptr(), td.data_ptr(), 128, 1e-3)
    assert np.allclose(net.get_params(), ref2, atol=4e-7, rtol=0)


def test_training_reduces_loss():
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    net = Q.Mlp(F, 64, seed=1)
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, size=(1024, F)).astype(np.float32)
    t = (3.0 * x[:, 0] - 2.0 * x[:, 5] + np.sin(4 * x[:, 7])).astype(np.float32)
    xd, td = _dev(x), _dev(t)
    l0, _ = net.gradient(xd.data_ptr(), td.data_ptr(), 1024)
    for _ in range(400):
        net.train_step(xd.data_ptr(), td.data_ptr(), 1024, 3e-3)
    l1, _ = net.gradient(xd.data_ptr(), td.data_ptr(), 1024)
    assert l1 < 0.05 * l0


@pytest.mark.parametrize("algo", [2, 3])
def test_learned_cost_plans_are_valid_and_correct(algo):
    need_gpu()
    from paper_2408_09055_gb300 import qsim as Q
    n = 14
    g = C.mixed_circuit(n, 300, 8)
    net = Q.Mlp(F, 64, seed=2)
    theta = net.get_params()
    theta[-1] = 7.0  # about 1 ms per kernel
    net.set_params(theta)
    plan = Q.Plan(n, g, algo=algo, mlp=net, fuse_kmax=6, precision=Q.QS_PREC_TF32X3)
    assert plan.opts.cost_kind == Q.QS_COST_LEARNED
    assert plan.validate() == 0
    OP.check_plan(g, plan.kernels())
    got, _, _ = run_plan_on_gpu(n, plan)
    assert_close_state(got, sim.apply(n, g))


def test_timing_generator_and_training_end_to_end():
    need_gpu()
    from paper_2408_09055_gb300 import costmodel as CM
    X, y, meta = CM.generate(n=18, count=48, seed=1, reps=2, batch=16, log=None)
    assert X.shape == (meta["count"], F) and meta["count"] >= 40
    assert np.all(np.isfinite(y))
    _, metrics = CM.train(X, y, hidden=32, epochs=20, batch=16)
    assert np.isfinite(metrics["train"]["mse"])
