"""GPU kernels of the learned-correction network against the FP64 oracle
(oracle/cnn.py).  FP32 mode: forward to 1e-5 and gradients to 1e-4 relative
(FP32 sums over up to ~10^4 terms); BF16-operand mode: forward and gradients
within 2e-2 relative (BF16 keeps 8 significand bits, products accumulate in
FP32).  Adam matches its definition; training lowers the loss."""
import numpy as np
import pytest

from oracle import cnn as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_01163_gb300 import asdsm
    return asdsm


def _dev32(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / max(np.linalg.norm(np.asarray(b, float)), 1e-300)


def _data(seed, B=2, H=19, W=23):
    rng = np.random.default_rng(seed)
    theta = orc.init_params(seed) + 0.02 * rng.normal(size=orc.n_params())
    x = rng.normal(size=(B, 6, H, W))
    t = rng.normal(size=(B, 1, H, W))
    return theta.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64), t.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("shape", [(2, 19, 23), (1, 16, 16), (3, 33, 7)])
def test_forward_matches_oracle_fp32(lib, shape):
    B, H, W = shape
    theta, x, t = _data(1, B, H, W)
    net = lib.Cnn(theta, bf16=False)
    y = net.forward(_dev32(x)).cpu().numpy()
    yo, _ = orc.forward(theta, x)
    assert _rel(y, yo) <= 1e-5, _rel(y, yo)
    net.close()


def test_gradient_matches_oracle_fp32(lib):
    theta, x, t = _data(2)
    net = lib.Cnn(theta, bf16=False)
    loss, g = net.backward(_dev32(x), _dev32(t), want_grad=True)
    lo, go = orc.grad(theta, x, t)
    assert abs(loss - lo) <= 1e-5 * lo
    for (W, b), (Wo, bo) in zip(orc.unpack(g.astype(np.float64)), orc.unpack(go)):
        assert _rel(W, Wo) <= 1e-4, _rel(W, Wo)
        assert _rel(b, bo) <= 1e-4, _rel(b, bo)
    net.close()


def test_bf16_operands_within_bound(lib):
    theta, x, t = _data(3)
    net = lib.Cnn(theta, bf16=True)
    y = net.forward(_dev32(x)).cpu().numpy()
    yo, _ = orc.forward(theta, x)
    assert _rel(y, yo) <= 2e-2, _rel(y, yo)
    loss, g = net.backward(_dev32(x), _dev32(t), want_grad=True)
    lo, go = orc.grad(theta, x, t)
    assert _rel(g, go) <= 2e-2, _rel(g, go)
    net.close()


def test_adam_step_matches_definition(lib):
    theta, x, t = _data(4)
    net = lib.Cnn(theta, bf16=False)
    _, g = net.backward(_dev32(x), _dev32(t), want_grad=True)
    net.adam(1e-3)
    opt = orc.Adam(theta.size, lr=1e-3)
    ref = opt.step(np.asarray(net_params := theta), g.astype(np.float64))
    got = net.params().astype(np.float64)
    assert _rel(got - theta, ref - theta) <= 1e-4
    net.close()


def test_training_lowers_the_loss(lib):
    rng = np.random.default_rng(5)
    theta = orc.init_params(5)
    x = rng.normal(size=(4, 6, 32, 32))
    # a learnable target: a smooth function of the input channels
    t = 0.5 * x[:, :1] - 0.25 * x[:, 1:2] + 0.1 * x[:, 2:3] ** 2
    net = lib.Cnn(theta, bf16=True)
    xd, td = _dev32(x), _dev32(t)
    l0, _ = net.backward(xd, td)
    for _ in range(200):
        net.backward(xd, td)
        net.adam(2e-3)
    l1, _ = net.backward(xd, td)
    assert l1 < 0.2 * l0, (l0, l1)
    net.close()


def test_weighted_loss_gradient_matches_oracle(lib):
    theta, x, t = _data(7)
    rng = np.random.default_rng(7)
    w = ((rng.random(size=t.shape) < 0.3) * 3.0).astype(np.float32).astype(np.float64)
    net = lib.Cnn(theta, bf16=False)
    loss, g = net.backward(_dev32(x), _dev32(t), want_grad=True, weights=_dev32(w))
    lo, go = orc.grad(theta, x, t, w=w)
    assert abs(loss - lo) <= 1e-5 * lo
    assert _rel(g, go) <= 1e-4
    net.close()
