"""The surrogate network's forward pass, gradients and training through the C ABI against the
FP64 reference in oracle/mlp.py (weights set from the test, so both sides see the same network)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import mlp as M  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_00011_gb300 import build
    build.build()


DIMS = [64, 256, 256, 136]
N_IN = 12


def _setup(seed=3, B=64):
    from paper_1904_00011_gb300.surrogate import Mlp
    rng = np.random.default_rng(seed)
    lo = -np.ones(N_IN)
    hi = np.ones(N_IN) * 3.0
    net = Mlp(DIMS, N_IN, lo, hi, max_batch=B, seed=1)
    Ws, bs = [], []
    for l in range(len(DIMS) - 1):
        K = DIMS[l]
        k_real = N_IN if l == 0 else K
        W = np.zeros((DIMS[l + 1], K), np.float32)
        W[:, :k_real] = rng.normal(0, 1 / np.sqrt(k_real), size=(DIMS[l + 1], k_real))
        b = rng.normal(0, 0.1, size=DIMS[l + 1]).astype(np.float32)
        net.set_layer(l, W, b)
        # the device computes with BF16 copies of the weights: give the reference the same values
        Ws.append(torch.from_numpy(W).to(torch.bfloat16).float().numpy().astype(np.float64))
        bs.append(b.astype(np.float64))
    theta = rng.uniform(lo, hi, size=(B, N_IN)).astype(np.float32)
    x = M.normalise(theta, lo, hi, DIMS[0])
    x = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)
    return net, Ws, bs, theta, x


def test_forward_matches_fp64_reference():
    net, Ws, bs, theta, x = _setup()
    got = net.predict(theta).cpu().numpy()
    ref, _, _ = M.forward(Ws, bs, x)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < 3e-2, err


@pytest.mark.parametrize("poisson", [False, True])
def test_gradients_match_fp64_reference(poisson):
    net, Ws, bs, theta, x = _setup(seed=4)
    rng = np.random.default_rng(9)
    if poisson:
        y = rng.poisson(1.5, size=(theta.shape[0], DIMS[-1])).astype(np.float32)
        net.set_loss(True)
    else:
        y = rng.normal(size=(theta.shape[0], DIMS[-1])).astype(np.float32)
    net.set_targets(torch.from_numpy(y).cuda(), theta.shape[0])
    net.train_step(theta, lr=0.0, update=False)
    loss = net.loss()
    ref_loss, gW, gb = M.loss_and_grads(Ws, bs, x, y.astype(np.float64), poisson)
    assert abs(loss - ref_loss) <= 3e-2 * ref_loss
    for l in range(len(DIMS) - 1):
        _, _, gw, gbb = net.get_layer(l)
        k_real = N_IN if l == 0 else DIMS[l]
        rel = np.linalg.norm(gw[:, :k_real] - gW[l][:, :k_real]) / np.linalg.norm(gW[l][:, :k_real])
        relb = np.linalg.norm(gbb - gb[l]) / np.linalg.norm(gb[l])
        assert rel < 5e-2 and relb < 5e-2, (l, rel, relb)


def test_training_reduces_loss_on_smooth_target():
    net, Ws, bs, theta, x = _setup(seed=5, B=128)
    rng = np.random.default_rng(10)
    A = rng.normal(size=(N_IN, DIMS[-1]))
    losses = []
    for step in range(300):
        th = rng.uniform(-1, 3, size=(128, N_IN)).astype(np.float32)
        xn = 2 * (th + 1) / 4 - 1
        y = np.tanh(xn @ A / 3).astype(np.float32)
        net.set_targets(torch.from_numpy(y).cuda(), 128)
        net.train_step(th, lr=1e-3)
        if step % 50 == 0 or step == 299:
            losses.append(net.loss())
    assert losses[-1] < 0.1 * losses[0], losses


@pytest.mark.parametrize("poisson", [True, False])
def test_surrogate_loglike_matches_fp64_reference(poisson):
    net, Ws, bs, theta, x = _setup(seed=6)
    net.set_loss(poisson)
    y = net.predict(theta)
    rng = np.random.default_rng(11)
    d = rng.poisson(3.0, size=DIMS[-1]).astype(np.uint32)
    d[::7] = 0
    d_dev = torch.from_numpy(d.astype(np.int32)).cuda()
    scale, ratio = 16.0, 0.7
    got = net.loglike(theta.shape[0], d_dev, scale, ratio)
    ref = M.surrogate_loglike(y.cpu().numpy(), d, scale, ratio, poisson)
    assert np.allclose(got, ref, rtol=1e-5, atol=1e-3), np.abs(got - ref).max()


@pytest.mark.parametrize("poisson", [True, False])
def test_fused_forward_loglike_matches_two_step_path(poisson):
    net, Ws, bs, theta, x = _setup(seed=7)
    net.set_loss(poisson)
    rng = np.random.default_rng(12)
    d = rng.poisson(2.0, size=DIMS[-1]).astype(np.uint32)
    d[::5] = 0
    d_dev = torch.from_numpy(d.astype(np.int32)).cuda()
    scale, ratio = 9.0, 1.3
    y = net.predict(theta)
    two = net.loglike(theta.shape[0], d_dev, scale, ratio)
    fused = net.forward_loglike(theta, d_dev, scale, ratio)
    ref = M.surrogate_loglike(y.cpu().numpy(), d, scale, ratio, poisson)
    assert np.allclose(fused, two, rtol=1e-5, atol=1e-3), np.abs(fused - two).max()
    assert np.allclose(fused, ref, rtol=1e-5, atol=1e-3)
