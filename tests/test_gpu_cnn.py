"""Warm-start network on the GPU (BF16 tensor cores, FP32 accumulate) vs the
FP64 oracle (oracle/cnn.py) fed the same BF16-rounded weights and inputs.

Tolerances: every layer rounds its activations (and the backward pass its
gradients) to BF16, relative rounding 2^-9; over 8 layers and the projection
the relative L2 error of the prediction stays below 3e-2, of the loss below
3e-2 and of each layer's gradient below 1e-1 (gradients pass through the
BF16-rounded ReLU masks and activations)."""
import numpy as np
import pytest

from oracle import cnn
from paper_1503_00757_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def bf16_round(a):
    import torch
    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def _data(n, B, seed):
    xs, ts = [], []
    for i in range(B):
        mT, mR, vs = synth.ellipses_pair(n, seed + i, vmax=0.1, kmax=min(16, n // 4))
        xs.append(np.stack([mT, mR]))
        ts.append(vs)
    return np.stack(xs), np.stack(ts)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _random_data(H, W, B, seed):
    """Smooth random images and a divergence-free random target on a non-square grid."""
    rng = np.random.default_rng(seed)
    x = np.stack([np.stack([synth.gaussian_smooth(rng.random((H, W)), 0.1) for _ in range(2)]) for _ in range(B)])
    t = cnn.leray(0.1 * np.stack([np.stack([synth.gaussian_smooth(rng.standard_normal((H, W)), 0.3)
                                            for _ in range(2)]) for _ in range(B)]))
    return x, t


@pytest.mark.parametrize("H,W,B", [(64, 64, 2), (64, 256, 1)])
def test_forward_and_gradients_match_oracle(H, W, B):
    """(64, 64): dilations 1, 2, ..., 2, 1; (64, 256): the full schedule 1, 2, 4, 8, 8, 4, 2, 1
    (8 x 32 sub-grids, one tile each at d = 8)."""
    import torch
    from paper_1503_00757_gb300.binding import Net, flatten_params, unflatten_params
    params = cnn.init_params(11)
    rng = np.random.default_rng(12)
    params = [(bf16_round(W_), rng.standard_normal(b.shape) * 0.05) for W_, b in params]
    if H == W:
        x, t = _data(H, B, 5000)
    else:
        x, t = _random_data(H, W, B, 5050)
    x = bf16_round(x)
    net = Net(H, W, B)
    flat = flatten_params(params)
    net.set_params(torch.tensor(flat, dtype=torch.float32, device="cuda"))
    xg = torch.tensor(x, dtype=torch.float32, device="cuda").contiguous()
    tg = torch.tensor(t, dtype=torch.float32, device="cuda").contiguous()
    v = torch.empty(B, 2, H, W, device="cuda")
    net.forward(xg, v)
    torch.cuda.synchronize()
    v_ref = cnn.predict(params, x)
    assert _rel(v.cpu().numpy(), v_ref) < 3e-2
    grads = torch.empty(net.nparams, device="cuda")
    loss = net.loss_grad(xg, tg, grads)
    loss_ref, g_ref = cnn.loss_and_grads(params, x, t)
    assert abs(loss - loss_ref) < 3e-2 * loss_ref
    g = unflatten_params(grads.cpu().numpy().astype(np.float64), cnn.CHANNELS)
    for l, ((dW, db), (dWr, dbr)) in enumerate(zip(g, g_ref)):
        assert _rel(dW, dWr) < 1e-1, (l, _rel(dW, dWr))
        assert _rel(db, dbr) < 1e-1, (l, _rel(db, dbr))
    net.close()


def test_training_reduces_loss_and_output_is_divergence_free():
    import torch
    from oracle import spectral as S
    from paper_1503_00757_gb300.binding import Net, flatten_params
    n, B = 64, 4
    x, t = _data(n, B, 5100)
    net = Net(n, n, B)
    net.set_params(torch.tensor(flatten_params(cnn.init_params(13)), dtype=torch.float32, device="cuda"))
    xg = torch.tensor(x, dtype=torch.float32, device="cuda").contiguous()
    tg = torch.tensor(t, dtype=torch.float32, device="cuda").contiguous()
    l0 = net.loss_grad(xg, tg)
    for _ in range(60):
        net.train_step(xg, tg, 1e-3)
    l1 = net.loss_grad(xg, tg)
    assert l1 < 0.5 * l0
    v = torch.empty(B, 2, n, n, device="cuda")
    net.forward(xg, v)
    vn = v.cpu().numpy().astype(np.float64)
    for i in range(B):
        assert np.abs(S.div(vn[i])).max() < 1e-3 * np.abs(vn[i]).max()
    net.close()


def test_output_scale_multiplies_the_prediction():
    import torch
    from paper_1503_00757_gb300.binding import Net, flatten_params
    n, B = 64, 2
    x, _ = _data(n, B, 5200)
    net = Net(n, n, B)
    net.set_params(torch.tensor(flatten_params(cnn.init_params(14)), dtype=torch.float32, device="cuda"))
    xg = torch.tensor(x, dtype=torch.float32, device="cuda").contiguous()
    v1, vs = torch.empty(B, 2, n, n, device="cuda"), torch.empty(B, 2, n, n, device="cuda")
    net.forward(xg, v1)
    net.set_output_scale(0.75)
    net.forward(xg, vs)
    torch.cuda.synchronize()
    assert torch.equal(vs, 0.75 * v1)
    net.set_output_scale(1.0)
    net.forward(xg, vs)
    torch.cuda.synchronize()
    assert torch.equal(vs, v1)
    with pytest.raises(Exception):
        net.set_output_scale(0.0)
    net.close()
