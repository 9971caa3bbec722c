"""Warm-start network on the GPU (BF16 tensor cores, FP32 accumulate) vs the
FP64 oracle (oracle/cnn.py), for both convolution kernels (tcgen05 / TMEM and
mma.sync).

Per layer (test_per_layer_parity): the oracle is fed the GPU's own BF16 layer
input (and, backward, the GPU's BF16 output gradient), so each comparison
sees one layer's arithmetic only.  A BF16 output differs from its FP64 value
by at most 2^-9 relative (rounding) plus the FP32 accumulation error of 9 Cin
products (~1e-6), so the relative L2 error of a layer's output and of its
input gradient stays below 1e-2; the FP32 raw output of the last layer and
the FP32 parameter gradients (sums of exact BF16 products over B H W pixels
in FP32) stay below 1e-4.

End to end (test_forward_and_gradients_match_oracle): the oracle runs in FP64
from the BF16-rounded weights and inputs, so the BF16 rounding of every
activation compounds over 8 layers and the projection: prediction and loss
within 3e-2, each layer's gradient within 1e-1 (it passes through the
BF16-rounded ReLU masks and activations)."""
import numpy as np
import pytest

from oracle import cnn
from paper_1503_00757_gb300 import synth

from .gpu_util import check

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


KINDS = ["tcgen05", "mma_sync"]


def _kind(name):
    from paper_1503_00757_gb300.binding import REG_CONV_MMA_SYNC, REG_CONV_TCGEN05
    return REG_CONV_TCGEN05 if name == "tcgen05" else REG_CONV_MMA_SYNC


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("H,W,B", [(64, 64, 2), (64, 256, 1)])
def test_forward_and_gradients_match_oracle(H, W, B, kind):
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
    net.set_conv_kernel(_kind(kind))
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


def _layer(net, kind, l, shape):
    import torch
    out = torch.empty(shape, device="cuda")
    net.layer_tensor(kind, l, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("H,W,B", [(64, 64, 2), (64, 256, 1), (256, 256, 3)])
def test_per_layer_parity(H, W, B, kind):
    """Every layer against the oracle fed the GPU's BF16 tensors of that layer.  (256, 256, 3):
    768 tiles, more than the persistent tcgen05 grid, so CTAs loop over several tiles."""
    import torch
    from paper_1503_00757_gb300.binding import (REG_NET_INPUT, REG_NET_OUTPUT, REG_NET_OUTPUT_GRAD, Net,
                                                flatten_params, unflatten_params)
    params = cnn.init_params(21)
    rng = np.random.default_rng(22)
    params = [(bf16_round(W_), bf16_round(rng.standard_normal(b.shape) * 0.05)) for W_, b in params]
    x, t = _random_data(H, W, B, 5300 + H)
    x = bf16_round(x)
    net = Net(H, W, B)
    net.set_conv_kernel(_kind(kind))
    net.set_record(True)
    net.set_params(torch.tensor(flatten_params(params), dtype=torch.float32, device="cuda"))
    xg = torch.tensor(x, dtype=torch.float32, device="cuda").contiguous()
    tg = torch.tensor(t, dtype=torch.float32, device="cuda").contiguous()
    grads = torch.empty(net.nparams, device="cuda")
    net.loss_grad(xg, tg, grads)
    g = unflatten_params(grads.cpu().numpy().astype(np.float64), cnn.CHANNELS)
    dil = cnn.dilations(H, W)
    M = 2 * B * H * W
    L = len(params)
    a0 = _layer(net, REG_NET_INPUT, 0, (B, 2, H, W))
    assert np.array_equal(a0, x)
    for l, (Wl, bl) in enumerate(params):
        cout, cin = Wl.shape[:2]
        a = _layer(net, REG_NET_INPUT, l, (B, cin, H, W))
        z = cnn.conv3x3(a, Wl, bl, dil[l])
        out = _layer(net, REG_NET_OUTPUT, l, (B, cout, H, W))
        if l < L - 1:
            check(f"network layer output, BF16 ({kind})", _rel(out, np.maximum(z, 0.0)), 1e-2, layer=l)
        else:
            check(f"network raw output, FP32 ({kind})", _rel(out, z), 1e-4, layer=l)
        dz = _layer(net, REG_NET_OUTPUT_GRAD, l, (B, cout, H, W))
        da, dW, db = cnn.conv3x3_backward(a, Wl, dz / M, dil[l])
        check(f"network weight gradient ({kind})", _rel(g[l][0], dW), 1e-4, layer=l)
        check(f"network bias gradient ({kind})", _rel(g[l][1], db), 1e-4, layer=l)
        if l > 0:
            dz_prev = _layer(net, REG_NET_OUTPUT_GRAD, l - 1, (B, cin, H, W))
            ref = M * da * (a > 0.0)
            check(f"network input gradient, BF16 ({kind})", _rel(dz_prev, ref), 1e-2, layer=l)
    net.close()


def test_conv_kernels_agree():
    """tcgen05 and mma.sync accumulate the same BF16 products in FP32: the raw outputs agree
    to FP32 summation order through 8 BF16-rounded layers."""
    import torch
    from paper_1503_00757_gb300.binding import REG_NET_OUTPUT, Net, flatten_params
    H, W, B = 128, 128, 2
    x, _ = _random_data(H, W, B, 5400)
    xg = torch.tensor(bf16_round(x), dtype=torch.float32, device="cuda").contiguous()
    flat = torch.tensor(flatten_params(cnn.init_params(23)), dtype=torch.float32, device="cuda")
    outs = []
    for kind in KINDS:
        net = Net(H, W, B)
        net.set_conv_kernel(_kind(kind))
        net.set_params(flat)
        v = torch.empty(B, 2, H, W, device="cuda")
        net.forward(xg, v)
        outs.append(_layer(net, REG_NET_OUTPUT, 7, (B, 2, H, W)))
        net.close()
    assert _rel(outs[0], outs[1]) < 1e-2


def test_forward_fine_matches_oracle():
    """Warm start on the doubled grid (reg_net_forward_fine): a 64^2 network applied to 128^2
    pairs.  Checked in three parts.  (1) The restricted images the network saw: the GPU's packed
    BF16 input of layer 0 against the oracle's FP64 full weighting rounded to BF16 (one BF16
    rounding apart at most: one unit in the last place, at most 2^-7 of the value).  (2) Everything after the network: the oracle applies
    the coarse output map, the bilinear prolongation, the fine output map and the scale to the
    GPU's own FP32 raw network output (FP32 spectral passes: 1e-5).  (3) End to end against
    oracle.cnn.predict_fine with BF16-rounded weights (3e-2, as for the coarse forward pass)."""
    import torch
    from paper_1503_00757_gb300.binding import REG_NET_INPUT, REG_NET_OUTPUT, Net, flatten_params
    H, B, s = 64, 2, 0.7
    params = cnn.init_params(31)
    rng = np.random.default_rng(32)
    params = [(bf16_round(W_), rng.standard_normal(b.shape) * 0.05) for W_, b in params]
    x = np.stack([np.stack(synth.ellipses_pair(2 * H, 5500 + i, vmax=0.098, kmax=8)[:2]) for i in range(B)])
    net = Net(H, H, B)
    net.set_params(torch.tensor(flatten_params(params), dtype=torch.float32, device="cuda"))
    net.set_output_scale(s)
    xg = torch.tensor(x, dtype=torch.float32, device="cuda").contiguous()
    v = torch.empty(B, 2, 2 * H, 2 * H, device="cuda")
    net.forward_fine(xg, v)
    torch.cuda.synchronize()
    vg = v.cpu().numpy().astype(np.float64)
    a0 = _layer(net, REG_NET_INPUT, 0, (B, 2, H, H))
    ref0 = bf16_round(cnn.restrict2(x.astype(np.float32).astype(np.float64)))
    check("doubled-grid warm start: restricted images (BF16)", float(np.abs(a0 - ref0).max() / np.abs(ref0).max()),
          1.01 * 2.0 ** -7)
    raw = _layer(net, REG_NET_OUTPUT, 7, (B, 2, H, H))
    ref_post = s * cnn.output_map(cnn.prolong2(cnn.output_map(raw)))
    check("doubled-grid warm start: prolongation and fine output map", _rel(vg, ref_post), 1e-5)
    check("doubled-grid warm start: end to end", _rel(vg, cnn.predict_fine(params, x, s)), 3e-2)
    net.close()
