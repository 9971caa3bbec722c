"""FP64 reference of the learned warm-start network (oracle; test
infrastructure only).

The paper has no learned component; this network is the warm-start predictor
the registration path is extended with: 8 convolution layers with 3x3
kernels and circular (periodic) padding, channel widths 2 -> 32 -> ... -> 32
-> 2, ReLU after every layer but the last.  The middle layers are dilated
(taps d apart) so that the receptive field covers the large-scale motion:
layer l uses dilation min(DILATION[l], H // 8, W // 32) (the cap keeps every
dilated sub-grid at least 8 x 32 points).  The raw output is smoothed by a
Gaussian low-pass G (symbol exp(-sigma^2 |k|^2 / 2), sigma = 2 h with
h = 2 pi / max(H, W), so the warm start carries no grid-scale noise, which the
Gauss-Newton-Krylov solve is expensive on) and projected onto divergence-free
fields with the Leray projection of the incompressible model
(Eq. (e:project-body-force) with w = 0), so that a warm start satisfies the
constraint div v = 0 exactly.

Convolution (cross-correlation) with periodic wrap and dilation d:
    z[b, o, y, x] = bias[o] + sum_{c, dy, dx in {-1,0,1}} W[o, c, dy+1, dx+1] a[b, c, (y+d dy) mod H, (x+d dx) mod W]
Loss: mean squared error between the filtered, projected prediction and the
target velocity, L = sum((P G out - t)^2) / (2 M), M = number of target
entries.  Backward passes are the adjoints of these maps written out (np.roll
is the periodic shift; P and G are symmetric Fourier multipliers that commute,
so (P G)^T = G P).
"""
import numpy as np

from .fft import fft2, ifft2
from .spectral import H1, apply_K, symbols

CHANNELS = (2, 32, 32, 32, 32, 32, 32, 32, 2)
DILATION = (1, 2, 4, 8, 8, 4, 2, 1)


def init_params(seed, channels=CHANNELS, scale=1.0):
    """He-style random initialisation: list of (W (Cout, Cin, 3, 3), b (Cout,))."""
    rng = np.random.default_rng(seed)
    params = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        std = scale * np.sqrt(2.0 / (9.0 * cin))
        params.append((rng.standard_normal((cout, cin, 3, 3)) * std, np.zeros(cout)))
    return params


def dilations(H, W, nlayers=len(DILATION)):
    """Per-layer dilation on an H x W grid (the schedule capped by H // 8 and W // 32)."""
    return [max(1, min(DILATION[l % len(DILATION)], H // 8, W // 32)) for l in range(nlayers)]


def _shift(a, dy, dx):
    """s[..., y, x] = a[..., (y + dy) mod H, (x + dx) mod W]."""
    return np.roll(a, shift=(-dy, -dx), axis=(-2, -1))


def conv3x3(a, W, b, d=1):
    out = np.zeros((a.shape[0], W.shape[0]) + a.shape[2:])
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            out += np.einsum("oc,bchw->bohw", W[:, :, dy + 1, dx + 1], _shift(a, d * dy, d * dx))
    return out + b[None, :, None, None]


def conv3x3_backward(a, W, dz, d=1):
    """Gradients of conv3x3 (dilation d) w.r.t. its input a, weights W and bias."""
    da = np.zeros_like(a)
    dW = np.zeros_like(W)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            da += np.roll(np.einsum("oc,bohw->bchw", W[:, :, dy + 1, dx + 1], dz), shift=(d * dy, d * dx),
                          axis=(-2, -1))
            dW[:, :, dy + 1, dx + 1] = np.einsum("bohw,bchw->oc", dz, _shift(a, d * dy, d * dx))
    return da, dW, dz.sum(axis=(0, 2, 3))


def leray(u):
    """Leray projection of each velocity u[b] (2, H, W)."""
    return np.stack([apply_K(u[i], H1, 1.0, np.inf) for i in range(u.shape[0])])


def gauss_sigma(H, W):
    """Width of the output low-pass: two grid spacings of the finer axis."""
    return 2.0 * (2.0 * np.pi / max(H, W))


def gauss(u):
    """Gaussian low-pass exp(-sigma^2 |k|^2 / 2) of each field u[b, c] (full |k|^2, Nyquist kept)."""
    H, W = u.shape[-2:]
    _, _, KK = symbols(H, W)
    s = gauss_sigma(H, W)
    mult = np.exp(-0.5 * s * s * KK)
    out = np.empty_like(u, dtype=np.float64)
    for i in np.ndindex(*u.shape[:-2]):
        out[i] = np.real(ifft2(mult * fft2(u[i])))
    return out


def output_map(u):
    """Divergence-free warm start from the raw network output: P G u."""
    return leray(gauss(u))


def forward(params, x, cache=False):
    """x: (B, 2, H, W) -> raw output (B, 2, H, W) and, if cache, the layer inputs."""
    acts = [x]
    a = x
    dil = dilations(x.shape[-2], x.shape[-1], len(params))
    for l, (W, b) in enumerate(params):
        z = conv3x3(a, W, b, dil[l])
        a = np.maximum(z, 0.0) if l < len(params) - 1 else z
        acts.append(a)
    return (a, acts) if cache else a


def predict(params, x):
    """Divergence-free warm-start velocity P G net(x)."""
    return output_map(forward(params, x))


def restrict2(u):
    """(..., 2H, 2W) -> (..., H, W): full weighting around fine node (2i, 2j), weights 1/4, 1/2, 1/4
    along each axis, periodic.  (Resampling of the warm-start pipeline; the paper has none.)"""
    out = np.zeros(u.shape[:-2] + (u.shape[-2] // 2, u.shape[-1] // 2))
    w = {-1: 0.25, 0: 0.5, 1: 0.25}
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            out += w[dy] * w[dx] * _shift(u, dy, dx)[..., ::2, ::2]
    return out


def prolong2(u):
    """(..., H, W) -> (..., 2H, 2W): bilinear interpolation, periodic; fine node (y, x) sits at
    coarse coordinates (y / 2, x / 2)."""
    H, W = u.shape[-2:]
    out = np.empty(u.shape[:-2] + (2 * H, 2 * W))
    right = _shift(u, 0, 1)
    down = _shift(u, 1, 0)
    diag = _shift(u, 1, 1)
    out[..., ::2, ::2] = u
    out[..., ::2, 1::2] = 0.5 * (u + right)
    out[..., 1::2, ::2] = 0.5 * (u + down)
    out[..., 1::2, 1::2] = 0.25 * (u + right + down + diag)
    return out


def predict_fine(params, x_fine, scale=1.0):
    """Warm start on the doubled grid from the network at the coarse grid: restrict the images,
    predict there, prolong, and apply the fine grid's own output map, times the output scale."""
    return scale * output_map(prolong2(predict(params, restrict2(x_fine))))


def loss_and_grads(params, x, t):
    """MSE loss of the filtered, projected prediction against t and its parameter gradients."""
    out, acts = forward(params, x, cache=True)
    dil = dilations(x.shape[-2], x.shape[-1], len(params))
    r = output_map(out) - t
    M = t.size
    loss = 0.5 * float(np.sum(r * r)) / M
    d = gauss(leray(r)) / M  # dL/d out = (P G)^T r / M = G P r / M
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, b = params[l]
        a_in = acts[l]
        da, dW, db = conv3x3_backward(a_in, W, d, dil[l])
        grads[l] = (dW, db)
        if l > 0:
            d = da * (acts[l] > 0.0)  # ReLU of layer l-1 (acts[l] is its output)
    return loss, grads
