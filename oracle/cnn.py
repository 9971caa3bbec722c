"""FP64 reference of the learned warm-start network (oracle; test
infrastructure only).

The paper has no learned component; this network is the warm-start predictor
the registration path is extended with: 8 convolution layers with 3x3
kernels and circular (periodic) padding, channel widths 2 -> 32 -> ... -> 32
-> 2, ReLU after every layer but the last, and the predicted velocity
projected onto divergence-free fields with the Leray projection of the
incompressible model (Eq. (e:project-body-force) with w = 0), so that a warm
start satisfies the constraint div v = 0 exactly.

Convolution (cross-correlation) with periodic wrap:
    z[b, o, y, x] = bias[o] + sum_{c, dy, dx in {-1,0,1}} W[o, c, dy+1, dx+1] a[b, c, (y+dy) mod H, (x+dx) mod W]
Loss: mean squared error between the projected prediction and the target
velocity, L = sum((P out - t)^2) / (2 M), M = number of target entries.
Backward passes are the adjoints of these maps written out (np.roll is the
periodic shift; the Leray projection is symmetric and idempotent).
"""
import numpy as np

from .spectral import H1, apply_K

CHANNELS = (2, 32, 32, 32, 32, 32, 32, 32, 2)


def init_params(seed, channels=CHANNELS, scale=1.0):
    """He-style random initialisation: list of (W (Cout, Cin, 3, 3), b (Cout,))."""
    rng = np.random.default_rng(seed)
    params = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        std = scale * np.sqrt(2.0 / (9.0 * cin))
        params.append((rng.standard_normal((cout, cin, 3, 3)) * std, np.zeros(cout)))
    return params


def _shift(a, dy, dx):
    """s[..., y, x] = a[..., (y + dy) mod H, (x + dx) mod W]."""
    return np.roll(a, shift=(-dy, -dx), axis=(-2, -1))


def conv3x3(a, W, b):
    out = np.zeros((a.shape[0], W.shape[0]) + a.shape[2:])
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            out += np.einsum("oc,bchw->bohw", W[:, :, dy + 1, dx + 1], _shift(a, dy, dx))
    return out + b[None, :, None, None]


def conv3x3_backward(a, W, dz):
    """Gradients of conv3x3 w.r.t. its input a, weights W and bias."""
    da = np.zeros_like(a)
    dW = np.zeros_like(W)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            da += np.roll(np.einsum("oc,bohw->bchw", W[:, :, dy + 1, dx + 1], dz), shift=(dy, dx), axis=(-2, -1))
            dW[:, :, dy + 1, dx + 1] = np.einsum("bohw,bchw->oc", dz, _shift(a, dy, dx))
    return da, dW, dz.sum(axis=(0, 2, 3))


def leray(u):
    """Leray projection of each velocity u[b] (2, H, W)."""
    return np.stack([apply_K(u[i], H1, 1.0, np.inf) for i in range(u.shape[0])])


def forward(params, x, cache=False):
    """x: (B, 2, H, W) -> raw output (B, 2, H, W) and, if cache, the layer inputs."""
    acts = [x]
    a = x
    for l, (W, b) in enumerate(params):
        z = conv3x3(a, W, b)
        a = np.maximum(z, 0.0) if l < len(params) - 1 else z
        acts.append(a)
    return (a, acts) if cache else a


def predict(params, x):
    """Divergence-free warm-start velocity P(net(x))."""
    return leray(forward(params, x))


def loss_and_grads(params, x, t):
    """MSE loss of the projected prediction against t and its parameter gradients."""
    out, acts = forward(params, x, cache=True)
    r = leray(out) - t
    M = t.size
    loss = 0.5 * float(np.sum(r * r)) / M
    d = leray(r) / M  # dL/d out (P symmetric and idempotent)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, b = params[l]
        a_in = acts[l]
        da, dW, db = conv3x3_backward(a_in, W, d)
        grads[l] = (dW, db)
        if l > 0:
            d = da * (acts[l] > 0.0)  # ReLU of layer l-1 (acts[l] is its output)
    return loss, grads
