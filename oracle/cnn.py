"""FP64 CPU oracle of the learned-correction network.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` alone; it shares no code
with the CUDA kernels.

The network is not in the paper (which only points to deep learning as
related work): a 4-layer convolutional net that maps per-point features of an
ASDSM sweep to a correction direction.  Definitions, written out plainly:

* conv3x3(a; W, b)[o, i, j] = b[o] + sum_c sum_{p,q in {0,1,2}}
  W[o, c, p, q] * a[c, i + p - 1, j + q - 1], with a = 0 outside the image
  (cross-correlation, zero "same" padding).
* layers: channels 6 -> 32 -> 32 -> 32 -> 1; a_l = relu(z_l) after layers
  1..3, the output y = z_4 is linear.
* loss L = 1/(2 n) * sum w (y - t)^2, n = number of output values, w optional
  per-point weights (1 when absent).
* Adam (Kingma and Ba, 2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
  theta -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Parameters are one flat vector [W1, b1, W2, b2, W3, b3, W4, b4], W_l of shape
(C_out, C_in, 3, 3) in C order.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (6, 32, 32, 32, 1)


def layer_shapes(channels=CHANNELS):
    shapes = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        shapes.append(((cout, cin, 3, 3), (cout,)))
    return shapes


def n_params(channels=CHANNELS) -> int:
    return sum(int(np.prod(w)) + int(np.prod(b)) for w, b in layer_shapes(channels))


def unpack(theta, channels=CHANNELS):
    """Flat vector -> list of (W, b) views."""
    out, off = [], 0
    for ws, bs in layer_shapes(channels):
        nw, nb = int(np.prod(ws)), int(np.prod(bs))
        out.append((theta[off:off + nw].reshape(ws), theta[off + nw:off + nw + nb]))
        off += nw + nb
    return out


def init_params(seed: int, channels=CHANNELS) -> np.ndarray:
    """He-normal weights (std sqrt(2 / (9 C_in))), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for (cout, cin, _, _), bs in layer_shapes(channels):
        parts.append(rng.normal(0.0, np.sqrt(2.0 / (9 * cin)), size=cout * cin * 9))
        parts.append(np.zeros(bs))
    return np.concatenate(parts)


def conv3x3(a, W, b):
    """a: (B, C_in, H, Wd); W: (C_out, C_in, 3, 3); b: (C_out,) -> (B, C_out, H, Wd)."""
    B, C, H, Wd = a.shape
    pad = np.zeros((B, C, H + 2, Wd + 2))
    pad[:, :, 1:-1, 1:-1] = a
    z = np.broadcast_to(b[None, :, None, None], (B, W.shape[0], H, Wd)).copy()
    for p in range(3):
        for q in range(3):
            # sum over input channels of W[o, c, p, q] * a[c, i + p - 1, j + q - 1]
            z += np.einsum("oc,bchw->bohw", W[:, :, p, q], pad[:, :, p:p + H, q:q + Wd])
    return z


def forward(theta, x, channels=CHANNELS):
    """Returns (y, activations): activations[0] = x, activations[l] = a_l."""
    acts = [x]
    layers = unpack(theta, channels)
    a = x
    for l, (W, b) in enumerate(layers):
        z = conv3x3(a, W, b)
        a = np.maximum(z, 0.0) if l + 1 < len(layers) else z
        acts.append(a)
    return acts[-1], acts


def loss(theta, x, t, channels=CHANNELS, w=None) -> float:
    y, _ = forward(theta, x, channels)
    wt = 1.0 if w is None else w
    return 0.5 * float(np.mean(wt * (y - t) ** 2))


def grad(theta, x, t, channels=CHANNELS, w=None):
    """(loss, dL/dtheta) by backpropagation through the definitions above."""
    y, acts = forward(theta, x, channels)
    layers = unpack(theta, channels)
    n = y.size
    g = np.zeros_like(theta)
    gl = unpack(g, channels)
    wt = 1.0 if w is None else w
    dz = wt * (y - t) / n                                # dL/dz_4
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        a_in = acts[l]
        B, C, H, Wd = a_in.shape
        pad = np.zeros((B, C, H + 2, Wd + 2))
        pad[:, :, 1:-1, 1:-1] = a_in
        gW, gb = gl[l]
        gb[:] = dz.sum(axis=(0, 2, 3))
        for p in range(3):
            for q in range(3):
                gW[:, :, p, q] = np.einsum("bohw,bchw->oc", dz, pad[:, :, p:p + H, q:q + Wd])
        if l == 0:
            break
        # dL/da_in: each a_in[c, i', j'] feeds z[o, i' - p + 1, j' - q + 1] with weight W[o, c, p, q]
        dpad = np.zeros_like(pad)
        for p in range(3):
            for q in range(3):
                dpad[:, :, p:p + H, q:q + Wd] += np.einsum("oc,bohw->bchw", W[:, :, p, q], dz)
        da = dpad[:, :, 1:-1, 1:-1]
        dz = da * (acts[l] > 0)                          # through relu of layer l
    return 0.5 * float(np.mean(wt * (y - t) ** 2)), g


class Adam:
    def __init__(self, n, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, theta, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)
