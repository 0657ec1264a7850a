"""CPU oracle of the residual CNN post-filter -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may use this module; the CUDA library never calls it.

The paper has no learned component; this network is an extension of the
decoder: a small residual CNN on the decoded viewport's luma that removes
quantisation artefacts.  Definition (plain fp64 numpy):

* input x = Y / 255 (H x W per image, batch first), zero padding at the
  image border for every 3x3 convolution ("same" size);
* layer 1: 3x3 convolution 1 -> 32 channels + bias, ReLU;
* layers 2-4: 3x3 convolution 32 -> 32 + bias, ReLU;
* layer 5: 3x3 convolution 32 -> 1 + bias: the residual r;
* output y = x + r; the loss of a batch is mean((y - t)^2) over all pixels.

Convolution is cross-correlation: out[co, i, j] = b[co] + sum over ci and
taps (dy, dx) in {-1, 0, 1}^2 of w[co, ci, dy + 1, dx + 1] x[ci, i + dy, j + dx].
The backward pass is the chain rule written out per layer.
"""
from __future__ import annotations

import numpy as np

CHANNELS = 32
SHAPES = [(CHANNELS, 1), (CHANNELS, CHANNELS), (CHANNELS, CHANNELS), (CHANNELS, CHANNELS), (1, CHANNELS)]


def init_params(seed: int = 0):
    """He-normal weights (fan-in 9 c_in), zero biases; last layer scaled down
    so the untrained network is close to the identity."""
    rng = np.random.default_rng(seed)
    params = []
    for k, (co, ci) in enumerate(SHAPES):
        std = np.sqrt(2.0 / (9 * ci)) * (0.1 if k == len(SHAPES) - 1 else 1.0)
        params.append((rng.standard_normal((co, ci, 3, 3)) * std, np.zeros(co)))
    return params


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x (n, ci, h, wd), w (co, ci, 3, 3), b (co,) -> (n, co, h, wd), zero
    padding, cross-correlation."""
    n, ci, h, wd = x.shape
    xp = np.zeros((n, ci, h + 2, wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    out = np.zeros((n, w.shape[0], h, wd))
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, :, dy:dy + h, dx:dx + wd]                  # x[ci, i + dy - 1, j + dx - 1]
            out += np.einsum("oc,nchw->nohw", w[:, :, dy, dx], patch)
    return out + b[None, :, None, None]


def forward(params, x: np.ndarray):
    """x (n, h, w) -> (y (n, h, w), activations): activations[k] is the
    input of layer k (a[0] = x with a channel axis)."""
    acts = [x[:, None].astype(np.float64)]
    h = acts[0]
    for k, (w, b) in enumerate(params):
        z = conv3x3(h, w, b)
        h = np.maximum(z, 0.0) if k < len(params) - 1 else z
        acts.append(h)
    return x + h[:, 0], acts


def loss(params, x, t) -> float:
    y, _ = forward(params, x)
    return float(np.mean((y - t) ** 2))


def conv3x3_grad_input(dz: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Gradient of conv3x3 with respect to its input: each output pixel
    (i, j) spreads dz[co, i, j] w[co, ci, dy, dx] back to input pixel
    (i + dy - 1, j + dx - 1); pixels outside the image are dropped."""
    n, co, h, wd = dz.shape
    dxp = np.zeros((n, w.shape[1], h + 2, wd + 2))
    for dy in range(3):
        for dx in range(3):
            dxp[:, :, dy:dy + h, dx:dx + wd] += np.einsum("oc,nohw->nchw", w[:, :, dy, dx], dz)
    return dxp[:, :, 1:-1, 1:-1]


def conv3x3_grad_weight(x: np.ndarray, dz: np.ndarray) -> np.ndarray:
    """Gradient of conv3x3 with respect to its weights:
    dw[co, ci, dy, dx] = sum over n, i, j of dz[co, i, j] x[ci, i + dy - 1, j + dx - 1]."""
    n, ci, h, wd = x.shape
    xp = np.zeros((n, ci, h + 2, wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    dw = np.zeros((dz.shape[1], ci, 3, 3))
    for dy in range(3):
        for dx in range(3):
            dw[:, :, dy, dx] = np.einsum("nohw,nchw->oc", dz, xp[:, :, dy:dy + h, dx:dx + wd])
    return dw


def backward(params, x: np.ndarray, t: np.ndarray):
    """Loss and its gradients [(dw, db), ...] for the mean squared error."""
    y, acts = forward(params, x)
    npx = y.size
    dy = 2.0 * (y - t) / npx                     # dL/dy; y = x + r, so dL/dr = dL/dy
    g = dy[:, None]                              # gradient at the output of layer 5 (pre-activation)
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        w, b = params[k]
        grads[k] = (conv3x3_grad_weight(acts[k], g), g.sum(axis=(0, 2, 3)))
        if k > 0:
            g = conv3x3_grad_input(g, w) * (acts[k] > 0)   # through the ReLU of layer k - 1's output
    return float(np.mean((y - t) ** 2)), grads


def psnr(a: np.ndarray, b: np.ndarray, peak: float = 255.0) -> float:
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(peak * peak / mse)
