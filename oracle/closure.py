"""FP64 oracle of the learned MPCD->LB closure network (test infrastructure).

Only tests, the smoke check and bench's CPU leg import this module.  It is a
plain numpy statement of the network the CUDA path evaluates with bf16
tensor-core kernels, so that the GPU forward pass and gradients can be
checked element by element.

Network (the closure is not in the paper; its form follows the problem
statement of the learned coupling): input one 16 x 16 patch of MPCD cells with
24 channels = 8 consecutive instantaneous frames x {density deviation
n/ppc - 1, u_x / sqrt(kT/m), u_y / sqrt(kT/m)} (frame f, field c at channel
3 f + c); three 3 x 3 convolutions with 64 channels and ReLU, a linear 3 x 3
convolution to 3 channels, zero padding; the last layer's output, less its
mean over the 16 rows of each patch column (per channel), is added to the
mean of the 8 input frames.  The network thus learns a correction to the
plain short window that redistributes each field along y within a patch
column but leaves the column's mean that of the 8-frame mean: fed back into
the flow, the closure cannot add or drain mass or momentum on average in any
column of the coupling strip, whatever its fit.  (Unconstrained, an
MSE-trained correction shrinks the predicted velocities towards the training
set's mean, most at the patch edges where the zero padding starts, and the
coupling loop amplifies that.)  Layout NHWC; weights W[l] of shape (cout, 3, 3, cin), biases b[l].

Loss: mean squared error over all output values.
"""
from __future__ import annotations

import numpy as np

LAYERS = [(24, 64), (64, 64), (64, 64), (64, 3)]


def n_params() -> int:
    return sum(co * 9 * ci + co for ci, co in LAYERS)


def unpack(theta: np.ndarray):
    """Flat parameter vector -> [(W (cout,3,3,cin), b (cout,))] in layer order,
    each layer's W (row-major over cout, ky, kx, cin) followed by its b."""
    out, o = [], 0
    for ci, co in LAYERS:
        W = theta[o:o + co * 9 * ci].reshape(co, 3, 3, ci)
        o += co * 9 * ci
        b = theta[o:o + co]
        o += co
        out.append((W, b))
    return out


def init_params(seed: int) -> np.ndarray:
    """He-normal weights, zero biases, last layer scaled by 0.1."""
    rng = np.random.default_rng(seed)
    parts = []
    for li, (ci, co) in enumerate(LAYERS):
        std = np.sqrt(2.0 / (9 * ci)) * (0.1 if li == len(LAYERS) - 1 else 1.0)
        parts.append(rng.normal(0.0, std, size=co * 9 * ci))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32).astype(np.float64)


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def conv3x3(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Same-size 3 x 3 convolution with zero padding: x (P,16,16,ci), W (co,3,3,ci)."""
    P, H, Wd, ci = x.shape
    xp = np.zeros((P, H + 2, Wd + 2, ci))
    xp[:, 1:-1, 1:-1] = x
    out = np.zeros((P, H, Wd, W.shape[0])) + b
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("pyxc,oc->pyxo", xp[:, ky:ky + H, kx:kx + Wd], W[:, ky, kx, :])
    return out


def forward(theta: np.ndarray, x: np.ndarray, emulate_bf16: bool = False, jitter=None):
    """Network output (P,16,16,3) and the per-layer cache for backward.
    emulate_bf16 rounds weights and stored activations to bf16 where the
    CUDA path stores them in bf16 (inputs, hidden activations, weights).
    jitter, if given, is applied to every layer's pre-activations z (a test
    uses it to measure how far rounding-order-sized changes of z move the
    bf16 and ReLU decisions downstream)."""
    r = bf16 if emulate_bf16 else (lambda a: a)
    layers = unpack(theta)
    a = r(x)
    cache = []
    for li, (W, b) in enumerate(layers):
        z = conv3x3(a, r(W), b)
        if jitter is not None:
            z = jitter(z)
        cache.append((a, z))
        a = r(np.maximum(z, 0.0)) if li < len(layers) - 1 else z
    centred = a - a.mean(axis=1, keepdims=True)      # over y in each patch column
    mean8 = x.reshape(*x.shape[:3], 8, 3).mean(axis=3)
    return centred + mean8, cache


def loss(theta, x, t, emulate_bf16=False) -> float:
    y, _ = forward(theta, x, emulate_bf16)
    return float(np.mean((y - t) ** 2))


def backward(theta: np.ndarray, x: np.ndarray, t: np.ndarray, emulate_bf16: bool = False, jitter=None):
    """Loss and its gradient with respect to the flat parameter vector
    (jitter: as in forward)."""
    r = bf16 if emulate_bf16 else (lambda a: a)
    layers = unpack(theta)
    y, cache = forward(theta, x, emulate_bf16, jitter)
    L = float(np.mean((y - t) ** 2))
    d = 2.0 * (y - t) / y.size                     # dL/dy
    d = d - d.mean(axis=1, keepdims=True)          # dL/dz of the last (linear) layer: through the centring
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        a, z = cache[li]
        if li < len(layers) - 1:
            d = d * (z > 0.0)                       # through the ReLU
        db = d.sum(axis=(0, 1, 2))
        dq = r(d)                                   # the CUDA path stores this gradient in bf16
        P, H, Wd, ci = a.shape
        ap = np.zeros((P, H + 2, Wd + 2, ci))
        ap[:, 1:-1, 1:-1] = a
        dW = np.zeros_like(W)
        for ky in range(3):
            for kx in range(3):
                dW[:, ky, kx, :] = np.einsum("pyxo,pyxc->oc", dq, ap[:, ky:ky + H, kx:kx + Wd])
        grads[li] = (dW, db)
        if li > 0:
            dp = np.zeros((P, H + 2, Wd + 2, ci))
            Wr = r(W)
            for ky in range(3):
                for kx in range(3):
                    dp[:, ky:ky + H, kx:kx + Wd] += np.einsum("pyxo,oc->pyxc", dq, Wr[:, ky, kx, :])
            d = dp[:, 1:-1, 1:-1]
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return L, flat


def mean8(x: np.ndarray) -> np.ndarray:
    """The plain short-window estimate: mean of the 8 input frames per field."""
    return x.reshape(*x.shape[:3], 8, 3).mean(axis=3)
