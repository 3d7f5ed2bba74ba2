"""FP64 CPU oracle of the residual corrector network (test infrastructure only).

pred = x + f(x), f = conv5 . relu . conv4 . relu . conv3 . relu . conv2 . relu . conv1,
each conv 3x3 with bias and periodic padding:
    y[co](p) = b[co] + sum_ci sum_{dy,dx in -1..1} w[co][ci][dy+1][dx+1] x[ci](p + (dy, dx)).
Loss L = mean over all pixels of (pred - hr)^2.  The backward pass is the chain rule
written out layer by layer.  Weights are taken as given (the tests pass the BF16-rounded
values the GPU uses)."""
from __future__ import annotations

import numpy as np

LAYERS = [(1, 32), (32, 32), (32, 32), (32, 32), (32, 1)]


def bf16_round(a):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(a, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unflatten(flat):
    out, k = [], 0
    for ci, co in LAYERS:
        w = np.asarray(flat[k:k + co * ci * 9], np.float64).reshape(co, ci, 3, 3)
        k += co * ci * 9
        b = np.asarray(flat[k:k + co], np.float64)
        k += co
        out.append((w, b))
    return out


def flatten(layers):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in layers])


def shifted(x, dy, dx):
    """x(p + (dy, dx)) with periodic wrap, x [..., H, W]."""
    return np.roll(x, (-dy, -dx), axis=(-2, -1))


def conv(x, w, b):
    """x [n, ci, H, W], w [co, ci, 3, 3] -> [n, co, H, W]."""
    n, ci, H, W = x.shape
    co = w.shape[0]
    y = np.broadcast_to(b[None, :, None, None], (n, co, H, W)).copy()
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            xs = shifted(x, dy, dx)
            y += np.einsum("oc,nchw->nohw", w[:, :, dy + 1, dx + 1], xs)
    return y


def forward(flat, x):
    """x [n, H, W] -> (pred [n, H, W], cache)."""
    layers = unflatten(flat)
    a = np.asarray(x, np.float64)[:, None]
    cache = [a]
    for l, (w, b) in enumerate(layers):
        z = conv(a, w, b)
        a = z if l == len(layers) - 1 else np.maximum(z, 0.0)
        cache.append(a)
    return np.asarray(x, np.float64) + a[:, 0], cache


def loss(flat, x, hr):
    pred, _ = forward(flat, x)
    return float(np.mean((pred - np.asarray(hr, np.float64)) ** 2))


def loss_grad(flat, x, hr):
    """(L, dL/dparams flat)."""
    layers = unflatten(flat)
    pred, cache = forward(flat, x)
    hr = np.asarray(hr, np.float64)
    n = pred.size
    g = (2.0 * (pred - hr) / n)[:, None]          # dL/d(output of the last conv)
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        w, b = layers[l]
        if l < len(layers) - 1:
            g = g * (cache[l + 1] > 0)                 # through the ReLU of layer l
        xin = cache[l]
        gw = np.zeros_like(w)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                gw[:, :, dy + 1, dx + 1] = np.einsum("nohw,nchw->oc", g, shifted(xin, dy, dx))
        grads[l] = (gw, g.sum(axis=(0, 2, 3)))
        if l > 0:
            gx = np.zeros_like(xin)
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    gx += shifted(np.einsum("oc,nohw->nchw", w[:, :, dy + 1, dx + 1], g), -dy, -dx)
            g = gx
    return float(np.mean((pred - hr) ** 2)), flatten(grads)
