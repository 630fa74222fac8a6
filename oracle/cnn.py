"""FP64 oracle of the learned residual CNN denoiser (App. C) and its faceting (App. D).

Network (DnCNN form, App. C): 8 convolution layers, 3 x 3 kernels, 'same'
zero padding, bias on every layer, channels 1 -> 64 -> ... -> 64 -> 1, ReLU
after every layer but the last, no batch normalisation.  The network N
predicts the noise; the denoiser is D(z) = z - N(z), and PnP applies
max(0, D(z)) (the final positivity is a reading: the paper is silent).

Convolutions are cross-correlations:
out[o, y, x] = b[o] + sum_{c, dy, dx} W[o, c, dy, dx] in[c, y + dy - 1, x + dx - 1].

With ``bf16=True`` the forward pass rounds what the network stores in BF16
(weights of every layer; hidden activations after bias and ReLU) to the
nearest BF16 value (ties to even) and accumulates in FP64; the input image,
the biases and the final layer's output stay in full precision.

Training loss (Eq. training_loss without the firm non-expansiveness term):
mean |D(u + sigma n) - u| over pixels and batch.
"""
from __future__ import annotations

import numpy as np

CHANNELS = 64
DEPTH = 8


def layer_shapes(channels: int = CHANNELS, depth: int = DEPTH):
    """(c_out, c_in) of each layer: 1 -> C, (depth-2) x C -> C, C -> 1."""
    return [(channels, 1)] + [(channels, channels)] * (depth - 2) + [(1, channels)]


def to_bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def im2col(x: np.ndarray) -> np.ndarray:
    """(B, C, H, W) -> (B, C*9, H*W) patches of the zero-padded input, tap index dy*3+dx."""
    B, C, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    cols = np.empty((B, C, 9, H, W), dtype=x.dtype)
    for dy in range(3):
        for dx in range(3):
            cols[:, :, dy * 3 + dx] = xp[:, :, dy:dy + H, dx:dx + W]
    return cols.reshape(B, C * 9, H * W)


def col2im(cols: np.ndarray, shape) -> np.ndarray:
    """Adjoint of im2col: (B, C*9, H*W) -> (B, C, H, W)."""
    B, C, H, W = shape
    cols = cols.reshape(B, C, 9, H, W)
    xp = np.zeros((B, C, H + 2, W + 2), dtype=cols.dtype)
    for dy in range(3):
        for dx in range(3):
            xp[:, :, dy:dy + H, dx:dx + W] += cols[:, :, dy * 3 + dx]
    return xp[:, :, 1:H + 1, 1:W + 1]


def conv_forward(x, Wt, b) -> np.ndarray:
    """3 x 3 'same' convolution with bias: (B, Ci, H, W) -> (B, Co, H, W)."""
    B, _, H, W = x.shape
    co = Wt.shape[0]
    out = np.einsum("ok,bkp->bop", Wt.reshape(co, -1), im2col(x)) + b[None, :, None]
    return out.reshape(B, co, H, W)


def conv_backward(x, Wt, dout):
    """Gradients (dx, dW, db) of ``conv_forward`` given dL/dout."""
    B, _, H, W = x.shape
    co = Wt.shape[0]
    d2 = dout.reshape(B, co, H * W)
    dW = np.einsum("bop,bkp->ok", d2, im2col(x)).reshape(Wt.shape)
    db = d2.sum(axis=(0, 2))
    dcols = np.einsum("ok,bop->bkp", Wt.reshape(co, -1), d2)
    return col2im(dcols, x.shape), dW, db


def network(params, z, bf16: bool = False, keep: bool = False):
    """N(z) for z of shape (B, 1, H, W) (or (H, W)); returns N(z) [and the activations]."""
    squeeze = z.ndim == 2
    h = z[None, None] if squeeze else z
    acts = [h]
    for i, (Wt, b) in enumerate(params):
        Wq = to_bf16(Wt) if bf16 else Wt
        h = conv_forward(h, Wq, b)
        if i < len(params) - 1:
            h = np.maximum(h, 0.0)
            if bf16:
                h = to_bf16(h)
        acts.append(h)
    out = h[0, 0] if squeeze else h
    return (out, acts) if keep else out


def denoise(params, z, bf16: bool = False, positivity: bool = True) -> np.ndarray:
    """D(z) = z - N(z), then max(0, .) when used inside PnP."""
    d = z - network(params, z, bf16)
    return np.maximum(d, 0.0) if positivity else d


def l1_loss_and_grads(params, u, noise, sigma: float, bf16: bool = False, with_abs: bool = False):
    """Loss mean|z - N(z) - u|, z = u + sigma n, and its gradients w.r.t. every (W, b).

    With ``bf16=True`` the forward pass is the BF16 one of ``network`` and the
    back-propagated pre-activation gradients of the hidden layers are rounded to
    BF16 after the ReLU mask (weights BF16 too); sums stay FP64.
    With ``with_abs=True`` also returns, per layer, the same sums taken over the
    absolute values of their terms (the scale of a floating-point error bound).
    """
    z = u + sigma * noise
    nz, acts = network(params, z, bf16=bf16, keep=True)
    resid = z - nz - u
    count = resid.size
    loss = float(np.abs(resid).sum() / count)
    g = -np.sign(resid) / count                    # dL/dN(z)
    grads = [None] * len(params)
    abs_grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        Wt, _ = params[i]
        if i < len(params) - 1:
            g = g * (acts[i + 1] > 0)              # ReLU
            if bf16:
                g = to_bf16(g)
        Wq = to_bf16(Wt) if bf16 else Wt
        dx, dW, db = conv_backward(acts[i], Wq, g)
        grads[i] = (dW, db)
        if with_abs:
            _, aW, ab = conv_backward(np.abs(acts[i]), np.abs(Wq), np.abs(g))
            abs_grads[i] = (aW, ab)
        g = dx
    return (loss, grads, abs_grads) if with_abs else (loss, grads)


def adam_step(params, grads, state, lr: float = 1e-4, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma & Ba 2015); ``state`` = dict(t, m, v) updated in place."""
    state["t"] += 1
    t = state["t"]
    out = []
    for i, ((Wt, b), (dW, db)) in enumerate(zip(params, grads)):
        new = []
        for j, (p, g) in enumerate(((Wt, dW), (b, db))):
            m = state["m"][i][j] = b1 * state["m"][i][j] + (1 - b1) * g
            v = state["v"][i][j] = b2 * state["v"][i][j] + (1 - b2) * g * g
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            new.append(p - lr * mh / (np.sqrt(vh) + eps))
        out.append(tuple(new))
    return out


def adam_init(params):
    return {"t": 0, "m": [[np.zeros_like(W), np.zeros_like(b)] for W, b in params],
            "v": [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]}


def facet_bounds(widths):
    e = np.concatenate([[0], np.cumsum(widths)])
    return list(zip(e[:-1], e[1:]))


def denoise_faceted(params, z, facet_rows, facet_cols, halo: int, bf16: bool = False,
                    positivity: bool = True) -> np.ndarray:
    """App. D: apply D independently on facets extended by a halo and keep each core.

    Each facet core [r0, r1) x [c0, c1) is extended by ``halo`` pixels (clipped
    at the image border) and denoised on its own; exact when the halo covers
    the receptive radius (8 px for 8 layers of 3 x 3).
    """
    n0, n1 = z.shape
    out = np.empty_like(z, dtype=np.float64)
    for r0, r1 in facet_bounds(facet_rows):
        for c0, c1 in facet_bounds(facet_cols):
            R0, R1 = max(0, r0 - halo), min(n0, r1 + halo)
            C0, C1 = max(0, c0 - halo), min(n1, c1 + halo)
            d = denoise(params, z[R0:R1, C0:C1], bf16, positivity)
            out[r0:r1, c0:c1] = d[r0 - R0:r1 - R0, c0 - C0:c1 - C0]
    return out
