"""FP64 oracle of the Jacobian of the residual CNN denoiser and of the firm non-expansiveness
measure of Eq. training_loss (App. C): ||grad (2D - I)||_S at an input z.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU baseline use this
module; the library never does.

With D(z) = z - N(z) (the denoiser of the training loss, before the PnP positivity) the Jacobian
of Q = 2D - I is J_Q = I - 2 J_N.  N is a ReLU network, so at z its Jacobian is the linear network
with the same weights, no biases, and every hidden layer multiplied by its ReLU mask [act > 0] at z:

* J_N v (forward-mode): t_0 = v, t_{l+1} = [act_{l+1} > 0] * (W_l * t_l) for the hidden layers,
  J_N v = W_last * t_last;
* J_N^T w (reverse-mode): the back-propagation of ``cnn.l1_loss_and_grads`` with cotangent w,
  down to the input image.

||J_Q||_S is the largest singular value, found by power iteration on J_Q^T J_Q: from a unit v,
w = J_Q v, u = J_Q^T w, sigma = ||w||, v = u / ||u||.  The constraint of Eq. training_loss asks
sigma <= 1 at every training input.

With ``bf16=True`` the products mirror the GPU's storage: weights BF16, and each hidden
tangent (after its mask) or back-propagated gradient (after its mask) rounded to BF16, as the
activations are in ``cnn.network``; sums stay FP64.
"""
from __future__ import annotations

import numpy as np

from .cnn import conv_backward, conv_forward, network, to_bf16


def _acts(params, z, bf16):
    _, acts = network(params, np.asarray(z, dtype=np.float64), bf16=bf16, keep=True)
    return acts


def jvp(params, z, v, bf16: bool = False, acts=None) -> np.ndarray:
    """J_N(z) v for an (H, W) input z and tangent image v."""
    acts = _acts(params, z, bf16) if acts is None else acts
    t = np.asarray(v, dtype=np.float64)[None, None]
    last = len(params) - 1
    for i, (Wt, b) in enumerate(params):
        Wq = to_bf16(Wt) if bf16 else Wt
        t = conv_forward(t, Wq, np.zeros_like(b))
        if i < last:
            t = t * (acts[i + 1] > 0)
            if bf16:
                t = to_bf16(t)
    return t[0, 0]


def vjp(params, z, w, bf16: bool = False, acts=None) -> np.ndarray:
    """J_N(z)^T w for an (H, W) input z and cotangent image w."""
    acts = _acts(params, z, bf16) if acts is None else acts
    g = np.asarray(w, dtype=np.float64)[None, None]
    last = len(params) - 1
    for i in range(last, -1, -1):
        Wt, _ = params[i]
        if i < last:
            g = g * (acts[i + 1] > 0)
            if bf16:
                g = to_bf16(g)
        Wq = to_bf16(Wt) if bf16 else Wt
        g, _, _ = conv_backward(acts[i], Wq, g)
    return g[0, 0]


def q_jacobian_norm(params, z, v0, iters: int, bf16: bool = False):
    """(sigma, v): power-iteration estimate of ||grad (2D - I)(z)||_S and its right singular vector."""
    acts = _acts(params, z, bf16)
    v = np.asarray(v0, dtype=np.float64)
    v = v / np.linalg.norm(v)
    sigma = 0.0
    for _ in range(iters):
        w = v - 2.0 * jvp(params, z, v, bf16, acts)
        u = w - 2.0 * vjp(params, z, w, bf16, acts)
        sigma = float(np.linalg.norm(w))
        v = u / np.linalg.norm(u)
    return sigma, v


def fne_penalty_and_grads(params, z, v, lam: float, eps: float, bf16: bool = False):
    """Soft firm non-expansiveness penalty and its weight gradients (Eq. training_loss relaxed).

    For a batch z (B, H, W) and unit vectors v (B, H, W) from the power iteration, held fixed:
        P = lam / B * sum_b max(||J_Q(z_b) v_b||^2, 1 - eps),   J_Q = I - 2 J_N.
    J_N v is the frozen-mask network without biases applied to v, so d||J_Q v||^2 / dW is the
    back-propagation of the cotangent -4 (J_Q v) through that tangent network (layer inputs: the
    tangents, layer 1's input: v).  The biases get no gradient (they enter only through the
    masks, which are locally constant), nor does an image whose ||J_Q v||^2 <= 1 - eps.
    Returns (P, [(dW, db)] per layer, [||J_Q v_b||^2 per image]).
    """
    z = np.asarray(z, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    B = z.shape[0]
    last = len(params) - 1
    grads = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    P, n2s = 0.0, []
    for bi in range(B):
        acts = _acts(params, z[bi], bf16)
        ts = [v[bi][None, None]]
        for i, (Wt, b) in enumerate(params):
            Wq = to_bf16(Wt) if bf16 else Wt
            t = conv_forward(ts[-1], Wq, np.zeros_like(b))
            if i < last:
                t = t * (acts[i + 1] > 0)
                if bf16:
                    t = to_bf16(t)
            ts.append(t)
        w = v[bi] - 2.0 * ts[-1][0, 0]
        n2 = float(np.sum(w * w))
        n2s.append(n2)
        P += lam / B * max(n2, 1.0 - eps)
        if n2 <= 1.0 - eps:
            continue
        g = (-4.0 * lam / B * w)[None, None]
        for i in range(last, -1, -1):
            Wt, _ = params[i]
            if i < last:
                g = g * (acts[i + 1] > 0)
                if bf16:
                    g = to_bf16(g)
            Wq = to_bf16(Wt) if bf16 else Wt
            dx, dW, _ = conv_backward(ts[i], Wq, g)
            grads[i] = (grads[i][0] + dW, grads[i][1])
            g = dx
    return P, grads, n2s
