"""FP64 CPU oracle of the learned-proposal network (test infrastructure only).

Nothing in the product path imports this module.  It defines, in plain
numpy, what the GPU training and inference kernels compute:

  h_0 = x,  z_l = h_{l-1} W_l + b_l,  h_l = GELU(z_l)  (l = 1..depth),
  logits = h_depth W_out + b_out,
  loss = mean_i [ -log softmax_valid(logits_i)[label_i] ],

where softmax_valid runs over the first n_valid[i] slots of row i only (the
neighbourhood of the stage-1 candidate; slots beyond it are not
candidates), GELU(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2, and parameters
are laid out flat as W_1 [n_in, width], b_1, ..., W_depth, b_depth, W_out
[width, n_out], b_out (row-major, input dimension first).  AdamW with
decoupled weight decay on every parameter.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def layer_shapes(n_in, width, depth, n_out):
    shapes = []
    d = n_in
    for _ in range(depth):
        shapes.append((d, width))
        d = width
    shapes.append((d, n_out))
    return shapes


def num_params(n_in, width, depth, n_out):
    return sum(a * b + b for a, b in layer_shapes(n_in, width, depth, n_out))


def unpack(theta, n_in, width, depth, n_out):
    out, o = [], 0
    for a, b in layer_shapes(n_in, width, depth, n_out):
        W = theta[o:o + a * b].reshape(a, b)
        o += a * b
        bias = theta[o:o + b]
        o += b
        out.append((W, bias))
    return out


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(theta, x, dims):
    """Returns logits and the per-layer (z, h) cache."""
    layers = unpack(np.asarray(theta, np.float64), *dims)
    h = np.asarray(x, np.float64)
    cache = [(None, h)]
    for W, b in layers[:-1]:
        z = h @ W + b
        h = gelu(z)
        cache.append((z, h))
    W, b = layers[-1]
    return h @ W + b, cache


def masked_ce(logits, n_valid, label):
    """Mean masked softmax cross-entropy and its gradient wrt the logits."""
    B, n_out = logits.shape
    valid = np.arange(n_out)[None, :] < np.asarray(n_valid)[:, None]
    l = np.where(valid, logits, -np.inf)
    m = l.max(axis=1, keepdims=True)
    e = np.where(valid, np.exp(l - m), 0.0)
    s = e.sum(axis=1, keepdims=True)
    p = e / s
    lab = np.asarray(label)
    loss = float(np.mean(-(l[np.arange(B), lab] - m[:, 0] - np.log(s[:, 0]))))
    g = p.copy()
    g[np.arange(B), lab] -= 1.0
    return loss, g / B


def loss_and_grad(theta, x, n_valid, label, dims):
    logits, cache = forward(theta, x, dims)
    loss, dlog = masked_ce(logits, n_valid, label)
    layers = unpack(np.asarray(theta, np.float64), *dims)
    grads = []
    dh = dlog
    # output layer
    h_prev = cache[-1][1]
    W, _ = layers[-1]
    grads.append((h_prev.T @ dh, dh.sum(axis=0)))
    dh = dh @ W.T
    for li in range(len(layers) - 2, -1, -1):
        z, _ = cache[li + 1]
        dz = dh * gelu_grad(z)
        h_prev = cache[li][1]
        W, _ = layers[li]
        grads.append((h_prev.T @ dz, dz.sum(axis=0)))
        dh = dz @ W.T
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def init_params(rng, dims):
    """He-style initialisation (normal, std sqrt(2 / fan_in)), zero biases."""
    parts = []
    for a, b in layer_shapes(*dims):
        parts.append(rng.standard_normal(a * b) * math.sqrt(2.0 / a))
        parts.append(np.zeros(b))
    return np.concatenate(parts)


def adamw(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW step (t counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    theta = theta - lr * (mh / (np.sqrt(vh) + eps) + wd * theta)
    return theta, m, v


def topk_valid(logits, n_valid, k):
    """Indices of the k largest valid logits per row (ties: lower slot first);
    rows with fewer than k valid slots are padded with -1."""
    B, n_out = logits.shape
    out = np.full((B, k), -1, dtype=np.int64)
    for i in range(B):
        nv = int(n_valid[i])
        order = sorted(range(nv), key=lambda j: (-logits[i, j], j))[:k]
        out[i, :len(order)] = order
    return out


def propose_mass(logits, n_valid, k, p_mass):
    """The proposal rule on top of the ranking: valid slots in decreasing
    logit order (ties: lower slot first), taken until their softmax
    probability over the valid slots reaches p_mass, or k slots are taken;
    rows padded with -1.  p_mass >= 1 gives topk_valid."""
    B, n_out = logits.shape
    out = np.full((B, k), -1, dtype=np.int64)
    for i in range(B):
        nv = int(n_valid[i])
        if nv <= 0:
            continue
        l = np.asarray(logits[i, :nv], np.float64)
        p = np.exp(l - l.max())
        p /= p.sum()
        order = sorted(range(nv), key=lambda j: (-l[j], j))
        cum = 0.0
        for r, j in enumerate(order[:k]):
            out[i, r] = j
            cum += p[j]
            if cum >= p_mass:
                break
    return out
