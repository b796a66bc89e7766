"""FP64 reference of the control-variate network (oracle; test infrastructure).

The control variate g(Omega, B) is a multilayer perceptron with SiLU hidden
activations and a linear output, trained by mean-squared error.  This module
computes, in plain NumPy FP64 from the definitions:

* the input features of a sample: for every nucleus k (input order) the unit
  vector n(Omega_k) = (sin t cos p, sin t sin p, cos t) of its coherent-state
  direction (Eq. 16), drawn with this project's Philox map; for each radical i
  the classical hyperfine field b_i = sum_{k in i} A_k (I_k n_k) / B_hyp,i
  (B_hyp,i of Eq. 21, with a_k^2 generalised to |A_k|_F^2 / 3); |b_1|, |b_2|,
  b_1 . b_2; and B / B_scale;
* the forward pass h_{l+1} = silu(W_l h_l + b_l), output W_L h_L + b_L,
  silu(z) = z / (1 + e^{-z});
* the loss 1/(2n) sum (g - y)^2 and its gradient by the chain rule
  (silu'(z) = s(z) (1 + z (1 - s(z))), s = logistic);
* the control-variate estimate mean(phi - beta (g - mu)), beta = cov(phi, g) /
  var(g), with standard error sqrt(var(phi - beta g)/M + beta^2 var(mu));
* one training step of Adam (D. P. Kingma and J. Ba, "Adam: a method for
  stochastic optimization", ICLR 2015, Algorithm 1: bias-corrected first and
  second moment estimates) with decoupled weight decay on the weights
  (I. Loshchilov and F. Hutter, "Decoupled weight decay regularization",
  ICLR 2019): theta <- theta - lr wd theta - lr m_hat / (sqrt(v_hat) + eps).

Parameters are a flat vector in the order W_0, b_0, W_1, b_1, ..., W_L, b_L,
W_l row-major of shape (out, in).
"""
from __future__ import annotations

import numpy as np

from .philox import draw_uniforms


def features(seed: int, pair: int, samples, system, B, B_scale: float):
    """(n_samples, 3 N + 10) features; B is a scalar or per-sample array."""
    samples = np.atleast_1d(samples)
    N = system.n_nuc
    u1, u2 = draw_uniforms(seed, pair, samples, N)
    ct = 1.0 - 2.0 * u1
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    ph = 2.0 * np.pi * u2
    n = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1)  # (S, N, 3)
    I = np.asarray(system.two_I, float) / 2.0
    b = np.zeros((samples.size, 2, 3))
    for i in range(2):
        ks = [k for k in range(N) if int(system.radical[k]) == i]
        bh2 = sum(np.sum(system.A[k] ** 2) / 3.0 * I[k] * (I[k] + 1.0) for k in ks)
        if not ks or bh2 <= 0.0:
            continue
        for k in ks:
            b[:, i] += I[k] * n[:, k] @ system.A[k].T
        b[:, i] /= np.sqrt(bh2)
    inv = np.stack([np.linalg.norm(b[:, 0], axis=1), np.linalg.norm(b[:, 1], axis=1),
                    np.sum(b[:, 0] * b[:, 1], axis=1)], axis=1)
    Bc = np.broadcast_to(np.asarray(B, float) / B_scale, (samples.size,)).reshape(-1, 1)
    return np.concatenate([n.reshape(samples.size, -1), b[:, 0], b[:, 1], inv, Bc], axis=1)


def shapes(d_in: int, hidden: int, layers: int):
    dims = [d_in] + [hidden] * layers + [1]
    return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]


def unflatten(params, d_in, hidden, layers):
    out, o = [], 0
    for (r, c) in shapes(d_in, hidden, layers):
        W = params[o:o + r * c].reshape(r, c)
        o += r * c
        b = params[o:o + r]
        o += r
        out.append((W, b))
    assert o == params.size
    return out


def forward(params, x, d_in, hidden, layers):
    """Output g (n,) and the cache of pre-activations / activations."""
    Wb = unflatten(np.asarray(params, float), d_in, hidden, layers)
    h = np.asarray(x, float)
    cache = []
    for i, (W, b) in enumerate(Wb):
        z = h @ W.T + b
        cache.append((h, z))
        if i < len(Wb) - 1:
            h = z / (1.0 + np.exp(-z))
        else:
            h = z
    return h[:, 0], cache


def loss_and_grad(params, x, y, d_in, hidden, layers):
    """Loss 1/(2n) sum (g - y)^2 and its gradient with respect to params."""
    Wb = unflatten(np.asarray(params, float), d_in, hidden, layers)
    g, cache = forward(params, x, d_in, hidden, layers)
    n = x.shape[0]
    r = g - np.asarray(y, float)
    loss = 0.5 * np.mean(r * r)
    grads = [None] * len(Wb)
    dz = (r / n)[:, None]
    for i in range(len(Wb) - 1, -1, -1):
        h, z = cache[i]
        W, _ = Wb[i]
        grads[i] = (dz.T @ h, dz.sum(axis=0))
        if i > 0:
            dh = dz @ W
            zp = cache[i - 1][1]
            s = 1.0 / (1.0 + np.exp(-zp))
            dz = dh * (s * (1.0 + zp * (1.0 - s)))
    flat = np.concatenate([np.concatenate([gW.ravel(), gb.ravel()]) for gW, gb in grads])
    return loss, flat


def cv_estimate(phi, g, mu, var_mu):
    """Control-variate mean and standard error for one field."""
    phi = np.asarray(phi, float)
    g = np.asarray(g, float)
    M = phi.size
    cg = np.cov(phi, g, ddof=1)
    beta = cg[0, 1] / cg[1, 1] if cg[1, 1] > 0 else 0.0
    est = phi.mean() - beta * (g.mean() - mu)
    resid = phi - beta * g
    se = np.sqrt(resid.var(ddof=1) / M + beta * beta * var_mu)
    return est, se, beta


def adam_step(params, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0,
              decay_mask=None):
    """One Adam update at step t >= 1 (Kingma and Ba, Algorithm 1) with
    decoupled weight decay wd on the entries where decay_mask is true.
    Returns the new (params, m, v)."""
    params = np.asarray(params, float)
    grad = np.asarray(grad, float)
    m = beta1 * np.asarray(m, float) + (1.0 - beta1) * grad
    v = beta2 * np.asarray(v, float) + (1.0 - beta2) * grad * grad
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    decay = np.zeros_like(params) if decay_mask is None else np.where(decay_mask, wd, 0.0)
    new = params - lr * decay * params - lr * m_hat / (np.sqrt(v_hat) + eps)
    return new, m, v


def weight_mask(d_in, hidden, layers):
    """True on the weight entries of the flat parameter vector, False on biases."""
    out = []
    for (r, c) in shapes(d_in, hidden, layers):
        out.append(np.ones(r * c, bool))
        out.append(np.zeros(r, bool))
    return np.concatenate(out)
