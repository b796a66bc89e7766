"""Pins of the FP64 control-variate reference (oracle/mlp.py) on the CPU."""
import math

import numpy as np

from oracle import mlp, philox


def _params(d_in, hidden, layers, seed=0):
    rng = np.random.default_rng(seed)
    n = sum(r * c + r for r, c in mlp.shapes(d_in, hidden, layers))
    return rng.normal(0, 0.5, n)


def test_gradient_by_central_differences():
    """The chain-rule gradient equals central finite differences of the loss."""
    d_in, hidden, layers = 7, 5, 3
    p = _params(d_in, hidden, layers, 1)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(11, d_in))
    y = rng.normal(size=11)
    loss, g = mlp.loss_and_grad(p, x, y, d_in, hidden, layers)
    num = np.zeros_like(p)
    h = 1e-6
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        num[i] = (mlp.loss_and_grad(p + e, x, y, d_in, hidden, layers)[0]
                  - mlp.loss_and_grad(p - e, x, y, d_in, hidden, layers)[0]) / (2 * h)
    assert np.max(np.abs(num - g)) < 1e-8 * max(1.0, np.max(np.abs(g)))
    # and the loss is the mean of the squared residuals over two
    gx, _ = mlp.forward(p, x, d_in, hidden, layers)
    assert abs(loss - 0.5 * np.mean((gx - y) ** 2)) < 1e-15


def test_features_are_directions_and_hyperfine_fields():
    """Eq. 16 directions of the Philox draws; b_i = sum_k a_k I_k n_k / B_hyp,i
    for isotropic couplings, whose mean square over the sphere is
    sum_k a_k^2 I_k^2 / B_hyp,i^2 = sum I_k / sum (I_k + 1) for equal a; B / B_scale last."""
    from paper_1612_09517_gb300 import workloads as wl
    s = wl.SpinSystem([0, 0, 1, 0], [1, 2, 1, 1], np.stack([0.3 * np.eye(3), -0.5 * np.eye(3),
                                                              0.8 * np.eye(3), 0.1 * np.eye(3)]), 1, 1, 0)
    feats = mlp.features(9, 3, np.arange(5, 25), s, 2.5, 10.0)
    th, ph = philox.draw_angles(9, 3, np.arange(5, 25), 4)
    n = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)
    assert feats.shape == (20, 3 * 4 + 10)
    assert np.allclose(feats[:, :12], n.reshape(20, -1), atol=1e-12)
    a = np.array([0.3, -0.5, 0.8, 0.1])
    I = np.array([0.5, 1.0, 0.5, 0.5])
    bh1 = np.sqrt(np.sum((a ** 2 * I * (I + 1))[[0, 1, 3]]))
    b1 = (a[0] * I[0] * n[:, 0] + a[1] * I[1] * n[:, 1] + a[3] * I[3] * n[:, 3]) / bh1
    b2 = (a[2] * I[2] * n[:, 2]) / abs(a[2]) / np.sqrt(I[2] * (I[2] + 1))
    assert np.allclose(feats[:, 12:15], b1) and np.allclose(feats[:, 15:18], b2)
    assert np.allclose(feats[:, 18], np.linalg.norm(b1, axis=1))
    assert np.allclose(feats[:, 20], np.sum(b1 * b2, axis=1))
    assert np.allclose(feats[:, 21], 0.25)
    big = mlp.features(1, 0, np.arange(40000), wl.SpinSystem([0, 0], [1, 1], np.stack([np.eye(3)] * 2), 1, 1, 0), 0.0, 1.0)
    assert abs(np.mean(np.sum(big[:, 6:9] ** 2, axis=1)) - 1.0 / 3.0) < 0.01


def test_control_variate_estimator_limits():
    """Perfect control variate: only the uncertainty of mu remains; an
    independent one: the plain estimate; a partial one: variance x (1 - rho^2)."""
    rng = np.random.default_rng(3)
    M = 20000
    phi = rng.normal(0.4, 0.1, M)
    est, se, beta = mlp.cv_estimate(phi, 2.0 * phi + 1.0, 2.0 * 0.4 + 1.0, 1e-10)
    assert abs(beta - 0.5) < 1e-12 and abs(est - 0.4) < 1e-9 and se < 1e-5
    est, se, beta = mlp.cv_estimate(phi, rng.normal(size=M), 0.0, 0.0)
    assert abs(beta) < 0.01 and abs(se - phi.std(ddof=1) / math.sqrt(M)) < 2e-5
    noise = rng.normal(0, 0.1, M)
    g = phi + noise  # rho^2 = 1/2
    est, se, beta = mlp.cv_estimate(phi, g, 0.4, 0.0)
    assert abs(se ** 2 / (phi.var(ddof=1) / M) - 0.5) < 0.03


def test_adam_step_closed_forms():
    """Adam's bias correction and the decoupled weight decay, from their
    definitions: (i) a constant gradient g gives m_hat = g and v_hat = g^2 at
    every step, so each step moves by exactly lr g / (|g| + eps) (without the
    correction the first step would be sqrt(1 - beta2) / (1 - beta1) = 0.316
    of it); (ii) a zero gradient leaves only the decay, theta (1 - lr wd), on
    the weights and nothing on the biases; (iii) on the quadratic
    f = |theta|^2 / 2 the first step is lr sign(theta)."""
    rng = np.random.default_rng(5)
    th = rng.normal(size=40)
    g = rng.normal(size=40)
    m = np.zeros(40)
    v = np.zeros(40)
    p = th.copy()
    lr, eps = 1e-2, 1e-8
    for t in range(1, 8):
        p_new, m, v = mlp.adam_step(p, m, v, g, t, lr, eps=eps)
        assert np.allclose(p - p_new, lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)
        p = p_new
    mask = mlp.weight_mask(3, 4, 2)
    assert mask.size == sum(r * c + r for r, c in mlp.shapes(3, 4, 2))
    assert mask.sum() == 3 * 4 + 4 * 4 + 4 * 1
    th = rng.normal(size=mask.size)
    p1, m1, v1 = mlp.adam_step(th, np.zeros_like(th), np.zeros_like(th), np.zeros_like(th), 1,
                               0.1, wd=0.5, decay_mask=mask)
    assert np.allclose(p1[mask], th[mask] * (1 - 0.05), rtol=1e-15)
    assert np.array_equal(p1[~mask], th[~mask])
    q, _, _ = mlp.adam_step(th, np.zeros_like(th), np.zeros_like(th), th, 1, 0.03)
    assert np.allclose(th - q, 0.03 * th / (np.abs(th) + 1e-8), rtol=1e-12)
