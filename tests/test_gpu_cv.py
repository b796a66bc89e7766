"""Control variate on the GPU: forward/backward against the FP64 reference, the
estimator, and what a trained network gains over the plain estimate."""
import math

import numpy as np
import pytest

from oracle import dense, mlp
from paper_1612_09517_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    torch.cuda.set_device(0)
    from paper_1612_09517_gb300 import rp
    rp.use_torch_allocator()
    yield


def _bf16(a):
    """Round FP32 values to the nearest BF16 (ties to even), kept in FP32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    r = ((u >> 16) & 1) + 0x7FFF
    return ((u + r) & 0xFFFF0000).astype(np.uint32).view(np.float32)


def _bf16_weights(p, d_in, hidden, layers):
    p = np.array(p, dtype=np.float32)
    o = 0
    for (r, c) in mlp.shapes(d_in, hidden, layers):
        p[o:o + r * c] = _bf16(p[o:o + r * c])
        o += r * c + r
    return p


def _net(hidden=32, layers=3, **kw):
    from paper_1612_09517_gb300 import rp
    s = wl.random_isotropic(2, 1, seed=3)
    sy = rp.System(s)
    return s, sy, rp.ControlVariate(sy, hidden=hidden, layers=layers, **kw)


def test_loss_and_gradient_match_reference():
    s, sy, cv = _net()
    d_in = cv.d_in
    rng = np.random.default_rng(0)
    p = _bf16_weights(rng.normal(0, 0.3, cv.n_params), d_in, 32, 3)
    cv.set_params(p)
    x = mlp.features(7, 0, np.arange(100), s, 1.5, 10.0)
    y = rng.normal(size=100)
    loss, g = cv.loss_grad(x.astype(np.float32), y.astype(np.float32))
    rl, rg = mlp.loss_and_grad(p.astype(np.float64), x.astype(np.float32).astype(np.float64),
                               y.astype(np.float32).astype(np.float64), d_in, 32, 3)
    assert abs(loss - rl) <= 1e-5 * abs(rl)
    assert np.max(np.abs(g - rg)) <= 1e-4 * np.max(np.abs(rg))


def test_adam_training_steps_match_reference():
    """Two full-batch epochs of rp_cv_train (two Adam steps on the FP32 master
    parameters, gradients through the BF16 weights, targets standardised per
    field) against the reference: loss gradient (mlp.loss_and_grad) and Adam
    with decoupled weight decay (mlp.adam_step, Kingma and Ba's update)."""
    lr, wd = 1e-2, 1e-2
    s, sy, cv = _net(hidden=16, layers=2, epochs=2, batch=64, lr=lr, weight_decay=wd)
    d_in = cv.d_in
    p0 = cv.get_params().astype(np.float64)
    samples = np.arange(200, 264)
    B = np.full(64, 2.0)
    phi = 0.3 + 0.05 * np.sin(np.arange(64) * 0.7)
    cv.train(B, samples, 77, phi)
    got = cv.get_params().astype(np.float64)
    x = mlp.features(77, 0, samples, s, 2.0, 10.0).astype(np.float32).astype(np.float64)
    y = ((phi - phi.mean()) / phi.std(ddof=1)).astype(np.float32).astype(np.float64)
    mask = mlp.weight_mask(d_in, 16, 2)
    p, m, v = p0, np.zeros_like(p0), np.zeros_like(p0)
    for t in (1, 2):
        fwd = _bf16_weights(p, d_in, 16, 2).astype(np.float64)
        _, grad = mlp.loss_and_grad(fwd, x, y, d_in, 16, 2)
        p, m, v = mlp.adam_step(p.astype(np.float32).astype(np.float64), m, v, grad, t, lr,
                                wd=wd, decay_mask=mask)
    err = np.abs(got - p)
    # a wrong bias correction moves the first step by 0.316 lr; a missing decay by lr wd |theta|
    assert np.quantile(err, 0.999) < 1e-3 * lr, np.sort(err)[-5:]
    assert err.max() < 2 * lr
    assert np.max(np.abs(got - p0)) > 1.5 * lr  # two steps were taken


def test_eval_and_mean_match_reference():
    """Features from the device Philox map + forward pass = reference forward."""
    s, sy, cv = _net(hidden=16, layers=2)
    rng = np.random.default_rng(1)
    p = _bf16_weights(rng.normal(0, 0.4, cv.n_params), cv.d_in, 16, 2)
    cv.set_params(p)
    samples = np.arange(10, 60)
    got = cv.eval(np.full(50, 3.0), samples, 1234)
    x = mlp.features(1234, 0, samples, s, 3.0, 10.0)
    ref, _ = mlp.forward(p.astype(np.float64), x, cv.d_in, 16, 2)
    assert np.max(np.abs(got - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))
    mu, vm = cv.mean([0.0, 3.0], 4096, 99)
    for i, B in enumerate([0.0, 3.0]):
        xr = mlp.features(99, 0, np.arange(4096), s, B, 10.0)
        gr, _ = mlp.forward(p.astype(np.float64), xr, cv.d_in, 16, 2)
        assert abs(mu[i] - gr.mean()) < 1e-5 * max(1.0, abs(gr.mean()))
        assert abs(vm[i] - gr.var(ddof=1) / 4096) < 1e-3 * vm[i] + 1e-12


def test_estimate_kernel_matches_reference():
    s, sy, cv = _net(hidden=8, layers=1)
    rng = np.random.default_rng(4)
    counts = np.array([50, 80, 33])
    offsets = np.array([0, 50, 130])
    ps = rng.normal(0.5, 0.05, (163, 3))
    # the network's outputs are FP32: compare on FP32-representable g
    g = (ps[:, 0] * 3.0 + rng.normal(0, 0.05, 163)).astype(np.float32).astype(np.float64)
    mu = np.array([1.4, 1.6, 1.5])
    vm = np.array([1e-8, 2e-8, 0.0])
    out = cv.estimate(offsets, counts, ps.ravel(), g, mu, vm)
    for f in range(3):
        sl = slice(offsets[f], offsets[f] + counts[f])
        est, se, beta = mlp.cv_estimate(ps[sl, 0], g[sl], mu[f], vm[f])
        assert np.allclose(out[f, [0, 1, 4]], [est, se, beta], rtol=1e-9, atol=1e-13)
        assert abs(out[f, 2] - ps[sl, 0].mean()) < 1e-13


def test_trained_control_variate_gains_and_stays_unbiased():
    """Config-1 system: a network trained on 6144 per-sample yields cuts the
    variance of the field estimates several-fold on fresh samples, and the
    control-variate estimate agrees with the exact trace (Eq. 14) within 4 SE."""
    from paper_1612_09517_gb300 import rp
    w = wl.config1()
    s = w.system
    sy = rp.System(s)
    fields = np.array([0.0, 1.0, 2.0])
    T = 3.0
    train = sy.yields(fields, 2048, 11, T, per_sample=True, precision="fp32")
    phi_tr = train["per_sample"][:, :, 0]
    cv = rp.ControlVariate(sy, hidden=64, layers=3, epochs=60, batch=256, lr=2e-3)
    B_tr = np.repeat(fields, 2048)
    samp_tr = np.tile(np.arange(2048), 3)
    losses = cv.train(B_tr, samp_tr, 11, phi_tr.ravel())
    assert losses[-1] < 0.5 * losses[0]
    M = 256
    est = sy.yields(fields, M, 22, T, per_sample=True, precision="fp32")
    ps = est["per_sample"].reshape(-1, 3)
    g = cv.eval(np.repeat(fields, M), np.tile(np.arange(M), 3), 22)
    mu, vm = cv.mean(fields, 1 << 16, 33)
    out = cv.estimate(np.arange(3) * M, np.full(3, M), ps.ravel(), g, mu, vm)
    gain = (out[:, 3] / out[:, 1]) ** 2
    assert np.all(gain > 3.0), gain
    for i, B in enumerate(fields):
        exact = dense.trace_yields(s, B, T)[0]
        assert abs(out[i, 0] - exact) < 4 * out[i, 1] + 1e-5
    print("variance reduction per field:", gain)


def test_converged_curve_with_control_variate():
    """rp_yields_cv: every field reaches the combined SE target, control-variate
    fields need fewer samples than their plain spread asks for, and every
    estimate agrees with the exact trace (Eq. 14) within 4 SE."""
    from paper_1612_09517_gb300 import rp
    w = wl.config1()
    s = w.system
    sy = rp.System(s)
    fields = np.array([0.0, 1.0, 2.0, 5.0])
    T, se = 3.0, 2e-3
    plan = rp.rp_cv_default_plan(M_train=128, cv_threshold=64,
                                 net=dict(hidden=64, layers=3, epochs=60, lr=2e-3))
    r = rp.rp_yields_cv(sy.handle, fields, se, 8, 20000, 7, T,
                        rp.rp_default_options(precision="fp32"), plan)
    out = r["out"]
    assert np.all(out[:, 1] <= se * 1.0001)
    used_cv = out[:, 7] > 0
    assert used_cv.any()
    for i, B in enumerate(fields):
        exact = dense.trace_yields(s, B, T)[0]
        assert abs(out[i, 0] - exact) < 4 * out[i, 1] + 1e-5
        if used_cv[i]:
            plain_need = (out[i, 3] ** 2 * r["M_plain"][i]) / se ** 2
            assert r["M_plain"][i] + r["M_cv"][i] < plain_need
    print("M_plain", r["M_plain"], "M_cv", r["M_cv"], "beta", out[:, 6])
