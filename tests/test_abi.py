"""C-ABI library: loads, exports every declared symbol, validates, plans (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest
import scipy.special

from paper_1612_09517_gb300 import rp
from paper_1612_09517_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "rp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(rp_\w+)\s*\(", src, flags=re.M))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_library_exports_every_declared_symbol():
    names = _declared_functions()
    assert len(names) >= 12, names
    lib = ctypes.CDLL(rp.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/rp.h but not exported"
    bound = {s[0] for s in rp.SIGNATURES}
    assert set(names) == bound, set(names) ^ bound


def test_status_strings_and_defaults():
    assert rp.LIB.rp_status_str(0) == b"RP_OK"
    assert rp.LIB.rp_status_str(7) == b"RP_ENODEV"
    o = rp.rp_default_options()
    assert o.precision == rp.RP_FP32 and o.n_cheb == 0 and o.stream is None


@pytest.mark.parametrize("kw,msg", [
    (dict(radical=[2], two_I=[1], A=np.eye(3)), "radical"),
    (dict(radical=[0], two_I=[0], A=np.eye(3)), "two_I"),
    (dict(radical=[0], two_I=[10], A=np.eye(3)), "two_I"),
    (dict(radical=[0], two_I=[1], A=np.array([[1, 2, 0], [0, 1, 0], [0, 0, 1.]])), "symmetric"),
    (dict(radical=[0], two_I=[1], A=np.eye(3) * np.nan), "finite"),
])
def test_create_validation(kw, msg):
    with pytest.raises(rp.RPError, match=msg):
        rp.rp_create(kw["radical"], kw["two_I"], kw["A"], 1.0, 1.0, 0.0)


def test_create_rate_validation():
    with pytest.raises(rp.RPError, match="RP_EINVAL"):
        rp.rp_create([0], [1], np.eye(3), 0.0, 0.0, 0.0)
    with pytest.raises(rp.RPError, match="RP_EINVAL"):
        rp.rp_create([0], [1], np.eye(3), -1.0, 1.0, 0.0)
    with pytest.raises(rp.RPError, match="exceeds"):
        rp.rp_create([0] * 24, [2] * 24, np.tile(np.eye(3), (24, 1)), 1.0, 1.0, 0.0)


def test_layout_orders_spin_half_first_and_permutes_states():
    s = wl.random_isotropic(2, 2, two_I=[2, 1, 3, 1], seed=1)
    sy = rp.System(s)
    assert list(sy.order) == [1, 3, 0, 2] and sy.Z == 2 * 3 * 4 * 2
    x = np.random.default_rng(0).normal(size=(3, 4 * sy.Z))
    assert np.array_equal(sy.to_input_order(sy.from_input_order(x)), x)


def test_plan_bounds_contain_the_spectrum():
    """Weyl bounds enclose the exact eigenvalues of H (oracle dense matrix)."""
    from oracle import spin
    for s in (wl.random_anisotropic(2, 1, two_I=[1, 2, 1], J=0.4, seed=2),
              wl.random_isotropic(1, 2, two_I=[3, 1, 2], J=-0.3, seed=3), wl.config1().system):
        sy = rp.System(s)
        for B in (0.0, 1.7, -4.0):
            p = sy.plan(B, 5.0)
            ev = np.linalg.eigvalsh(spin.hamiltonian(s, B))
            assert p["E_min"] <= ev[0] + 1e-9 and p["E_max"] >= ev[-1] - 1e-9
            assert p["E_c"] - p["dE"] <= ev[0] and p["E_c"] + p["dE"] >= ev[-1]
            assert abs(p["h"] * p["n_macro"] - 5.0) < 1e-12


def test_plan_coefficients_match_scipy_bessel():
    s = wl.random_isotropic(2, 2, k_S=2.0, k_T=0.5, seed=4)
    sy = rp.System(s)
    for prec, tol in ((rp.RP_FP64, 1e-15), (rp.RP_FP32, 1e-9)):
        p = sy.plan(3.0, 7.0, precision=prec, with_coef=True)
        n = np.arange(p["n_cheb"])
        x = p["dE"] * p["h"]
        # J_n(x) at x ~ 46: SciPy's jv is off by up to ~2e-15 there, so the
        # reference is 40-digit mpmath when it is installed
        try:
            import mpmath
            mpmath.mp.dps = 40
            jn = np.array([float(mpmath.besselj(int(k), mpmath.mpf(float(x)))) for k in n])
            atol = 1e-15
        except ImportError:
            jn = scipy.special.jv(n, x)
            atol = 3e-15
        ref = (np.where(n == 0, 1, 2) * (-1j) ** n * jn
               * np.exp(-0.5 * p["kbar"] * p["h"] - 1j * p["E_c"] * p["h"]))
        assert np.allclose(p["coef"], ref, rtol=0, atol=atol)
        assert p["tail"] <= tol
        # time-integral weights: Hermitian and equal to a SciPy quadrature
        W = p["W"]
        assert np.allclose(W, W.conj().T, atol=1e-16)
        q, w = np.polynomial.legendre.leggauss(200)
        tau = 0.5 * p["h"] * (q + 1)
        wt = 0.5 * p["h"] * w * np.exp(-p["kbar"] * tau)
        c = (np.where(n == 0, 1, 2) * (-1j) ** n)[None, :] * scipy.special.jv(n[None, :], p["dE"] * tau[:, None])
        Wref = np.einsum("q,qn,qm->nm", wt, c.conj(), c)
        assert np.max(np.abs(W - Wref)) < 1e-15 * p["h"] * 50


def test_plan_rejects_bad_arguments():
    sy = rp.System(wl.config1().system)
    with pytest.raises(rp.RPError):
        sy.plan(1.0, -1.0)
    with pytest.raises(rp.RPError):
        sy.plan(1.0, 1.0, n_cheb=4)


def test_yields_argument_checks_without_gpu():
    sy = rp.System(wl.config1().system)
    r = sy.yields(np.zeros(0), 4, 0, 1.0)  # empty sweep is a no-op
    assert r["out"].shape == (0, 5)
    with pytest.raises(rp.RPError, match="M must be"):
        sy.yields([0.0], 1, 0, 1.0)
    with pytest.raises(rp.RPError, match="t_max"):
        sy.yields([0.0], 4, 0, 0.0)
    with pytest.raises(rp.RPError, match="finite"):
        sy.yields([np.inf], 4, 0, 1.0)


def test_yields_reports_missing_device_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    sy = rp.System(wl.config1().system)
    with pytest.raises(rp.RPError, match="RP_ENODEV"):
        sy.yields([0.0], 4, 0, 1.0)


def test_time_trace_size_query_and_capacity():
    """rp_time_trace reports n_macro + 1 time points without a GPU and refuses a
    too small output buffer before any device work."""
    s = wl.random_isotropic(2, 1, seed=9)
    sy = rp.System(s)
    p = sy.plan(1.5, 2.0)
    o = rp.rp_default_options(precision=rp.RP_FP64)
    n = ctypes.c_int(0)
    assert rp.LIB.rp_time_trace(sy.handle, 1.5, 4, ctypes.c_uint64(0), 2.0, ctypes.byref(o), 0,
                                ctypes.byref(n), None, None) == 0
    assert n.value == p["n_macro"] + 1
    t = np.zeros(n.value)
    out = np.zeros(3 * n.value)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = rp.LIB.rp_time_trace(sy.handle, 1.5, 4, ctypes.c_uint64(0), 2.0, ctypes.byref(o),
                              n.value - 1, ctypes.byref(n), dp(t), dp(out))
    assert st == 1  # RP_EINVAL


def test_basis_indices_bit_exact_with_oracle():
    """The library's host draw of basis indices (deterministic = 2) equals the
    oracle's Philox draw bit for bit."""
    from oracle import philox
    for seed, pair, off, Z in ((0, 0, 0, 16), (12345678901, 7, 2 ** 33 + 5, 20736),
                               (3, 1, 1000, 1048576), (2 ** 63 + 11, 2 ** 31, 17, 3)):
        got = rp.rp_basis_indices(seed, pair, off, 64, Z)
        ref = philox.draw_basis_indices(seed, pair, np.arange(off, off + 64, dtype=np.uint64), Z)
        assert np.array_equal(got, ref), (seed, pair, off, Z)


def test_option_validation_without_gpu():
    """Execution options outside their ranges are refused before any device
    work: kernel path, time-integral path, graph replay, sampling mode; the
    autotuner needs two rows; basis-index draws need a positive Z."""
    sy = rp.System(wl.config1().system)
    for kw, msg in ((dict(kernel=6), "kernel"), (dict(kernel=-1), "kernel"), (dict(gram=3), "gram"),
                    (dict(graph=2), "graph"), (dict(deterministic=4), "deterministic")):
        with pytest.raises(rp.RPError, match=msg):
            sy.yields([0.0], 4, 0, 1.0, **kw)
    with pytest.raises(rp.RPError, match="rows"):
        rp.rp_tune(sy.handle, 1.0, 1)
    with pytest.raises(rp.RPError, match="RP_EINVAL"):
        rp.rp_basis_indices(0, 0, 0, 4, 0)
    with pytest.raises(rp.RPError, match="coherent"):
        sy.yields_converged([0.0], 1e-3, 8, 100, 0, 1.0, deterministic=1)


def test_static_entry_point_refuses_other_launch_choices_without_gpu():
    """rp_yields_static always runs the per-term kernels with the CUDA-core
    integral, eagerly: other kernel, gram and graph choices, and random
    basis-state sampling, are refused before any device work."""
    sy = rp.System(wl.config1().system)
    for kw, msg in ((dict(kernel=2), "kernel"), (dict(kernel=3), "kernel"), (dict(gram=2), "gram"),
                    (dict(graph=1), "graph"), (dict(deterministic=2), "basis-state"),
                    (dict(max_rows=-1), "max_rows")):
        with pytest.raises(rp.RPError, match=msg):
            rp.rp_yields_static(sy.handle, [0.0], 4, 0, 1.0, rp.rp_default_options(**kw))


def test_trace_propagations_count_sector_classes():
    """deterministic = 3 needs as many propagations as the largest class of
    nuclear configurations with equal total M (counted here by brute force);
    deterministic = 1 needs Z; anisotropic systems are refused."""
    import itertools
    for s in (wl.config1().system, wl.config2().system,
              wl.random_isotropic(2, 2, two_I=[1, 2, 3, 1], seed=3)):
        sy = rp.System(s)
        counts = {}
        for ms in itertools.product(*[range(int(t) + 1) for t in s.two_I]):
            two_M = sum(int(t) - 2 * j for t, j in zip(s.two_I, ms))
            counts[two_M] = counts.get(two_M, 0) + 1
        assert rp.rp_trace_propagations(sy.handle, 3) == max(counts.values())
        assert rp.rp_trace_propagations(sy.handle, 1) == s.Z
    assert rp.rp_trace_propagations(rp.System(wl.config1().system).handle, 3) == 6
    an = rp.System(wl.random_anisotropic(1, 1, seed=2))
    with pytest.raises(rp.RPError, match="isotropic"):
        rp.rp_trace_propagations(an.handle, 3)
    with pytest.raises(rp.RPError, match="isotropic"):
        an.yields([0.0], 2, 0, 1.0, deterministic=3)
