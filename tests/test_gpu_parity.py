"""GPU parity: the sm_103a path through the C ABI against the FP64 CPU oracle.

Tolerances (per-sample yields phi_S, phi_T of Eq. 22 truncated at T):
* FP64 path: 1e-10 relative.  The plan bounds the Chebyshev truncation by
  1e-15 per macro-step; FP64 rounding over ~1e2-1e4 macro-steps stays far below.
* FP32 path: 1e-5 relative.  FP32 storage rounds each term at 6e-8; the
  accumulated random walk over the macro-steps of these horizons stays below.
Survival |psi(T)|^2 is compared in absolute terms at the same levels.
"""
import math

import numpy as np
import pytest

from oracle import chebyshev, coherent, dense, philox, spin
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


def _rp():
    from paper_1612_09517_gb300 import rp
    return rp


TOL = {"fp64": 1e-10, "fp32": 1e-5}


def _cmp_per_sample(got, phS, phT, surv, prec):
    tol = TOL[prec]
    eS = np.max(np.abs(got[:, 0] - phS) / np.maximum(np.abs(phS), 1e-3))
    # phi_T = 1 - survival - phi_S is derived by conservation, so its error is
    # measured on the scale of the yields (max(|phi_T|, |phi_S|))
    eT = np.max(np.abs(got[:, 1] - phT) / np.maximum(np.maximum(np.abs(phT), np.abs(phS)), 1e-3))
    eU = np.max(np.abs(got[:, 2] - surv))
    assert eS < tol and eT < tol and eU < tol, (eS, eT, eU)
    return max(eS, eT)


MIXED = [
    ("config1", lambda: wl.config1().system),
    ("aniso_mixed", lambda: wl.random_anisotropic(2, 1, two_I=[1, 2, 1], k_S=2.0, k_T=0.5, J=0.3, seed=40)),
    ("spin3half_J", lambda: wl.random_isotropic(1, 2, two_I=[3, 1, 2], k_S=0.2, k_T=5.0, J=-0.5, seed=41)),
    ("no_nuclei", lambda: wl.SpinSystem([], [], np.zeros((0, 3, 3)), 1.5, 0.7, 0.4)),
    ("ragged_z", lambda: wl.random_isotropic(3, 2, two_I=[2, 1, 2, 2, 1], k_S=1.0, k_T=2.0, seed=42)),
    # five anisotropic spin-1/2 nuclei, Z = 32: a 32-thread block holds the
    # per-block U / U-dagger table of 40 entries (strided fill)
    ("aniso_5half", lambda: wl.random_anisotropic(3, 2, two_I=[1] * 5, k_S=1.2, k_T=0.4, J=0.2,
                                                  seed=48)),
]


# ------------------------------------------------------------ initial states

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,mk", MIXED, ids=[m[0] for m in MIXED])
def test_initial_states_match_oracle(name, mk, prec):
    rp = _rp()
    s = mk()
    sy = rp.System(s)
    n, sample0, seed, pair = 5, 3, 12345678901, 7
    dt = torch.float64 if prec == "fp64" else torch.float32
    psi = torch.zeros(n * 4 * sy.Z * 2, dtype=dt, device="cuda")
    uv = rp.rp_init_states(sy.handle, rp.RP_FP64 if prec == "fp64" else rp.RP_FP32, seed, pair,
                           sample0, n, psi.data_ptr(), sy.n_nuc)
    if sy.n_nuc:
        u1, u2 = philox.draw_uniforms(seed, pair, np.arange(sample0, sample0 + n), sy.n_nuc)
        # integer work: the 53-bit uniforms must agree bit for bit
        assert np.array_equal(uv[..., 0], u1) and np.array_equal(uv[..., 1], u2)
    got = psi.cpu().numpy().view(np.complex128 if prec == "fp64" else np.complex64)
    got = sy.to_input_order(got.reshape(n, 4 * sy.Z))
    ref = coherent.sample_states(s, seed, np.arange(sample0, sample0 + n), pair=pair)
    assert np.max(np.abs(got - ref)) < (1e-14 if prec == "fp64" else 2e-7)


# --------------------------------------------------------------------- H psi

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,mk", MIXED, ids=[m[0] for m in MIXED])
def test_apply_h_matches_dense(name, mk, prec):
    """(H - iK) x of the kernel against the oracle's dense Eq. 1 - Eq. 2 matrix."""
    rp = _rp()
    s = mk()
    sy = rp.System(s)
    rng = np.random.default_rng(5)
    n_vec = 3
    x = rng.normal(size=(n_vec, 4 * sy.Z)) + 1j * rng.normal(size=(n_vec, 4 * sy.Z))
    for B in (0.0, 2.3, -7.1):
        Heff = spin.hamiltonian(s, B) - 1j * spin.haberkorn(s)
        ref = x @ Heff.T
        cdt = np.complex128 if prec == "fp64" else np.complex64
        xl = np.ascontiguousarray(sy.from_input_order(x).astype(cdt))
        dt = torch.float64 if prec == "fp64" else torch.float32
        xd = torch.from_numpy(xl.view(np.float64 if prec == "fp64" else np.float32).copy()).to("cuda")
        yd = torch.zeros_like(xd)
        rp.rp_apply_h(sy.handle, B, rp.RP_FP64 if prec == "fp64" else rp.RP_FP32, n_vec,
                      xd.data_ptr(), yd.data_ptr())
        got = sy.to_input_order(yd.cpu().numpy().view(cdt).reshape(n_vec, -1))
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err < (1e-13 if prec == "fp64" else 2e-6), err


# ----------------------------------------------------------- yields, config 1

@pytest.mark.parametrize("kernel", [0, 5])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_config1_per_sample_parity(prec, kernel):
    """Config 1 in full (11 fields in 0-5 mT, M = 64, seed 0, T = 10 us), in
    the default launch form and in one persistent launch (kernel 5)."""
    rp = _rp()
    w = wl.config1()
    s = w.system
    sy = rp.System(s)
    res = sy.yields(w.fields, w.M, w.seed, w.t_max, per_sample=True, precision=prec, kernel=kernel)
    if kernel == 5:
        assert res["stats"]["kernel_path"] == 5 and res["stats"]["step_launches"] == 1
    psi0 = coherent.sample_states(s, w.seed, range(w.M))
    worst = 0.0
    for i, B in enumerate(w.fields):
        phS, phT, surv = dense.sample_yields(s, B, w.t_max, psi0)
        worst = max(worst, _cmp_per_sample(res["per_sample"][i], phS, phT, surv, prec))
        # per-field mean and standard error (Eq. 18, Eq. 23) of the device reduction
        mS, seS = dense.estimate(res["per_sample"][i][:, 0])
        assert abs(res["out"][i, 0] - mS) < 1e-14 and abs(res["out"][i, 2] - seS) < 1e-14
        mO, _ = dense.estimate(phS)
        assert abs(res["out"][i, 0] - mO) < TOL[prec]
    print(f"config1 {prec}: worst relative per-sample error {worst:.2e}")


def test_side_case_closed_form():
    """One spin-1/2, a = 1 mT, k = 1 us^-1, T = 10 us: Phi_S = 0.6249838157 (closed form)."""
    rp = _rp()
    sy = rp.System(wl.one_nucleus(1.0, 1, 1.0))
    for prec, tol in (("fp64", 1e-10), ("fp32", 1e-5)):
        r = sy.yields([0.0], 2, 0, 10.0, precision=prec, deterministic=1)
        assert abs(r["out"][0, 0] - 0.6249838157) < tol
        r = sy.yields([0.0], 8, 3, 10.0, per_sample=True, precision=prec)
        assert np.max(np.abs(r["per_sample"][0, :, 0] - 0.6249838157)) < tol


def test_deterministic_trace_matches_oracle():
    """Eq. 14 on the GPU (Z basis states) against tr[Y P_S]/Z of the oracle."""
    rp = _rp()
    s = wl.random_anisotropic(2, 1, two_I=[1, 2, 1], k_S=2.0, k_T=0.5, J=0.3, seed=40)
    sy = rp.System(s)
    fields = np.array([0.0, 1.5, -1.5])
    r = sy.yields(fields, 2, 0, 3.0, precision="fp64", deterministic=1)
    for i, B in enumerate(fields):
        ref = dense.trace_yields(s, B, 3.0)
        assert abs(r["out"][i, 0] - ref[0]) < 1e-10 * abs(ref[0])
        assert abs(r["out"][i, 1] - ref[1]) < 1e-10 * abs(ref[1])
        assert abs(r["out"][i, 4] - ref[2]) < 1e-12
    # field-reversal symmetry of the trace
    assert abs(r["out"][1, 0] - r["out"][2, 0]) < 1e-10


SECTOR = [
    ("config1", lambda: wl.config1().system),
    ("spin1_J", lambda: wl.random_isotropic(2, 2, two_I=[1, 2, 1, 2], k_S=2.0, k_T=0.4, J=0.3,
                                            seed=46)),
    ("spin32", lambda: wl.random_isotropic(1, 2, two_I=[3, 1, 2], k_S=0.2, k_T=5.0, J=-0.5,
                                           seed=41)),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,mk", SECTOR, ids=[c[0] for c in SECTOR])
def test_sector_trace_matches_oracle_and_basis_states(name, mk, prec):
    """The J_z-sector trace (deterministic = 3) equals tr[Y P_S]/Z of the
    oracle (Eq. 14) with fewer propagations, and each propagation's yield is
    the mean of the yields of the basis states it carries (run one by one
    with deterministic = 1): the cross terms between J_z classes vanish."""
    rp = _rp()
    s = mk()
    sy = rp.System(s)
    fields = np.array([0.0, 1.2, 4.0])
    T = 2.5
    r3 = sy.yields(fields, 2, 0, T, per_sample=True, precision=prec, deterministic=3)
    r1 = sy.yields(fields, 2, 0, T, per_sample=True, precision=prec, deterministic=1)
    n3 = rp.rp_trace_propagations(sy.handle, 3)
    assert r3["per_sample"].shape == (3, n3, 3) and n3 < sy.Z
    assert r3["stats"]["propagations"] == 3 * n3
    tol = TOL[prec]
    for i, B in enumerate(fields):
        ref = dense.trace_yields(s, B, T)
        assert abs(r3["out"][i, 0] - ref[0]) < tol * abs(ref[0])
        assert abs(r3["out"][i, 1] - ref[1]) < tol * max(abs(ref[1]), abs(ref[0]))
        assert abs(r3["out"][i, 4] - ref[2]) < tol
        assert r3["out"][i, 2] == 0.0 and r3["out"][i, 3] == 0.0
    # class of every layout configuration: total 2M from the layout digits
    dims = [int(s.two_I[k]) + 1 for k in sy.order]
    rank, seen = np.zeros(sy.Z, int), {}
    for m in range(sy.Z):
        q, two_M = m, 0
        for d in dims:
            two_M += (d - 1) - 2 * (q % d)
            q //= d
        rank[m] = seen.get(two_M, 0)
        seen[two_M] = rank[m] + 1
    for i in range(n3):
        members = np.flatnonzero(rank == i)
        want = r1["per_sample"][:, members, :].mean(axis=1)
        assert np.allclose(r3["per_sample"][:, i, :], want, rtol=tol, atol=tol * 1e-2), i


@pytest.mark.parametrize("kernel", [1, 2, 5])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,mk", MIXED[1:], ids=[m[0] for m in MIXED[1:]])
def test_mixed_systems_per_sample(name, mk, prec, kernel):
    """Anisotropic tensors, spin 1 and 3/2, J != 0, k_S != k_T, no nuclei, ragged Z;
    per-term launches (kernel 1), whole macro-steps on chip (kernel 2) and
    whole propagations in one persistent launch (kernel 5)."""
    rp = _rp()
    s = mk()
    sy = rp.System(s)
    fields = np.array([0.0, 0.8, 3.0])
    T, M = 2.5, 6
    r = sy.yields(fields, M, 11, T, per_sample=True, precision=prec, kernel=kernel)
    psi0 = coherent.sample_states(s, 11, range(M))
    for i, B in enumerate(fields):
        phS, phT, surv = dense.sample_yields(s, B, T, psi0)
        _cmp_per_sample(r["per_sample"][i], phS, phT, surv, prec)


def test_no_nuclei_closed_form():
    rp = _rp()
    sy = rp.System(wl.SpinSystem([], [], np.zeros((0, 3, 3)), 1.5, 0.7, 0.4))
    r = sy.yields([0.0, 4.0], 2, 0, 1.3, precision="fp64")
    assert np.allclose(r["out"][:, 0], 1 - math.exp(-1.5 * 1.3), atol=1e-12)
    assert np.allclose(r["out"][:, 1], 0.0, atol=1e-12)


# ------------------------------------------------------- execution invariance

def test_batching_and_offset_invariance():
    """Row batching (max_rows) and sample_offset do not change any sample's result."""
    rp = _rp()
    s = wl.random_isotropic(2, 2, two_I=[1, 2, 1, 1], k_S=1.0, k_T=3.0, J=0.2, seed=7)
    sy = rp.System(s)
    fields = [0.0, 1.0, 4.0]
    a = sy.yields(fields, 8, 5, 2.0, per_sample=True, precision="fp64")
    b = sy.yields(fields, 8, 5, 2.0, per_sample=True, precision="fp64", max_rows=5)
    assert np.allclose(a["per_sample"], b["per_sample"], rtol=1e-13, atol=1e-15)
    c = sy.yields(fields, 4, 5, 2.0, per_sample=True, precision="fp64", sample_offset=4)
    assert np.allclose(a["per_sample"][:, 4:], c["per_sample"], rtol=1e-13, atol=1e-15)


def test_edge_cases():
    rp = _rp()
    sy = rp.System(wl.config1().system)
    # horizon shorter than one macro-step, minimal M
    r = sy.yields([0.0, 5.0], 2, 0, 1e-4, per_sample=True, precision="fp64")
    psi0 = coherent.sample_states(wl.config1().system, 0, range(2))
    for i, B in enumerate([0.0, 5.0]):
        phS, phT, surv = dense.sample_yields(wl.config1().system, B, 1e-4, psi0)
        assert np.allclose(r["per_sample"][i, :, 0], phS, rtol=1e-10, atol=1e-16)
    # k_S = 0: no singlet yield at all
    s0 = wl.random_isotropic(2, 0, k_S=0.0, k_T=1.0, seed=3)
    r = rp.System(s0).yields([1.0], 3, 0, 2.0, per_sample=True, precision="fp64")
    assert np.all(r["per_sample"][0, :, 0] == 0.0)
    assert r["stats"]["kernel_launches"] > 0


# -------------------------------------------- config 2 at full size, sampled

@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_config2_full_size_sampled(prec):
    """Config 2 (Z = 20736, 12 nuclei, k_S != k_T) in the bench's launch form:
    all rows of a field sweep run together; sampled rows against the oracle's
    matrix-free FP64 propagation (horizon shortened so the CPU finishes)."""
    rp = _rp()
    w = wl.config2()
    sy = rp.System(w.system)
    fields = np.array([0.0, 10.0, 3.0, 30.0])
    M, T = 4, 0.15
    r = sy.yields(fields, M, 0, T, per_sample=True, precision=prec)
    psi0 = coherent.sample_states(w.system, 0, [0, 3])
    for fi, si in ((0, 0), (1, 3)):
        ref = chebyshev.propagate_yields(w.system, fields[fi], T, psi0[0 if si == 0 else 1])
        got = r["per_sample"][fi, si]
        assert abs(got[0] - ref[0]) < TOL[prec] * abs(ref[0])
        # phi_T comes from conservation: error on the scale of the yields
        assert abs(got[1] - ref[1]) < TOL[prec] * max(abs(ref[1]), abs(ref[0]))
        assert abs(got[2] - ref[2]) < TOL[prec]


# ----------------------------------------------- converged curve (Eq. 23 target)

def test_converged_curve_meets_target_and_matches_plain_runs():
    """rp_yields_converged: every field reaches SE <= target (or M_max), and each
    field's estimate equals rp_yields over the same sample indices 0..M_f-1."""
    rp = _rp()
    s = wl.random_isotropic(3, 1, k_S=1.0, k_T=1.0, seed=21)
    sy = rp.System(s)
    fields = np.array([0.0, 1.0, 3.0, 8.0])
    se_target, M_min, M_max = 4e-3, 8, 600
    r = sy.yields_converged(fields, se_target, M_min, M_max, 5, 3.0, precision="fp64", max_rows=37)
    used = r["M_used"]
    assert np.all(used >= M_min) and np.all(used <= M_max)
    for i, B in enumerate(fields):
        assert r["out"][i, 2] <= se_target or used[i] == M_max
        plain = sy.yields([B], int(used[i]), 5, 3.0, precision="fp64")
        assert np.allclose(r["out"][i], plain["out"][0], rtol=1e-12, atol=1e-14)
    # the oracle agrees on the samples it can check cheaply
    psi0 = coherent.sample_states(s, 5, range(int(used[0])))
    phS, _, _ = dense.sample_yields(s, fields[0], 3.0, psi0)
    assert abs(r["out"][0, 0] - phS.mean()) < 1e-10


# ------------------------------------------- several systems of uneven size

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_of_uneven_systems_matches_single_runs(prec):
    """rp_yields_batch over systems of different Z, spins, tensors, rates and
    horizons equals rp_yields of each system with pair word pair_id + s."""
    rp = _rp()
    systems = [wl.config1().system,
               wl.random_anisotropic(2, 1, two_I=[1, 2, 1], k_S=2.0, k_T=0.5, J=0.3, seed=40),
               wl.random_isotropic(1, 2, two_I=[3, 1, 2], k_S=0.2, k_T=5.0, J=-0.5, seed=41),
               wl.random_isotropic(5, 4, seed=43, k_S=1.0, k_T=0.3)]
    sys_h = [rp.System(s) for s in systems]
    fields = [np.array([0.0, 2.0]), np.array([1.0]), np.array([0.5, 3.0, 7.0]), np.array([0.0, 4.0])]
    M = [5, 3, 4, 2]
    T = [2.0, 1.5, 1.0, 0.8]
    o = rp.rp_default_options(precision=prec, pair_id=10)
    r = rp.rp_yields_batch(sys_h, fields, M, T, 77, o)
    tol = TOL[prec]
    for s in range(len(systems)):
        single = sys_h[s].yields(fields[s], M[s], 77, T[s], precision=prec, pair_id=10 + s)
        assert np.allclose(r["out"][s], single["out"], rtol=tol, atol=tol * 1e-2), s
    # and the oracle agrees for the smallest system
    psi0 = coherent.sample_states(systems[1], 77, range(3), pair=11)
    phS, _, _ = dense.sample_yields(systems[1], 1.0, 1.5, psi0)
    assert abs(r["out"][1][0, 0] - phS.mean()) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_kernel_paths_agree(prec):
    """The on-chip macro-step kernel and the per-term kernels give the same
    per-sample yields (largest Z that fits on chip included)."""
    rp = _rp()
    big = wl.random_isotropic(6, 4, two_I=[1] * 10, seed=44, k_S=1.0, k_T=0.4, J=0.1)  # Z = 1024
    for s in (wl.config1().system, big):
        sy = rp.System(s)
        a = sy.yields([0.0, 2.0], 4, 3, 1.0, per_sample=True, precision=prec, kernel=1)
        b = sy.yields([0.0, 2.0], 4, 3, 1.0, per_sample=True, precision=prec, kernel=2)
        c = sy.yields([0.0, 2.0], 4, 3, 1.0, per_sample=True, precision=prec, kernel=5)
        tol = 1e-12 if prec == "fp64" else 2e-6
        assert np.allclose(a["per_sample"], b["per_sample"], rtol=tol, atol=tol * 1e-2)
        assert np.allclose(a["per_sample"], c["per_sample"], rtol=tol, atol=tol * 1e-2)
        assert b["stats"]["step_launches"] < a["stats"]["step_launches"]
        assert c["stats"]["kernel_path"] == 5 and c["stats"]["step_launches"] == 1


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_persistent_launch_edges(prec):
    """One persistent launch (kernel 5): the largest Z it takes (2048 FP32,
    1024 FP64), more items than CTAs with uneven horizons (fields of different
    step counts share the launch), the basis-state trace (deterministic 1),
    an uneven batch, and a system too large for it (selects as kernel 0)."""
    rp = _rp()
    tol = 1e-12 if prec == "fp64" else 2e-6
    n_half = 11 if prec == "fp32" else 10
    top = wl.random_isotropic(6, n_half - 6, two_I=[1] * n_half, seed=45, k_S=0.8, k_T=2.0, J=0.2)
    sy = rp.System(top)
    a = sy.yields([0.0, 6.0], 3, 9, 0.6, per_sample=True, precision=prec, kernel=1)
    c = sy.yields([0.0, 6.0], 3, 9, 0.6, per_sample=True, precision=prec, kernel=5)
    assert c["stats"]["kernel_path"] == 5
    assert np.allclose(a["per_sample"], c["per_sample"], rtol=tol, atol=tol * 1e-2)
    # many items per CTA, fields with different macro-step counts
    s = wl.random_isotropic(2, 2, two_I=[1, 2, 1, 1], k_S=1.0, k_T=3.0, J=0.2, seed=7)
    sy = rp.System(s)
    fields = [0.0, 1.0, 4.0, 20.0]
    a = sy.yields(fields, 400, 5, 2.0, per_sample=True, precision=prec, kernel=2)
    c = sy.yields(fields, 400, 5, 2.0, per_sample=True, precision=prec, kernel=5)
    assert c["stats"]["propagations"] > c["stats"]["rows"]
    assert np.allclose(a["per_sample"], c["per_sample"], rtol=tol, atol=tol * 1e-2)
    # basis-state trace (Eq. 14) against the oracle's trace
    a = sy.yields(fields[:2], 0, 0, 2.0, per_sample=True, precision=prec, deterministic=1, kernel=5)
    for i, B in enumerate(fields[:2]):
        ref = dense.trace_yields(s, B, 2.0)
        assert abs(a["out"][i, 0] - ref[0]) < TOL[prec]
    # uneven batch in one launch per group
    systems = [wl.config1().system, wl.random_anisotropic(2, 1, two_I=[1, 2, 1], k_S=2.0, k_T=0.5,
                                                          J=0.3, seed=40)]
    sys_h = [rp.System(x) for x in systems]
    fl = [np.array([0.0, 2.0]), np.array([1.0])]
    o5 = rp.rp_default_options(precision=prec, pair_id=10, kernel=5)
    o2 = rp.rp_default_options(precision=prec, pair_id=10, kernel=2)
    r5 = rp.rp_yields_batch(sys_h, fl, [5, 3], [2.0, 1.5], 77, o5)
    r2 = rp.rp_yields_batch(sys_h, fl, [5, 3], [2.0, 1.5], 77, o2)
    for x in range(2):
        assert np.allclose(r5["out"][x], r2["out"][x], rtol=tol, atol=tol * 1e-2)
    # too large for one CTA: kernel 5 selects as kernel 0
    big = wl.random_isotropic(5, 5, two_I=[1, 1, 2, 1, 1, 2, 1, 2, 1, 1], k_S=1.5, k_T=0.6, seed=49)
    r = rp.System(big).yields([1.0], 2, 3, 0.2, precision=prec, kernel=5)
    assert r["stats"]["kernel_path"] != 5


# systems the cluster macro-step kernel splits over 1, 2, 4 and 8 CTAs
# (isotropic spin-1/2 and spin-1 nuclei; J and k_S != k_T; 1 to 3
# configurations per thread)
CLUSTER = [
    ("c1_kpt1", lambda: wl.random_isotropic(4, 4, two_I=[1, 1, 2, 1, 1, 2, 1, 2], k_S=1.5,
                                            k_T=0.6, J=0.4, seed=49)),              # Z = 864
    ("c1_kpt2", lambda: wl.random_isotropic(5, 4, two_I=[1, 1, 1, 2, 2, 1, 1, 1, 2], k_S=1.0,
                                            k_T=3.0, J=0.2, seed=50)),              # Z = 1728
    ("c2_one_half", lambda: wl.random_isotropic(4, 4, two_I=[1, 2, 2, 2, 2, 2, 2, 2], k_S=0.5,
                                                k_T=2.0, seed=51)),                 # Z = 4374
    ("c4", lambda: wl.random_isotropic(6, 5, two_I=[1, 1, 1, 1, 2, 2, 1, 1, 1, 2, 2], k_S=2.0,
                                       k_T=0.7, J=-0.3, seed=52)),                  # Z = 10368
    ("c8_config2", lambda: wl.config2().system),                                    # Z = 20736
]


@pytest.mark.parametrize("name,mk", CLUSTER, ids=[c[0] for c in CLUSTER])
def test_cluster_macro_step_matches_per_term_and_oracle(name, mk):
    """The cluster macro-step kernel (kernel = 4: a row's Chebyshev vectors in
    the distributed shared memory of 2^c CTAs) gives the per-term kernels'
    per-sample yields at the FP32 tolerance, with the tensor-core and the
    CUDA-core time integrals, and one row agrees with the FP64 oracle."""
    rp = _rp()
    s = mk()
    sy = rp.System(s)
    fields = np.array([0.0, 3.0, 12.0])
    M, T = 3, 0.12
    ref = sy.yields(fields, M, 5, T, per_sample=True, precision="fp32", kernel=1)
    for gram in (2, 1):
        got = sy.yields(fields, M, 5, T, per_sample=True, precision="fp32", kernel=4, gram=gram)
        assert got["stats"]["step_launches"] < ref["stats"]["step_launches"], "cluster path not taken"
        e = _cmp_per_sample(got["per_sample"].reshape(-1, 3), ref["per_sample"][..., 0].ravel(),
                            ref["per_sample"][..., 1].ravel(), ref["per_sample"][..., 2].ravel(),
                            "fp32")
        assert e < 1e-5
    psi0 = coherent.sample_states(s, 5, [2])
    o = chebyshev.propagate_yields(s, fields[2], T, psi0[0])
    g = got["per_sample"][2, 2]
    assert abs(g[0] - o[0]) < TOL["fp32"] * abs(o[0])
    assert abs(g[1] - o[1]) < TOL["fp32"] * max(abs(o[1]), abs(o[0]))
    assert abs(g[2] - o[2]) < TOL["fp32"]


def test_cluster_macro_step_graph_replay_and_refill():
    """Cluster macro-steps replayed from CUDA graphs, with rows refilled
    between macro-steps, equal the eager cluster launches."""
    rp = _rp()
    sy = rp.System(CLUSTER[2][1]())
    fields = [0.0, 2.0, 6.0]
    a = sy.yields(fields, 5, 3, 0.3, per_sample=True, precision="fp32", kernel=4, max_rows=4)
    b = sy.yields(fields, 5, 3, 0.3, per_sample=True, precision="fp32", kernel=4, max_rows=4,
                  graph=1)
    assert np.allclose(a["per_sample"], b["per_sample"], rtol=1e-12, atol=1e-14)
    assert b["stats"]["graph_launches"] > 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_replay_matches_eager(prec):
    """Macro-steps replayed from CUDA graphs (kernels reading the macro-step
    index from the device counter) give the eager launches' results, with row
    refills between replays; uneven systems in one batch too."""
    rp = _rp()
    big = wl.random_isotropic(6, 4, two_I=[1] * 10, seed=44, k_S=1.0, k_T=0.4, J=0.1)  # Z = 1024
    mid = wl.random_isotropic(4, 3, two_I=[1, 1, 1, 2, 1, 1, 2], seed=45, k_S=2.0, k_T=0.5)
    fields = [0.0, 2.0, 6.0]
    for s, kern in ((wl.config1().system, 2), (big, 1), (big, 2), (mid, 1)):
        sy = rp.System(s)
        a = sy.yields(fields, 5, 3, 1.0, per_sample=True, precision=prec, kernel=kern, max_rows=4)
        b = sy.yields(fields, 5, 3, 1.0, per_sample=True, precision=prec, kernel=kern, max_rows=4,
                      graph=1)
        # the state vectors are bitwise equal; only the order of the FP64
        # atomics of the time integral may differ
        assert np.allclose(a["per_sample"], b["per_sample"], rtol=1e-12, atol=1e-14), kern
        assert b["stats"]["graph_launches"] > 0 and a["stats"]["graph_launches"] == 0
        assert b["stats"]["step_launches"] == a["stats"]["step_launches"]
    systems = [wl.config1().system, mid, big]
    sys_h = [rp.System(s) for s in systems]
    fl = [np.array([0.0, 2.0]), np.array([1.0, 5.0]), np.array([3.0])]
    M, T = [4, 3, 2], [1.0, 0.7, 0.5]
    ra = rp.rp_yields_batch(sys_h, fl, M, T, 9, rp.rp_default_options(precision=prec, max_rows=3))
    rb = rp.rp_yields_batch(sys_h, fl, M, T, 9,
                            rp.rp_default_options(precision=prec, max_rows=3, graph=1))
    for s in range(3):
        assert np.allclose(ra["out"][s], rb["out"][s], rtol=1e-12, atol=1e-14), s
    assert rb["stats"]["graph_launches"] > 0


def test_autotuner_choice_and_cache(tmp_path, monkeypatch):
    """rp_tune times its candidates, returns valid settings whose yields agree
    with the oracle at the FP64 tolerance, and reuses its cache file."""
    rp = _rp()
    s = wl.random_isotropic(3, 2, two_I=[1, 2, 1, 1, 1], k_S=1.0, k_T=2.0, seed=46)
    sy = rp.System(s)
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("RP_TUNE_CACHE", str(cache))
    base = rp.rp_default_options(precision="fp64")
    tuned, res = rp.rp_tune(sy.handle, 3.0, 6, base)
    # Z = 48 fits on chip: kernels 1 and 2 with and without graph replay, and
    # the persistent launch (eager only), at four n_cheb each
    assert res["candidates"] == 20 and res["from_cache"] == 0
    assert res["kernel"] in (1, 2, 5) and res["n_cheb"] in (32, 48, 64, 88) and res["graph"] in (0, 1)
    assert res["rate"] > 0 and res["rate"] >= res["base_rate"] > 0
    assert tuned.max_rows == 6 and tuned.precision == rp.RP_FP64
    tuned2, res2 = rp.rp_tune(sy.handle, 3.0, 6, base)
    assert res2["from_cache"] == 1 and res2["candidates"] == 0
    assert (res2["kernel"], res2["n_cheb"], res2["graph"]) == (res["kernel"], res["n_cheb"], res["graph"])
    assert cache.read_text().count("\n") == 1
    got = rp.rp_yields(sy.handle, [3.0], 6, 21, 1.5, tuned, True, Z=sy.Z)
    psi0 = coherent.sample_states(s, 21, range(6))
    phS, phT, surv = dense.sample_yields(s, 3.0, 1.5, psi0)
    _cmp_per_sample(got["per_sample"][0], phS, phT, surv, "fp64")


@pytest.mark.parametrize("aniso", [False, True])
def test_bulk_staged_step_matches_direct_and_oracle(aniso):
    """The FP32 step kernel that stages partner tiles by bulk async copies
    (kernel 3 with >= 8 spin-1/2 nuclei: here one outer spin-1/2, a spin-1 and
    a spin-3/2 nucleus outside the 256-configuration tile) equals the kernel
    that reads partners directly (kernel 1), and the oracle at the FP32
    tolerance."""
    rp = _rp()
    two_I = [1] * 9 + [2, 3]  # Z = 512 * 3 * 4 = 6144
    gen = wl.random_anisotropic if aniso else wl.random_isotropic
    s = gen(6, 5, two_I=two_I, k_S=2.0, k_T=0.5, J=0.2, seed=47)
    sy = rp.System(s)
    fields = [0.0, 4.0]
    a = sy.yields(fields, 3, 8, 0.2, per_sample=True, precision="fp32", kernel=1)
    b = sy.yields(fields, 3, 8, 0.2, per_sample=True, precision="fp32", kernel=3)
    assert np.allclose(a["per_sample"], b["per_sample"], rtol=1e-12, atol=1e-14)
    psi0 = coherent.sample_states(s, 8, [1])
    ref = chebyshev.propagate_yields(s, fields[1], 0.2, psi0[0])
    got = b["per_sample"][1, 1]
    assert abs(got[0] - ref[0]) < TOL["fp32"] * abs(ref[0])
    assert abs(got[1] - ref[1]) < TOL["fp32"] * max(abs(ref[1]), abs(ref[0]))
    assert abs(got[2] - ref[2]) < TOL["fp32"]


@pytest.mark.parametrize("n_cheb", [32, 64, 84, 88])
def test_tensor_core_time_integral_matches_cuda_core(n_cheb):
    """The tcgen05 time integral (3xTF32 split, FP64 contraction; gram=2) equals
    the CUDA-core Gram (gram=1) at FP32 rounding level, for 2 n_cheb below,
    at and above 128 rows, with padded rows (n_cheb = 84) and a Z that is not
    a multiple of the 16-configuration chunk; and the oracle at the FP32
    tolerance."""
    rp = _rp()
    s = wl.random_isotropic(4, 3, two_I=[1, 1, 1, 2, 2, 2, 4], k_S=2.0, k_T=0.5, J=0.1, seed=48)
    sy = rp.System(s)  # Z = 8 * 27 * 5 = 1080
    fields = [0.0, 3.0]
    kw = dict(per_sample=True, precision="fp32", kernel=1, n_cheb=n_cheb, max_rows=5)
    a = sy.yields(fields, 4, 12, 0.5, gram=1, **kw)["per_sample"]
    b = sy.yields(fields, 4, 12, 0.5, gram=2, **kw)["per_sample"]
    # phi_S relative; phi_T = 1 - survival - phi_S on the scale of the yields;
    # survival does not involve the time integral
    scale = np.maximum(np.abs(a[..., 0]), np.abs(a[..., 1]))
    assert np.max(np.abs(a[..., 0] - b[..., 0]) / np.abs(a[..., 0])) < 1e-6
    assert np.max(np.abs(a[..., 1] - b[..., 1]) / scale) < 1e-6
    assert np.array_equal(a[..., 2], b[..., 2])
    psi0 = coherent.sample_states(s, 12, [2])
    ref = chebyshev.propagate_yields(s, fields[1], 0.5, psi0[0])
    got = b[1, 2]
    assert abs(got[0] - ref[0]) < TOL["fp32"] * abs(ref[0])
    assert abs(got[2] - ref[2]) < TOL["fp32"]


def test_tensor_core_time_integral_long_accumulation():
    """Config 2 with few rows, so each CTA of the tensor-core integral covers
    many chunks: the result stays at FP32 rounding level of the CUDA-core Gram
    and of the FP64 path (the tensor core's own accumulation is kept to two
    chunks between drains into FP32 partial sums)."""
    rp = _rp()
    sy = rp.System(wl.config2().system)
    f = [3.0, 20.0]
    kw = dict(per_sample=True, max_rows=2)
    a = sy.yields(f, 2, 0, 0.5, precision="fp32", gram=1, **kw)["per_sample"]
    b = sy.yields(f, 2, 0, 0.5, precision="fp32", gram=2, **kw)["per_sample"]
    c = sy.yields(f, 2, 0, 0.5, precision="fp64", **kw)["per_sample"]
    assert np.max(np.abs(b[..., 0] - a[..., 0]) / np.abs(a[..., 0])) < 1e-6
    assert np.max(np.abs(b[..., 0] - c[..., 0]) / np.abs(c[..., 0])) < 5e-6


def test_tensor_core_time_integral_uneven_batch():
    """rp_yields_batch with systems of different Z (none a multiple of the
    16-configuration chunk) sharing rows that are refilled across systems: the
    tensor-core integral (each row over its own Z, zero padding kept by the
    step kernel) equals the CUDA-core Gram at FP32 rounding level."""
    rp = _rp()
    systems = [wl.random_isotropic(4, 3, two_I=[1, 1, 1, 2, 2, 2, 4], seed=50, k_S=2.0, k_T=0.5),
               wl.random_isotropic(5, 4, two_I=[1] * 7 + [2, 2], seed=51, k_S=1.0, k_T=1.0),
               wl.random_anisotropic(4, 4, two_I=[1, 1, 1, 1, 2, 2, 2, 2], seed=52, k_S=0.5,
                                     k_T=3.0, J=0.2)]
    assert sorted(s.Z for s in systems) == [1080, 1152, 1296]
    sys_h = [rp.System(s) for s in systems]
    fl = [np.array([0.0, 4.0]), np.array([1.0, 6.0]), np.array([2.0])]
    M, T = [3, 3, 4], [0.4, 0.3, 0.5]
    kw = dict(precision="fp32", kernel=1, max_rows=3)
    a = rp.rp_yields_batch(sys_h, fl, M, T, 5, rp.rp_default_options(gram=1, **kw))
    b = rp.rp_yields_batch(sys_h, fl, M, T, 5, rp.rp_default_options(gram=2, **kw))
    for s in range(3):
        A, B = a["out"][s], b["out"][s]
        assert np.max(np.abs(A[:, 0] - B[:, 0]) / np.abs(A[:, 0])) < 1e-6, s
        assert np.max(np.abs(A[:, 1] - B[:, 1]) / np.maximum(np.abs(A[:, 1]), np.abs(A[:, 0]))) < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_time_trace_closed_form_one_nucleus(prec):
    """P_S(t), P_T(t), survival at the macro-step boundaries for one spin-1/2
    (a = 1 mT, k_S = k_T = 1, B = 0): the trace over the Z = 2 basis states
    equals e^{-kt} (5/8 + 3/8 cos(a t)) and the survival e^{-kt}."""
    rp = _rp()
    s = wl.one_nucleus(1.0, k=1.0)
    sy = rp.System(s)
    t, out = rp.rp_time_trace(sy.handle, 0.0, 2, 0, 2.0,
                              rp.rp_default_options(precision=prec, deterministic=1))
    a = 176.085963023
    ps = np.exp(-t) * (5 / 8 + 3 / 8 * np.cos(a * t))
    tol = TOL[prec]
    assert abs(t[-1] - 2.0) < 1e-12 and t.size > 3
    assert np.max(np.abs(out[:, 0] - ps)) < tol
    assert np.max(np.abs(out[:, 2] - np.exp(-t))) < tol
    assert np.max(np.abs(out[:, 1] - (np.exp(-t) - ps))) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_time_trace_matches_dense_oracle(prec):
    """Sample means of P_S(t) and survival on the config-1 system (k_S != k_T
    variant) at B = 2 mT against direct matrix exponentials of the oracle."""
    rp = _rp()
    s = wl.random_isotropic(3, 1, two_I=[1, 2, 1, 1], k_S=2.0, k_T=0.5, J=0.2, seed=53)
    sy = rp.System(s)
    M, B, T = 5, 2.0, 1.0
    t, out = rp.rp_time_trace(sy.handle, B, M, 7, T, rp.rp_default_options(precision=prec))
    psi0 = coherent.sample_states(s, 7, range(M))
    ps = np.mean([dense.singlet_probability(s, B, p, t) for p in psi0], axis=0)
    A = spin.generator(s, B)
    import scipy.linalg
    surv = np.array([np.mean([np.linalg.norm(scipy.linalg.expm(A * ti) @ p) ** 2 for p in psi0])
                     for ti in t])
    tol = TOL[prec]
    assert np.max(np.abs(out[:, 0] - ps)) < tol
    assert np.max(np.abs(out[:, 2] - surv)) < tol
    assert np.max(np.abs(out[:, 1] - (surv - ps))) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_basis_state_sampling_matches_oracle(prec):
    """deterministic = 2: M basis states |S, M> drawn at random; per-sample
    yields equal the oracle's for the same drawn indices, and the draw is the
    library's own rp_basis_indices."""
    from oracle import philox
    rp = _rp()
    s = wl.random_isotropic(3, 1, two_I=[1, 2, 1, 1], k_S=2.0, k_T=0.5, J=0.2, seed=54)
    sy = rp.System(s)
    M, B, T = 6, 1.5, 1.0
    r = sy.yields([B], M, 21, T, per_sample=True, precision=prec, deterministic=2, pair_id=4,
                  sample_offset=10)
    idx = philox.draw_basis_indices(21, 4, np.arange(10, 10 + M), s.Z)
    assert np.array_equal(idx, rp.rp_basis_indices(21, 4, 10, M, s.Z))
    # |S> x |m> in the library layout (configuration m, electron index e = 2 e1 + e2
    # innermost: <S| = (<ab| - <ba|)/sqrt 2), then in the oracle's kron order
    lib = np.zeros((M, 4 * s.Z), complex)
    for k, m in enumerate(idx):
        lib[k, 4 * m + 1], lib[k, 4 * m + 2] = 2 ** -0.5, -(2 ** -0.5)
    psi0 = sy.to_input_order(lib)
    assert np.allclose(np.abs(psi0 @ coherent.basis_states(s).conj().T).max(axis=1), 1.0)
    phS, phT, surv = dense.sample_yields(s, B, T, psi0)
    _cmp_per_sample(r["per_sample"][0], phS, phT, surv, prec)


# ------------------------------------------------ field direction (rp_rotate)

def _rot_to_z(theta, phi):
    """R_y(-theta) R_z(-phi), the rotation taking n(theta, phi) to z."""
    ct, st, cp, sp = math.cos(theta), math.sin(theta), math.cos(phi), math.sin(phi)
    Rz = np.array([[cp, sp, 0.0], [-sp, cp, 0.0], [0.0, 0.0, 1.0]])
    Ry = np.array([[ct, 0.0, -st], [0.0, 1.0, 0.0], [st, 0.0, ct]])
    return Ry @ Rz


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_field_direction_matches_oracle(prec):
    """A field along n(theta, phi) for an anisotropic pair (rp_rotate): the
    deterministic trace equals the oracle's with the Zeeman term omega n.S
    (Eq. 1), and each coherent-state sample equals the oracle's lab-frame
    sample whose directions are R^T n_k."""
    rp = _rp()
    s = wl.random_anisotropic(2, 1, two_I=[1, 2, 1], k_S=2.0, k_T=0.5, J=0.3, seed=40)
    sy = rp.System(s)
    th, ph = 0.7, 1.9
    n = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    sr = rp.System.rotated(sy, th, ph)
    fields = np.array([0.5, 2.0])
    T = 2.0
    tr = sr.yields(fields, 2, 0, T, precision=prec, deterministic=1)
    for i, B in enumerate(fields):
        ref = dense.trace_yields(s, B, T, direction=n)
        assert abs(tr["out"][i, 0] - ref[0]) < TOL[prec] * abs(ref[0])
    r = sr.yields(fields, 5, 9, T, per_sample=True, precision=prec)
    th_k, ph_k = philox.draw_angles(9, 0, np.arange(5), s.n_nuc)
    R = _rot_to_z(th, ph)
    psi0 = []
    for i in range(5):
        nk = np.stack([np.sin(th_k[i]) * np.cos(ph_k[i]), np.sin(th_k[i]) * np.sin(ph_k[i]),
                       np.cos(th_k[i])], -1) @ R  # rows: R^T n_k
        lt = np.arccos(np.clip(nk[:, 2], -1, 1))
        lp = np.arctan2(nk[:, 1], nk[:, 0])
        psi0.append(coherent.sample_state(s, lt, lp))
    for i, B in enumerate(fields):
        phS, phT, surv = dense.sample_yields(s, B, T, np.array(psi0), direction=n)
        _cmp_per_sample(r["per_sample"][i], phS, phT, surv, prec)


# ------------------------------------------ time-resolved electron observables

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_time_observable_matches_oracle(prec):
    """rp_time_observable: <psi(t)| A_e x 1 |psi(t)> averaged over samples at
    the macro-step boundaries (Eq. 18 with a general electron operator)
    against the oracle's dense propagation, for S_1z, S_1x S_2y + h.c. and the
    triplet projector T_0; A_e = P_S reproduces rp_time_trace."""
    rp = _rp()
    s = wl.random_isotropic(2, 1, two_I=[1, 2, 1], k_S=2.0, k_T=0.5, J=0.3, seed=45)
    sy = rp.System(s)
    B, M, T = 1.7, 4, 0.6
    sx = np.array([[0, 0.5], [0.5, 0]], complex)
    sy_ = np.array([[0, -0.5j], [0.5j, 0]])
    sz = np.diag([0.5, -0.5]).astype(complex)
    e2 = np.eye(2)
    t0 = np.zeros((4, 4), complex)
    v = np.array([0, 1, 1, 0]) / math.sqrt(2)
    t0 = np.outer(v, v).astype(complex)
    singlet = np.array([0, 1, -1, 0]) / math.sqrt(2)
    ops_e = {"S1z": np.kron(sz, e2), "mix": np.kron(sx, sy_) + np.kron(sy_, sx).conj().T,
             "T0": t0, "PS": np.outer(singlet, singlet).astype(complex)}
    o = rp.rp_default_options(precision=prec)
    psi0 = coherent.sample_states(s, 6, range(M))
    Z = s.Z
    tol = 1e-10 if prec == "fp64" else 1e-5
    for name, Ae in ops_e.items():
        t, val = rp.rp_time_observable(sy.handle, B, M, 6, T, Ae, o)
        ref = dense.expectation_traces(s, B, psi0, t, [np.kron(Ae, np.eye(Z))])[:, 0]
        assert np.max(np.abs(val - ref)) < tol, (name, np.max(np.abs(val - ref)))
    t2, tr = rp.rp_time_trace(sy.handle, B, M, 6, T, o)
    _, ps = rp.rp_time_observable(sy.handle, B, M, 6, T, ops_e["PS"], o)
    assert np.allclose(t2, t) and np.max(np.abs(ps.real - tr[:, 0])) < 1e-12
