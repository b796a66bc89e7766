"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here touches the CUDA path.  Every check compares the oracle with
something other than itself: closed forms, invariants, symmetry, quadrature
identities, brute force, values printed in the paper, or its other
independent path (dense Van Loan vs matrix-free Chebyshev).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.special

from oracle import chebyshev, coherent, dense, philox, spin
from paper_1612_09517_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
G = spin.GAMMA_E


# ----------------------------------------------------------------- spin algebra

@pytest.mark.parametrize("two_I", [1, 2, 3, 4, 5])
def test_spin_algebra(two_I):
    """[I_x, I_y] = i I_z (cyclic) and I^2 = I(I+1)."""
    Ix, Iy, Iz = spin.spin_matrices(two_I)
    I = two_I / 2
    assert np.allclose(Ix @ Iy - Iy @ Ix, 1j * Iz, atol=1e-14)
    assert np.allclose(Iy @ Iz - Iz @ Iy, 1j * Ix, atol=1e-14)
    assert np.allclose(Iz @ Ix - Ix @ Iz, 1j * Iy, atol=1e-14)
    assert np.allclose(Ix @ Ix + Iy @ Iy + Iz @ Iz, I * (I + 1) * np.eye(two_I + 1), atol=1e-13)
    assert np.allclose(np.diag(Iz).real, I - np.arange(two_I + 1))


def test_projectors():
    """Eqs. 3-4: P_S, P_T are complementary projectors; |S> spans P_S per nuclear state."""
    s = wl.random_isotropic(1, 1, two_I=[1, 2], seed=3)
    PS, PT = spin.projectors(s)
    assert np.allclose(PS @ PS, PS, atol=1e-14)
    assert np.allclose(PS + PT, np.eye(s.dim), atol=1e-14)
    assert abs(np.trace(PS).real - s.Z) < 1e-12
    v = np.kron(spin.singlet_vector(), np.ones(s.Z) / math.sqrt(s.Z))
    assert np.allclose(PS @ v, v, atol=1e-14)


def test_exchange_sign_singlet_energy():
    """Eq. 1 uses +2J S1.S2: the singlet lies at -3J/2, the triplets at +J/2,
    so the S-T_- crossing sits at omega = 2J (Sec. V, Fig. 3 discussion)."""
    s = spin.spin_matrices(1)
    dot = sum(np.kron(s[a], np.eye(2)) @ np.kron(np.eye(2), s[a]) for a in range(3))
    J = 0.7
    He = 2 * J * dot
    S = spin.singlet_vector()
    assert np.allclose(He @ S, -1.5 * J * S)
    omega = 2 * J
    Hz = He + omega * (np.kron(s[2], np.eye(2)) + np.kron(np.eye(2), s[2]))
    ev = np.sort(np.linalg.eigvalsh(Hz))
    assert np.isclose(ev[0], -1.5 * J) and np.isclose(ev[1], -1.5 * J)  # S and T_- degenerate


# ------------------------------------------------------------ coherent states

@pytest.mark.parametrize("two_I", [1, 2, 3, 4])
def test_coherent_state_components(two_I):
    """Eq. 15 expanded: c_n = sqrt(C(2J,n)) cos^{2J-n}(t/2) sin^n(t/2) e^{i n phi}."""
    rng = np.random.default_rng(two_I)
    for _ in range(5):
        th, ph = rng.uniform(0, np.pi), rng.uniform(0, 2 * np.pi)
        v = coherent.coherent_state(two_I, th, ph)
        n = np.arange(two_I + 1)
        ref = (np.sqrt(scipy.special.comb(two_I, n)) * np.cos(th / 2) ** (two_I - n)
               * np.sin(th / 2) ** n * np.exp(1j * n * ph))
        assert np.allclose(v, ref, atol=1e-14)
        assert abs(np.vdot(v, v).real - 1) < 1e-14


@pytest.mark.parametrize("two_I", [1, 2, 3, 5])
def test_coherent_expectation_eq16(two_I):
    """Eq. 16: <Omega|J|Omega> = J n(Omega)."""
    rng = np.random.default_rng(10 + two_I)
    Ix, Iy, Iz = spin.spin_matrices(two_I)
    J = two_I / 2
    for _ in range(5):
        th, ph = rng.uniform(0, np.pi), rng.uniform(0, 2 * np.pi)
        v = coherent.coherent_state(two_I, th, ph)
        n = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
        got = np.array([np.vdot(v, O @ v).real for O in (Ix, Iy, Iz)])
        assert np.allclose(got, J * n, atol=1e-13)


def _sphere_quadrature(n_theta, n_phi):
    x, w = np.polynomial.legendre.leggauss(n_theta)  # x = cos(theta)
    phis = 2 * np.pi * np.arange(n_phi) / n_phi
    th = np.arccos(x)
    T, P = np.meshgrid(th, phis, indexing="ij")
    W = np.outer(w, np.full(n_phi, 2 * np.pi / n_phi))
    return T.ravel(), P.ravel(), W.ravel()  # weights sum to 4 pi


@pytest.mark.parametrize("two_I", [1, 2, 3])
def test_completeness_eq17(two_I):
    """Eq. 17: (2J+1)/(4 pi) int dOmega |Omega><Omega| = 1, by exact quadrature."""
    T, P, W = _sphere_quadrature(two_I + 2, 2 * two_I + 3)
    acc = np.zeros((two_I + 1, two_I + 1), complex)
    for t, p, w in zip(T, P, W):
        v = coherent.coherent_state(two_I, t, p)
        acc += w * np.outer(v, v.conj())
    assert np.allclose((two_I + 1) / (4 * np.pi) * acc, np.eye(two_I + 1), atol=1e-13)


# ------------------------------------------------------------------- Philox

def test_philox_weyl_constants():
    """The key schedule constants are floor(2^32 (golden ratio - 1)) and floor(2^32 (sqrt3 - 1))."""
    from decimal import Decimal, getcontext
    getcontext().prec = 50
    golden = (Decimal(5).sqrt() - 1) / 2
    assert philox.PHILOX_W0 == int(golden * (1 << 32))
    assert philox.PHILOX_W1 == int((Decimal(3).sqrt() - 1) * (1 << 32))


def test_philox_known_answer_vectors():
    """Known-answer vectors of Philox4x32-10 published with the Random123
    library of Salmon et al. (SC'11): (counter, key) -> four output words.
    A wrong multiplier, a wrong Weyl constant, a missing round or swapped
    output words each change all of them."""
    kat = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in kat:
        got = philox.philox4x32_10(np.array(ctr, dtype=np.uint64), np.array(key, dtype=np.uint64))
        assert [int(x) for x in got] == list(want), (ctr, key, [hex(int(x)) for x in got])
    # vectorised form gives the same words
    c = np.array([k[0] for k in kat], dtype=np.uint64)
    k = np.array([k[1] for k in kat], dtype=np.uint64)
    assert np.array_equal(philox.philox4x32_10(c, k), np.array([k_[2] for k_ in kat], dtype=np.uint64))


def test_philox_round_is_bijective_on_sample():
    """Distinct counters give distinct outputs (Philox is a keyed bijection)."""
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(20000, 4), dtype=np.uint64)
    ctr[:, 3] = np.arange(20000)  # make counters distinct
    out = philox.philox4x32_10(ctr, np.array([[123, 456]], dtype=np.uint64))
    assert len({tuple(r) for r in out.tolist()}) == 20000


def test_philox_uniformity_and_sphere_moments():
    """u in [0,1) is uniform (chi^2) and directions have <n> = 0, <n n^T> = 1/3."""
    u1, u2 = philox.draw_uniforms(7, 0, np.arange(20000), 5)
    u = np.concatenate([u1.ravel(), u2.ravel()])
    assert u.min() >= 0 and u.max() < 1
    hist, _ = np.histogram(u, bins=50, range=(0, 1))
    exp = u.size / 50
    chi2 = np.sum((hist - exp) ** 2 / exp)
    assert chi2 < 49 + 6 * math.sqrt(2 * 49)
    th, ph = philox.draw_angles(7, 0, np.arange(20000), 5)
    n = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1).reshape(-1, 3)
    N = n.shape[0]
    assert np.all(np.abs(n.mean(0)) < 5 / math.sqrt(3 * N))
    assert np.allclose(n.T @ n / N, np.eye(3) / 3, atol=5 * math.sqrt(0.1 / N))
    # different nuclei / samples / seeds / pairs decorrelated
    a, _ = philox.draw_uniforms(7, 1, np.arange(20000), 1)
    assert abs(np.corrcoef(u1[:, 0], a[:, 0])[0, 1]) < 0.04
    assert abs(np.corrcoef(u1[:, 0], u1[:, 1])[0, 1]) < 0.04


# ------------------------------------------------------------- closed forms

def _phi_closed(a, k, T, weight_const, weight_cos, freq):
    b = freq
    return (weight_const * (1 - math.exp(-k * T))
            + weight_cos * k * (k - math.exp(-k * T) * (k * math.cos(b * T) - b * math.sin(b * T))) / (k * k + b * b))


@pytest.mark.parametrize("a_mT,k,T", [(1.0, 1.0, 10.0), (0.37, 2.5, 3.0), (-0.8, 0.3, 7.0)])
def test_closed_form_one_spin_half(a_mT, k, T):
    """One I=1/2 nucleus, B=0, J=0, k_S=k_T=k: P_S(t) = e^{-kt}(5/8 + 3/8 cos at)."""
    s = wl.one_nucleus(a_mT, 1, k)
    a = G * a_mT
    PhiS, PhiT, surv = dense.trace_yields(s, 0.0, T)
    ref = _phi_closed(a, k, T, 5 / 8, 3 / 8, a)
    assert abs(PhiS - ref) < 1e-12
    assert abs(surv - math.exp(-k * T)) < 1e-12
    psi0 = coherent.sample_states(s, 0, range(3))
    ts = np.array([0.0, 0.013, 0.5, 2.0])
    for i in range(3):
        ps = dense.singlet_probability(s, 0.0, psi0[i], ts)
        assert np.allclose(ps, np.exp(-k * ts) * (5 / 8 + 3 / 8 * np.cos(a * ts)), atol=1e-12)


def test_closed_form_config1_side_case_value():
    """a = 1 mT, k = 1 us^-1, T = 10 us: Phi_S(T) = 0.6249838157 (closed form)."""
    PhiS, _, _ = dense.trace_yields(wl.one_nucleus(1.0, 1, 1.0), 0.0, 10.0)
    assert abs(PhiS - 0.6249838157) < 1e-10


def test_closed_form_one_spin_one():
    """One I=1 nucleus, B=0: P_S(t) = 5/9 + 4/9 cos(3at/2)."""
    a_mT, k, T = 0.6, 0.8, 6.0
    s = wl.one_nucleus(a_mT, 2, k)
    a = G * a_mT
    PhiS, _, _ = dense.trace_yields(s, 0.0, T)
    assert abs(PhiS - _phi_closed(a, k, T, 5 / 9, 4 / 9, 1.5 * a)) < 1e-12
    psi0 = coherent.sample_states(s, 1, range(2))
    ts = np.array([0.0, 0.01, 0.3])
    ps = dense.singlet_probability(s, 0.0, psi0[0], ts)
    assert np.allclose(ps, np.exp(-k * ts) * (5 / 9 + 4 / 9 * np.cos(1.5 * a * ts)), atol=1e-12)


@pytest.mark.parametrize("B,J,kS,kT", [(0.0, 0.0, 1.0, 1.0), (3.0, 0.4, 2.0, 0.5), (-7.0, -1.0, 0.3, 4.0)])
def test_no_nuclei(B, J, kS, kT):
    """No nuclei: |S> is an eigenstate, P_S(t) = e^{-k_S t}, Phi_S(T) = 1 - e^{-k_S T}."""
    s = wl.SpinSystem([], [], np.zeros((0, 3, 3)), kS, kT, J)
    T = 1.7
    PhiS, PhiT, surv = dense.trace_yields(s, B, T)
    # FP64 rounding after ~log2(|A| T) doublings of the exponential: 1e-12
    assert abs(PhiS - (1 - math.exp(-kS * T))) < 1e-12
    assert abs(PhiT) < 1e-12 and abs(surv - math.exp(-kS * T)) < 1e-12


# --------------------------------------------------------------- invariants

def test_norm_decay_and_conservation():
    """k_S = k_T: |psi(T)|^2 = e^{-kT}.  Always: Phi_S + Phi_T + survival = 1."""
    s = wl.random_isotropic(2, 1, two_I=[1, 2, 1], k_S=1.3, k_T=1.3, J=0.2, seed=5)
    psi0 = coherent.sample_states(s, 3, range(4))
    phS, phT, surv = dense.sample_yields(s, 1.5, 2.5, psi0)
    assert np.allclose(surv, math.exp(-1.3 * 2.5), atol=1e-12)
    assert np.allclose(phS + phT + surv, 1.0, atol=1e-12)
    s2 = wl.random_anisotropic(1, 2, two_I=[1, 1, 2], k_S=2.0, k_T=0.4, J=0.3, seed=6)
    psi0 = coherent.sample_states(s2, 3, range(4))
    phS, phT, surv = dense.sample_yields(s2, 0.8, 3.0, psi0)
    assert np.allclose(phS + phT + surv, 1.0, atol=1e-12)
    assert np.all((phS >= 0) & (phS <= 1)) and np.all(surv <= 1)


def test_field_reversal_symmetry_anisotropic():
    """Phi_S(B) = Phi_S(-B), also with anisotropic tensors and J."""
    s = wl.random_anisotropic(2, 1, k_S=1.0, k_T=0.5, J=0.25, seed=8)
    for B in (0.4, 2.0):
        a = dense.trace_yields(s, B, 3.0)
        b = dense.trace_yields(s, -B, 3.0)
        assert np.allclose(a, b, atol=1e-12)


def test_zero_field_rotational_invariance_anisotropic():
    """At B = 0 the trace is invariant under rotating every tensor A -> R A R^T;
    a rotation about z leaves it invariant at any field along z."""
    rng = np.random.default_rng(2)
    A0 = np.stack([np.diag([0.3, -0.7, 1.1]), np.diag([0.9, 0.2, -0.4])])
    base = wl.SpinSystem([0, 1], [1, 2], A0, 1.0, 0.6, 0.2)
    R = wl.haar_rotation(rng)
    rot = wl.SpinSystem([0, 1], [1, 2], np.einsum("ij,kjl,ml->kim", R, A0, R), 1.0, 0.6, 0.2)
    assert np.allclose(dense.trace_yields(base, 0.0, 2.0), dense.trace_yields(rot, 0.0, 2.0), atol=1e-12)
    c, sn = math.cos(0.9), math.sin(0.9)
    Rz = np.array([[c, -sn, 0], [sn, c, 0], [0, 0, 1]])
    rotz = wl.SpinSystem([0, 1], [1, 2], np.einsum("ij,kjl,ml->kim", Rz, A0, Rz), 1.0, 0.6, 0.2)
    assert np.allclose(dense.trace_yields(base, 1.3, 2.0), dense.trace_yields(rotz, 1.3, 2.0), atol=1e-12)
    # ... but a generic rotation changes it once the field picks a direction
    assert abs(dense.trace_yields(base, 1.3, 2.0)[0] - dense.trace_yields(rot, 1.3, 2.0)[0]) > 1e-6


def test_total_Jz_conserved_isotropic():
    """Isotropic H commutes with J_z (Sec. V): <J_z>(t) = e^{-kt} <J_z>(0) for k_S = k_T."""
    s = wl.random_isotropic(2, 1, two_I=[1, 2, 1], k_S=0.7, k_T=0.7, J=0.3, seed=9)
    dims = spin.dims_of(s)
    Jz = np.zeros((s.dim, s.dim), complex)
    for p, d in enumerate(dims):
        ops = spin.spin_matrices(d - 1)
        term = np.ones((1, 1))
        for q, dq in enumerate(dims):
            term = np.kron(term, ops[2] if q == p else np.eye(dq))
        Jz += term
    psi0 = coherent.sample_states(s, 2, [0])[0]
    T = 1.1
    psiT = scipy.linalg.expm(spin.generator(s, 2.0) * T) @ psi0
    assert abs(np.vdot(psiT, Jz @ psiT).real - math.exp(-0.7 * T) * np.vdot(psi0, Jz @ psi0).real) < 1e-12


# ------------------------------------------------------------- unbiasedness

def test_unbiased_exact_by_quadrature():
    """Eq. 17 -> Eq. 18: the sphere average of phi_S(Omega) equals the trace (Eq. 14)
    exactly; the integrand is a low-degree trigonometric polynomial, so a product
    Gauss quadrature over both nuclear spheres is exact."""
    s = wl.random_anisotropic(1, 1, two_I=[1, 2], k_S=1.5, k_T=0.5, J=0.2, seed=12)
    YS, YT, F = dense.yield_operators(s, 0.9, 2.0)
    quads = [_sphere_quadrature(int(t) + 2, 2 * int(t) + 3) for t in s.two_I]
    states = [[coherent.coherent_state(int(s.two_I[k]), t, p) for t, p in zip(*quads[k][:2])]
              for k in range(2)]
    acc = 0.0
    for i, w1 in enumerate(quads[0][2]):
        for j, w2 in enumerate(quads[1][2]):
            psi = np.kron(spin.singlet_vector(), np.kron(states[0][i], states[1][j]))
            acc += w1 * w2 * np.vdot(psi, YS @ psi).real
    acc /= (4 * np.pi) ** 2
    PhiS, _, _ = dense.trace_yields(s, 0.9, 2.0)
    assert abs(acc - PhiS) < 1e-12


def test_unbiased_statistical():
    """Monte Carlo estimates over several seeds agree with the trace within their SE."""
    s = wl.random_isotropic(3, 1, seed=21, k_S=1.0, k_T=1.0)
    YS, YT, F = dense.yield_operators(s, 0.5, 5.0)
    PS, _ = spin.projectors(s)
    trace = np.trace(YS @ PS).real / s.Z
    zs = []
    for seed in range(6):
        psi = coherent.sample_states(s, seed, range(300))
        phi = np.einsum("si,ij,sj->s", psi.conj(), YS, psi).real
        m, se = dense.estimate(phi)
        zs.append((m - trace) / se)
        assert phi.std(ddof=1) <= 0.5  # Sec. V: sigma <= 1/2
    zs = np.array(zs)
    assert np.all(np.abs(zs) < 4.0)
    assert np.sum(zs ** 2) < 6 + 5 * math.sqrt(12)


def test_trace_equals_basis_state_average():
    """Eq. 14: the trace is the mean of the Z single-wavepacket yields from |S, M>."""
    s = wl.random_isotropic(2, 1, two_I=[1, 2, 1], k_S=1.0, k_T=3.0, J=0.1, seed=4)
    basis = coherent.basis_states(s)
    phS, phT, surv = dense.sample_yields(s, 1.0, 2.0, basis)
    tr = dense.trace_yields(s, 1.0, 2.0)
    assert np.allclose([phS.mean(), phT.mean(), surv.mean()], tr, atol=1e-13)


# ------------------------------------------------------------- brute force

def test_yield_by_brute_force_time_quadrature():
    """Van Loan yield == k_S times a composite Gauss-Legendre quadrature of P_S(t)."""
    s = wl.random_isotropic(2, 0, seed=30, k_S=2.0, k_T=0.5, J=0.2)
    psi0 = coherent.sample_states(s, 0, [0])[0]
    B, T = 0.7, 1.0
    A = spin.generator(s, B)
    PS, _ = spin.projectors(s)
    x, w = np.polynomial.legendre.leggauss(20)
    n_pan = 40
    edges = np.linspace(0, T, n_pan + 1)
    acc = 0.0
    Fstep = scipy.linalg.expm(A * (T / n_pan))
    psi_start = psi0.copy()
    for p in range(n_pan):
        for xi, wi in zip(x, w):
            tau = 0.5 * (edges[1] - edges[0]) * (xi + 1)
            psi = scipy.linalg.expm(A * tau) @ psi_start
            acc += 0.5 * (edges[1] - edges[0]) * wi * np.vdot(psi, PS @ psi).real
        psi_start = Fstep @ psi_start
    phS, _, _ = dense.sample_yields(s, B, T, psi0)
    assert abs(s.k_S * acc - phS[0]) < 1e-11


# ----------------------------------------------- matrix-free path vs dense

SYSTEMS = [
    ("config1", lambda: wl.config1().system, 2.5, 10.0),
    ("aniso_spin1", lambda: wl.random_anisotropic(2, 1, two_I=[1, 2, 1], k_S=2.0, k_T=0.5, J=0.3, seed=40), 3.0, 2.0),
    ("spin3half", lambda: wl.random_isotropic(1, 1, two_I=[3, 1], k_S=0.2, k_T=5.0, J=-0.5, seed=41), 1.0, 1.5),
]


@pytest.mark.parametrize("name,mk,B,T", SYSTEMS, ids=[x[0] for x in SYSTEMS])
def test_chebyshev_matches_dense(name, mk, B, T):
    s = mk()
    psi0 = coherent.sample_states(s, 11, range(2))
    ref = dense.sample_yields(s, B, T, psi0)
    for i in range(2):
        got = chebyshev.propagate_yields(s, B, T, psi0[i])
        for g, r in zip(got, (ref[0][i], ref[1][i], ref[2][i])):
            assert abs(g - r) <= 1e-11 * max(abs(r), 1e-3)


def test_chebyshev_weights_converged():
    dE, Ec, h, n_c = 900.0, 37.0, 0.04, 48
    W1 = chebyshev.weights(dE, Ec, h, n_c)
    W2 = chebyshev.weights(dE, Ec, h, n_c, n_nodes=2 * n_c + int(dE * h) + 120)
    assert np.max(np.abs(W1 - W2)) < 1e-15 * h * 10


# ----------------------------------------------------------- paper values

def _read_golden():
    rows, vals = [], {}
    with open(os.path.join(GOLDEN, "table1_hyperfine.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            parts = line.split()
            if parts[0].isdigit():
                rows.append([float(x) for x in parts[1:]])
            else:
                vals[parts[0]] = float(parts[1])
    return np.array(rows), vals


def test_table1_effective_hyperfine_fields():
    """Eq. 21 on Table I reproduces B_hyp,1 = 1.72 mT and B_hyp,2 = 1.74 mT (Sec. IV)."""
    rows, vals = _read_golden()
    b1 = spin.effective_hyperfine_field(rows[:, 0], [1] * 10)
    b2 = spin.effective_hyperfine_field(rows[:, 1], [1] * 10)
    assert round(b1, 2) == vals["B_hyp_1"] and round(b2, 2) == vals["B_hyp_2"]
    # the workload module carries the same table
    assert np.allclose(rows[:, 0], wl.TABLE1_A1) and np.allclose(rows[:, 1], wl.TABLE1_A2)


def test_resonance_minimum_at_omega_2J():
    """Sec. V: with weak hyperfine coupling the singlet yield dips where omega = 2J."""
    s = wl.random_isotropic(2, 1, a_scale=0.15, seed=50, k_S=1.0, k_T=1.0, J=1.0)
    Bs = np.linspace(0.0, 4.0, 41)
    phi = np.array([dense.trace_yields(s, B, 3.0)[0] for B in Bs])
    assert abs(Bs[np.argmin(phi)] - 2.0) <= 0.2


def test_basis_index_draw_is_uniform_and_disjoint_from_angles():
    """Basis-state sampling draws: every index in range, uniform over Z bins
    (chi-square at the 1e-4 level), and a different stream from the angles
    (counter word 0 is 0xFFFFFFFF, never a nucleus index)."""
    from oracle import philox
    Z = 48
    idx = philox.draw_basis_indices(5, 3, np.arange(96000), Z)
    assert idx.min() >= 0 and idx.max() <= Z - 1
    counts = np.bincount(idx, minlength=Z)
    exp = idx.size / Z
    chi2 = float(np.sum((counts - exp) ** 2 / exp))
    assert chi2 < 100.0  # 47 dof: P(chi2 > 100) < 1e-5
    u1, _ = philox.draw_uniforms(5, 3, np.arange(8), 1)
    assert not np.array_equal(np.floor(u1[:, 0] * Z).astype(np.int64), idx[:8])


# ------------------------------------------- field direction, general observables

def _rot_to_z(theta, phi):
    """R_y(-theta) R_z(-phi): the rotation taking n(theta, phi) to z."""
    ct, st, cp, sp = math.cos(theta), math.sin(theta), math.cos(phi), math.sin(phi)
    Rz = np.array([[cp, sp, 0.0], [-sp, cp, 0.0], [0.0, 0.0, 1.0]])
    Ry = np.array([[ct, 0.0, -st], [0.0, 1.0, 0.0], [st, 0.0, ct]])
    return Ry @ Rz


def test_field_direction_hamiltonian():
    """Eq. 1 with omega = |gamma_e| B n: n = z gives the z Hamiltonian exactly;
    an isotropic system's trace does not depend on the direction (a global
    rotation of every spin leaves P_S / Z invariant); an anisotropic system
    with the field along n has the trace of the system with tensors R A R^T
    and the field along z (R n = z)."""
    s = wl.random_anisotropic(2, 1, two_I=[1, 2, 1], k_S=2.0, k_T=0.5, J=0.3, seed=40)
    assert np.array_equal(spin.hamiltonian(s, 1.3), spin.hamiltonian(s, 1.3, [0, 0, 1]))
    th, ph = 0.7, 1.9
    n = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    R = _rot_to_z(th, ph)
    assert np.allclose(R @ n, [0, 0, 1], atol=1e-15)
    iso = wl.random_isotropic(2, 1, two_I=[1, 2, 1], k_S=2.0, k_T=0.5, J=0.3, seed=40)
    a = dense.trace_yields(iso, 1.5, 2.0)
    b = dense.trace_yields(iso, 1.5, 2.0, direction=n)
    assert np.allclose(a, b, rtol=1e-11, atol=1e-13)
    rot = wl.SpinSystem(s.radical, s.two_I, np.einsum("ij,kjl,ml->kim", R, s.A, R), s.k_S, s.k_T,
                        s.J)
    a = dense.trace_yields(s, 1.5, 2.0, direction=n)
    b = dense.trace_yields(rot, 1.5, 2.0)
    assert np.allclose(a, b, rtol=1e-11, atol=1e-13)
    # and the direction matters for the anisotropic system
    assert abs(a[0] - dense.trace_yields(s, 1.5, 2.0)[0]) > 1e-4


def test_expectation_traces_closed_forms():
    """<P_S>(t) = e^{-kt}(5/8 + 3/8 cos at) and <1>(t) = e^{-kt} for one
    spin-1/2 nucleus at zero field with k_S = k_T = k; <S_1z>(t) = 0 at zero
    field (the singlet and the isotropic coupling are rotation invariant)."""
    a_mT, k = 1.0, 1.0
    s = wl.one_nucleus(a_mT, 1, k)
    a = spin.GAMMA_E * a_mT
    PS, _ = spin.projectors(s)
    S1, _ = spin.electron_ops(s)
    psi0 = coherent.sample_states(s, 3, range(6))
    times = np.array([0.0, 0.013, 0.2, 1.1])
    out = dense.expectation_traces(s, 0.0, psi0, times, [PS, np.eye(PS.shape[0]), S1[2]])
    for i, t in enumerate(times):
        assert abs(out[i, 0] - math.exp(-k * t) * (5 / 8 + 3 / 8 * math.cos(a * t))) < 1e-10
        assert abs(out[i, 1] - math.exp(-k * t)) < 1e-12
    assert np.max(np.abs(out[:, 0].imag)) < 1e-14
    # a single sample has <S_1z> != 0 in general; the mean over the sphere is 0
    full = coherent.sample_states(s, 3, range(4000))
    m = dense.expectation_traces(s, 0.0, full, [0.2], [S1[2]])
    assert abs(m[0, 0]) < 5e-3
