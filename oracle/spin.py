"""Dense spin operators of the radical-pair model (oracle; test infrastructure).

Eq. 1:  H = H_1 + H_2 + 2 J S_1.S_2,  H_i = omega.S_i + sum_k I_ik . A_ik . S_i
        (isotropic in the paper, a_ik I_ik.S_i; the anisotropic form with a
        symmetric tensor A_ik reduces to it for A = a 1).
        omega = -gamma B with gamma the (negative) electron gyromagnetic ratio,
        so for B along z, omega = |gamma_e| B z.  Nuclear Zeeman terms are
        neglected, both electrons share one g, hbar = 1.
Eq. 2:  K = k_S/2 P_S + k_T/2 P_T  (Haberkorn).
Eq. 3:  P_S = 1/4 - S_1.S_2;   Eq. 4:  P_T = 3/4 + S_1.S_2.

Basis order (kron, left = slowest): electron 1, electron 2, then the nuclei in
the order the system lists them.  Each spin uses |M> with M = +I, I-1, ..., -I
(Condon-Shortley phases).

Units: energies in rad/us, so every mT value is multiplied by GAMMA_E.
"""
from __future__ import annotations

import numpy as np

# |gamma_e| in rad us^-1 mT^-1 (CODATA 2018: 1.76085963023e11 rad s^-1 T^-1).
GAMMA_E = 176.085963023


def spin_matrices(two_I: int):
    """(I_x, I_y, I_z) for spin I = two_I / 2 in the basis M = I ... -I."""
    I = two_I / 2.0
    d = two_I + 1
    M = I - np.arange(d)
    Iz = np.diag(M).astype(complex)
    Iplus = np.zeros((d, d), complex)
    for j in range(1, d):
        m = M[j]  # I_+ |m> = sqrt(I(I+1) - m(m+1)) |m+1>, and |m+1> is row j-1
        Iplus[j - 1, j] = np.sqrt(I * (I + 1) - m * (m + 1))
    Iminus = Iplus.conj().T
    Ix = 0.5 * (Iplus + Iminus)
    Iy = -0.5j * (Iplus - Iminus)
    return Ix, Iy, Iz


def _embed(op, pos, dims):
    out = np.ones((1, 1), complex)
    for p, d in enumerate(dims):
        out = np.kron(out, op if p == pos else np.eye(d))
    return out


def dims_of(system):
    return [2, 2] + [int(t) + 1 for t in system.two_I]


def electron_ops(system):
    """S_1 and S_2 as lists [x, y, z] of full-space matrices."""
    dims = dims_of(system)
    s = spin_matrices(1)
    return ([_embed(s[a], 0, dims) for a in range(3)],
            [_embed(s[a], 1, dims) for a in range(3)])


def projectors(system):
    """(P_S, P_T) of Eqs. 3-4 on the full space."""
    S1, S2 = electron_ops(system)
    dot = sum(S1[a] @ S2[a] for a in range(3))
    one = np.eye(dot.shape[0])
    return 0.25 * one - dot, 0.75 * one + dot


def hamiltonian(system, B, direction=None):
    """Eq. 1 as a dense matrix in rad/us, field B (mT) along z, or along the
    unit vector `direction` (the Zeeman term omega . S_i of Eq. 1 with
    omega = |gamma_e| B direction)."""
    dims = dims_of(system)
    S1, S2 = electron_ops(system)
    S = (S1, S2)
    omega = GAMMA_E * float(B)
    if direction is None:
        H = omega * (S1[2] + S2[2])
    else:
        n = np.asarray(direction, float)
        n = n / np.linalg.norm(n)
        H = sum(omega * n[a] * (S1[a] + S2[a]) for a in range(3))
    H = H + 2.0 * GAMMA_E * system.J * sum(S1[a] @ S2[a] for a in range(3))
    for k in range(system.n_nuc):
        Ik = spin_matrices(int(system.two_I[k]))
        Ifull = [_embed(Ik[b], 2 + k, dims) for b in range(3)]
        Si = S[int(system.radical[k])]
        for a in range(3):
            for b in range(3):
                Aab = system.A[k, a, b]
                if Aab != 0.0:
                    H = H + GAMMA_E * Aab * (Si[a] @ Ifull[b])
    return H


def haberkorn(system):
    """Eq. 2, K = k_S/2 P_S + k_T/2 P_T (rates in us^-1)."""
    PS, PT = projectors(system)
    return 0.5 * system.k_S * PS + 0.5 * system.k_T * PT


def generator(system, B, direction=None):
    """A = -i H - K, so that d psi/dt = A psi (Eq. 13, Eq. 6)."""
    return -1j * hamiltonian(system, B, direction) - haberkorn(system)


def singlet_vector():
    """|S> = (|alpha beta> - |beta alpha>)/sqrt 2 on electron 1 x electron 2."""
    v = np.zeros(4, complex)
    v[1] = 1.0 / np.sqrt(2.0)
    v[2] = -1.0 / np.sqrt(2.0)
    return v


def effective_hyperfine_field(a_mT, two_I):
    """Eq. 21: B_hyp = sqrt(sum_k a_k^2 I_k (I_k + 1)), in mT."""
    a = np.asarray(a_mT, float)
    I = np.asarray(two_I, float) / 2.0
    return float(np.sqrt(np.sum(a * a * I * (I + 1.0))))
