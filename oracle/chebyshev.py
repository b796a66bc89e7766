"""Matrix-free FP64 propagation with an exact time integral (oracle; test infrastructure).

For systems whose 4Z x 4Z matrices are too large for ``oracle.dense``.  It
computes the same per-sample quantities -- phi_S^T = k_S int_0^T |P_S psi(t)|^2 dt
(Eq. 22 truncated at T), phi_T^T likewise, and |psi(T)|^2 -- for
psi(t) = exp(-i H_eff t) psi(0), H_eff = H - i K (Eq. 1, Eq. 2, Eq. 13).

Steps:
1. The state is a tensor of shape (2, 2, d_1, ..., d_N) (electron 1, electron 2,
   nuclei in listed order).  H_eff psi is applied term by term: the 4x4
   electron operator omega (S_1z + S_2z) + 2J S_1.S_2 - i K on the two electron
   axes, and for each nucleus k the dense block sum_ab A_k,ab S_a I_b on the
   axes (electron of its radical, nucleus k) (Eq. 1).
2. The horizon is cut into equal steps h.  On each step
   psi(t0 + tau) = sum_n c_n(tau) phi_n with phi_n = T_n(Ht) psi(t0),
   Ht = (H_eff - E_c)/dE and c_n(tau) = (2 - delta_n0)(-i)^n J_n(dE tau) e^{-i E_c tau}
   (the Chebyshev expansion of exp(-i tau (E_c + dE x)); Tal-Ezer and Kosloff,
   J. Chem. Phys. 81, 3967 (1984)).  E_c and dE come from Weyl's inequality on
   the Hermitian part, so the real part of every eigenvalue of Ht lies in [-1, 1].
3. The integral over the step is exact up to truncation:
   int_0^h |P_S psi|^2 dtau = sum_nm W_nm <P_S phi_n | P_S phi_m>,
   W_nm = int_0^h conj(c_n(tau)) c_m(tau) dtau, evaluated by Gauss-Legendre
   quadrature with many more nodes than the integrand's effective degree.
   The triplet integral uses the full Gram minus the singlet Gram (P_T = 1 - P_S).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special

from .spin import GAMMA_E, spin_matrices


class TensorHamiltonian:
    """H_eff = H - i K applied to a state tensor of shape (2, 2, d_1, ..., d_N)."""

    def __init__(self, system, B):
        self.system = system
        self.dims = [2, 2] + [int(t) + 1 for t in system.two_I]
        s = spin_matrices(1)
        e1 = [np.kron(s[a], np.eye(2)) for a in range(3)]
        e2 = [np.kron(np.eye(2), s[a]) for a in range(3)]
        dot = sum(e1[a] @ e2[a] for a in range(3))
        PS4 = 0.25 * np.eye(4) - dot
        PT4 = 0.75 * np.eye(4) + dot
        omega = GAMMA_E * float(B)
        self.He = omega * (e1[2] + e2[2]) + 2.0 * GAMMA_E * system.J * dot
        self.K4 = 0.5 * system.k_S * PS4 + 0.5 * system.k_T * PT4
        self.PS4 = PS4
        self.blocks = []
        for k in range(system.n_nuc):
            I = spin_matrices(int(system.two_I[k]))
            h = np.zeros((2 * (int(system.two_I[k]) + 1),) * 2, complex)
            for a in range(3):
                for b in range(3):
                    h += GAMMA_E * system.A[k, a, b] * np.kron(s[a], I[b])
            self.blocks.append(h)

    def spectral_bounds(self):
        """Weyl bounds [E_min, E_max] on the spectrum of the Hermitian part H."""
        ev = np.linalg.eigvalsh(self.He)
        lo, hi = ev[0], ev[-1]
        for h in self.blocks:
            evk = np.linalg.eigvalsh(h)
            lo += evk[0]
            hi += evk[-1]
        return lo, hi

    def apply(self, psi):
        n = len(self.dims)
        v = psi.reshape(4, -1)
        y = ((self.He - 1j * self.K4) @ v).reshape(psi.shape)
        for k, h in enumerate(self.blocks):
            r = int(self.system.radical[k])
            ax = 2 + k
            t = np.moveaxis(psi, (r, ax), (0, 1))
            shp = t.shape
            t = (h @ t.reshape(shp[0] * shp[1], -1)).reshape(shp)
            y += np.moveaxis(t, (0, 1), (r, ax))
        return y

    def singlet_component(self, psi):
        """<S|psi> on the electron axes, a tensor over the nuclear axes."""
        v = psi.reshape(4, -1)
        return ((v[1] - v[2]) / math.sqrt(2.0))


def _tail(x, n_c, rho):
    n = np.arange(n_c, n_c + 200)
    return float(np.sum(2.0 * np.abs(scipy.special.jv(n, x)) * rho ** n))


def plan(dE, kmax, T, n_c=64, tol=1e-15):
    """Largest step h with truncation tail below tol; returns (h, n_steps)."""
    rho = 1.0 + kmax / max(dE, 1e-300)
    lo, hi = 0.0, float(n_c)
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if _tail(mid, n_c, rho) < tol:
            lo = mid
        else:
            hi = mid
    h_max = lo / dE
    n_steps = max(1, int(math.ceil(T / h_max)))
    return T / n_steps, n_steps


def coefficients(dE, Ec, tau, n_c):
    """c_n(tau) = (2 - delta_n0)(-i)^n J_n(dE tau) e^{-i Ec tau}, shape (len(tau), n_c)."""
    tau = np.atleast_1d(tau)
    n = np.arange(n_c)
    J = scipy.special.jv(n[None, :], dE * tau[:, None])
    eps = np.where(n == 0, 1.0, 2.0)
    return eps[None, :] * ((-1j) ** n)[None, :] * J * np.exp(-1j * Ec * tau)[:, None]


def weights(dE, Ec, h, n_c, n_nodes=None):
    """W_nm = int_0^h conj(c_n(tau)) c_m(tau) dtau by Gauss-Legendre quadrature."""
    if n_nodes is None:
        n_nodes = 2 * n_c + int(dE * h) + 40
    x, w = np.polynomial.legendre.leggauss(n_nodes)
    tau = 0.5 * h * (x + 1.0)
    wt = 0.5 * h * w
    c = coefficients(dE, Ec, tau, n_c)
    return np.einsum("q,qn,qm->nm", wt, c.conj(), c)


def propagate_yields(system, B, T, psi0, n_c=64, tol=1e-15, return_state=False):
    """Per-sample (phi_S, phi_T, survival) for one initial state psi0 (4Z,)."""
    Hm = TensorHamiltonian(system, B)
    lo, hi = Hm.spectral_bounds()
    Ec = 0.5 * (hi + lo)
    dE = 0.5 * (hi - lo) * (1.0 + 1e-12) + 1e-9
    kmax = 0.5 * max(system.k_S, system.k_T)
    h, n_steps = plan(dE, kmax, T, n_c, tol)
    W = weights(dE, Ec, h, n_c)
    c_end = coefficients(dE, Ec, h, n_c)[0]
    psi = np.asarray(psi0, complex).reshape(Hm.dims).copy()
    intS = 0.0
    intT = 0.0
    for _ in range(n_steps):
        phis = [psi]
        prev, cur = None, psi
        for n in range(1, n_c):
            Hc = (Hm.apply(cur) - Ec * cur) / dE
            nxt = Hc if n == 1 else 2.0 * Hc - prev
            phis.append(nxt)
            prev, cur = cur, nxt
        X = np.stack([p.reshape(-1) for p in phis])          # (n_c, 4Z)
        Xs = np.stack([Hm.singlet_component(p) for p in phis])  # (n_c, Z)
        G_all = X.conj() @ X.T
        G_S = Xs.conj() @ Xs.T
        iS = np.sum(W * G_S).real
        intS += iS
        intT += np.sum(W * (G_all - G_S)).real
        psi = np.tensordot(c_end, X, axes=1).reshape(Hm.dims)
    surv = float(np.vdot(psi, psi).real)
    out = (system.k_S * intS, system.k_T * intT, surv)
    if return_state:
        return out + (psi.reshape(-1),)
    return out
