"""Exact truncated yields by dense matrix exponentials (oracle; test infrastructure).

Definitions followed (paper section / equation):

* Eq. 13, Eq. 6: a wavepacket evolves as psi(t) = exp(A t) psi(0) with
  A = -i H - K (Eq. 1, Eq. 2).
* Eq. 22: the single-wavepacket singlet yield
  phi_S = k_S int_0^inf <psi(t)| P_S |psi(t)> dt.  The integral is truncated at
  a horizon T (the reading used throughout this project), so
  phi_S^T(psi0) = <psi0| Y_S(T) |psi0>,  Y_S(T) = k_S int_0^T exp(A^H s) P_S exp(A s) ds,
  and likewise phi_T^T with k_T and P_T; survival(T) = |exp(A T) psi0|^2.
* Eq. 14 / Eq. 20: the deterministic trace with rho(0) = P_S / Z:
  Phi_S^T = tr[Y_S(T) P_S] / Z  (the sum over the Z states |S, M_1, M_2>).
* Eq. 18 with Eq. 23: the stochastic estimate is the mean of phi_S^T over M
  coherent-state samples, with standard error sigma / sqrt(M) (sigma from the
  M samples, denominator M - 1).

Y(T) and exp(A T) come from Van Loan's block exponential (C. F. Van Loan,
IEEE Trans. Autom. Control 23, 395 (1978)): for C = [[-A^H, P], [0, A]],
exp(C t) = [[exp(-A^H t), int_0^t exp(-A^H (t-s)) P exp(A s) ds], [0, exp(A t)]],
so Y = exp(A t)^H times the upper-right block.  The exponential is taken on a
short interval h = T / 2^n (scipy's expm is a library primitive) and the
horizon is reached by doubling, using only the additivity of the integral:
Y(2t) = Y(t) + exp(A t)^H Y(t) exp(A t),  exp(2 A t) = exp(A t)^2.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

from .spin import generator, projectors


def _vanloan_block(A, P, t):
    n = A.shape[0]
    C = np.zeros((2 * n, 2 * n), complex)
    C[:n, :n] = -A.conj().T
    C[:n, n:] = P
    C[n:, n:] = A
    E = scipy.linalg.expm(C * t)
    F = E[n:, n:]
    return F, F.conj().T @ E[:n, n:]


def yield_operators(system, B, T, max_norm_step=0.5, direction=None):
    """(Y_S, Y_T, F) with Y_X = k_X int_0^T e^{A^H s} P_X e^{A s} ds and F = e^{A T};
    the field is B along z, or along the unit vector `direction`."""
    A = generator(system, B, direction)
    PS, PT = projectors(system)
    norm = max(np.abs(A).sum(axis=0).max(), 1.0)  # 1-norm of A
    n_double = max(0, int(math.ceil(math.log2(max(norm * T / max_norm_step, 1.0)))))
    h = T / (2 ** n_double)
    F, YS = _vanloan_block(A, PS, h)
    _, YT = _vanloan_block(A, PT, h)
    for _ in range(n_double):
        FH = F.conj().T
        YS = YS + FH @ YS @ F
        YT = YT + FH @ YT @ F
        F = F @ F
    return system.k_S * YS, system.k_T * YT, F


def sample_yields(system, B, T, psi0, direction=None):
    """Per-sample (phi_S, phi_T, survival) for initial states psi0 (n, 4Z)."""
    YS, YT, F = yield_operators(system, B, T, direction=direction)
    psi0 = np.atleast_2d(psi0)
    phiS = np.einsum("si,ij,sj->s", psi0.conj(), YS, psi0).real
    phiT = np.einsum("si,ij,sj->s", psi0.conj(), YT, psi0).real
    surv = np.sum(np.abs(psi0 @ F.T) ** 2, axis=1)
    return phiS, phiT, surv


def trace_yields(system, B, T, direction=None):
    """Deterministic trace (Eq. 14 with rho(0) = P_S/Z): (Phi_S, Phi_T, survival)."""
    YS, YT, F = yield_operators(system, B, T, direction=direction)
    PS, _ = projectors(system)
    Z = system.Z
    surv = np.trace(F.conj().T @ F @ PS).real / Z
    return np.trace(YS @ PS).real / Z, np.trace(YT @ PS).real / Z, surv


def singlet_probability(system, B, psi0, times):
    """P_S(t) = <psi(t)|P_S|psi(t)> at the given times by direct exponentials."""
    A = generator(system, B)
    PS, _ = projectors(system)
    out = []
    for t in np.atleast_1d(times):
        psi = scipy.linalg.expm(A * t) @ psi0
        out.append(np.vdot(psi, PS @ psi).real)
    return np.array(out)


def estimate(per_sample):
    """Eq. 18 mean and Eq. 23 standard error over the last axis."""
    x = np.asarray(per_sample, float)
    M = x.shape[-1]
    return x.mean(axis=-1), x.std(axis=-1, ddof=1) / math.sqrt(M)


def expectation_traces(system, B, psi0, times, ops, direction=None):
    """Eqs. 7-9 and 18 per initial state: <psi(t)| O |psi(t)> for each full-space
    operator O in `ops` at each time, psi(t) = exp(A t) psi0 (Eq. 13), averaged
    over the rows of psi0.  Returns an array (len(times), len(ops)), complex."""
    A = generator(system, B, direction)
    psi0 = np.atleast_2d(psi0)
    out = np.zeros((len(times), len(ops)), complex)
    for i, t in enumerate(times):
        P = scipy.linalg.expm(A * float(t)) @ psi0.T  # (4Z, n)
        for j, O in enumerate(ops):
            out[i, j] = np.mean(np.einsum("in,ij,jn->n", P.conj(), O, P))
    return out
