"""Spin coherent states and sample initial states (oracle; test infrastructure).

Eq. 15: |Omega_J> = (cos theta/2)^{2J} exp{tan(theta/2) e^{i phi} J_-} |J, J>,
        0 <= theta <= pi, 0 <= phi < 2 pi.  Built here literally, with the
        matrix exponential of the (nilpotent) lowering operator J_-.
Eq. 16: <Omega_J| J |Omega_J> = J n(Omega)      (checked by the tests)
Eq. 17: 1 = (2J+1)/(4 pi) int dOmega |Omega_J><Omega_J|   (checked by the tests)
Eq. 19: |Omega_i> = prod_k |Omega_ik>;  the sample state of Eq. 18 is
        |S> x |Omega_1> x |Omega_2>, in the basis order of ``oracle.spin``.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .spin import spin_matrices, singlet_vector
from .philox import draw_angles


def coherent_state(two_I: int, theta: float, phi: float):
    """|Omega_J> of Eq. 15 for J = two_I/2, in the basis M = J ... -J."""
    Ix, Iy, Iz = spin_matrices(two_I)
    Jminus = Ix - 1j * Iy
    top = np.zeros(two_I + 1, complex)
    top[0] = 1.0  # |J, J>
    z = np.tan(theta / 2.0) * np.exp(1j * phi)
    return np.cos(theta / 2.0) ** two_I * (scipy.linalg.expm(z * Jminus) @ top)


def sample_state(system, theta_row, phi_row):
    """|S> x prod_k |Omega_k> for one sample (angles per nucleus)."""
    psi = singlet_vector()
    for k in range(system.n_nuc):
        psi = np.kron(psi, coherent_state(int(system.two_I[k]), theta_row[k], phi_row[k]))
    return psi


def sample_states(system, seed: int, samples, pair: int = 0):
    """Initial states of the given sample indices, shape (n_samples, 4 Z)."""
    samples = np.asarray(samples).reshape(-1)
    theta, phi = draw_angles(seed, pair, samples, system.n_nuc)
    return np.stack([sample_state(system, theta[i], phi[i]) for i in range(samples.size)])


def basis_states(system):
    """|S, M_1, M_2> for every nuclear basis state (Eq. 13), shape (Z, 4 Z)."""
    Z = system.Z
    s = singlet_vector()
    out = np.zeros((Z, 4 * Z), complex)
    for m in range(Z):
        e = np.zeros(Z, complex)
        e[m] = 1.0
        out[m] = np.kron(s, e)
    return out
