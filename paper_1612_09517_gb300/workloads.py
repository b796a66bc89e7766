"""Seeded synthetic radical-pair workloads.

This module only *describes* inputs: which nuclei sit on which radical, their
spins, hyperfine tensors, rate constants, exchange coupling, field grids and
sample counts.  It holds none of the method's arithmetic (no Hamiltonian, no
propagation, no yields), so both the CUDA path and the CPU oracle may take
their inputs from it.

Units follow the paper's tables: hyperfine tensors, exchange J and fields in
mT; rate constants in inverse microseconds; times in microseconds.

Workloads (all seeded; the generator seed of workload c is 1000 + c):

* ``config1`` -- 4 spin-1/2 nuclei on radical 1, isotropic a ~ U[-1, 1] mT,
  J = 0, k_S = k_T = 1 us^-1, 11 fields in [0, 5] mT, t_max = 10 us, M = 64.
* ``one_nucleus`` -- a single spin-I nucleus on radical 1 (closed-form side case).
* ``config2`` -- 8 spin-1/2 + 4 spin-1 nuclei; radical 1 holds 5 x 1/2 + 2 x 1,
  radical 2 holds 3 x 1/2 + 2 x 1 (Z = 20736); isotropic a ~ N(0, 0.5 mT);
  J = 0; k_S = 2, k_T = 0.5 us^-1; 64 fields in [0, 50] mT; t_max = 20 us; M = 200.
* ``config3`` -- 18 spin-1/2 + 2 spin-1, 9 x 1/2 + 1 x 1 on each radical
  (Z = 2359296); anisotropic symmetric tensors R diag(lambda) R^T with
  lambda ~ N(0, 0.8 mT) and R Haar-random; J = 0.1 mT; k_S = k_T = 1 us^-1;
  128 fields in [0, 10] mT; t_max = 10 us; M = 200.
* ``config4`` -- 256 pairs, N ~ U{6..16} nuclei, each spin-1/2 with
  probability 0.8 else spin-1, ceil(N/2) on radical 1; a ~ N(0, 0.5 mT);
  k_S, k_T ~ LogUniform[0.1, 10] us^-1 independently; J = 0; 32 fields in
  [0, 10] mT; t_max = 10 / min(k_S, k_T); M = 64.
* ``table1`` -- the paper's own model (Table I; Sec. IV): 10 + 10 spin-1/2
  nuclei with the listed couplings, J/gamma = 1.75 mT, k_S/gamma = 0.1 mT,
  k_T/gamma = 1.0 mT.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np


@dataclass
class SpinSystem:
    """A radical pair: nuclei, hyperfine tensors, recombination rates, exchange.

    ``radical[k]`` is 0 or 1 (the electron nucleus k couples to), ``two_I[k]``
    is twice the nuclear spin, ``A[k]`` is the 3x3 real symmetric hyperfine
    tensor in mT (isotropic coupling a is ``a * eye(3)``), ``k_S`` / ``k_T``
    are in us^-1 and ``J`` in mT.
    """

    radical: np.ndarray
    two_I: np.ndarray
    A: np.ndarray
    k_S: float
    k_T: float
    J: float
    name: str = ""

    def __post_init__(self):
        self.radical = np.asarray(self.radical, dtype=np.int32).reshape(-1)
        self.two_I = np.asarray(self.two_I, dtype=np.int32).reshape(-1)
        self.A = np.asarray(self.A, dtype=np.float64).reshape(-1, 3, 3)
        self.k_S = float(self.k_S)
        self.k_T = float(self.k_T)
        self.J = float(self.J)

    @property
    def n_nuc(self) -> int:
        return int(self.radical.size)

    @property
    def Z(self) -> int:
        """Number of nuclear spin states, prod(2 I_k + 1)."""
        return int(np.prod(self.two_I + 1)) if self.n_nuc else 1

    @property
    def dim(self) -> int:
        """Dimension of the electron x nuclear Hilbert space, 4 Z."""
        return 4 * self.Z


@dataclass
class Workload:
    system: SpinSystem
    fields: np.ndarray
    M: int
    t_max: float
    seed: int = 0
    extra: dict = field(default_factory=dict)


def _iso(a):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    return a[:, None, None] * np.eye(3)[None]


def one_nucleus(a_mT: float = 1.0, two_I: int = 1, k: float = 1.0, J: float = 0.0,
                radical: int = 0) -> SpinSystem:
    """One spin-I nucleus with isotropic coupling a on one radical."""
    return SpinSystem([radical], [two_I], _iso([a_mT]), k, k, J, name="one_nucleus")


def random_isotropic(n1: int, n2: int, two_I=None, a_scale=1.0, k_S=1.0, k_T=1.0,
                     J=0.0, seed=0, dist="uniform") -> SpinSystem:
    """Small random isotropic system used by tests (n1 nuclei on radical 1, n2 on 2)."""
    rng = np.random.default_rng(seed)
    n = n1 + n2
    if two_I is None:
        two_I = [1] * n
    if dist == "uniform":
        a = rng.uniform(-a_scale, a_scale, n)
    else:
        a = rng.normal(0.0, a_scale, n)
    return SpinSystem([0] * n1 + [1] * n2, two_I, _iso(a), k_S, k_T, J,
                      name=f"iso_{n1}_{n2}_s{seed}")


def haar_rotation(rng) -> np.ndarray:
    """Haar-random rotation from a normalised Gaussian quaternion."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def random_anisotropic(n1: int, n2: int, two_I=None, scale=0.8, k_S=1.0, k_T=1.0,
                       J=0.0, seed=0) -> SpinSystem:
    """Random symmetric tensors R diag(lambda) R^T, lambda ~ N(0, scale)."""
    rng = np.random.default_rng(seed)
    n = n1 + n2
    if two_I is None:
        two_I = [1] * n
    A = np.empty((n, 3, 3))
    for k in range(n):
        lam = rng.normal(0.0, scale, 3)
        R = haar_rotation(rng)
        A[k] = R @ np.diag(lam) @ R.T
        A[k] = 0.5 * (A[k] + A[k].T)
    return SpinSystem([0] * n1 + [1] * n2, two_I, A, k_S, k_T, J,
                      name=f"aniso_{n1}_{n2}_s{seed}")


def config1() -> Workload:
    rng = np.random.default_rng(1001)
    a = rng.uniform(-1.0, 1.0, 4)
    sys_ = SpinSystem([0] * 4, [1] * 4, _iso(a), 1.0, 1.0, 0.0, name="config1")
    return Workload(sys_, np.linspace(0.0, 5.0, 11), 64, 10.0, seed=0,
                    extra={"side_case": one_nucleus(1.0, 1, 1.0)})


def config2() -> Workload:
    rng = np.random.default_rng(1002)
    # radical 1: 5 x 1/2 + 2 x 1 ; radical 2: 3 x 1/2 + 2 x 1
    two_I = [1] * 5 + [2] * 2 + [1] * 3 + [2] * 2
    radical = [0] * 7 + [1] * 5
    a = rng.normal(0.0, 0.5, 12)
    sys_ = SpinSystem(radical, two_I, _iso(a), 2.0, 0.5, 0.0, name="config2")
    return Workload(sys_, np.linspace(0.0, 50.0, 64), 200, 20.0, seed=0)


def config3() -> Workload:
    rng = np.random.default_rng(1003)
    two_I = [1] * 9 + [2] + [1] * 9 + [2]
    radical = [0] * 10 + [1] * 10
    A = np.empty((20, 3, 3))
    for k in range(20):
        lam = rng.normal(0.0, 0.8, 3)
        R = haar_rotation(rng)
        A[k] = R @ np.diag(lam) @ R.T
        A[k] = 0.5 * (A[k] + A[k].T)
    sys_ = SpinSystem(radical, two_I, A, 1.0, 1.0, 0.1, name="config3")
    return Workload(sys_, np.linspace(0.0, 10.0, 128), 200, 10.0, seed=0)


def config4(n_pairs: int = 256) -> list[Workload]:
    rng = np.random.default_rng(1004)
    out = []
    for p in range(n_pairs):
        n = int(rng.integers(6, 17))
        two_I = np.where(rng.uniform(size=n) < 0.8, 1, 2)
        n1 = int(math.ceil(n / 2))
        radical = [0] * n1 + [1] * (n - n1)
        a = rng.normal(0.0, 0.5, n)
        k_S = float(10.0 ** rng.uniform(-1.0, 1.0))
        k_T = float(10.0 ** rng.uniform(-1.0, 1.0))
        sys_ = SpinSystem(radical, two_I, _iso(a), k_S, k_T, 0.0, name=f"config4_{p}")
        out.append(Workload(sys_, np.linspace(0.0, 10.0, 32), 64,
                            10.0 / min(k_S, k_T), seed=p))
    return out


def config5() -> Workload:
    w = config2()
    return Workload(w.system, np.linspace(0.0, 50.0, 128), 2000, 20.0, seed=0,
                    extra={"train_yields": 200000, "se_target": 1e-3})


# Table I of the paper: a_1k/gamma and a_2k/gamma in mT, k = 1..10.
TABLE1_A1 = [-0.999985, -0.736925, 0.511210, -0.0826998, 0.0655341,
             -0.562082, -0.905911, 0.357729, 0.358593, 0.869386]
TABLE1_A2 = [-0.232996, 0.0388327, 0.661931, -0.930856, -0.893077,
             0.0594001, 0.342299, -0.984604, -0.233169, -0.866316]


def table1(gamma: float) -> SpinSystem:
    """The paper's model radical pair (Table I and Sec. IV).

    ``gamma`` converts the paper's k/gamma values (in mT) to us^-1; the caller
    supplies its own electron gyromagnetic ratio in rad us^-1 mT^-1.
    """
    a = TABLE1_A1 + TABLE1_A2
    return SpinSystem([0] * 10 + [1] * 10, [1] * 20, _iso(a), 0.1 * gamma,
                      1.0 * gamma, 1.75, name="table1")
