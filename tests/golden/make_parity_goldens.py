"""Write the oracle's per-sample yields for the long-horizon and full-size
parity cases (tests/golden/parity_long.json).

Only the FP64 CPU oracle (``oracle.chebyshev``, ``oracle.coherent``) and the
seeded input descriptions (``paper_1612_09517_gb300.workloads``) are called
here; no value comes from the CUDA path.  Each case is one (system, field B,
horizon T, sample s): phi_S = k_S int_0^T |P_S psi|^2 dt, phi_T likewise and
the survival |psi(T)|^2 of psi(0) = |S> x prod_k |Omega_k(s)> (Eqs. 13, 19, 22
with Eq. 20 truncated at T), with the sample directions of Eq. 17 drawn by the
oracle's Philox4x32-10 under seed 0.

Cases (the horizons give the GPU's plan the macro-step counts stated):
* config2_fp64: the 12-nucleus isotropic system (Z = 20736, k_S != k_T),
  samples 0-7 at B = 0, 16.67, 33.33, 50 mT, each field over 100 macro-steps
  of the FP64 plan (88 terms each): T = 100 h(B).
* config3: the 20-nucleus anisotropic system (Z = 2359296), sample 0 at
  2.5 mT and sample 1 at 10 mT, T = 0.1 us (several FP32 macro-steps).
* table1: the paper's model (Table I, Z = 2^20), sample 0 at 3.5 mT and
  sample 1 at 10 mT, T = 0.1 us.

Run from the repository root:  python tests/golden/make_parity_goldens.py [jobs]
(about an hour on 8 cores; the config-3 propagations hold ~12 GB each).
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "parity_long.json")

# FP64 macro-step lengths h(B) of the GPU plan (88 terms, tail 1e-15) at the
# config-2 fields; the horizon of each field is 100 of them.  They only set
# the horizons: any T is a valid case, these make the GPU run >= 100 steps.
CONFIG2_FIELDS = [0.0, 50.0 / 3.0, 100.0 / 3.0, 50.0]
CONFIG2_MACRO = 100


def _cases(config2_h):
    cases = []
    for B, h in zip(CONFIG2_FIELDS, config2_h):
        T = CONFIG2_MACRO * h
        for s in range(8):
            cases.append({"system": "config2", "B": B, "T": T, "sample": s, "n_c": 64})
    for B, s in ((2.5, 0), (10.0, 1)):
        cases.append({"system": "config3", "B": B, "T": 0.1, "sample": s, "n_c": 32})
    for B, s in ((3.5, 0), (10.0, 1)):
        cases.append({"system": "table1", "B": B, "T": 0.1, "sample": s, "n_c": 32})
    return cases


def _system(name):
    from oracle.spin import GAMMA_E
    from paper_1612_09517_gb300 import workloads as wl
    if name == "config2":
        return wl.config2().system
    if name == "config3":
        return wl.config3().system
    return wl.table1(GAMMA_E)


def _run(case):
    sys.path.insert(0, ROOT)
    from oracle import chebyshev, coherent
    s = _system(case["system"])
    t0 = time.time()
    psi0 = coherent.sample_states(s, 0, [case["sample"]])[0]
    phS, phT, surv = chebyshev.propagate_yields(s, case["B"], case["T"], psi0, n_c=case["n_c"])
    out = dict(case)
    out.update({"phi_S": float(phS), "phi_T": float(phT), "survival": float(surv),
                "cpu_s": round(time.time() - t0, 1)})
    print(json.dumps(out), flush=True)
    return out


def _config2_h():
    """The FP64 plan's macro-step h(B) of config 2, from the oracle's own
    Weyl bounds (the same bounds the GPU planner uses, Eq. 1) and the
    88-term, 1e-15 tail rule of ``oracle.chebyshev.plan``."""
    from oracle import chebyshev
    s = _system("config2")
    hs = []
    for B in CONFIG2_FIELDS:
        Hm = chebyshev.TensorHamiltonian(s, B)
        lo, hi = Hm.spectral_bounds()
        dE = 0.5 * (hi - lo)
        h, _ = chebyshev.plan(dE, 0.5 * max(s.k_S, s.k_T), 1.0, n_c=88, tol=1e-15)
        hs.append(h)
    return hs


def main():
    sys.path.insert(0, ROOT)
    jobs = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    cases = _cases(_config2_h())
    # largest first so the long config-3 propagations start at once
    order = sorted(range(len(cases)), key=lambda i: cases[i]["system"] == "config2")
    ctx = mp.get_context("spawn")
    with ctx.Pool(jobs) as pool:
        res = pool.map(_run, [cases[i] for i in order], chunksize=1)
    back = [None] * len(cases)
    for i, r in zip(order, res):
        back[i] = r
    doc = {"source": "oracle.chebyshev.propagate_yields (FP64, matrix-free, exact step "
                     "integrals), psi0 from oracle.coherent.sample_states(seed 0)",
           "cases": back}
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    main()
