#!/usr/bin/env python
"""Benchmark: time to a converged singlet-yield curve Phi_S(B) on one GB300.

Workload (config 2 of this project): 12 nuclei (8 spin-1/2 + 4 spin-1, 7 on
radical 1 and 5 on radical 2, Z = 20736, state dimension 82944), isotropic
a ~ N(0, 0.5 mT), J = 0, k_S = 2 us^-1, k_T = 0.5 us^-1 (decay not factorable),
64 fields in 0-50 mT, horizon T = 20 us, complex FP32 state with FP64 time
integrals and averages; target SE <= 1e-3 at every field (Eq. 23).

One step = one rp_yields call through the C ABI on half of the 64 fields
(alternate halves: fields 0, 2, 4, ... then 1, 3, 5, ...) x
``--samples-per-step`` coherent-state samples each, every sample propagated
over the full horizon; steps and ranks use disjoint sample ranges
(sample_offset).  The timed steps give (a) the throughput in Chebyshev
row-terms per second on the curve's own field mix and (b) the spread sigma_f
of phi_S at every field, pooled over the timed steps.

Reported ``value``: seconds to the converged 64-field curve =
sum_f M_f x (Chebyshev terms of one sample at field f, exact from the plan) /
(measured row-terms per second of device time), with M_f the per-field sample
counts rp_yields_converged asks for the measured sigma_f
(max(8, ceil(1.15 sigma_f^2 / SE^2) + 1)).  ``e2e`` is the same with the wall
time of the C-ABI calls (host planning, host<->device copies and
synchronisation inside).  At one GPU the line also carries, measured once
each after the timed steps:
* ``converged_measured``: the whole 64-field curve through rp_yields_converged
  and through rp_yields_cv (learned control variate), wall time;
* ``fp64_plain.measured_reduced``: the plain FP64 form against the FP32 +
  control-variate form end to end on a reduced workload (4 fields, 1 us);
  ``fp64_plain.projected_full`` projects the FP64 form to the full curve from
  its measured throughput;
* ``cpu_baseline``: the FP64 oracle on the host cores, bounded sample,
  projected to the same curve.

``--impl reference`` times the FP64 CPU oracle (matrix-free Chebyshev,
NumPy) on the host cores on bounded samples of the same workload and reports
the same metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("time to converged Φ_S(B) at SE≤1e-3 vs FP64 plain; "
          "H·ψ HBM GB/s vs peak")
WORKLOAD = ("config2: 12 nuclei (8x1/2 + 4x1, split 7/5), Z=20736, isotropic a~N(0,0.5 mT), "
            "J=0, k_S=2, k_T=0.5 us^-1, 64 fields 0-50 mT, t_max=20 us, SE target 1e-3")
SE_TARGET = 1e-3
# Per-field standard deviation of phi_S over the 64 fields of this workload,
# measured on GB300 by `python bench.py --converge` (rp_yields_converged,
# SE <= 1e-3 everywhere; 16 to 991 samples per field).  Only the reference
# arm uses it: the CPU oracle cannot afford enough full-horizon samples to
# measure the spread itself, so it turns its throughput into the time for a
# converged curve with these per-field sample counts.
SIGMA_REFERENCE = [
    0.01636, 0.02267, 0.02981, 0.02294, 0.01538, 0.0101, 0.00761, 0.00606, 0.00459, 0.00434,
    0.00371, 0.00346, 0.00296, 0.00253, 0.00227, 0.00203, 0.00183, 0.00164, 0.00146, 0.00132,
    0.00119, 0.00109, 0.00099, 0.00091, 0.00085, 0.0008, 0.00076, 0.00074, 0.00071, 0.0007,
    0.00068, 0.00066, 0.00065, 0.00063, 0.00062, 0.00061, 0.0006, 0.00059, 0.00059, 0.00058,
    0.00057, 0.00057, 0.00057, 0.00056, 0.00056, 0.00056, 0.00056, 0.00056, 0.00056, 0.00056,
    0.00056, 0.00056, 0.00055, 0.00055, 0.00055, 0.00055, 0.00055, 0.00055, 0.00055, 0.00055,
    0.00056, 0.00056, 0.00056, 0.00056]
M_MIN = 8


def samples_per_field(sigmas=SIGMA_REFERENCE):
    """M_f of rp_yields_converged for SE <= SE_TARGET (Eq. 23), per field."""
    return [max(M_MIN, int(math.ceil(1.15 * s * s / (SE_TARGET * SE_TARGET))) + 1) for s in sigmas]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback 6.8 TB/s"


def _kernel_source_hash():
    h = hashlib.sha256()
    for f in ("rp_kernels.cu", "rp_kernels.cuh", "rp_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1612_09517_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _profile_traffic(kernel, key="dram_bytes_per_row"):
    """A committed ncu figure of `kernel` (profiles/traffic.json): by default
    the DRAM bytes (read + write) per row of one launch; None when absent or
    captured on a different kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel)
    if not d or d.get("kernel_source_sha256_16") != _kernel_source_hash() or key not in d:
        return None
    return float(d[key])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()

    def summary(self):
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _field_terms(sy, fields, t_max, precision):
    """Chebyshev terms of one sample at each field (exact, from the plan)."""
    out = []
    for B in fields:
        p = sy.plan(B, t_max, precision=precision)
        out.append(p["n_macro"] * p["n_cheb"])
    return out


def _curve_terms(sy, fields, t_max, precision):
    """Chebyshev terms of one sample over all fields."""
    return sum(_field_terms(sy, fields, t_max, precision))


# ---------------------------------------------------------------- CPU oracle

def _oracle_worker(args):
    B, T, sample = args
    sys.path.insert(0, ROOT)
    import numpy as np  # noqa: F401
    from oracle import chebyshev, coherent
    from paper_1612_09517_gb300 import workloads as wl
    s = wl.config2().system
    psi0 = coherent.sample_states(s, 0, [sample])[0]
    Hm = chebyshev.TensorHamiltonian(s, B)
    lo, hi = Hm.spectral_bounds()
    dE = 0.5 * (hi - lo) * (1.0 + 1e-12) + 1e-9
    h, n_steps = chebyshev.plan(dE, 0.5 * max(s.k_S, s.k_T), T)
    t0 = time.perf_counter()
    chebyshev.propagate_yields(s, B, T, psi0)
    return time.perf_counter() - t0, n_steps * 64


def _oracle_field_terms(t_max, fields):
    from oracle import chebyshev
    from paper_1612_09517_gb300 import workloads as wl
    s = wl.config2().system
    out = []
    for B in fields:
        Hm = chebyshev.TensorHamiltonian(s, B)
        lo, hi = Hm.spectral_bounds()
        dE = 0.5 * (hi - lo) * (1.0 + 1e-12) + 1e-9
        h, n = chebyshev.plan(dE, 0.5 * max(s.k_S, s.k_T), t_max)
        out.append(n * 64)
    return out


def cpu_oracle_throughput(cores, T_sample, B_list):
    """Row-terms per second of the FP64 oracle over `cores` spawned processes
    (one BLAS thread each, so the processes do not oversubscribe the cores)."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    ctx = mp.get_context("spawn")
    jobs = [(B_list[i % len(B_list)], T_sample, i) for i in range(cores)]
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    wall = time.perf_counter() - t0
    terms = sum(r[1] for r in res)
    busy = max(r[0] for r in res)
    return terms / busy, wall, terms


# ---------------------------------------------------------------------- main

def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--samples-per-step", type=int, default=2,
                    help="samples per field in each step (each step runs half of the 64 fields)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the measured converged curves, the FP64 comparisons and the CPU "
                         "baseline")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--kernel", type=int, default=0,
                    help="rp_options.kernel of the timed steps and the profiling cases (0: choose)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--converge", action="store_true",
                    help="run the whole converged curve (rp_yields_converged, SE <= 1e-3) once "
                         "and print its measured time")
    ap.add_argument("--cv", action="store_true",
                    help="with --converge: use the learned control variate (rp_yields_cv)")
    ap.add_argument("--cv-bias", action="store_true",
                    help="config 5: the 128-field curve to SE <= 1e-3 with the learned control "
                         "variate, then an independent plain M = 2000 estimate at four fields "
                         "to check its bias; prints one JSON line")
    ap.add_argument("--config5", action="store_true",
                    help="config 5 (the config-2 system over 128 fields 0-50 mT): the converged "
                         "curve plain (rp_yields_converged) and with the learned control "
                         "variate (rp_yields_cv), both end to end; one JSON line")
    ap.add_argument("--config4", action="store_true",
                    help="config 4 (256 radical pairs of uneven size) through rp_yields_batch on "
                         "a stated subset: every pair at --c4-fields fields of its sweep x "
                         "--c4-samples samples; time, work and the projection to the full "
                         "workload by the plan's exact work; one JSON line")
    ap.add_argument("--c4-fields", type=int, default=2)
    ap.add_argument("--c4-samples", type=int, default=4)
    ap.add_argument("--table1", action="store_true",
                    help="the paper's model problem (Table I couplings, Z = 2^20): Phi_S(B) at 21 "
                         "fields 0-10 mT with M = 400 (and the first 100 and 200 samples, as in "
                         "Fig. 2), the field of the minimum, per-sample histograms at three "
                         "fields (Fig. 4); one JSON line")
    ap.add_argument("--basis-sampling", action="store_true",
                    help="config-2 system, 3 fields x 200 samples: spread of phi_S with "
                         "coherent-state samples vs random basis states (deterministic = 2); "
                         "one JSON line")
    ap.add_argument("--trace", action="store_true",
                    help="config 2 at 1.59 and 3.17 mT: the deterministic trace (Eq. 14) by J_z "
                         "sectors against the stochastic estimate to SE <= 1e-3, measured wall "
                         "times and the trace-level error; one JSON line")
    ap.add_argument("--basis-aniso", action="store_true",
                    help="config-3 system (anisotropic, Z = 2359296), 1 and 5 mT over 1 us: "
                         "spread of phi_S with 64 coherent-state samples vs 64 random basis "
                         "states; one JSON line")
    ap.add_argument("--cv-size", action="store_true",
                    help="config-2 system at 1.6 / 3.2 / 4.8 mT: variance reduction of the "
                         "learned control variate on 1000 fresh samples per field as a function "
                         "of the training-set size; one JSON line")
    ap.add_argument("--grouped-prototype", action="store_true",
                    help="config-3 system: time of the grouped dense-block H.psi on the tensor "
                         "cores (the group's (8 x 2^g)^2 real block times the state, as a plain "
                         "GEMM by the vendor library: TF32 x3 for the FP32 accuracy, BF16 for "
                         "reference) against the matrix-free per-term kernel; one JSON line")
    ap.add_argument("--ncu-case3", action="store_true",
                    help="profiling case of the anisotropic config-3 system (Z = 2359296): "
                         "2 rows, two macro-steps, ~4 GB on the device")
    ap.add_argument("--ncu-case5", action="store_true",
                    help="profiling case of the persistent launch (kernel 5): the first 8 "
                         "config-4 pairs with Z <= 2048, 4 fields x 8 samples each, one "
                         "rp_yields_batch call")
    ap.add_argument("--ncu-case", action="store_true",
                    help="run one small profiling case (192 rows, two macro-steps) and exit")
    return ap.parse_args()


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    import numpy as np
    world, rank, _ = _dist()
    if rank != 0:
        return
    from paper_1612_09517_gb300 import workloads as wl
    w = wl.config2()
    cores = os.cpu_count() or 1
    # bounded sample: each core propagates one (field, sample) for T_sample us
    B_list = list(w.fields[[0, 21, 42, 63]])
    T_sample = 0.1
    fterms = _oracle_field_terms(w.t_max, w.fields)
    Mf = samples_per_field()
    conv_terms = sum(m * t for m, t in zip(Mf, fterms))
    times = []
    rates = []
    for i in range(args.warmup + args.steps):
        rate, wall, terms = cpu_oracle_throughput(cores, T_sample, B_list)
        if i >= args.warmup:
            times.append(wall)
            rates.append(rate)
    rate = statistics.median(rates)
    value = conv_terms / rate
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.median(times) * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "oracle": "matrix-free FP64 Chebyshev (NumPy)",
                   "samples_total": int(sum(Mf)), "oracle_terms_converged_curve": int(conv_terms),
                   "note": "value = oracle Chebyshev terms of the converged curve (per-field "
                           "sample counts M_f, SE <= 1e-3) / oracle row-terms per second on the "
                           "host cores"},
        "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} processes, each one (field, sample) propagation over "
                                   f"{T_sample} us at B in {[round(float(b), 2) for b in B_list]} mT; "
                                   f"row-terms/s {rate:.0f} extrapolated to the {conv_terms} oracle "
                                   "terms of the converged 64-field curve"},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)  # before the process group, so NCCL binds this GPU
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_1612_09517_gb300 import rp
    from paper_1612_09517_gb300 import workloads as wl
    rp.use_torch_allocator()

    w = wl.config2()
    sy = rp.System(w.system)
    prec = rp.RP_FP32 if args.precision == "fp32" else rp.RP_FP64
    if args.converge:
        sy.yields([0.0], 2, 0, 0.05)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        o = rp.rp_default_options(precision=prec, stream=torch.cuda.current_stream().cuda_stream)
        if args.cv:
            plan = rp.rp_cv_default_plan()
            r = rp.rp_yields_cv(sy.handle, w.fields, SE_TARGET, M_MIN, 4000, 0, w.t_max, o, plan)
            wall = time.perf_counter() - t0
            st = r["stats"]
            print(json.dumps({"mode": "converge+cv", "workload": WORKLOAD, "wall_s": wall,
                              "propagations": st["propagations"], "row_terms": st["row_terms"],
                              "kernel_launches": st["kernel_launches"], "rows": st["rows"],
                              "M_min": M_MIN, "max_SE": float(r["out"][:, 1].max()),
                              "M_plain": r["M_plain"].tolist(), "M_cv": r["M_cv"].tolist(),
                              "beta": [round(float(x), 5) for x in r["out"][:, 6]],
                              "PhiS": r["out"][:, 0].tolist()}), flush=True)
            return
        r = rp.rp_yields_converged(sy.handle, w.fields, SE_TARGET, M_MIN, 4000, 0, w.t_max, o)
        wall = time.perf_counter() - t0
        st = r["stats"]
        sig = r["out"][:, 2] * np.sqrt(r["M_used"])
        print(json.dumps({"mode": "converge", "workload": WORKLOAD, "wall_s": wall,
                          "device_ms": st["device_ms"], "propagations": st["propagations"],
                          "row_terms": st["row_terms"], "kernel_launches": st["kernel_launches"],
                          "rows": st["rows"], "M_min": M_MIN, "max_SE": float(r["out"][:, 2].max()),
                          "M_used": r["M_used"].tolist(),
                          "sigma": [round(float(x), 5) for x in sig],
                          "PhiS": r["out"][:, 0].tolist()}), flush=True)
        return
    if args.config5:
        w5 = wl.config5()
        o = rp.rp_default_options(precision=prec, stream=torch.cuda.current_stream().cuda_stream)
        sy.yields([0.0], 2, 0, 0.05)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rpl = rp.rp_yields_converged(sy.handle, w5.fields, SE_TARGET, M_MIN, 4000, 0, w5.t_max, o)
        wall_plain = time.perf_counter() - t0
        t0 = time.perf_counter()
        rcv = rp.rp_yields_cv(sy.handle, w5.fields, SE_TARGET, M_MIN, 4000, 0, w5.t_max, o,
                              rp.rp_cv_default_plan())
        wall_cv = time.perf_counter() - t0
        print(json.dumps({
            "mode": "config5", "workload": "config5: " + WORKLOAD.split(": ", 1)[1]
            .replace("64 fields", "128 fields"),
            "plain": {"wall_s": wall_plain, "samples": int(rpl["M_used"].sum()),
                      "row_terms": int(rpl["stats"]["row_terms"]),
                      "max_SE": float(rpl["out"][:, 2].max())},
            "cv": {"wall_s": wall_cv, "samples_plain": int(rcv["M_plain"].sum()),
                   "samples_cv": int(rcv["M_cv"].sum()),
                   "fields_with_cv": int(rcv["out"][:, 7].sum()),
                   "control_variate_s": rcv["stats"]["cv_ms"] * 1e-3,
                   "max_SE": float(rcv["out"][:, 1].max())},
            "max_abs_diff_PhiS": float(np.max(np.abs(rcv["out"][:, 0] - rpl["out"][:, 0])))}),
              flush=True)
        return
    if args.cv_bias:
        w5 = wl.config5()
        o = rp.rp_default_options(precision=prec, stream=torch.cuda.current_stream().cuda_stream)
        sy.yields([0.0], 2, 0, 0.05)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = rp.rp_yields_cv(sy.handle, w5.fields, SE_TARGET, M_MIN, 4000, 0, w5.t_max, o,
                            rp.rp_cv_default_plan())
        wall_cv = time.perf_counter() - t0
        # independent plain estimate (seed 1: other directions) at four low fields,
        # where the spread and the control-variate gain are largest
        idx = [3, 8, 13, 20]
        t0 = time.perf_counter()
        p = rp.rp_yields(sy.handle, w5.fields[idx], 2000, 1, w5.t_max, o)
        wall_plain = time.perf_counter() - t0
        est, se = r["out"][idx, 0], r["out"][idx, 1]
        z = (est - p["out"][:, 0]) / np.sqrt(se ** 2 + p["out"][:, 2] ** 2)
        print(json.dumps({"mode": "cv-bias", "workload": "config5: " + WORKLOAD.split(": ", 1)[1]
                          .replace("64 fields", "128 fields"),
                          "wall_cv_s": wall_cv, "max_SE": float(r["out"][:, 1].max()),
                          "M_plain": r["M_plain"].tolist(), "M_cv": r["M_cv"].tolist(),
                          "used_cv": [int(x) for x in r["out"][:, 7]],
                          "bias_fields_mT": [round(float(b), 4) for b in w5.fields[idx]],
                          "PhiS_cv": est.tolist(), "SE_cv": se.tolist(),
                          "PhiS_plain_M2000": p["out"][:, 0].tolist(),
                          "SE_plain_M2000": p["out"][:, 2].tolist(),
                          "z": z.tolist(), "chi2": float(np.sum(z ** 2)), "dof": len(idx),
                          "wall_plain_s": wall_plain}), flush=True)
        return
    if args.basis_sampling:
        fb = w.fields[[1, 4, 12]]
        res = {}
        for name, det in (("coherent", 0), ("basis", 2)):
            o = rp.rp_default_options(precision=prec, deterministic=det,
                                      stream=torch.cuda.current_stream().cuda_stream)
            t0 = time.perf_counter()
            r = rp.rp_yields(sy.handle, fb, 200, 0, w.t_max, o, per_sample=True)
            ps = r["per_sample"][:, :, 0]
            res[name] = {"PhiS": ps.mean(1).round(6).tolist(),
                         "sigma": ps.std(1, ddof=1).round(6).tolist(),
                         "wall_s": time.perf_counter() - t0}
        ratio = [(b / c) ** 2 for b, c in zip(res["basis"]["sigma"], res["coherent"]["sigma"])]
        print(json.dumps({"mode": "basis-sampling", "workload": WORKLOAD, "fields_mT":
                          [round(float(b), 4) for b in fb], "M": 200, **res,
                          "variance_ratio_basis_over_coherent": [round(x, 3) for x in ratio]}),
              flush=True)
        return
    if args.grouped_prototype:
        # The grouped tier would apply the g innermost nuclei and both electrons
        # as one dense complex block of dimension D = 4 x 2^g: in the layout the
        # state is then a (Z / 2^g) x D complex matrix (the group's indices
        # innermost), i.e. a real (Z / 2^g) x 2D matrix X, and the block a real
        # 2D x 2D matrix; Y = X Hb^T is one plain GEMM.  Its time on the tensor
        # cores (cuBLAS) bounds what a hand-written tcgen05 version could reach.
        w3 = wl.config3()
        s3 = rp.System(w3.system)
        Z3 = s3.Z
        st = torch.cuda.current_stream()
        o = rp.rp_default_options(precision=rp.RP_FP32, profile=1, stream=st.cuda_stream)
        B3 = 10.0
        h = s3.plan(B3, w3.t_max, precision=rp.RP_FP32)["h"]
        rp.rp_yields(s3.handle, np.array([B3]), 2, 0, h, o)  # warm-up
        r = rp.rp_yields(s3.handle, np.array([B3]), 2, 0, 3 * h, o)
        per_term_ms = r["stats"]["step_ms"] / max(r["stats"]["step_launches_timed"], 1)
        row_term_us = per_term_ms * 1e3 / 2  # two rows per launch
        n_nuc = w3.system.n_nuc
        res = []
        torch.backends.cuda.matmul.allow_tf32 = True
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for g in (4, 5, 6, 8):
            D2 = 2 * 4 * (1 << g)
            cols = Z3 // (1 << g)
            X = torch.randn(cols, D2, device="cuda")
            Hb = torch.randn(D2, D2, device="cuda")
            Y = torch.empty(cols, D2, device="cuda")
            times = {}
            for name, dt in (("tf32", torch.float32), ("bf16", torch.bfloat16)):
                Xc, Hc = X.to(dt), Hb.to(dt)
                Yc = Y.to(dt)
                for _ in range(3):
                    torch.matmul(Xc, Hc.t(), out=Yc)
                ev0.record(st)
                for _ in range(10):
                    torch.matmul(Xc, Hc.t(), out=Yc)
                ev1.record(st)
                torch.cuda.synchronize()
                times[name] = ev0.elapsed_time(ev1) / 10 * 1e3  # us per GEMM
            gemm_3x = 3 * times["tf32"]
            share = g / n_nuc  # the group's share of the nuclei the per-term kernel applies
            res.append({"g": g, "block_dim_real": D2, "columns": cols,
                        "gflop_per_gemm": 2.0 * D2 * D2 * cols / 1e9,
                        "tf32_gemm_us": times["tf32"], "tf32x3_us": gemm_3x,
                        "bf16_gemm_us": times["bf16"],
                        "matrix_free_share_us": share * row_term_us,
                        "grouped_row_term_us_bound": gemm_3x + (1 - share) * row_term_us,
                        "pays": bool(gemm_3x + (1 - share) * row_term_us < row_term_us)})
            del X, Hb, Y
        torch.backends.cuda.matmul.allow_tf32 = False
        print(json.dumps({"mode": "grouped-prototype", "Z": int(Z3), "n_nuc": n_nuc,
                          "field_mT": B3, "matrix_free_row_term_us": row_term_us,
                          "results": res,
                          "note": "grouped bound = 3 TF32 GEMMs (hi.hi + hi.lo + lo.hi for the "
                                  "1e-5 FP32 bar, splits not counted) + the remaining nuclei's "
                                  "share of the measured matrix-free term; BF16 (one GEMM) "
                                  "misses the 1e-5 bar by orders of magnitude"}), flush=True)
        return
    if args.basis_aniso:
        w3 = wl.config3()
        s3 = rp.System(w3.system)
        fb = np.array([1.0, 5.0])
        T3, M3 = 1.0, 64
        res = {}
        for name, det in (("coherent", 0), ("basis", 2)):
            o = rp.rp_default_options(precision=prec, deterministic=det,
                                      stream=torch.cuda.current_stream().cuda_stream)
            t0 = time.perf_counter()
            r = rp.rp_yields(s3.handle, fb, M3, 0, T3, o, per_sample=True)
            ps = r["per_sample"][:, :, 0]
            res[name] = {"PhiS": ps.mean(1).round(6).tolist(),
                         "sigma": ps.std(1, ddof=1).round(6).tolist(),
                         "wall_s": time.perf_counter() - t0}
        ratio = [(b / c) ** 2 for b, c in zip(res["basis"]["sigma"], res["coherent"]["sigma"])]
        print(json.dumps({"mode": "basis-aniso", "workload": "config3 system (18x1/2 + 2x1, "
                          "anisotropic, J = 0.1 mT, k = 1 us^-1, Z = 2359296)", "t_max_us": T3,
                          "fields_mT": fb.tolist(), "M": M3, **res,
                          "variance_ratio_basis_over_coherent": [round(x, 3) for x in ratio],
                          "note": "the variance ratio carries a relative error of ~0.25 at "
                                  "M = 64"}), flush=True)
        return
    if args.cv_size:
        fb = np.array([1.6, 3.2, 4.8])
        o = rp.rp_default_options(precision=prec, stream=torch.cuda.current_stream().cuda_stream)
        n_max, n_test = 2400, 1000
        t0 = time.perf_counter()
        tr = rp.rp_yields(sy.handle, fb, n_max, 0, w.t_max, o, per_sample=True)
        te = rp.rp_yields(sy.handle, fb, n_test, 0,
                          w.t_max, rp.rp_default_options(precision=prec, sample_offset=1 << 30,
                                                         stream=torch.cuda.current_stream().cuda_stream),
                          per_sample=True)
        t_prop = time.perf_counter() - t0
        phi_tr, phi_te = tr["per_sample"][:, :, 0], te["per_sample"][:, :, 0]
        res = []
        for n in (150, 600, 2400):
            cv = rp.ControlVariate(sy)
            t1 = time.perf_counter()
            cv.train(np.repeat(fb, n), np.tile(np.arange(n), len(fb)), 0, phi_tr[:, :n].ravel())
            g = cv.eval(np.repeat(fb, n_test), np.tile(np.arange(n_test) + (1 << 30), len(fb)), 0)
            mu, vm = cv.mean(fb, 1 << 18, 0, pair_id=1 << 30)
            out = cv.estimate(np.arange(len(fb)) * n_test, np.full(len(fb), n_test),
                              te["per_sample"].ravel(), g, mu, vm)
            res.append({"train_per_field": n, "train_total": n * len(fb),
                        "variance_reduction": [round(float(x), 3) for x in (out[:, 3] / out[:, 1]) ** 2],
                        "beta": [round(float(x), 4) for x in out[:, 4]],
                        "train_eval_mean_s": time.perf_counter() - t1})
        print(json.dumps({"mode": "cv-size", "workload": WORKLOAD, "fields_mT": fb.tolist(),
                          "test_samples_per_field": n_test, "propagation_s": t_prop,
                          "results": res}), flush=True)
        return
    if args.config4:
        w4 = wl.config4()
        systems = [rp.System(x.system) for x in w4]
        nf = args.c4_fields
        # evenly spaced fields of each pair's 32-field sweep, both ends included
        fsel = np.unique(np.round(np.linspace(0, len(w4[0].fields) - 1, nf)).astype(int))
        fields = [x.fields[fsel] for x in w4]
        Ms = [args.c4_samples] * len(w4)
        T4 = [x.t_max for x in w4]

        def cfg_terms(sy_, x, flds, m):
            # configuration-terms (Z x Chebyshev terms) of m samples at each field
            return sum(sy_.plan(B, x.t_max, precision=prec)["n_macro"] * 88 * m * x.system.Z
                       for B in flds)
        sub = sum(cfg_terms(s_, x, f, m) for s_, x, f, m in zip(systems, w4, fields, Ms))
        full = sum(cfg_terms(s_, x, x.fields, x.M) for s_, x in zip(systems, w4))
        o = rp.rp_default_options(precision=prec, profile=1,
                                  stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = rp.rp_yields_batch(systems, fields, Ms, T4, 4, o)
        wall = time.perf_counter() - t0
        st = r["stats"]
        Zs = np.array([x.system.Z for x in w4])
        print(json.dumps({
            "mode": "config4", "pairs": len(w4), "Z_range": [int(Zs.min()), int(Zs.max())],
            "fields_per_pair": int(len(fsel)), "samples": args.c4_samples,
            "propagations": int(st["propagations"]), "row_terms": int(st["row_terms"]),
            "config_terms": sub, "wall_s": wall, "device_s": st["device_ms"] * 1e-3,
            "kernel_launches": int(st["kernel_launches"]),
            "step_kernels_hbm_GBps": (st["step_bytes"] / (st["step_ms"] * 1e-3) / 1e9)
            if st["step_ms"] else None,
            "fraction_of_full_workload": sub / full,
            "full_workload_projected_s": wall * full / sub,
            "note": "projection by the exact configuration-terms of the plans (Z x Chebyshev "
                    "terms summed over pairs, fields and samples); the subset covers every "
                    "pair, so every size class and kernel path of the full workload"}),
              flush=True)
        return
    if args.table1:
        gam = 176.085963023
        s1 = wl.table1(gam)
        sy1 = rp.System(s1)
        T1 = 10.0 / min(s1.k_S, s1.k_T)  # survival e^-10 at the horizon
        B1 = np.linspace(0.0, 10.0, 21)
        M1 = 400
        o = rp.rp_default_options(precision=prec, stream=torch.cuda.current_stream().cuda_stream)
        t0 = time.perf_counter()
        r = rp.rp_yields(sy1.handle, B1, M1, 0, T1, o, per_sample=True)
        wall = time.perf_counter() - t0
        ps = r["per_sample"][:, :, 0]
        curve = {}
        for M in (100, 200, 400):
            x = ps[:, :M]
            mean, se = x.mean(1), x.std(1, ddof=1) / np.sqrt(M)
            curve[M] = {"PhiS": mean.round(6).tolist(), "SE": se.round(6).tolist(),
                        "B_min_mT": float(B1[int(np.argmin(mean))])}
        # Fig. 2: the M = 100 and M = 200 curves against the M = 400 curve, in
        # units of their own error bars (the samples are nested, so this is a
        # consistency check, not an independent test)
        ref = np.array(curve[400]["PhiS"])
        dev = {M: (np.abs(np.array(curve[M]["PhiS"]) - ref) / np.array(curve[M]["SE"])).round(3).tolist()
               for M in (100, 200)}
        hist = {}
        for b in (0.0, 3.5, 10.0):
            j = int(np.argmin(np.abs(B1 - b)))
            h, edges = np.histogram(ps[j], bins=20, range=(0.0, 1.0))
            hist[str(b)] = {"counts": h.tolist(), "mean": float(ps[j].mean()),
                            "sd": float(ps[j].std(ddof=1)), "min": float(ps[j].min()),
                            "max": float(ps[j].max())}
        print(json.dumps({"mode": "table1", "Z": int(s1.Z), "t_max_us": T1, "fields_mT": B1.tolist(),
                          "two_J_over_gamma_mT": 2 * s1.J, "M": M1, "wall_s": wall,
                          "device_ms": r["stats"]["device_ms"], "row_terms": r["stats"]["row_terms"],
                          "mean_survival": float(r["out"][:, 4].max()),
                          "M100": curve[100], "M200": curve[200], "M400": curve[400],
                          "deviation_from_M400_in_SE": dev, "hist": hist}), flush=True)
        return
    if args.trace:
        fb = w.fields[[2, 4]]
        o = rp.rp_default_options(precision=prec, stream=torch.cuda.current_stream().cuda_stream)
        sy.yields([0.0], 2, 0, 0.05)  # warm-up
        n3 = rp.rp_trace_propagations(sy.handle, 3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        o3 = rp.rp_default_options(precision=prec, deterministic=3,
                                   stream=torch.cuda.current_stream().cuda_stream)
        tr = rp.rp_yields(sy.handle, fb, 2, 0, w.t_max, o3)
        t_trace = time.perf_counter() - t0
        t0 = time.perf_counter()
        st = rp.rp_yields_converged(sy.handle, fb, SE_TARGET, M_MIN, 4000, 3, w.t_max, o)
        t_stoch = time.perf_counter() - t0
        z = (st["out"][:, 0] - tr["out"][:, 0]) / st["out"][:, 2]
        print(json.dumps({"mode": "trace", "workload": WORKLOAD, "fields_mT": fb.round(4).tolist(),
                          "precision": args.precision, "Z": int(sy.Z), "sector_propagations": n3,
                          "trace_PhiS": tr["out"][:, 0].tolist(), "trace_wall_s": t_trace,
                          "trace_row_terms": tr["stats"]["row_terms"],
                          "stochastic_PhiS": st["out"][:, 0].tolist(),
                          "stochastic_SE": st["out"][:, 2].tolist(),
                          "stochastic_M": st["M_used"].tolist(), "stochastic_wall_s": t_stoch,
                          "z_stochastic_vs_trace": z.tolist(),
                          "speedup_vs_sector_trace_measured": t_trace / t_stoch,
                          "speedup_vs_full_trace_projected": t_trace * sy.Z / n3 / t_stoch,
                          "note": "full trace (Z propagations per field) projected from the "
                                  "sector trace by the exact ratio of propagations, Z / n3; "
                                  "every propagation costs the same Chebyshev terms"}), flush=True)
        return
    if args.ncu_case5:
        w4 = [x for x in wl.config4() if x.system.Z <= 2048][:8]
        o = rp.rp_default_options(precision=rp.RP_FP32, kernel=5,
                                  stream=torch.cuda.current_stream().cuda_stream)
        r = rp.rp_yields_batch([rp.System(x.system) for x in w4], [x.fields[::8] for x in w4],
                               [8] * len(w4), [x.t_max for x in w4], 3, o)
        torch.cuda.synchronize()
        print(json.dumps({"mode": "ncu-case5", "Z": [int(x.system.Z) for x in w4],
                          "row_terms": int(r["stats"]["row_terms"]),
                          "device_ms": r["stats"]["device_ms"]}), flush=True)
        return
    if args.ncu_case3:
        w3 = wl.config3()
        s3 = rp.System(w3.system)
        o = rp.rp_default_options(precision=rp.RP_FP32, stream=torch.cuda.current_stream().cuda_stream)
        h = s3.plan(10.0, w3.t_max, precision=rp.RP_FP32)["h"]
        rp.rp_yields(s3.handle, np.array([10.0]), 2, 0, 2 * h, o)
        torch.cuda.synchronize()
        return
    if args.ncu_case:
        # config-2 system, 3 fields x 64 samples = 192 rows (127 MB per state
        # vector, ~2 GB on the device), horizon of two macro-steps at 50 mT
        o = rp.rp_default_options(precision=rp.RP_FP32, stream=torch.cuda.current_stream().cuda_stream,
                                  kernel=args.kernel)
        h50 = sy.plan(50.0, w.t_max, precision=rp.RP_FP32)["h"]
        rp.rp_yields(sy.handle, np.array([0.0, 25.0, 50.0]), 64, 0, 2 * h50, o)
        torch.cuda.synchronize()
        return
    n_f = len(w.fields)
    # two interleaved halves of the 64-field sweep; step i runs half i % 2
    halves = [np.arange(g, n_f, 2) for g in range(2)]
    m = args.samples_per_step
    stream = torch.cuda.current_stream()
    fterms = _field_terms(sy, w.fields, w.t_max, prec)
    curve_terms = sum(fterms)

    def step(i, profile):
        idx = halves[i % 2]
        o = rp.rp_default_options(precision=prec, sample_offset=(i * world + rank) * m,
                                  profile=int(profile), stream=stream.cuda_stream,
                                  kernel=args.kernel)
        t0 = time.perf_counter()
        r = rp.rp_yields(sy.handle, w.fields[idx], m, 0, w.t_max, o, per_sample=True)
        return idx, r, time.perf_counter() - t0

    for i in range(args.warmup):
        step(i, False)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # per-field sums of phi_S over the timed steps: n, sum, sum of squares
    acc = np.zeros((n_f, 3))
    dev_ms, wall_s, row_terms, launches = 0.0, 0.0, 0, 0
    step_ms, step_bytes, step_launches_timed = 0.0, 0.0, 0
    h2d = 0
    d2h = 0
    paths = set()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t_all = time.perf_counter()
        ev0.record(stream)
        for i in range(args.warmup, args.warmup + args.steps):
            idx, r, wall = step(i, True)
            st = r["stats"]
            dev_ms += st["device_ms"]
            wall_s += wall
            row_terms += st["row_terms"]
            launches += st["kernel_launches"]
            step_ms += st["step_ms"]
            step_bytes += st["step_bytes"]
            step_launches_timed += st["step_launches_timed"]
            paths.add(st["kernel_path"])
            h2d += st["h2d_bytes"] + w.fields[idx].nbytes
            d2h += st["d2h_bytes"]
            phi = r["per_sample"][:, :, 0]
            acc[idx, 0] += phi.shape[1]
            acc[idx, 1] += phi.sum(axis=1)
            acc[idx, 2] += (phi * phi).sum(axis=1)
        ev1.record(stream)
        barrier()
        t_all = time.perf_counter() - t_all
    region_ms = ev0.elapsed_time(ev1)
    clocks = clk.summary()

    # max over ranks of the timed quantities, sums of work and of the samples
    row_terms_all, launches_all = row_terms, launches
    if world > 1:
        from paper_1612_09517_gb300 import shard
        dev_ms, wall_s, region_ms, step_ms = shard.max_over_ranks(
            [dev_ms, wall_s, region_ms, step_ms]).tolist()
        work = torch.tensor([row_terms, launches], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(work, op=torch.distributed.ReduceOp.SUM)
        row_terms_all, launches_all = work[0].item(), work[1].item()
        a = torch.tensor(acc, dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(a, op=torch.distributed.ReduceOp.SUM)
        acc = a.cpu().numpy()

    sigma, sigma_src = _sigma_from_sums(acc)
    Mf = samples_per_field(sigma)
    conv_terms = sum(mf * t for mf, t in zip(Mf, fterms))
    sigma_max = max(sigma)
    m_uniform = max(2, int(math.ceil((sigma_max / SE_TARGET) ** 2)))
    rate_dev = row_terms_all / (dev_ms * 1e-3)
    rate_e2e = row_terms_all / wall_s
    value = conv_terms / rate_dev
    e2e = conv_terms / rate_e2e

    extras = rank == 0 and world == 1 and not args.no_extras
    peak, peak_src = _peaks()
    path = max(paths) if paths else 1
    n_c = r["stats"]["n_cheb"]
    if path == 4:
        # on-chip macro-steps: the Chebyshev vectors stream through shared
        # memory; algorithmic shared-memory bytes per configuration and term
        # (phi_{n-1} and phi_{n-2} of the configuration, 16 B per flip-flop
        # partner, phi_n written)
        nh = int(np.sum(w.system.two_I == 1))
        n1 = int(np.sum(w.system.two_I == 2))
        b_cfg = 96.0 + 16.0 * (nh + 4.0 / 3.0 * n1)
        sm_bytes = row_terms * (n_c - 1) / n_c * sy.Z * b_cfg
        n_sm = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
        peak_sm = n_sm * 128.0 * mhz * 1e6 / 1e9
        achieved = sm_bytes / (step_ms * 1e-3) / 1e9 if step_ms > 0 else None
        traffic = _profile_traffic("k_macro_cluster")
        rows_per_launch = row_terms / n_c / max(step_launches_timed, 1)
        roofline = {
            "bound": "smem", "kernel": "k_macro_cluster (whole macro-step, vectors in "
                                      "distributed shared memory)",
            "achieved": achieved, "peak": peak_sm, "unit": "GB/s",
            "frac": (achieved / peak_sm) if achieved else None,
            "traffic": (traffic * rows_per_launch) if traffic else None,
            "peak_source": f"derived: {n_sm} SMs x 128 B/clk x {mhz:.0f} MHz (median SM clock "
                           "in the timed region)",
            "algorithmic_bytes_per_launch": sm_bytes / max(step_launches_timed, 1),
            "algorithmic_bytes_per_config_term": b_cfg,
            "avg_launch_ms": step_ms / max(step_launches_timed, 1),
            "hbm_algorithmic_GBps": step_bytes / (step_ms * 1e-3) / 1e9 if step_ms > 0 else None,
            "hbm_peak": peak, "hbm_peak_source": peak_src,
        }
        # the kernel is bound by instruction issue (ncu: issue slots ~60 % busy
        # on the active SMs): warp instructions per second from the committed
        # per-configuration-term count against 4 issue slots per SM and clock
        instr = _profile_traffic("k_macro_cluster", "thread_instructions_per_config_term")
        if instr and step_ms > 0:
            cfg_terms = row_terms * (n_c - 1) / n_c * sy.Z
            issue = instr / 32.0 * cfg_terms / (step_ms * 1e-3)
            peak_issue = n_sm * 4 * mhz * 1e6
            roofline["issue"] = {
                "achieved": issue, "peak": peak_issue, "unit": "warp instructions/s",
                "frac": issue / peak_issue,
                "source": f"{instr:.1f} thread instructions per configuration and term (ncu, "
                          f"profiles/traffic.json) x configuration-terms / step time; peak "
                          f"{n_sm} SMs x 4 issue slots x {mhz:.0f} MHz; clusters of 8 CTAs "
                          "occupy 120 of the 152 SMs"}
    else:
        achieved = step_bytes / (step_ms * 1e-3) / 1e9 if step_ms > 0 else None
        traffic_per_row = _profile_traffic("k_cheb_step")
        avg_rows = row_terms / max(step_launches_timed, 1) / n_c * (n_c - 1) \
            if step_launches_timed else None
        # the same launches at the minimum count of 4.25 vector passes per
        # term (the accumulator read-modify-write not counted as useful)
        passes = 3.5 + 4.25 + 5.25 * (n_c - 3)
        achieved_min = achieved * 4.25 * (n_c - 1) / passes if achieved else None
        roofline = {
            "bound": "hbm", "kernel": "k_cheb_step (fused H.psi + Chebyshev term)",
            "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "achieved_min_count": achieved_min,
            "frac_min": (achieved_min / peak) if achieved_min else None,
            "min_count_note": "4.25 vector passes per term instead of the kernel's 3.5 / 5.25 / 4.25",
            "traffic": (traffic_per_row * avg_rows) if (traffic_per_row and avg_rows) else None,
            "peak_source": peak_src,
            "algorithmic_bytes_per_launch": step_bytes / max(step_launches_timed, 1),
            "avg_launch_ms": step_ms / max(step_launches_timed, 1),
        }

    # plain FP64 form on the same GPU: measured end to end on a reduced
    # workload beside the FP32 + control-variate form, and projected to the full curve
    fp64 = None
    if args.precision == "fp32" and extras:
        o64 = rp.rp_default_options(precision=rp.RP_FP64, stream=stream.cuda_stream)
        rp.rp_yields(sy.handle, w.fields[1:7], 43, 0, 0.02, o64)
        torch.cuda.synchronize()
        r64 = rp.rp_yields(sy.handle, w.fields[1:7], 43, 0, 0.2, o64)
        st64 = r64["stats"]
        rate64 = st64["row_terms"] / (st64["device_ms"] * 1e-3)
        curve64 = _curve_terms(sy, w.fields, w.t_max, rp.RP_FP64)
        t64 = m_uniform * curve64 / rate64
        fp64 = {"projected_full": {
            "time_to_converged_s": t64, "row_terms_per_s": rate64,
            "form": "FP64, one M for every field (M = (sigma_max / 1e-3)^2 from the sigma "
                    "measured in the timed steps), rate measured over 0.2 us of 258 rows",
            "ratio_ours_over_fp64_plain": value / t64}}
        fp64["measured_reduced"] = _reduced_ratio(rp, sy, w, stream)

    converged = None
    if extras:
        converged = _converged_runs(rp, sy, w, prec, stream)

    cpu = None
    if extras and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        T_sample = 0.1
        B_list = list(w.fields[[0, 21, 42, 63]])
        rate_cpu, wall_cpu, terms_cpu = cpu_oracle_throughput(cores, T_sample, B_list)
        conv_o = sum(mf * t for mf, t in zip(Mf, _oracle_field_terms(w.t_max, w.fields)))
        cpu = {"value": conv_o / rate_cpu, "unit": "s", "cores": cores,
               "kind": "oracle",
               "sample": f"{cores} spawned processes, each one (field, sample) FP64 matrix-free "
                         f"propagation over {T_sample} us (B in {[round(float(b), 1) for b in B_list]} mT); "
                         f"{rate_cpu:.0f} row-terms/s over {wall_cpu:.1f} s, extrapolated to "
                         f"the {conv_o} oracle terms of the converged curve (per-field M_f from "
                         "the sigma measured in the timed steps)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 state / f64 integrals" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "step": f"rp_yields on 32 of the 64 fields (alternate halves) x {m} "
                               "samples per rank, full 20 us horizon",
                       "samples_per_step_per_rank": m, "rows": r["stats"]["rows"],
                       "kernel_path": path,
                       "l2": "working set per step > 129 MB L2 (state vectors + singlet slices)",
                       "se_target": SE_TARGET, "sigma_source": sigma_src,
                       "sigma_max": sigma_max, "samples_converged_curve": int(sum(Mf)),
                       "terms_converged_curve": int(conv_terms),
                       "uniform_M": m_uniform,
                       "uniform_M_time_s": m_uniform * curve_terms / rate_dev,
                       "curve_terms_per_sample": curve_terms,
                       "row_terms_per_s": rate_dev, "timed_region_ms": region_ms},
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": int(h2d / max(args.steps, 1)),
                    "d2h_bytes_per_step": int(d2h / max(args.steps, 1))},
            "gpu_launches": int(launches_all),
            "roofline": roofline,
            "clocks": clocks,
            "converged_measured": converged,
            "fp64_plain": fp64,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _sigma_from_sums(acc):
    """Per-field sample standard deviation of phi_S (M - 1 denominator) from
    (n, sum, sum of squares); a field without two samples takes its nearest
    measured neighbour's value."""
    import numpy as np
    n, s1, s2 = acc[:, 0], acc[:, 1], acc[:, 2]
    sig = np.full(len(n), np.nan)
    ok = n >= 2
    sig[ok] = np.sqrt(np.maximum(s2[ok] - s1[ok] ** 2 / n[ok], 0.0) / (n[ok] - 1))
    src = (f"measured in the timed steps: {int(n[ok].min()) if ok.any() else 0}-"
           f"{int(n.max())} samples per field")
    if not ok.all():
        good = np.flatnonzero(ok)
        for f in np.flatnonzero(~ok):
            sig[f] = sig[good[np.argmin(np.abs(good - f))]]
        src += f"; {int((~ok).sum())} fields without samples take the nearest field's value"
    return [float(x) for x in sig], src


def _converged_runs(rp, sy, w, prec, stream):
    """The converged 64-field curve measured end to end through the C ABI:
    rp_yields_converged (plain, per-field sample counts) and rp_yields_cv (the
    learned control variate where it pays); seed 7 (directions independent of
    the timed steps)."""
    import torch
    out = {}
    o = rp.rp_default_options(precision=prec, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = rp.rp_yields_converged(sy.handle, w.fields, SE_TARGET, M_MIN, 4000, 7, w.t_max, o)
    wall = time.perf_counter() - t0
    out["plain"] = {"wall_s": wall, "device_s": r["stats"]["device_ms"] * 1e-3,
                    "samples": int(r["M_used"].sum()), "max_SE": float(r["out"][:, 2].max()),
                    "row_terms": r["stats"]["row_terms"], "kernel_path": r["stats"]["kernel_path"]}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c = rp.rp_yields_cv(sy.handle, w.fields, SE_TARGET, M_MIN, 4000, 7, w.t_max, o,
                        rp.rp_cv_default_plan())
    wall = time.perf_counter() - t0
    out["cv"] = {"wall_s": wall, "samples_plain": int(c["M_plain"].sum()),
                 "samples_cv": int(c["M_cv"].sum()), "max_SE": float(c["out"][:, 1].max()),
                 "fields_with_cv": int(c["out"][:, 7].sum()),
                 "control_variate_s": c["stats"]["cv_ms"] * 1e-3,
                 "control_variate_share": c["stats"]["cv_ms"] * 1e-3 / wall}
    out["note"] = ("one run each, after the timed steps, 64 fields to SE <= 1e-3 (Eq. 23); "
                   "wall time of the C-ABI call")
    return out


def _reduced_ratio(rp, sy, w, stream):
    """The ratio the goal names, measured end to end on a reduced workload:
    the four fields 0.79-3.17 mT of the sweep over t_max = 1 us to SE <= 1e-3,
    FP32 + control variate (rp_yields_cv) against the plain FP64 form
    (rp_yields_converged in FP64), and plain FP32 beside them."""
    import torch
    fields = w.fields[1:5]
    T = 1.0
    res = {"workload": "config-2 system, fields " + str([round(float(b), 3) for b in fields]) +
                       " mT, t_max = 1 us, SE <= 1e-3 at every field"}
    for name, prec, cv in (("fp64_plain", rp.RP_FP64, False), ("fp32_plain", rp.RP_FP32, False),
                           ("fp32_cv", rp.RP_FP32, True)):
        o = rp.rp_default_options(precision=prec, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if cv:
            r = rp.rp_yields_cv(sy.handle, fields, SE_TARGET, M_MIN, 4000, 11, T, o,
                                rp.rp_cv_default_plan())
            se = float(r["out"][:, 1].max())
        else:
            r = rp.rp_yields_converged(sy.handle, fields, SE_TARGET, M_MIN, 4000, 11, T, o)
            se = float(r["out"][:, 2].max())
        res[name] = {"wall_s": time.perf_counter() - t0, "max_SE": se}
    res["ratio_fp32_cv_over_fp64_plain"] = res["fp32_cv"]["wall_s"] / res["fp64_plain"]["wall_s"]
    res["ratio_fp32_plain_over_fp64_plain"] = (res["fp32_plain"]["wall_s"] /
                                               res["fp64_plain"]["wall_s"])
    return res


if __name__ == "__main__":
    main()
