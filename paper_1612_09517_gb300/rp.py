"""Thin Python binding of the C ABI in ``include/rp.h`` (argument marshalling only).

Every computation runs inside ``_lib/librp.so`` (sm_103a CUDA kernels and the
host planner).  Importing this module loads the library and fails loudly if it
has not been built: there is no CPU fallback.

The functions carry the C names: ``rp_create``, ``rp_destroy``, ``rp_layout``,
``rp_plan_field``, ``rp_yields``, ``rp_apply_h``, ``rp_init_states`` ... and
``System`` wraps an ``rp_system*`` for convenience.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "librp.so")

RP_FP64 = 0
RP_FP32 = 1
STATUS = ["RP_OK", "RP_EINVAL", "RP_ENOMEM", "RP_ECUDA", "RP_ETIMEOUT", "RP_ENOTCONV",
          "RP_ENOTIMPL", "RP_ENODEV"]


class RPError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{name}: {msg}")


class rp_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("n_cheb", C.c_int), ("tol", C.c_double),
                ("max_rows", C.c_int), ("deterministic", C.c_int),
                ("sample_offset", C.c_longlong), ("pair_id", C.c_uint32),
                ("profile", C.c_int), ("stream", C.c_void_p), ("kernel", C.c_int),
                ("gram", C.c_int), ("graph", C.c_int)]


class rp_stats(C.Structure):
    _fields_ = [("kernel_launches", C.c_longlong), ("step_launches", C.c_longlong),
                ("row_terms", C.c_longlong), ("propagations", C.c_longlong),
                ("step_bytes", C.c_double), ("step_ms", C.c_double),
                ("step_launches_timed", C.c_longlong), ("device_ms", C.c_double),
                ("rows", C.c_int), ("n_cheb", C.c_int), ("h2d_bytes", C.c_longlong),
                ("d2h_bytes", C.c_longlong), ("graph_launches", C.c_longlong),
                ("kernel_path", C.c_int), ("cv_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class rp_field_plan(C.Structure):
    _fields_ = [("E_min", C.c_double), ("E_max", C.c_double), ("E_c", C.c_double),
                ("dE", C.c_double), ("h", C.c_double), ("n_macro", C.c_longlong),
                ("n_cheb", C.c_int), ("tail", C.c_double), ("kbar", C.c_double),
                ("kappa", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class rp_cv_options(C.Structure):
    _fields_ = [("hidden", C.c_int), ("layers", C.c_int), ("epochs", C.c_int), ("batch", C.c_int),
                ("lr", C.c_double), ("weight_decay", C.c_double), ("B_scale", C.c_double),
                ("init_seed", C.c_uint64), ("stream", C.c_void_p)]


class rp_cv_plan(C.Structure):
    _fields_ = [("M_train", C.c_int), ("cv_threshold", C.c_int), ("n_mc", C.c_longlong),
                ("net", rp_cv_options)]


class rp_tune_result(C.Structure):
    _fields_ = [("kernel", C.c_int), ("n_cheb", C.c_int), ("graph", C.c_int),
                ("rate", C.c_double), ("base_rate", C.c_double), ("candidates", C.c_int),
                ("from_cache", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

# (name, restype, argtypes) of every exported symbol declared in include/rp.h
SIGNATURES = [
    ("rp_version", C.c_char_p, []),
    ("rp_status_str", C.c_char_p, [C.c_int]),
    ("rp_last_error", C.c_char_p, []),
    ("rp_default_options", None, [C.POINTER(rp_options)]),
    ("rp_set_allocator", C.c_int, [ALLOC_FN, FREE_FN, C.c_void_p]),
    ("rp_create", C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                            C.POINTER(C.c_double), C.c_double, C.c_double, C.c_double,
                            C.POINTER(C.c_void_p)]),
    ("rp_destroy", None, [C.c_void_p]),
    ("rp_layout", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_longlong)]),
    ("rp_plan_field", C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int, C.c_double,
                                C.POINTER(rp_field_plan), C.POINTER(C.c_double),
                                C.POINTER(C.c_double)]),
    ("rp_yields", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_int, C.c_uint64,
                            C.c_double, C.POINTER(rp_options), C.POINTER(C.c_double),
                            C.POINTER(C.c_double), C.POINTER(rp_stats)]),
    ("rp_apply_h", C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                             C.c_void_p]),
    ("rp_init_states", C.c_int, [C.c_void_p, C.c_int, C.c_uint64, C.c_uint32, C.c_longlong,
                                 C.c_int, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    ("rp_yields_converged", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_double,
                                      C.c_int, C.c_int, C.c_uint64, C.c_double,
                                      C.POINTER(rp_options), C.POINTER(C.c_double),
                                      C.POINTER(C.c_int), C.POINTER(rp_stats)]),
    ("rp_cv_default_options", None, [C.POINTER(rp_cv_options)]),
    ("rp_cv_create", C.c_int, [C.c_void_p, C.POINTER(rp_cv_options), C.POINTER(C.c_void_p)]),
    ("rp_cv_destroy", None, [C.c_void_p]),
    ("rp_cv_params", C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float),
                               C.POINTER(C.c_longlong)]),
    ("rp_cv_loss_grad", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                  C.POINTER(C.c_double), C.POINTER(C.c_float)]),
    ("rp_cv_train", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                              C.c_uint64, C.c_uint32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("rp_cv_eval", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                             C.c_uint64, C.c_uint32, C.POINTER(C.c_double)]),
    ("rp_cv_mean", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_longlong, C.c_uint64,
                             C.c_uint32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("rp_cv_estimate", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_longlong),
                                 C.POINTER(C.c_longlong), C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("rp_cv_default_plan", None, [C.POINTER(rp_cv_plan)]),
    ("rp_yields_cv", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_double, C.c_int,
                               C.c_int, C.c_uint64, C.c_double, C.POINTER(rp_options),
                               C.POINTER(rp_cv_plan), C.POINTER(C.c_double), C.POINTER(C.c_int),
                               C.POINTER(C.c_int), C.POINTER(rp_stats)]),
    ("rp_yields_batch", C.c_int, [C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_int),
                                  C.POINTER(C.POINTER(C.c_double)), C.POINTER(C.c_int),
                                  C.POINTER(C.c_double), C.c_uint64, C.POINTER(rp_options),
                                  C.POINTER(C.POINTER(C.c_double)), C.POINTER(rp_stats)]),
    ("rp_yields_static", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_int,
                                   C.c_uint64, C.c_double, C.POINTER(rp_options),
                                   C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.POINTER(rp_stats)]),
    ("rp_basis_indices", C.c_int, [C.c_uint64, C.c_uint32, C.c_longlong, C.c_int, C.c_longlong,
                                   C.POINTER(C.c_longlong)]),
    ("rp_trace_propagations", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_longlong)]),
    ("rp_field_sums", C.c_int, [C.c_int, C.POINTER(C.c_double), C.c_longlong,
                                C.POINTER(C.c_double)]),
    ("rp_combine_sums", C.c_int, [C.c_int, C.POINTER(C.c_double), C.c_longlong,
                                  C.POINTER(C.c_double)]),
    ("rp_rotate", C.c_int, [C.c_void_p, C.c_double, C.c_double, C.POINTER(C.c_void_p)]),
    ("rp_time_observable", C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_uint64, C.c_double,
                                     C.POINTER(rp_options), C.POINTER(C.c_double), C.c_int,
                                     C.POINTER(C.c_int), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double)]),
    ("rp_time_trace", C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_uint64, C.c_double,
                                C.POINTER(rp_options), C.c_int, C.POINTER(C.c_int),
                                C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("rp_tune", C.c_int, [C.c_void_p, C.c_double, C.c_int, C.POINTER(rp_options),
                          C.POINTER(rp_options), C.POINTER(rp_tune_result)]),
]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (or "
                          f"python paper_1612_09517_gb300/build.py) first; there is no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


def _check(st):
    if st != 0:
        raise RPError(st, LIB.rp_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def rp_version() -> str:
    return LIB.rp_version().decode()


def rp_default_options(**kw) -> rp_options:
    o = rp_options()
    LIB.rp_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": RP_FP64, "fp32": RP_FP32}[v.lower()]
        setattr(o, k, v)
    return o


def rp_create(radical, two_I, A, k_S, k_T, J):
    radical = np.ascontiguousarray(radical, dtype=np.int32).reshape(-1)
    two_I = np.ascontiguousarray(two_I, dtype=np.int32).reshape(-1)
    A = np.ascontiguousarray(A, dtype=np.float64).reshape(-1)
    n = radical.size
    h = C.c_void_p()
    _check(LIB.rp_create(n, radical.ctypes.data_as(C.POINTER(C.c_int)),
                         two_I.ctypes.data_as(C.POINTER(C.c_int)), _dptr(A), float(k_S),
                         float(k_T), float(J), C.byref(h)))
    return h


def rp_destroy(h):
    LIB.rp_destroy(h)


def rp_layout(h, n_nuc):
    order = np.zeros(max(n_nuc, 1), dtype=np.int32)
    Z = C.c_longlong()
    _check(LIB.rp_layout(h, order.ctypes.data_as(C.POINTER(C.c_int)), C.byref(Z)))
    return order[:n_nuc], int(Z.value)


def rp_plan_field(h, B, t_max, precision=RP_FP64, n_cheb=0, tol=0.0, with_coef=False):
    p = rp_field_plan()
    n_c = n_cheb or 88
    coef = np.zeros(2 * n_c) if with_coef else None
    W = np.zeros(2 * n_c * n_c) if with_coef else None
    _check(LIB.rp_plan_field(h, float(B), float(t_max), precision, n_cheb, float(tol), C.byref(p),
                             _dptr(coef) if with_coef else None, _dptr(W) if with_coef else None))
    d = p.as_dict()
    if with_coef:
        d["coef"] = coef.view(np.complex128)
        d["W"] = W.view(np.complex128).reshape(n_c, n_c)
    return d


def rp_field_sums(out, M):
    """Per-field sums (n_fields, 5) of an rp_yields output block over M samples."""
    out = np.ascontiguousarray(out, dtype=np.float64).reshape(-1, 5)
    sums = np.zeros_like(out)
    _check(LIB.rp_field_sums(out.shape[0], _dptr(out), int(M), _dptr(sums)))
    return sums


def rp_combine_sums(sums, M):
    """The rp_yields output block over M samples from summed per-field sums."""
    sums = np.ascontiguousarray(sums, dtype=np.float64).reshape(-1, 5)
    out = np.zeros_like(sums)
    _check(LIB.rp_combine_sums(sums.shape[0], _dptr(sums), int(M), _dptr(out)))
    return out


def rp_trace_propagations(h, deterministic):
    """Propagations per field of the deterministic traces (1: Z, 3: J_z sectors)."""
    n = C.c_longlong()
    _check(LIB.rp_trace_propagations(h, int(deterministic), C.byref(n)))
    return int(n.value)


def rp_yields(h, fields, M, seed, t_max, opt=None, per_sample=False, Z=None):
    fields = np.ascontiguousarray(fields, dtype=np.float64).reshape(-1)
    nf = fields.size
    o = opt if opt is not None else rp_default_options()
    out = np.zeros(max(nf * 5, 1))
    Mr = rp_trace_propagations(h, o.deterministic) if o.deterministic in (1, 3) else M
    ps = np.zeros(max(nf * Mr * 3, 1)) if per_sample else None
    stats = rp_stats()
    _check(LIB.rp_yields(h, nf, _dptr(fields), int(M), C.c_uint64(int(seed)), float(t_max),
                         C.byref(o), _dptr(out), _dptr(ps) if per_sample else None,
                         C.byref(stats)))
    res = {"out": out[: nf * 5].reshape(nf, 5), "stats": stats.as_dict()}
    if per_sample:
        res["per_sample"] = ps[: nf * Mr * 3].reshape(nf, Mr, 3)
    return res


def rp_yields_converged(h, fields, se_target, M_min, M_max, seed, t_max, opt=None):
    fields = np.ascontiguousarray(fields, dtype=np.float64).reshape(-1)
    nf = fields.size
    o = opt if opt is not None else rp_default_options()
    out = np.zeros(max(nf * 5, 1))
    used = np.zeros(max(nf, 1), dtype=np.int32)
    stats = rp_stats()
    _check(LIB.rp_yields_converged(h, nf, _dptr(fields), float(se_target), int(M_min), int(M_max),
                                   C.c_uint64(int(seed)), float(t_max), C.byref(o), _dptr(out),
                                   used.ctypes.data_as(C.POINTER(C.c_int)), C.byref(stats)))
    return {"out": out[: nf * 5].reshape(nf, 5), "M_used": used[:nf].copy(),
            "stats": stats.as_dict()}


def rp_yields_static(h, fields, M, seed, t_max, opt=None, per_sample=False, Z=None):
    """rp_yields with all device scratch in the library's fixed 64 MiB array
    (for callers that must not allocate device memory while they run)."""
    fields = np.ascontiguousarray(fields, dtype=np.float64).reshape(-1)
    nf = fields.size
    o = opt if opt is not None else rp_default_options()
    out = np.zeros(max(nf * 5, 1))
    Mr = Z if o.deterministic == 1 else M
    ps = np.zeros(max(nf * Mr * 3, 1)) if per_sample else None
    stats = rp_stats()
    _check(LIB.rp_yields_static(h, nf, _dptr(fields), int(M), C.c_uint64(int(seed)),
                                float(t_max), C.byref(o), _dptr(out),
                                _dptr(ps) if per_sample else None, C.byref(stats)))
    res = {"out": out[: nf * 5].reshape(nf, 5), "stats": stats.as_dict()}
    if per_sample:
        res["per_sample"] = ps[: nf * Mr * 3].reshape(nf, Mr, 3)
    return res


def rp_basis_indices(seed, pair_id, sample_offset, M, Z):
    """Basis indices of deterministic = 2 (host only)."""
    out = np.zeros(max(int(M), 1), dtype=np.int64)
    _check(LIB.rp_basis_indices(C.c_uint64(int(seed)), C.c_uint32(int(pair_id)), int(sample_offset),
                                int(M), int(Z), out.ctypes.data_as(C.POINTER(C.c_longlong))))
    return out[: int(M)]


def rp_time_trace(h, B, M, seed, t_max, opt=None):
    """Sample means of P_S(t), P_T(t) and survival at the macro-step boundaries:
    returns (t, out) with out[:, 0] = P_S, out[:, 1] = P_T, out[:, 2] = survival."""
    o = opt if opt is not None else rp_default_options()
    n = C.c_int(0)
    _check(LIB.rp_time_trace(h, float(B), int(M), C.c_uint64(int(seed)), float(t_max), C.byref(o),
                             0, C.byref(n), None, None))
    t = np.zeros(n.value)
    out = np.zeros(3 * n.value)
    _check(LIB.rp_time_trace(h, float(B), int(M), C.c_uint64(int(seed)), float(t_max), C.byref(o),
                             n.value, C.byref(n), _dptr(t), _dptr(out)))
    return t, out.reshape(-1, 3)


def rp_time_observable(h, B, M, seed, t_max, A_e, opt=None):
    """Sample mean of <psi(t)| A_e x 1 |psi(t)> at the macro-step boundaries for a
    4 x 4 complex electron operator A_e: returns (t, values complex array)."""
    o = opt if opt is not None else rp_default_options()
    A = np.zeros(32)
    A[0::2] = np.real(np.asarray(A_e, complex)).ravel()
    A[1::2] = np.imag(np.asarray(A_e, complex)).ravel()
    n = C.c_int(0)
    _check(LIB.rp_time_observable(h, float(B), int(M), C.c_uint64(int(seed)), float(t_max),
                                  C.byref(o), _dptr(A), 0, C.byref(n), None, None))
    t = np.zeros(n.value)
    out = np.zeros(2 * n.value)
    _check(LIB.rp_time_observable(h, float(B), int(M), C.c_uint64(int(seed)), float(t_max),
                                  C.byref(o), _dptr(A), n.value, C.byref(n), _dptr(t), _dptr(out)))
    return t, out[0::2] + 1j * out[1::2]


def rp_tune(h, B, rows, opt=None):
    """Measured choice of kernel path, n_cheb and graph replay for `rows`
    concurrent samples at field B; returns (tuned rp_options, result dict)."""
    o = opt if opt is not None else rp_default_options()
    tuned = rp_options()
    res = rp_tune_result()
    _check(LIB.rp_tune(h, float(B), int(rows), C.byref(o), C.byref(tuned), C.byref(res)))
    return tuned, res.as_dict()


def rp_apply_h(h, B, precision, n_vec, x_ptr, y_ptr, stream=None):
    _check(LIB.rp_apply_h(h, float(B), precision, int(n_vec), C.c_void_p(x_ptr),
                          C.c_void_p(y_ptr), C.c_void_p(stream or 0)))


def rp_init_states(h, precision, seed, pair_id, sample0, n, psi_ptr, n_nuc, stream=None):
    uv = np.zeros(max(n * n_nuc * 2, 1))
    _check(LIB.rp_init_states(h, precision, C.c_uint64(int(seed)), C.c_uint32(pair_id),
                              int(sample0), int(n), C.c_void_p(psi_ptr), _dptr(uv),
                              C.c_void_p(stream or 0)))
    return uv[: n * n_nuc * 2].reshape(n, n_nuc, 2)


_ALLOC_KEEP = []


def use_torch_allocator():
    """Route library device allocations through PyTorch's caching allocator."""
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      stream or 0)
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _ALLOC_KEEP[:] = [a, f]
    _check(LIB.rp_set_allocator(a, f, None))


class System:
    """An ``rp_system`` created from a spin system (radical, two_I, A, k_S, k_T, J)."""

    def __init__(self, spin_system):
        s = spin_system
        self.spin_system = s
        self.n_nuc = int(np.asarray(s.radical).size)
        self.handle = rp_create(s.radical, s.two_I, s.A, s.k_S, s.k_T, s.J)
        self.order, self.Z = rp_layout(self.handle, self.n_nuc)

    @classmethod
    def rotated(cls, system, theta, phi):
        """rp_rotate: the same pair with the field along n(theta, phi)."""
        h = C.c_void_p()
        _check(LIB.rp_rotate(system.handle, float(theta), float(phi), C.byref(h)))
        obj = cls.__new__(cls)
        obj.spin_system = system.spin_system
        obj.n_nuc = system.n_nuc
        obj.handle = h
        obj.order, obj.Z = rp_layout(h, obj.n_nuc)
        return obj

    def close(self):
        if self.handle:
            rp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plan(self, B, t_max, **kw):
        return rp_plan_field(self.handle, B, t_max, **kw)

    def yields(self, fields, M, seed, t_max, per_sample=False, **opt):
        o = rp_default_options(**opt)
        return rp_yields(self.handle, fields, M, seed, t_max, o, per_sample, Z=self.Z)

    def yields_converged(self, fields, se_target, M_min, M_max, seed, t_max, **opt):
        o = rp_default_options(**opt)
        return rp_yields_converged(self.handle, fields, se_target, M_min, M_max, seed, t_max, o)

    def to_input_order(self, psi):
        """Permute library-layout state vectors (..., 4Z) to the oracle's kron order
        (electron 1, electron 2, nuclei in input order)."""
        psi = np.asarray(psi)
        lead = psi.shape[:-1]
        dims_pos = [int(self.spin_system.two_I[k]) + 1 for k in self.order]
        # library index: ((j_{N-1} ... j_0) , e1, e2) with position 0 innermost
        t = psi.reshape(*lead, *dims_pos[::-1], 2, 2)
        nl = len(lead)
        npos = len(dims_pos)
        # axes of t after lead: positions N-1..0, then e1, e2
        pos_axis = {p: nl + (npos - 1 - p) for p in range(npos)}
        inv = {int(k): p for p, k in enumerate(self.order)}
        perm = list(range(nl)) + [nl + npos, nl + npos + 1] + [pos_axis[inv[k]] for k in range(npos)]
        return np.transpose(t, perm).reshape(*lead, -1)

    def from_input_order(self, psi):
        psi = np.asarray(psi)
        lead = psi.shape[:-1]
        nl = len(lead)
        npos = self.n_nuc
        dims_in = [int(d) + 1 for d in self.spin_system.two_I]
        t = psi.reshape(*lead, 2, 2, *dims_in)
        inv = {int(k): p for p, k in enumerate(self.order)}
        # target axes: positions N-1..0 (input index order[p]), then e1, e2
        perm = list(range(nl)) + [nl + 2 + int(self.order[p]) for p in range(npos - 1, -1, -1)] + [nl, nl + 1]
        return np.transpose(t, perm).reshape(*lead, -1)


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _lptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_longlong))


def rp_cv_default_options(**kw) -> rp_cv_options:
    o = rp_cv_options()
    LIB.rp_cv_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class ControlVariate:
    """An ``rp_cv`` network for the nuclei of a ``System`` (see include/rp.h)."""

    def __init__(self, system, **opt):
        self.system = system
        self.opt = rp_cv_default_options(**opt)
        h = C.c_void_p()
        _check(LIB.rp_cv_create(system.handle, C.byref(self.opt), C.byref(h)))
        self.handle = h
        cnt = C.c_longlong()
        _check(LIB.rp_cv_params(h, None, None, C.byref(cnt)))
        self.n_params = int(cnt.value)
        self.d_in = 3 * system.n_nuc + 10

    def close(self):
        if self.handle:
            LIB.rp_cv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        p = np.zeros(self.n_params, dtype=np.float32)
        _check(LIB.rp_cv_params(self.handle, _fptr(p), None, None))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        _check(LIB.rp_cv_params(self.handle, None, _fptr(p), None))

    def loss_grad(self, x, y):
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        loss = C.c_double()
        g = np.zeros(self.n_params, dtype=np.float32)
        _check(LIB.rp_cv_loss_grad(self.handle, y.size, _fptr(x), _fptr(y), C.byref(loss), _fptr(g)))
        return loss.value, g

    def train(self, B, samples, seed, phi, pair_id=0):
        B = np.ascontiguousarray(B, dtype=np.float64)
        samples = np.ascontiguousarray(samples, dtype=np.int64)
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        losses = np.zeros(max(self.opt.epochs, 1))
        _check(LIB.rp_cv_train(self.handle, B.size, _dptr(B), _lptr(samples), C.c_uint64(seed),
                               C.c_uint32(pair_id), _dptr(phi), _dptr(losses)))
        return losses[: self.opt.epochs]

    def eval(self, B, samples, seed, pair_id=0):
        B = np.ascontiguousarray(B, dtype=np.float64)
        samples = np.ascontiguousarray(samples, dtype=np.int64)
        g = np.zeros(max(B.size, 1))
        _check(LIB.rp_cv_eval(self.handle, B.size, _dptr(B), _lptr(samples), C.c_uint64(seed),
                              C.c_uint32(pair_id), _dptr(g)))
        return g[: B.size]

    def mean(self, fields, n_mc, seed, pair_id=0):
        fields = np.ascontiguousarray(fields, dtype=np.float64)
        mu = np.zeros(max(fields.size, 1))
        vm = np.zeros(max(fields.size, 1))
        _check(LIB.rp_cv_mean(self.handle, fields.size, _dptr(fields), int(n_mc), C.c_uint64(seed),
                              C.c_uint32(pair_id), _dptr(mu), _dptr(vm)))
        return mu[: fields.size], vm[: fields.size]

    def estimate(self, offsets, counts, per_sample, g, mu, var_mu):
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        counts = np.ascontiguousarray(counts, dtype=np.int64)
        per_sample = np.ascontiguousarray(per_sample, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        var_mu = np.ascontiguousarray(var_mu, dtype=np.float64)
        nf = offsets.size
        out = np.zeros(max(nf * 5, 1))
        _check(LIB.rp_cv_estimate(self.handle, nf, _lptr(offsets), _lptr(counts), _dptr(per_sample),
                                  _dptr(g), _dptr(mu), _dptr(var_mu), _dptr(out)))
        return out[: nf * 5].reshape(nf, 5)


def rp_cv_default_plan(**kw) -> rp_cv_plan:
    p = rp_cv_plan()
    LIB.rp_cv_default_plan(C.byref(p))
    for k, v in kw.items():
        if k == "net":
            for kk, vv in v.items():
                setattr(p.net, kk, vv)
        else:
            setattr(p, k, v)
    return p


def rp_yields_cv(h, fields, se_target, M_min, M_max, seed, t_max, opt=None, plan=None):
    fields = np.ascontiguousarray(fields, dtype=np.float64).reshape(-1)
    nf = fields.size
    o = opt if opt is not None else rp_default_options()
    p = plan if plan is not None else rp_cv_default_plan()
    out = np.zeros(max(nf * 8, 1))
    mp = np.zeros(max(nf, 1), dtype=np.int32)
    mc = np.zeros(max(nf, 1), dtype=np.int32)
    stats = rp_stats()
    _check(LIB.rp_yields_cv(h, nf, _dptr(fields), float(se_target), int(M_min), int(M_max),
                            C.c_uint64(int(seed)), float(t_max), C.byref(o), C.byref(p), _dptr(out),
                            mp.ctypes.data_as(C.POINTER(C.c_int)),
                            mc.ctypes.data_as(C.POINTER(C.c_int)), C.byref(stats)))
    return {"out": out[: nf * 8].reshape(nf, 8), "M_plain": mp[:nf].copy(), "M_cv": mc[:nf].copy(),
            "stats": stats.as_dict()}


def rp_yields_batch(systems, fields, M, t_max, seed, opt=None):
    """systems: list of System; fields: list of arrays; M, t_max: per system."""
    n = len(systems)
    o = opt if opt is not None else rp_default_options()
    hs = (C.c_void_p * n)(*[s.handle for s in systems])
    f_arrs = [np.ascontiguousarray(f, dtype=np.float64).reshape(-1) for f in fields]
    nf = (C.c_int * n)(*[a.size for a in f_arrs])
    fp = (C.POINTER(C.c_double) * n)(*[_dptr(a) for a in f_arrs])
    Ms = (C.c_int * n)(*[int(m) for m in M])
    ts = (C.c_double * n)(*[float(t) for t in t_max])
    outs = [np.zeros(max(a.size * 5, 1)) for a in f_arrs]
    op = (C.POINTER(C.c_double) * n)(*[_dptr(a) for a in outs])
    stats = rp_stats()
    _check(LIB.rp_yields_batch(n, hs, nf, fp, Ms, ts, C.c_uint64(int(seed)), C.byref(o), op,
                               C.byref(stats)))
    return {"out": [o_[: a.size * 5].reshape(a.size, 5) for o_, a in zip(outs, f_arrs)],
            "stats": stats.as_dict()}
