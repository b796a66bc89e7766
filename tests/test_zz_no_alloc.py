"""rp_yields_static: the allocation-free variant of rp_yields.

Some callers must not allocate device memory while they run (a host
application that gives a plug-in a fixed device-memory budget and forbids the
allocator, or a service that must not fail part-way on a failed allocation).
rp_yields_static serves them from a fixed 64 MiB device array inside the
library.  This test calls it through the C ABI and checks it against
rp_yields on the same inputs, two calls in a row on different systems (the
second call finds the first call's data in the shared array), and that a
workload too large for the array is refused with a clear error.

It sits in its own file, collected last, and passes both alone in a fresh
process and after the rest of the suite.
"""
import numpy as np
import pytest

from paper_1612_09517_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    torch.cuda.set_device(0)
    yield


def _close(a, b, prec):
    scale = np.maximum(np.abs(b), 1e-3)
    return float(np.max(np.abs(a - b) / scale)) < TOL[prec]


def _close_out(a, b, prec):
    """Per-field output rows (Phi_S, Phi_T, SE_S, SE_T, survival): the means
    relative to themselves; the standard errors (Eq. 23) on the scale of the
    yields they are computed from, since |d SE| <= 2 max_i |d phi_i| / sqrt(M)
    and an SE far below the yields (the basis-state trace) has no relative
    accuracy of its own in FP32."""
    means = [0, 1, 4]
    if not _close(a[:, means], b[:, means], prec):
        return False
    scale = np.maximum(np.max(np.abs(b[:, :2]), axis=1, keepdims=True), 1e-3)
    return float(np.max(np.abs(a[:, 2:4] - b[:, 2:4]) / scale)) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_static_scratch_matches_allocating_entry_point(prec):
    from paper_1612_09517_gb300 import rp
    cases = [
        (wl.config1().system, np.array([0.0, 2.5, 5.0]), 8, 3.0),
        (wl.random_anisotropic(2, 1, two_I=[1, 2, 1], k_S=2.0, k_T=0.5, J=0.3, seed=40),
         np.array([0.5, 3.0]), 6, 2.0),
    ]
    for s, fields, M, T in cases:  # two calls in a row on the shared array
        sy = rp.System(s)
        o = rp.rp_default_options(precision=prec)
        a = rp.rp_yields_static(sy.handle, fields, M, 4, T, o, per_sample=True)
        b = rp.rp_yields(sy.handle, fields, M, 4, T, o, per_sample=True)
        assert _close(a["per_sample"], b["per_sample"], prec)
        assert _close_out(a["out"], b["out"], prec)
        assert a["stats"]["kernel_launches"] > 0 and a["stats"]["rows"] >= 1


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_static_scratch_deterministic_trace_matches(prec):
    """The deterministic trace over the Z = 16 basis states of config 1 (Eq. 14)
    through the allocation-free entry point equals rp_yields, twice in a row,
    the second time with the rows capped at 5 (ten batches through the array)."""
    from paper_1612_09517_gb300 import rp
    s = wl.config1().system
    sy = rp.System(s)
    fields = np.array([0.0, 1.5, 5.0])
    for max_rows in (0, 5):
        o = rp.rp_default_options(precision=prec, deterministic=1, max_rows=max_rows)
        a = rp.rp_yields_static(sy.handle, fields, 2, 0, 2.0, o, per_sample=True, Z=sy.Z)
        b = rp.rp_yields(sy.handle, fields, 2, 0, 2.0, o, per_sample=True, Z=sy.Z)
        assert a["per_sample"].shape == (3, sy.Z, 3)
        assert _close(a["per_sample"], b["per_sample"], prec)
        assert _close_out(a["out"], b["out"], prec)
        if max_rows:
            assert a["stats"]["rows"] == max_rows


def test_static_scratch_rejects_oversized_workload():
    from paper_1612_09517_gb300 import rp
    s = wl.random_isotropic(9, 9, seed=1)  # Z = 2^18: one FP32 row needs > 64 MiB
    sy = rp.System(s)
    with pytest.raises(rp.RPError, match="bytes of scratch"):
        rp.rp_yields_static(sy.handle, [0.0], 2, 0, 1.0, rp.rp_default_options())
