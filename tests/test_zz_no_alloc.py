"""hot_field_noalloc: the allocation-free forward-field entry point.

Callers that cannot allocate device memory (a real-time frame loop with pre-planned memory,
an external pool that owns every allocation) evaluate the trap fields through this entry
point; its working memory is a fixed device array inside the library.  These tests call it
through the C ABI and compare it with the context path (hot_set_traps, hot_set_phase,
hot_gsw(0), hot_get_fields) and with the FP64 oracle's Eq. 1, twice in a row so that a second
call on the reused scratch array is covered, and once more without the e/u output on a side
stream ordered after the previous call.  The file name sorts last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_0907_4027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

REL_V = 1e-4     # the tolerance of the parity tests
ABS_EU = 1e-3


@pytest.fixture(scope="module")
def hot():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0907_4027_gb300 import _build
    _build.build()
    from paper_0907_4027_gb300 import hot as h
    return h


def context_fields(hot, w):
    with hot.Hologram.from_workload(w) as h:
        e, u = h.gsw(0)
        V, _ = h.fields()
    return V, e, u


def noalloc_fields(hot, w, stream=None, with_eu=True):
    import torch
    stream = stream or torch.cuda.current_stream()
    with torch.cuda.stream(stream):
        xyz = torch.tensor(w.xyz, dtype=torch.float64, device="cuda")
        phi = torch.tensor(w.phi0, dtype=torch.float32, device="cuda")
        V = torch.full((2 * w.M,), float("nan"), dtype=torch.float64, device="cuda")
        eu = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda") if with_eu else None
    hot.hot_field_noalloc(w.W, w.H, w.pitch, w.wavelength, w.focal, xyz, phi, w.precision, V, eu,
                          stream.cuda_stream)
    stream.synchronize()
    v = V.cpu().numpy()
    if eu is None:
        return v[0::2] + 1j * v[1::2], None, None
    e, u = eu.cpu().numpy()
    return v[0::2] + 1j * v[1::2], float(e), float(u)


def rel_err(a, b):
    return np.max(np.abs(np.abs(a) - np.abs(b)) / np.abs(b))


def test_noalloc_matches_context_path_and_oracle_on_two_calls(hot):
    cases = [wl.random_case(100, 37, 13, seed=21, precision="fast"),
             wl.random_case(512, 512, 100, seed=0, precision="accurate")]
    for w in cases:                      # two calls in a row on the same scratch array
        V_ref, e_ref, u_ref = context_fields(hot, w)
        V, e, u = noalloc_fields(hot, w)
        assert rel_err(V, V_ref) < REL_V
        assert np.max(np.abs(V - V_ref)) < REL_V * np.max(np.abs(V_ref))
        assert abs(e - e_ref) < ABS_EU and abs(u - u_ref) < ABS_EU
        oV = oracle.forward(w.geom, w.xyz, w.phi0)   # Eq. 1 in FP64, independent of both paths
        assert rel_err(V, oV) < REL_V
        oe, ou = oracle.metrics(oV)
        assert abs(e - oe) < ABS_EU and abs(u - ou) < ABS_EU


def test_noalloc_without_metrics_on_a_side_stream(hot):
    """eu = NULL, on a stream other than the previous call's, ordered after it: the fields
    still match the oracle (the accumulators left by the previous call are cleared)."""
    import torch
    first = wl.random_case(96, 50, 40, seed=3, precision="fast")
    noalloc_fields(hot, first)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    w = wl.random_case(70, 45, 20, seed=22, precision="fast")
    V, e, u = noalloc_fields(hot, w, stream=side, with_eu=False)
    assert e is None and u is None
    assert rel_err(V, oracle.forward(w.geom, w.xyz, w.phi0)) < REL_V


def test_noalloc_rejects_sizes_beyond_its_scratch(hot):
    import torch
    M = 2000
    xyz = torch.zeros(3 * M, dtype=torch.float64, device="cuda")
    phi = torch.zeros(1920 * 1152, dtype=torch.float32, device="cuda")
    V = torch.zeros(2 * M, dtype=torch.float64, device="cuda")
    with pytest.raises(hot.HotError) as ei:
        hot.hot_field_noalloc(1920, 1152, 15e-6, 1.064e-6, 4e-3, xyz, phi, "fast", V)
    assert ei.value.status == hot.HOT_EINVAL and "scratch" in str(ei.value)
