"""hot_field_noalloc: the allocation-free forward-field entry point.

Callers that cannot allocate device memory (a real-time frame loop with pre-planned memory,
an external pool that owns every allocation) evaluate the trap fields through this entry
point; its working memory is a fixed device array inside the library.  These tests call it
through the C ABI and compare it with the context path (hot_set_traps, hot_set_phase,
hot_gsw(0), hot_get_fields), twice in a row so that a second call on the reused scratch array
is covered.  The file name sorts last so that a run stopping at the first failure has already
run every other test.
"""
import numpy as np
import pytest

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


def noalloc_fields(hot, w):
    import torch
    xyz = torch.tensor(w.xyz, dtype=torch.float64, device="cuda")
    phi = torch.tensor(w.phi0, dtype=torch.float32, device="cuda")
    V = torch.full((2 * w.M,), float("nan"), dtype=torch.float64, device="cuda")
    eu = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    hot.hot_field_noalloc(w.W, w.H, w.pitch, w.wavelength, w.focal, xyz, phi, w.precision, V, eu,
                          stream.cuda_stream)
    torch.cuda.synchronize()
    v = V.cpu().numpy()
    e, u = eu.cpu().numpy()
    return v[0::2] + 1j * v[1::2], float(e), float(u)


def test_noalloc_matches_context_path_on_two_calls(hot):
    cases = [wl.random_case(100, 37, 13, seed=21, precision="fast"),
             wl.random_case(512, 512, 100, seed=0, precision="accurate")]
    for w in cases:                      # two calls in a row on the same scratch array
        V_ref, e_ref, u_ref = context_fields(hot, w)
        V, e, u = noalloc_fields(hot, w)
        rel = np.max(np.abs(np.abs(V) - np.abs(V_ref)) / np.abs(V_ref))
        assert rel < REL_V, rel
        assert np.max(np.abs(V - V_ref)) < REL_V * np.max(np.abs(V_ref))
        assert abs(e - e_ref) < ABS_EU and abs(u - u_ref) < ABS_EU


def test_noalloc_rejects_sizes_beyond_its_scratch(hot):
    import torch
    M = 2000
    xyz = torch.zeros(3 * M, dtype=torch.float64, device="cuda")
    phi = torch.zeros(1920 * 1152, dtype=torch.float32, device="cuda")
    V = torch.zeros(2 * M, dtype=torch.float64, device="cuda")
    with pytest.raises(hot.HotError) as ei:
        hot.hot_field_noalloc(1920, 1152, 15e-6, 1.064e-6, 4e-3, xyz, phi, "fast", V)
    assert ei.value.status == hot.HOT_EINVAL and "scratch" in str(ei.value)
