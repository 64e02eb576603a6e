"""Row-band sharded GSW on one GPU: the bands of one hologram as separate contexts whose
partial sums are added on the device between launches (the all-reduce of a multi-GPU run,
emulated in one process).  Against the unsharded context and the FP64 oracle, with the
parity tolerances (|V_m| 1e-4 relative after one iteration, e and u 1e-3 after three)."""
import numpy as np
import pytest

import oracle
from paper_0907_4027_gb300 import sharded
from paper_0907_4027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

REL_V = 1e-4
ABS_EU = 1e-3


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0907_4027_gb300 import _build
    _build.build()
    from paper_0907_4027_gb300 import hot
    return torch, hot


def make_bands(torch, hot, w, world):
    st = torch.cuda.current_stream().cuda_stream
    bands = []
    for r in range(world):
        y0, rows = sharded.band_rows(w.H, world, r)
        h = hot.Hologram(w.W, rows, w.pitch, w.wavelength, w.focal, st, w.precision)
        h.set_band(w.H, y0)
        h.set_traps(w.xyz, w.w0)
        h.set_phase(w.phi0.reshape(w.H, w.W)[y0:y0 + rows].reshape(-1))
        bands.append(h)
    return bands


def emulate(bands, iters):
    """The launch sequence of run_sharded over all bands in lockstep, partial sums added on
    the device (int64, exact) in place of the all-reduce."""
    def exchange(k):
        s = [h.sharded_sums(k) for h in bands]
        total = sum(s[1:], s[0].clone())
        for t in s:
            t.copy_(total)
    for h in bands:
        h.sharded_begin()
    exchange(0)
    for k in range(1, iters + 1):
        for h in bands:
            h.sharded_step(k)
        exchange(k)
    return [h.sharded_end(iters) for h in bands]


@pytest.mark.parametrize("precision", ["accurate", "fast", "separable", "tensor"])
@pytest.mark.parametrize("W,H,M,world", [(100, 37, 13, 2), (64, 64, 130, 3), (33, 20, 3, 4)])
def test_bands_match_unsharded_and_oracle(env, W, H, M, world, precision):
    torch, hot = env
    w = wl.random_case(W, H, M, seed=W + M, precision=precision)
    bands = make_bands(torch, hot, w, world)
    try:
        emulate(bands, 1)
        fields = [h.fields() for h in bands]
        eus = emulate(bands, 2)        # resumes: three iterations in all
        phi = np.concatenate([h.phase("f32") for h in bands])
    finally:
        for h in bands:
            h.close()
    V1, w1 = fields[0]
    for V, wt in fields[1:]:           # every band derives the same field and weights
        assert np.array_equal(V, V1) and np.array_equal(wt, w1)
    assert all(eu == eus[0] for eu in eus)
    r1 = oracle.gsw(w.geom, w.xyz, 1, w.phi0)
    assert np.max(np.abs(np.abs(V1) - np.abs(r1["V"])) / np.abs(r1["V"])) < REL_V
    np.testing.assert_allclose(w1, r1["w"], rtol=REL_V)
    r3 = oracle.gsw(w.geom, w.xyz, 3, w.phi0)
    e, u = eus[0]
    assert abs(e - r3["e"]) < ABS_EU and abs(u - r3["u"]) < ABS_EU, (e, u, r3["e"], r3["u"])
    with hot.Hologram.from_workload(w) as h:   # the unsharded context
        h.gsw(1)
        Vu, _ = h.fields()
        eu_u = h.gsw(2)
    assert np.max(np.abs(np.abs(V1) - np.abs(Vu)) / np.abs(Vu)) < REL_V
    assert abs(e - eu_u[0]) < ABS_EU and abs(u - eu_u[1]) < ABS_EU
    assert phi.shape == (w.N,)


@pytest.mark.parametrize("precision", ["fast", "tensor"])
def test_single_band_is_the_plain_context(env, precision):
    """A band covering the whole hologram gives hot_gsw's result bit for bit."""
    torch, hot = env
    w = wl.random_case(64, 48, 20, seed=2, precision=precision)
    bands = make_bands(torch, hot, w, 1)
    try:
        eu = emulate(bands, 3)[0]
        phi_b, V_b = bands[0].phase("f32"), bands[0].fields()[0]
    finally:
        bands[0].close()
    with hot.Hologram.from_workload(w) as h:
        h.use_graphs(False)
        eu_p = h.gsw(3)
        phi_p, V_p = h.phase("f32"), h.fields()[0]
    assert np.array_equal(phi_b, phi_p) and np.array_equal(V_b, V_p) and eu == eu_p


def test_sharded_calls_out_of_order_and_bad_bands(env):
    torch, hot = env
    w = wl.random_case(32, 16, 4, seed=3, precision="fast")
    with hot.Hologram.from_workload(w) as h:
        with pytest.raises(hot.HotError, match="HOT_ESTATE"):
            h.sharded_step(1)
        h.sharded_begin()
        with pytest.raises(hot.HotError, match="HOT_ESTATE"):
            h.sharded_step(2)
        with pytest.raises(hot.HotError, match="HOT_ESTATE"):
            h.sharded_sums(1)
        with pytest.raises(hot.HotError, match="HOT_ESTATE"):
            h.sharded_end(1)
        h.sharded_end(0)
        for total, y0 in ((15, 0), (16, 1), (40, -1), (40, 25)):
            with pytest.raises(hot.HotError, match="HOT_EINVAL"):
                h.set_band(total, y0)
