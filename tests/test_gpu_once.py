"""GPU: the one-exponential GSW step (hot_set_once) -- each pixel-trap exponential evaluated once
per iteration and kept in registers between the back-projection and the forward field.  Checked
against the FP64 oracle (Eq. 1, Sec. 3; tolerances as in test_gpu_parity) and against the direct
kernels, on shapes that cover the kernel's forms (8, 4, 3 and 2 rows per sub-tile, with and without
the fused forward field, padding), ragged strips, both column staging paths and runs of a block
that cross from one 32-pixel strip into the next."""
import numpy as np
import pytest

import oracle
from paper_0907_4027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

REL_V = 1e-4
ABS_EU = 1e-3
TOL_S = {"accurate": 2e-6, "fast": 2e-5}


@pytest.fixture(scope="module")
def hot():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0907_4027_gb300 import _build
    _build.build()
    from paper_0907_4027_gb300 import hot as h
    return h


def rel_err(a, b):
    return np.max(np.abs(np.abs(a) - np.abs(b)) / np.maximum(np.abs(b), 1e-300))


@pytest.mark.parametrize("precision", ["accurate", "fast"])
@pytest.mark.parametrize("W,H,M", [
    (96, 64, 32),     # 4 traps per warp, 8 rows per sub-tile
    (70, 45, 64),     # W not a multiple of 4: column parts copied one by one; 8 traps x 4 rows
    (1024, 40, 100),  # runs that cross strip boundaries; 13 traps x 2 rows, padding on four warps
    (300, 60, 104),   # a ragged last strip (12 columns); 13 traps x 2 rows, a remainder sub-tile of one row
    (128, 30, 128),   # 16 traps x 2 rows
    (37, 29, 9),      # one ragged strip, fewer traps than warps (2 x 8 with padding)
    (160, 33, 89),    # 12 traps x 2 rows, padding on seven warps; an odd row count
    (64, 47, 122),    # 16 traps x 2 rows, padding on six warps
    (200, 21, 88),    # 11 traps x 3 rows
    (96, 50, 77),     # 10 traps x 3 rows, padding on three warps
])
def test_once_matches_oracle_and_direct_kernels(hot, W, H, M, precision):
    w = wl.random_case(W, H, M, seed=W * 7 + H + M, precision=precision)
    out = {}
    for once in (True, False):
        with hot.Hologram.from_workload(w) as h:
            h.set_once(once)
            assert h.tiling()["once"] == once
            h.gsw(0)
            V0, _ = h.fields()
            h.gsw(1)
            V1, w1 = h.fields()
            phi1 = h.phase("f32")
            eu3 = h.gsw(2)  # resumes: three iterations in all
            out[once] = (V0, V1, w1, phi1, eu3)
    V0, V1, w1, phi1, (e3, u3) = out[True]
    assert rel_err(V0, oracle.forward(w.geom, w.xyz, w.phi0)) < REL_V
    r1 = oracle.gsw(w.geom, w.xyz, 1, w.phi0)
    assert rel_err(V1, r1["V"]) < REL_V
    np.testing.assert_allclose(w1, r1["w"], rtol=REL_V)
    r3 = oracle.gsw(w.geom, w.xyz, 3, w.phi0)
    assert abs(e3 - r3["e"]) < ABS_EU and abs(u3 - r3["u"]) < ABS_EU
    # the phases of the first iteration from the oracle's coefficients (conditioning-aware)
    _, coef = oracle.update_weights(oracle.forward(w.geom, w.xyz, w.phi0), np.ones(M))
    ophi, S = oracle.backproject(w.geom, w.xyz, coef, want_S=True)
    d = np.abs(np.angle(np.exp(1j * (phi1.astype(np.float64) - ophi))))
    assert not (np.abs(S) * d > TOL_S[precision] * np.sum(np.abs(coef))).any()
    # and the direct kernels agree to the same tolerance
    assert rel_err(V1, out[False][1]) < REL_V and rel_err(out[False][1], r1["V"]) < REL_V


@pytest.mark.parametrize("precision", ["accurate", "fast"])
def test_once_bits_resume_graphs_persistent(hot, precision):
    """Resumed calls, launches without graphs and the persistent form give the bits of one
    graph-replayed call (the forward field of stored phases is the step's own arithmetic)."""
    w = wl.random_case(200, 90, 100, seed=11, precision=precision)
    res = []
    for mode in ("one", "split", "nographs", "persistent"):
        with hot.Hologram.from_workload(w) as h:
            assert h.tiling()["once"]
            if mode == "nographs":
                h.use_graphs(False)
            if mode == "persistent":
                h.use_persistent(True)
            if mode == "split":
                h.gsw(2)
                eu = h.gsw(3)
            else:
                eu = h.gsw(5)
            res.append((h.phase("f32"), *h.fields(), eu))
    for p, V, wt, eu in res[1:]:
        assert np.array_equal(res[0][0], p) and np.array_equal(res[0][1], V) and np.array_equal(res[0][2], wt)
        assert eu == res[0][3]


def test_once_applies_where_it_can(hot):
    w = wl.random_case(64, 32, 128, seed=3, precision="fast")
    with hot.Hologram.from_workload(w) as h:
        assert h.tiling()["once"]
        h.set_precision("accurate")
        assert h.tiling()["once"]
        h.set_precision("separable")
        assert not h.tiling()["once"]
        h.set_precision("fast")
        assert h.tiling()["once"]
        h.set_once(False)
        assert not h.tiling()["once"] and not hot.hot_get_once(h.ctx)["requested"]
        h.set_once(True)
        assert h.tiling()["once"]
        assert hot.lib.hot_set_once(h.ctx, 2) == hot.HOT_EINVAL
    w = wl.random_case(64, 32, 129, seed=3, precision="fast")
    with hot.Hologram.from_workload(w) as h:
        assert not h.tiling()["once"] and hot.hot_get_once(h.ctx)["requested"]


@pytest.mark.parametrize("precision", ["accurate", "fast"])
def test_once_full_hd_slm_against_oracle(hot, precision):
    """A 1920 x 1152 SLM with 100 traps: about 76 sub-tiles per block and runs that change strips,
    against the oracle (|V| after one iteration, weights, e and u after two)."""
    w = wl.random_case(1920, 1152, 100, seed=17, precision=precision)
    with hot.Hologram.from_workload(w) as h:
        assert h.tiling()["once"]
        h.gsw(1)
        V1, w1 = h.fields()
        e2, u2 = h.gsw(1)
    r1 = oracle.gsw(w.geom, w.xyz, 1, w.phi0)
    assert rel_err(V1, r1["V"]) < REL_V
    np.testing.assert_allclose(w1, r1["w"], rtol=REL_V)
    r2 = oracle.gsw(w.geom, w.xyz, 2, w.phi0)
    assert abs(e2 - r2["e"]) < ABS_EU and abs(u2 - r2["u"]) < ABS_EU


def test_once_stored_phasors_follow_the_phases(hot):
    """The unit phasors that the last step of a call leaves for the next call serve only the phases
    that step wrote: after hot_set_phase the next call starts from e^{i phi} of the new phases
    (against the oracle), and hot_get_phasors reports none; a resumed call uses them."""
    w = wl.random_case(160, 64, 40, seed=5, precision="fast")
    other = np.random.default_rng(9).uniform(-np.pi, np.pi, w.W * w.H).astype(np.float32)
    with hot.Hologram.from_workload(w) as h:
        assert hot.hot_get_phasors(h.ctx, h.N) is None  # phases set by the caller
        h.gsw(2)
        u = hot.hot_get_phasors(h.ctx, h.N)
        assert u is not None
        phi = h.phase("f32")
        np.testing.assert_allclose(u[0::2] + 1j * u[1::2], np.exp(1j * phi.astype(np.float64)), atol=2e-6)
        h.set_phase(other)
        assert hot.hot_get_phasors(h.ctx, h.N) is None
        h.gsw(0)
        V, _ = h.fields()
        h.gsw(0)  # still no phasors: the same bits again
        assert np.array_equal(h.fields()[0], V)
    assert rel_err(V, oracle.forward(w.geom, w.xyz, other.astype(np.float64))) < REL_V


def test_once_phasors_dropped_by_other_phase_writers(hot):
    """hot_superposition and a batch write the phases of a context with kept unit phasors: the
    phasors are dropped, and the next call's forward field is that of the new phases."""
    w = wl.random_case(96, 40, 30, seed=8, precision="fast")
    coef = np.exp(1j * np.random.default_rng(4).uniform(-np.pi, np.pi, w.xyz.shape[0]))
    with hot.Hologram.from_workload(w) as h:
        h.gsw(2)
        assert hot.hot_get_phasors(h.ctx, h.N) is not None
        h.superposition(coef)
        assert hot.hot_get_phasors(h.ctx, h.N) is None
        phi_sr = h.phase("f32")
        h.gsw(0)
        V_sr, _ = h.fields()
        h.gsw(2)
        assert hot.hot_get_phasors(h.ctx, h.N) is not None
        with hot.Batch([h]) as b:
            b.gsw(1)
        assert hot.hot_get_phasors(h.ctx, h.N) is None
        phi_b = h.phase("f32")
        h.gsw(0)
        V_b, _ = h.fields()
    assert rel_err(V_sr, oracle.forward(w.geom, w.xyz, phi_sr.astype(np.float64))) < REL_V
    assert rel_err(V_b, oracle.forward(w.geom, w.xyz, phi_b.astype(np.float64))) < REL_V


def test_once_phasor_calls_where_they_do_not_apply(hot):
    """hot_set_phasors needs the one-exponential step in effect; get_state carries no phasors in
    the other modes, and set_state without them starts from e^{i phi}."""
    w = wl.random_case(64, 24, 20, seed=2, precision="separable")
    with hot.Hologram.from_workload(w) as h:
        h.gsw(1)
        phi, wt, u = h.get_state()
        assert u is None
        with pytest.raises(hot.HotError, match="HOT_ESTATE"):
            hot.hot_set_phasors(h.ctx, np.zeros(2 * h.N, dtype=np.float32))
        h.set_state(phi, wt)
        h.gsw(0)
    w = wl.random_case(64, 24, 20, seed=2, precision="fast")
    with hot.Hologram.from_workload(w) as h:
        h.gsw(1)
        _, _, u = h.get_state()
        assert u is not None and u.shape == (2 * h.N,)
        with pytest.raises(hot.HotError, match="HOT_EINVAL"):
            hot.hot_set_phasors(h.ctx, np.full(2 * h.N, 3.0, dtype=np.float32))
        assert hot.hot_get_phasors(h.ctx, h.N) is not None  # a rejected call leaves them
