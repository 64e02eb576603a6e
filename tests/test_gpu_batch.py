"""Batched GSW (hot_batch_*), tiling and autotuning, through the C ABI: holograms of uneven
size and trap count in one launch per group and iteration, against the same holograms run one
by one and against the FP64 oracle.  Tolerances as in the parity tests: |V_m| 1e-4 relative
after one iteration; e and u 1e-3 after the run (here three iterations, resumed after the
first: hot_gsw(1) then hot_gsw(2) is hot_gsw(3))."""
import numpy as np
import pytest

import oracle
from paper_0907_4027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

REL_V = 1e-4
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


def cases(precision):
    # ragged tiles, several trap chunks, fewer traps than warps, a wide one
    return [wl.random_case(100, 37, 13, seed=1, precision=precision),
            wl.random_case(64, 64, 130, seed=2, precision=precision),
            wl.random_case(33, 20, 3, seed=3, precision=precision),
            wl.random_case(256, 128, 40, seed=4, precision=precision)]


def rel_err(a, b):
    return np.max(np.abs(np.abs(a) - np.abs(b)) / np.abs(b))


def check_against_oracle(w, V1, w1, eu3):
    """V1, w1: after one iteration; eu3: (e, u) after three."""
    r1 = oracle.gsw(w.geom, w.xyz, 1, w.phi0)
    assert rel_err(V1, r1["V"]) < REL_V
    np.testing.assert_allclose(w1, r1["w"], rtol=REL_V)
    r3 = oracle.gsw(w.geom, w.xyz, 3, w.phi0)
    assert abs(eu3[0] - r3["e"]) < ABS_EU and abs(eu3[1] - r3["u"]) < ABS_EU, (eu3, r3["e"], r3["u"])


def run_batch(hot, ws, configure=None):
    """Per hologram: (V, w) after one batched iteration, (e, u) after two more, phases."""
    holos = [hot.Hologram.from_workload(w) for w in ws]
    try:
        with hot.Batch(holos) as b:
            if configure:
                configure(b)
            b.gsw(1)
            one = [h.fields() for h in holos]
            b.gsw(2)
            out = [(V, wt, h.metrics(), h.phase("f32")) for (V, wt), h in zip(one, holos)]
            lat = b.latency()
            tiling = b.tiling()
    finally:
        for h in holos:
            h.close()
    return out, lat, tiling


@pytest.mark.parametrize("precision", ["accurate", "fast", "separable"])
def test_batch_matches_single_runs_and_oracle(hot, precision):
    ws = cases(precision)
    got, _, _ = run_batch(hot, ws)
    for w, (V, wt, eu, phi) in zip(ws, got):
        with hot.Hologram.from_workload(w) as h:
            h.gsw(1)
            V1, w1 = h.fields()
            eu1 = h.gsw(2)
        assert rel_err(V, V1) < REL_V
        np.testing.assert_allclose(wt, w1, rtol=REL_V)
        assert abs(eu[0] - eu1[0]) < ABS_EU and abs(eu[1] - eu1[1]) < ABS_EU
        check_against_oracle(w, V, wt, eu)
        assert phi.shape == (w.N,)


def test_batch_resume_is_bit_identical(hot):
    ws = cases("fast")
    out = []
    for split in ((4,), (3, 1)):
        holos = [hot.Hologram.from_workload(w) for w in ws]
        with hot.Batch(holos) as b:
            for k in split:
                b.gsw(k)
            out.append([(h.phase("f32"), h.fields()[0]) for h in holos])
        for h in holos:
            h.close()
    for (pa, Va), (pb, Vb) in zip(*out):
        assert np.array_equal(pa, pb) and np.array_equal(Va, Vb)


@pytest.mark.parametrize("group_pairs", [1.0, 1e18])
def test_batch_groups_and_latency(hot, group_pairs):
    """Shortest-first groups: one group per hologram (group_pairs = 1) and all holograms in
    lockstep (a threshold above the total) compute the same GSW; completion stamps are positive
    and, with one group per hologram, grow with the work order."""
    ws = cases("fast")
    pairs = [w.N * w.M for w in ws]
    got, lat, tiling = run_batch(hot, ws, lambda b: b.set_tiling(group_pairs=group_pairs))
    assert tiling["groups"] == (len(ws) if group_pairs == 1.0 else 1)
    assert np.all(lat > 0), lat
    if group_pairs == 1.0:
        order = np.argsort(pairs, kind="stable")
        assert np.all(np.diff(lat[order]) >= 0), (lat, pairs)
    for w, (V, wt, eu, _) in zip(ws, got):
        check_against_oracle(w, V, wt, eu)


@pytest.mark.parametrize("tiling", [(3, 2, 32), (14, 1, 64), (1, 4, 8), (7, 3, 128)])
def test_tiling_matches_oracle(hot, tiling):
    """Any tiling (rows per sub-tile, blocks per SM, trap chunk) computes the same GSW."""
    w = wl.random_case(100, 37, 130, seed=7, precision="fast")
    with hot.Hologram.from_workload(w) as h:
        h.set_tiling(*tiling)
        t = h.tiling()
        assert (t["rows"], t["chunk"]) == (tiling[0], tiling[2]) and 1 <= t["blocks_per_sm"] <= tiling[1]
        h.gsw(1)
        V1, w1 = h.fields()
        eu = h.gsw(2)
    check_against_oracle(w, V1, w1, eu)


@pytest.mark.parametrize("precision", ["accurate", "separable"])
@pytest.mark.parametrize("tiling", [(5, 2, 16), (14, 1, 128)])
def test_batch_tiling_matches_oracle(hot, tiling, precision):
    ws = cases(precision)
    got, _, t = run_batch(hot, ws, lambda b: b.set_tiling(*tiling))
    assert (t["rows"], t["chunk"]) == (tiling[0], tiling[2])
    for w, (V, wt, eu, _) in zip(ws, got):
        check_against_oracle(w, V, wt, eu)


def test_tiling_rejects_out_of_range(hot):
    w = wl.random_case(64, 64, 5, seed=1, precision="fast")
    with hot.Hologram.from_workload(w) as h:
        for bad in ((15, 0, 0), (0, 33, 0), (0, 0, 129), (-1, 0, 0)):
            with pytest.raises(hot.HotError, match="HOT_EINVAL"):
                h.set_tiling(*bad)


def test_autotune_keeps_state(hot):
    """The autotuner returns a valid tiling and leaves phases and weights as they were; GSW
    afterwards still matches the oracle."""
    w = wl.random_case(128, 96, 40, seed=5, precision="fast")
    with hot.Hologram.from_workload(w) as h:
        phi_before = h.phase("f32")
        t = h.autotune(4)
        assert 1 <= t["rows"] <= 14 and 1 <= t["blocks_per_sm"] <= 4 and 1 <= t["chunk"] <= 128
        assert t["us_per_iter"] > 0
        assert h.tiling() == {k: t[k] for k in ("rows", "blocks_per_sm", "chunk", "merge", "once")}
        assert np.array_equal(h.phase("f32"), phi_before)
        with pytest.raises(hot.HotError, match="HOT_ESTATE"):
            h.fields()
        h.gsw(1)
        V1, w1 = h.fields()
        eu = h.gsw(2)
    check_against_oracle(w, V1, w1, eu)


def test_batch_autotune_keeps_state(hot):
    ws = cases("fast")
    holos = [hot.Hologram.from_workload(w) for w in ws]
    try:
        with hot.Batch(holos) as b:
            before = [h.phase("f32") for h in holos]
            t = b.autotune(2)
            assert 1 <= t["rows"] <= 14 and t["us_per_iter"] > 0
            assert all(np.array_equal(h.phase("f32"), p) for h, p in zip(holos, before))
            with pytest.raises(hot.HotError, match="HOT_ESTATE"):
                b.latency()
            b.gsw(1)
            one = [h.fields() for h in holos]
            b.gsw(2)
            got = [(V, wt, h.metrics()) for (V, wt), h in zip(one, holos)]
    finally:
        for h in holos:
            h.close()
    for w, (V, wt, eu) in zip(ws, got):
        check_against_oracle(w, V, wt, eu)


def test_row_bands_are_not_batched(hot):
    w = wl.random_case(64, 32, 5, seed=1, precision="fast")
    with hot.Hologram(w.W, 16, w.pitch, w.wavelength, w.focal, precision="fast") as h:
        h.set_band(32, 16)
        h.set_traps(w.xyz)
        with pytest.raises(hot.HotError, match="HOT_EINVAL"):
            hot.Batch([h]).close()


@pytest.mark.slow
def test_largest_batch64_member_fast(hot):
    """The largest hologram of the batch64 workload (1920 x 1152 px, 1818 traps; fast mode) run
    through hot_batch_gsw beside a small one: the fields of the GPU's final phase against the
    oracle forward on a seeded 64-trap subset, and one step from the GPU's state (its fields and
    weights, Sec. 3 update and Sec. 4 back-projection in FP64) on that subset, after 3 iterations;
    e and u against the oracle forward of the GPU's final phase (all traps)."""
    big = max(wl.batch64(), key=lambda w: w.N * w.M)
    assert (big.W, big.H, big.M) == (1920, 1152, 1818)
    small = wl.random_case(100, 37, 13, seed=1, precision="fast")
    holos = [hot.Hologram.from_workload(w) for w in (big, small)]
    try:
        with hot.Batch(holos) as b:
            b.gsw(2)
            VK, wK1 = holos[0].fields()
            b.gsw(1)
            VK1, _ = holos[0].fields()
            e, u = holos[0].metrics()
            phiK = holos[0].phase("f32")
    finally:
        for h in holos:
            h.close()
    sub = np.sort(np.random.default_rng(0).choice(big.M, 64, replace=False))
    assert rel_err(VK1[sub], oracle.forward(big.geom, big.xyz[sub], phiK)) < REL_V
    _, coef = oracle.update_weights(VK, wK1)
    ophi = oracle.backproject(big.geom, big.xyz, coef)
    assert rel_err(VK1[sub], oracle.forward(big.geom, big.xyz[sub], ophi)) < REL_V
    oe, ou = oracle.metrics(oracle.forward(big.geom, big.xyz, phiK))
    assert abs(e - oe) < ABS_EU and abs(u - ou) < ABS_EU
