"""HOT_PREC_TENSOR: the separable GSW iteration as complex matrix products on the tcgen05
tensor cores (operands split in two FP16 parts), through the C ABI.

- the GEMM alone (hot_tc_gemm), both operand types: bit-exact on small integers (every product
  and partial sum is exact in TF32/FP16 and FP32, so any slip of layout, transposition, swizzle
  or K order shows), and within the split's error bound of the FP64 product on random data (a
  dropped low part gives ~5e-4 relative errors, 100x over the bound);
- GSW in the tensor mode against the FP64 oracle with the tolerances of every other mode
  (|V_m| 1e-4 relative after one iteration, e and u 1e-3, conditioning-aware phases);
- bit-identical resume, graph replay vs direct launches, the convergence trace, and the calls
  the mode rejects.
"""
import numpy as np
import pytest

import oracle
from paper_0907_4027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

REL_V = 1e-4
ABS_EU = 1e-3
TOL_S = 4e-6


@pytest.fixture(scope="module")
def hot():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0907_4027_gb300 import _build
    _build.build()
    from paper_0907_4027_gb300 import hot as h
    return h


def gemm(hot, A, B, tile_n, operands):
    import torch
    a = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(B, dtype=np.float32)).cuda()
    c = torch.full((A.shape[0], B.shape[0]), float("nan"), dtype=torch.float32, device="cuda")
    hot.hot_tc_gemm(a, b, c, tile_n, operands)
    return c.cpu().numpy()


OPERANDS = [0, 1]  # HOT_TC_TF32, HOT_TC_FP16


@pytest.mark.parametrize("operands", OPERANDS)
@pytest.mark.parametrize("tile_n", [32, 64, 128, 256])
@pytest.mark.parametrize("rows,cols,K", [(128, 64, 32), (200, 130, 75), (1, 1, 1), (257, 300, 96), (300, 520, 200)])
def test_gemm_exact_on_small_integers(hot, rows, cols, K, tile_n, operands):
    rng = np.random.default_rng(rows * 7 + cols + K)
    A = rng.integers(-8, 9, size=(rows, K)).astype(np.float32)
    B = rng.integers(-8, 9, size=(cols, K)).astype(np.float32)
    C = gemm(hot, A, B, tile_n, operands)
    assert np.array_equal(C, (A.astype(np.int64) @ B.astype(np.int64).T).astype(np.float32))


@pytest.mark.parametrize("operands", OPERANDS)
@pytest.mark.parametrize("tile_n", [32, 64, 128, 256])
@pytest.mark.parametrize("rows,cols,K", [(300, 200, 1000), (130, 70, 33)])
def test_gemm_within_split_bound(hot, rows, cols, K, tile_n, operands):
    """Operands of magnitude ~1 (uniform on [0.5, 1] with random sign: the FP16 split keeps its
    full precision there, as on the mode's unit phasors)."""
    rng = np.random.default_rng(rows + cols + K)
    A = (rng.uniform(0.5, 1.0, (rows, K)) * rng.choice([-1, 1], (rows, K))).astype(np.float32)
    B = (rng.uniform(0.5, 1.0, (cols, K)) * rng.choice([-1, 1], (cols, K))).astype(np.float32)
    C = gemm(hot, A, B, tile_n, operands).astype(np.float64)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    # per product ~2^-20 relative (split), plus FP32 accumulation over K terms
    assert np.all(np.abs(C - ref) <= 4e-6 * scale), np.max(np.abs(C - ref) / scale)


def rel_err(a, b):
    return np.max(np.abs(np.abs(a) - np.abs(b)) / np.maximum(np.abs(b), 1e-300))


def check_phase_step(gpu_phi, w, coef):
    ophi, S = oracle.backproject(w.geom, w.xyz, coef, want_S=True)
    d = np.abs(np.angle(np.exp(1j * (gpu_phi.astype(np.float64) - ophi))))
    bad = np.abs(S) * d > TOL_S * np.sum(np.abs(coef))
    assert not bad.any(), f"{bad.sum()} pixels"


@pytest.mark.parametrize("W,H,M", [(100, 37, 13), (64, 16, 1), (33, 9, 7), (40, 24, 300), (1, 1, 5),
                                   (257, 3, 9), (5, 70, 129), (300, 260, 70), (2048, 1280, 64),
                                   (1600, 1300, 128)])
def test_one_iteration_matches_oracle(hot, W, H, M):
    """Ragged tiles in both directions, one and several K splits, the tile widths (2048 x 1280
    takes 256-wide back-projection tiles and 128-wide forward tiles, 1600 x 1300 with 128 traps
    256-wide tiles in both, the small cases 32-wide tiles)."""
    w = wl.random_case(W, H, M, seed=W + H + M, precision="tensor")
    with hot.Hologram.from_workload(w) as h:
        e0, u0 = h.gsw(0)
        V0, _ = h.fields()
        e1, u1 = h.gsw(1)
        V1, w1 = h.fields()
        phi1 = h.phase("f32")
    oV0 = oracle.forward(w.geom, w.xyz, w.phi0)
    assert rel_err(V0, oV0) < REL_V
    oe, ou = oracle.metrics(oV0)
    assert abs(e0 - oe) < ABS_EU and abs(u0 - ou) < ABS_EU
    r = oracle.gsw(w.geom, w.xyz, 1, w.phi0)
    np.testing.assert_allclose(w1, r["w"], rtol=REL_V)
    assert rel_err(V1, r["V"]) < REL_V
    assert abs(e1 - r["e"]) < ABS_EU and abs(u1 - r["u"]) < ABS_EU
    # the phases from the coefficients of the GPU's own V0: with 2.6e6 pixels the smallest |V_m|
    # of random phases is ~30x below the mean, its weight ~30x above, and the coefficient error
    # that V0's rounding leaves there would dominate a comparison against the oracle's own
    _, coef = oracle.update_weights(V0, np.ones(M))
    check_phase_step(phi1, w, coef)


def test_rand100_512_full_run_matches_oracle(hot):
    w = wl.rand100_512()
    w.precision = "tensor"
    with hot.Hologram.from_workload(w) as h:
        h.gsw(1)
        V1, _ = h.fields()
        e, u = h.gsw(w.iters - 1)
    r1 = oracle.gsw(w.geom, w.xyz, 1, w.phi0)
    assert rel_err(V1, r1["V"]) < REL_V
    r = oracle.gsw(w.geom, w.xyz, w.iters, w.phi0)
    assert abs(e - r["e"]) < ABS_EU and abs(u - r["u"]) < ABS_EU, (e, r["e"], u, r["u"])


def test_resume_graphs_and_determinism(hot):
    w = wl.random_case(70, 45, 20, seed=5, precision="tensor")
    with hot.Hologram.from_workload(w) as a, hot.Hologram.from_workload(w) as b, \
            hot.Hologram.from_workload(w) as c:
        a.gsw(5)
        b.gsw(3)
        b.gsw(2)
        c.use_graphs(False)
        c.gsw(5)
        pa, pb, pc = (x.phase("f32") for x in (a, b, c))
        (Va, wa), (Vb, wb), (Vc, wc) = (x.fields() for x in (a, b, c))
        a.set_phase(w.phi0)
        a.set_weights(np.ones(w.M))
        a.gsw(5)                                 # graph replay
        assert np.array_equal(a.phase("f32"), pa)
    for p, V, wt in ((pb, Vb, wb), (pc, Vc, wc)):
        assert np.array_equal(pa, p) and np.array_equal(Va, V) and np.array_equal(wa, wt)


def test_trace_and_new_traps(hot):
    """The convergence trace in the tensor mode; new traps of the same count rebuild the
    operands in place."""
    w = wl.random_case(100, 37, 13, seed=21, precision="tensor")
    with hot.Hologram.from_workload(w) as h:
        h.set_trace(True)
        eK, uK = h.gsw(4)
        e, u = h.trace(4)
        assert e[-1] == np.float32(eK) and u[-1] == np.float32(uK)
        w2 = wl.random_case(100, 37, 13, seed=22, precision="tensor")
        h.set_traps(w2.xyz)
        h.set_phase(w2.phi0)
        e2, u2 = h.gsw(1)
    for k in range(5):
        r = oracle.gsw(w.geom, w.xyz, k, w.phi0)
        assert abs(e[k] - r["e"]) < ABS_EU and abs(u[k] - r["u"]) < ABS_EU, k
    r = oracle.gsw(w2.geom, w2.xyz, 1, w2.phi0)
    assert abs(e2 - r["e"]) < ABS_EU and abs(u2 - r["u"]) < ABS_EU


def test_rejected_calls_and_other_entry_points(hot):
    w = wl.random_case(64, 40, 10, seed=3, precision="tensor")
    with hot.Hologram.from_workload(w) as h:
        h.use_persistent(True)
        with pytest.raises(hot.HotError, match="HOT_EINVAL"):
            h.gsw(1)
        h.use_persistent(False)
        with pytest.raises(hot.HotError, match="HOT_EINVAL"):
            h.autotune(2)
        with hot.Batch([h]) as b:              # tensor batches: no tiling to set or tune
            with pytest.raises(hot.HotError, match="HOT_EINVAL"):
                b.set_tiling(rows=7)
            with pytest.raises(hot.HotError, match="HOT_EINVAL"):
                b.autotune(2)
        import torch
        phi = torch.from_numpy(np.asarray(w.phi0, dtype=np.float32)).cuda()
        Vd = torch.empty(2 * w.M, dtype=torch.float32, device="cuda")
        hot.hot_field(h.ctx, phi, Vd)            # the separable kernels serve hot_field
        h.sync()
        V = Vd.cpu().numpy().astype(np.float64).view(np.complex128)
        e, u = h.gsw(2)
    assert rel_err(V, oracle.forward(w.geom, w.xyz, w.phi0)) < REL_V
    r = oracle.gsw(w.geom, w.xyz, 2, w.phi0)
    assert abs(e - r["e"]) < ABS_EU and abs(u - r["u"]) < ABS_EU


def test_tensor_batch_equals_single_runs(hot):
    """A HOT_PREC_TENSOR batch runs every member's own launch sequence on concurrent chains: each
    member's phases, fields and weights equal its hot_gsw run bit for bit (also across a resumed
    call), and every member gets a completion stamp."""
    ws = [wl.random_case(W, H, M, seed=W + M, precision="tensor")
          for (W, H, M) in [(100, 37, 13), (256, 128, 40), (64, 64, 130), (33, 20, 3), (300, 200, 200),
                            (128, 96, 7), (200, 90, 37), (96, 64, 65), (160, 120, 300), (40, 24, 300)]]
    ref = []
    for w in ws:
        with hot.Hologram.from_workload(w) as h:
            h.gsw(3)
            ref.append((h.phase("f32"), *h.fields()))
    holos = [hot.Hologram.from_workload(w) for w in ws]
    try:
        with hot.Batch(holos) as b:
            assert b.tiling()["groups"] == 8              # chains
            b.gsw(2)
            b.gsw(1)
            lat = b.latency()
            got = [(h.phase("f32"), *h.fields()) for h in holos]
            eu = [h.metrics() for h in holos]
    finally:
        for h in holos:
            h.close()
    for (p0, V0, w0), (p1, V1, w1) in zip(ref, got):
        assert np.array_equal(p0, p1) and np.array_equal(V0, V1) and np.array_equal(w0, w1)
    assert np.all(lat > 0) and len(lat) == len(ws)
    for w, (e, u) in zip(ws, eu):
        r = oracle.gsw(w.geom, w.xyz, 3, w.phi0)
        assert abs(e - r["e"]) < ABS_EU and abs(u - r["u"]) < ABS_EU
