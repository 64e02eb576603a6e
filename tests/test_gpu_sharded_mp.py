"""Row-band sharded GSW across processes: two ranks, each a separate process with its own CUDA
context on the same GPU, each holding one band of rows of the hologram (hot_set_band) and
running the launch sequence of sharded.run_sharded; the 2M int64 fixed-point partial sums of
every launch are copied to the host, added over the ranks by a gloo all-reduce and copied back
before the next launch (no kernel waits on another process: the host orders every exchange, and
no NCCL, NVLS or multicast memory is involved).

Checks: the two-process run equals, bit for bit, the same bands run in one process with the sums
added on the device (the exchange is exact integer addition, so the process boundary changes
nothing); and it matches the unsharded hot_gsw within the parity tolerances (|V_m| 1e-4 relative,
e and u 1e-3) and the FP64 oracle.  Bit equality with the unsharded context is not expected: each
band's schedule groups its pixels into sub-tiles differently, and the FP32 partial sums of a
sub-tile depend on that grouping before they are rounded to fixed point."""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle
from paper_0907_4027_gb300 import sharded
from paper_0907_4027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

REL_V = 1e-4
ABS_EU = 1e-3
ITERS = 3


def _case(precision):
    return wl.random_case(200, 90, 37, seed=17, precision=precision)


def _band(hot, w, world, rank, stream):
    y0, rows = sharded.band_rows(w.H, world, rank)
    h = hot.Hologram(w.W, rows, w.pitch, w.wavelength, w.focal, stream, w.precision)
    h.set_band(w.H, y0)
    h.set_traps(w.xyz, w.w0)
    h.set_phase(w.phi0.reshape(w.H, w.W)[y0:y0 + rows].reshape(-1))
    return h


def host_exchange():
    """run_sharded's exchange over gloo: device sums -> host, all-reduce (int64 addition), back."""
    import torch.distributed as dist

    def exchange(t):
        h = t.cpu()                      # ordered after the launch on the current stream
        dist.all_reduce(h, op=dist.ReduceOp.SUM)
        t.copy_(h)                       # ordered before the next launch
    return exchange


def _worker(rank, world, port, precision, out_dir):
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        from paper_0907_4027_gb300 import hot
        w = _case(precision)
        band = _band(hot, w, world, rank, torch.cuda.current_stream().cuda_stream)
        e, u = sharded.run_sharded(band, ITERS, host_exchange())
        phi = band.phase("f32")
        V, wt = band.fields()
        band.close()
        phis = [None] * world
        dist.all_gather_object(phis, phi)
        if rank == 0:
            np.savez(os.path.join(out_dir, f"{precision}.npz"), phi=np.concatenate(phis), V=V, w=wt, e=e, u=u)
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _one_process(hot, torch, w, world):
    """The same bands in one process, partial sums added on the device between launches."""
    st = torch.cuda.current_stream().cuda_stream
    bands = [_band(hot, w, world, r, st) for r in range(world)]

    def exchange(k):
        s = [h.sharded_sums(k) for h in bands]
        total = sum(s[1:], s[0].clone())
        for t in s:
            t.copy_(total)
    for h in bands:
        h.sharded_begin()
    exchange(0)
    for k in range(1, ITERS + 1):
        for h in bands:
            h.sharded_step(k)
        exchange(k)
    eu = [h.sharded_end(ITERS) for h in bands]
    phi = np.concatenate([h.phase("f32") for h in bands])
    V, wt = bands[0].fields()
    for h in bands:
        h.close()
    return phi, V, wt, eu[0]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0907_4027_gb300 import _build
    _build.build()
    from paper_0907_4027_gb300 import hot
    return torch, hot


@pytest.mark.parametrize("precision", ["fast", "tensor"])
def test_two_process_bands_equal_one_process_and_unsharded(env, precision):
    import torch.multiprocessing as mp
    torch, hot = env
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_worker, args=(world, _free_port(), precision, d), nprocs=world, join=True)
        r = dict(np.load(os.path.join(d, f"{precision}.npz")))
    w = _case(precision)
    # bit for bit against the same bands in one process
    phi1, V1, w1, (e1, u1) = _one_process(hot, torch, w, world)
    assert np.array_equal(r["phi"], phi1) and np.array_equal(r["V"], V1) and np.array_equal(r["w"], w1)
    assert float(r["e"]) == e1 and float(r["u"]) == u1
    # the unsharded context and the oracle, within the parity tolerances
    with hot.Hologram.from_workload(w) as h:
        e0, u0 = h.gsw(ITERS)
        V0, w0 = h.fields()
    ref = oracle.gsw(w.geom, w.xyz, ITERS, w.phi0)
    for V, e, u in ((r["V"], float(r["e"]), float(r["u"])), (V0, e0, u0)):
        assert np.max(np.abs(np.abs(V) - np.abs(ref["V"])) / np.abs(ref["V"])) < REL_V
        assert abs(e - ref["e"]) < ABS_EU and abs(u - ref["u"]) < ABS_EU
    np.testing.assert_allclose(r["w"], w0, rtol=REL_V)
