"""Multi-rank host logic on CPU (gloo, world size 2): band and replica partitions, the
max-over-ranks timing, and the row-band sharded GSW driver with an all-reduce exchange.

The sharded driver is run with a CPU stand-in for the CUDA band context: an FP64 band engine
that takes Eq. 2 from oracle.delta, forms the band's partial sums of Eq. 1, applies the
Sec. 3 weight update of oracle.update_weights to the summed field and back-projects its own
rows (Sec. 4).  Summed over the two ranks by gloo, the result must equal the unsharded
oracle GSW to FP64 rounding."""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle
from paper_0907_4027_gb300 import sharded
from paper_0907_4027_gb300 import workloads as wl


@pytest.mark.parametrize("H,world", [(37, 2), (1, 1), (5, 8), (1152, 3), (512, 4)])
def test_bands_cover_rows_once(H, world):
    rows = []
    for r in range(world):
        y0, n = sharded.band_rows(H, world, r)
        rows += list(range(y0, y0 + n))
        assert n in (H // world, H // world + 1)
    assert rows == list(range(H))


def test_band_rows_rejects_bad_rank():
    with pytest.raises(ValueError):
        sharded.band_rows(10, 2, 2)


class CpuBand:
    """FP64 stand-in with the sharded interface (rows y0 .. y0+rows-1 of the hologram)."""

    def __init__(self, w, y0, rows):
        import torch
        self.torch = torch
        self.N, self.M = w.N, w.M
        pix = [(ix, iy) for iy in range(y0, y0 + rows) for ix in range(w.W)]
        D = np.array([[oracle.delta(w.geom, t, ix, iy) for t in w.xyz] for ix, iy in pix])
        self.E = np.exp(1j * D)                      # e^{i Delta_j^m}, [band pixels, M]
        self.phi = w.phi0.reshape(w.H, w.W)[y0:y0 + rows].reshape(-1).astype(np.float64)
        self.w = np.ones(w.M)
        self.sums = {}

    def _forward(self, k):  # Eq. 1 over the band's pixels
        V = (np.exp(1j * self.phi) @ np.conj(self.E)) / self.N
        self.sums[k] = self.torch.tensor(np.concatenate([V.real, V.imag]))

    def _V(self, k):
        s = self.sums[k].numpy()
        return s[:self.M] + 1j * s[self.M:]

    def sharded_begin(self):
        self._forward(0)

    def sharded_sums(self, k):
        return self.sums[k]

    def sharded_step(self, k):
        self.w, c = oracle.update_weights(self._V(k - 1), self.w)   # Sec. 3, summed field
        self.phi = np.angle(self.E @ c)                             # Sec. 4, this band
        self._forward(k)

    def sharded_end(self, iters):
        self.V = self._V(iters)
        return oracle.metrics(self.V)


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        w = wl.random_case(12, 7, 5, seed=11, precision="accurate")
        y0, rows = sharded.band_rows(w.H, world, rank)
        band = CpuBand(w, y0, rows)
        e, u = sharded.run_sharded(band, 3, sharded.allreduce_exchange())
        phis = [None] * world
        dist.all_gather_object(phis, band.phi)
        t = sharded.max_over_ranks(1.5 + rank)
        if rank == 0:
            np.savez(os.path.join(out_dir, "r.npz"), phi=np.concatenate(phis), V=band.V, w=band.w,
                     e=e, u=u, t=t)
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_sharded_gsw_over_gloo_equals_unsharded_oracle():
    import torch.multiprocessing as mp
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_worker, args=(world, _free_port(), d), nprocs=world, join=True)
        r = dict(np.load(os.path.join(d, "r.npz")))
    w = wl.random_case(12, 7, 5, seed=11, precision="accurate")
    ref = oracle.gsw(w.geom, w.xyz, 3, w.phi0)
    assert float(r["t"]) == 2.5                                    # max over ranks
    np.testing.assert_allclose(r["V"], ref["V"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["w"], ref["w"], rtol=1e-10)
    d = np.angle(np.exp(1j * (r["phi"] - ref["phi"])))
    assert np.max(np.abs(d)) < 1e-9
    assert abs(float(r["e"]) - ref["e"]) < 1e-12 and abs(float(r["u"]) - ref["u"]) < 1e-12


def test_max_over_ranks_without_process_group():
    assert sharded.max_over_ranks(3.25) == 3.25
