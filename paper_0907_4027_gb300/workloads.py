"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws numbers and nothing else: it holds no arithmetic of the GSW method, so
both the CUDA path and the FP64 oracle may take their inputs from it.

Optics shared by every workload: SLM pitch p = 15 um, wavelength 1.064 um, effective focal
length f = 4 mm.  Random numbers come from numpy's PCG64 (``default_rng``); trap positions
and initial phases use separate streams of the same seed so that changing M does not
change phi0.  Initial phases are rounded to float32 and handed to both sides as the same
float64 values, so parity never depends on how either side rounds its inputs.

Named workloads (sizes as quoted with the method's published configurations):
  grid16_256    256 x 256 px, 4 x 4 grid of traps in z = 0 at +-2, +-6 um, w = 1, 10 iterations
  rand100_512   512 x 512 px, 100 traps, x, y ~ U[-40, 40] um, z ~ U[-10, 10] um, 30 iterations,
                fast sincos, 8-bit output
  rand1000_1920 1920 x 1152 px, 1000 traps, x, y ~ U[-60, 60] um, z ~ U[-15, 15] um, 50 iterations
  diff256_1024  1024 x 1024 px, 256 traps as rand1000_1920 (differentiable form)
  batch64       64 holograms, sizes from {512^2, 1024^2, 1920 x 1152}, M ~ U{8..2000}
Paper-shaped extras: n x n square grids (spacing 4 um) and the 8-trap cube of side 5 um
(Sec. 5), on a 768 x 768 SLM (the SR hologram size quoted in Sec. 4).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

PITCH = 15e-6
WAVELENGTH = 1.064e-6
FOCAL = 4e-3
TWO_PI = 2.0 * np.pi


@dataclass
class Workload:
    name: str
    W: int
    H: int
    xyz: np.ndarray                 # (M, 3) float64, metres
    phi0: np.ndarray                # (H*W,) float64 holding float32 values, radians in [0, 2pi)
    iters: int
    w0: np.ndarray = None           # (M,) float64; None -> all ones
    precision: str = "accurate"     # "accurate" | "fast" | "separable" | "tensor"
    quantize: bool = False
    pitch: float = PITCH
    wavelength: float = WAVELENGTH
    focal: float = FOCAL
    meta: dict = field(default_factory=dict)

    def __post_init__(self):
        self.xyz = np.ascontiguousarray(self.xyz, dtype=np.float64).reshape(-1, 3)
        if self.w0 is None:
            self.w0 = np.ones(len(self.xyz))

    @property
    def M(self) -> int:
        return len(self.xyz)

    @property
    def N(self) -> int:
        return self.W * self.H

    @property
    def geom(self):
        return (self.W, self.H, self.pitch, self.wavelength, self.focal)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


def phases(N: int, seed: int = 0) -> np.ndarray:
    """phi0 ~ U[0, 2pi), rounded to float32, returned as float64."""
    return _rng(seed, 2).uniform(0.0, TWO_PI, N).astype(np.float32).astype(np.float64)


def random_traps(M: int, xy_um: float, z_um: float, seed: int = 0) -> np.ndarray:
    """M traps with x, y ~ U[-xy_um, xy_um] um and z ~ U[-z_um, z_um] um (metres)."""
    g = _rng(seed, 1)
    x = g.uniform(-xy_um, xy_um, M) * 1e-6
    y = g.uniform(-xy_um, xy_um, M) * 1e-6
    z = g.uniform(-z_um, z_um, M) * 1e-6 if z_um > 0 else np.zeros(M)
    return np.stack([x, y, z], axis=1)


def square_grid(n: int, spacing_um: float = 4.0, z_um: float = 0.0) -> np.ndarray:
    """n x n traps in the plane z, spacing_um apart, centred on the optical axis."""
    c = (np.arange(n) - (n - 1) / 2.0) * spacing_um * 1e-6
    X, Y = np.meshgrid(c, c, indexing="xy")
    return np.stack([X.ravel(), Y.ravel(), np.full(n * n, z_um * 1e-6)], axis=1)


def cube(side_um: float = 5.0) -> np.ndarray:
    """8 traps on the vertices of a cube of the given side, centred on the focus."""
    h = side_um / 2.0 * 1e-6
    v = [(sx * h, sy * h, sz * h) for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)]
    return np.array(v, dtype=np.float64)


def random_case(W: int, H: int, M: int, iters: int = 1, xy_um: float = 40.0, z_um: float = 10.0,
                seed: int = 0, precision: str = "accurate", name: str = None) -> Workload:
    return Workload(name or f"rand{M}_{W}x{H}", W, H, random_traps(M, xy_um, z_um, seed),
                    phases(W * H, seed), iters, precision=precision)


def grid16_256(seed: int = 0) -> Workload:
    return Workload("grid16_256", 256, 256, square_grid(4, 4.0), phases(256 * 256, seed), 10,
                    precision="accurate")


def rand100_512(seed: int = 0) -> Workload:
    return Workload("rand100_512", 512, 512, random_traps(100, 40.0, 10.0, seed),
                    phases(512 * 512, seed), 30, precision="fast", quantize=True)


def rand1000_1920(seed: int = 0) -> Workload:
    return Workload("rand1000_1920", 1920, 1152, random_traps(1000, 60.0, 15.0, seed),
                    phases(1920 * 1152, seed), 50, precision="accurate")


def diff256_1024(seed: int = 0) -> Workload:
    return Workload("diff256_1024", 1024, 1024, random_traps(256, 60.0, 15.0, seed),
                    phases(1024 * 1024, seed), 200, precision="accurate")


def batch64(seed: int = 0, count: int = 64):
    """Independent holograms of uneven size and trap count (batched form)."""
    g = _rng(seed, 3)
    sizes = [(512, 512), (1024, 1024), (1920, 1152)]
    out = []
    for b in range(count):
        W, H = sizes[int(g.integers(0, len(sizes)))]
        M = int(g.integers(8, 2001))
        out.append(Workload(f"batch{b}", W, H, random_traps(M, 60.0, 15.0, seed * 1000 + b + 1),
                            phases(W * H, seed * 1000 + b + 1), 30, precision="fast"))
    return out


def paper_grid(n: int, W: int = 768, iters: int = 1, seed: int = 0) -> Workload:
    """Sec. 5: n x n square grid (4 um spacing) on a 768 x 768 SLM."""
    return Workload(f"grid{n}x{n}_{W}", W, W, square_grid(n, 4.0), phases(W * W, seed), iters)


def paper_cube(W: int = 768, iters: int = 5, seed: int = 0) -> Workload:
    """Sec. 5: the 8-bead cube of side 5 um, 5 GSW iterations per frame."""
    return Workload(f"cube8_{W}", W, W, cube(5.0), phases(W * W, seed), iters)


NAMED = {
    "grid16_256": grid16_256,
    "rand100_512": rand100_512,
    "rand1000_1920": rand1000_1920,
    "diff256_1024": diff256_1024,
}
