"""FP64 CPU oracle for GSW hologram generation by direct superposition.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The CUDA product path never
imports this package and this package never imports the product.

The arithmetic lives in ``hot_oracle.c`` (plain C, double precision, OpenMP over rows);
this module compiles it with gcc on first use and exposes numpy-level wrappers.
Each wrapper names the passage of Bianchi & Di Leonardo it follows:

  delta           Eq. 2   lens + grating phase Delta_j^m
  forward         Eq. 1   trap fields V_m
  backproject     Sec. 4  back-propagation S_j = sum_m c_m e^{i Delta_j^m}, phi_j = arg S_j
  update_weights  Sec. 3  w_m <- w_m <|V|>/|V_m|, c_m = w_m V_m/|V_m|
  metrics         Eq. 4   efficiency e and uniformity u
  gsw             Sec. 3 / Fig. 2  K GSW iterations
  quantize        Sec. 5  8-bit grey levels mapped linearly onto 0..2pi
  adjoint         derivative of Eq. 1 (gradient of a real loss of V w.r.t. phi)

Parity status: every function here is pinned by closed forms or library routines in
``tests/test_oracle_pins.py`` (none is "parity unpinned").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hot_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile hot_oracle.c into liboracle.so next to it (gcc, -O2, no fast math)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-fno-fast-math", "-fPIC", "-shared", "-std=c11", "-Wall"]
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        # No OpenMP runtime: the oracle still works, single threaded.
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True, capture_output=True, text=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i, d = ctypes.c_int, ctypes.c_double
        lib.oracle_threads.argtypes = [i]
        lib.oracle_threads.restype = i
        lib.oracle_delta.argtypes = [i, i, d, d, d, d, d, d, i, i]
        lib.oracle_delta.restype = d
        geo = [i, i, d, d, d, i, _dp]
        lib.oracle_forward.argtypes = geo + [_dp, _dp]
        lib.oracle_forward.restype = i
        lib.oracle_backproject.argtypes = geo + [_dp, _dp, _dp]
        lib.oracle_backproject.restype = i
        lib.oracle_update_weights.argtypes = [i, _dp, _dp, _dp, i]
        lib.oracle_update_weights.restype = i
        lib.oracle_metrics.argtypes = [i, _dp, _dp, _dp]
        lib.oracle_metrics.restype = None
        lib.oracle_gsw.argtypes = geo + [i, _dp, _dp, _dp, _dp, _dp]
        lib.oracle_gsw.restype = i
        lib.oracle_quantize.argtypes = [ctypes.c_long, _dp, _u8p]
        lib.oracle_quantize.restype = None
        lib.oracle_adjoint.argtypes = geo + [_dp, _dp, _dp]
        lib.oracle_adjoint.restype = i
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp) if a is not None else None


def _cplx_in(c) -> np.ndarray:
    """Complex (or real) values -> interleaved (Re, Im) float64."""
    c = np.asarray(c, dtype=np.complex128).reshape(-1)
    return _f64(np.stack([c.real, c.imag], axis=-1).reshape(-1))


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle_{what}: invalid arguments")


def set_threads(n: int = 0) -> int:
    """Set (n > 0) and return the number of OpenMP threads the oracle uses."""
    return int(_load().oracle_threads(int(n)))


def delta(geom, xyz_m, ix: int, iy: int) -> float:
    """Eq. 2 for one pixel (ix, iy) and one trap xyz_m = (x_m, y_m, z_m) in metres."""
    W, H, p, lam, f = geom
    x, y, z = (float(v) for v in xyz_m)
    return float(_load().oracle_delta(W, H, p, lam, f, x, y, z, int(ix), int(iy)))


def forward(geom, xyz, phi) -> np.ndarray:
    """Eq. 1: complex trap fields V (M,) for pixel phases phi (H*W,)."""
    W, H, p, lam, f = geom
    xyz = _f64(xyz).reshape(-1, 3)
    phi = _f64(phi).reshape(-1)
    assert phi.size == W * H
    V = np.empty(2 * len(xyz))
    _check(_load().oracle_forward(W, H, p, lam, f, len(xyz), _ptr(xyz), _ptr(phi), _ptr(V)), "forward")
    return V[0::2] + 1j * V[1::2]


def backproject(geom, xyz, coef, want_S: bool = False):
    """Sec. 4 back-propagation: phi = arg S with S_j = sum_m coef_m e^{i Delta_j^m}.

    Returns phi (H*W,), or (phi, S) when want_S."""
    W, H, p, lam, f = geom
    xyz = _f64(xyz).reshape(-1, 3)
    c = _cplx_in(coef)
    assert c.size == 2 * len(xyz)
    phi = np.empty(W * H)
    S = np.empty(2 * W * H) if want_S else None
    _check(_load().oracle_backproject(W, H, p, lam, f, len(xyz), _ptr(xyz), _ptr(c), _ptr(phi),
                                      _ptr(S)), "backproject")
    if want_S:
        return phi, S[0::2] + 1j * S[1::2]
    return phi


def update_weights(V, w, update: bool = True):
    """Sec. 3 weight update.  Returns (w_new, coef) without touching the inputs."""
    Vi = _cplx_in(V)
    w = _f64(w).reshape(-1).copy()
    assert Vi.size == 2 * w.size
    coef = np.empty(Vi.size)
    _check(_load().oracle_update_weights(w.size, _ptr(Vi), _ptr(w), _ptr(coef), int(update)), "update_weights")
    return w, coef[0::2] + 1j * coef[1::2]


def metrics(V):
    """Eq. 4: (e, u) of the trap fields V."""
    Vi = _cplx_in(V)
    e, u = ctypes.c_double(), ctypes.c_double()
    _load().oracle_metrics(Vi.size // 2, _ptr(Vi), ctypes.byref(e), ctypes.byref(u))
    return e.value, u.value


def gsw(geom, xyz, K: int, phi0, w0=None):
    """K GSW iterations (Sec. 3, Fig. 2) from phi0 and w0 (default 1).

    Returns dict(phi, w, V, e, u) where V, e, u come from the forward of the final phi."""
    W, H, p, lam, f = geom
    xyz = _f64(xyz).reshape(-1, 3)
    M = len(xyz)
    phi = _f64(phi0).reshape(-1).copy()
    assert phi.size == W * H
    w = np.ones(M) if w0 is None else _f64(w0).reshape(-1).copy()
    V = np.empty(2 * M)
    e, u = ctypes.c_double(), ctypes.c_double()
    _check(_load().oracle_gsw(W, H, p, lam, f, M, _ptr(xyz), int(K), _ptr(phi), _ptr(w), _ptr(V),
                              ctypes.byref(e), ctypes.byref(u)), "gsw")
    return dict(phi=phi, w=w, V=V[0::2] + 1j * V[1::2], e=e.value, u=u.value)


def quantize(phi) -> np.ndarray:
    """Sec. 5 8-bit encoding: g = rint(phi * 256 / 2pi) mod 256."""
    phi = _f64(phi).reshape(-1)
    g = np.empty(phi.size, dtype=np.uint8)
    _load().oracle_quantize(phi.size, _ptr(phi), g.ctypes.data_as(_u8p))
    return g


def adjoint(geom, xyz, phi, G) -> np.ndarray:
    """Gradient dL/dphi (H*W,) for upstream G_m = 2 dL/d conj(V_m) (derivative of Eq. 1)."""
    W, H, p, lam, f = geom
    xyz = _f64(xyz).reshape(-1, 3)
    phi = _f64(phi).reshape(-1)
    Gi = _cplx_in(G)
    assert Gi.size == 2 * len(xyz) and phi.size == W * H
    grad = np.empty(W * H)
    _check(_load().oracle_adjoint(W, H, p, lam, f, len(xyz), _ptr(xyz), _ptr(phi), _ptr(Gi),
                                  _ptr(grad)), "adjoint")
    return grad
