"""ctypes binding of the C ABI in include/hot.h (argument marshalling only).

Every computation runs in libhot.so's CUDA kernels.  Importing this module loads the
library and raises ImportError if it has not been built (``__graft_entry__.build()`` or
``python -m paper_0907_4027_gb300._build``): there is no CPU fallback.

Module-level functions carry the C names (``hot_create`` ... ``hot_last_error``) and take
numpy arrays for host memory or CUDA tensors (anything with ``data_ptr()``) for device
memory.  ``Hologram`` is a small convenience class over them.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libhot.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: build it with __graft_entry__.build() "
                      "(the engine has no CPU fallback)")
lib = ctypes.CDLL(_LIB_PATH)

HOT_OK, HOT_EINVAL, HOT_ENOMEM, HOT_ECUDA, HOT_ETIMEOUT, HOT_ESTATE = 0, -1, -2, -3, -4, -5
HOT_PREC_ACCURATE, HOT_PREC_FAST, HOT_PREC_SEPARABLE, HOT_PREC_TENSOR = 0, 1, 2, 3
PRECISIONS = {"accurate": HOT_PREC_ACCURATE, "fast": HOT_PREC_FAST, "separable": HOT_PREC_SEPARABLE,
              "tensor": HOT_PREC_TENSOR}
HOT_FMT_F32, HOT_FMT_U8 = 0, 1
HOT_MAX_TRAPS = 4096
_STATUS = {0: "HOT_OK", -1: "HOT_EINVAL", -2: "HOT_ENOMEM", -3: "HOT_ECUDA", -4: "HOT_ETIMEOUT",
           -5: "HOT_ESTATE"}

_c_int, _c_double, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)

# Every symbol declared in include/hot.h with its C signature.
SIGNATURES = {
    "hot_create": (_c_int, [ctypes.POINTER(_vp), _c_int, _c_int, _c_double, _c_double, _c_double, _vp]),
    "hot_set_traps": (_c_int, [_vp, _c_int, _vp, _vp]),
    "hot_set_weights": (_c_int, [_vp, _vp]),
    "hot_set_phase": (_c_int, [_vp, _vp, _c_int]),
    "hot_set_precision": (_c_int, [_vp, _c_int]),
    "hot_gsw": (_c_int, [_vp, _c_int, _dp, _dp]),
    "hot_phase_out": (_c_int, [_vp, _vp, _c_int, _c_int]),
    "hot_get_fields": (_c_int, [_vp, _vp, _vp]),
    "hot_sync": (_c_int, [_vp]),
    "hot_get_metrics": (_c_int, [_vp, _dp, _dp]),
    "hot_batch_create": (_c_int, [ctypes.POINTER(_vp), _c_int, _vp, _vp]),
    "hot_batch_gsw": (_c_int, [_vp, _c_int]),
    "hot_batch_destroy": (None, [_vp]),
    "hot_batch_set_tiling": (_c_int, [_vp, _c_int, _c_int, _c_int, _c_double]),
    "hot_batch_get_tiling": (_c_int, [_vp, _ip, _ip, _ip, _dp, _ip]),
    "hot_batch_autotune": (_c_int, [_vp, _c_int, _ip, _ip, _ip, _dp]),
    "hot_batch_latency": (_c_int, [_vp, _vp, _c_int]),
    "hot_set_tiling": (_c_int, [_vp, _c_int, _c_int, _c_int]),
    "hot_set_band": (_c_int, [_vp, _c_int, _c_int]),
    "hot_sharded_begin": (_c_int, [_vp]),
    "hot_sharded_step": (_c_int, [_vp, _c_int]),
    "hot_sharded_sums": (_c_int, [_vp, _c_int, ctypes.POINTER(_vp), _ip]),
    "hot_sharded_end": (_c_int, [_vp, _c_int, _dp, _dp]),
    "hot_get_tiling": (_c_int, [_vp, _ip, _ip, _ip]),
    "hot_set_block_merge": (_c_int, [_vp, _c_int]),
    "hot_get_block_merge": (_c_int, [_vp, _ip, _ip]),
    "hot_set_once": (_c_int, [_vp, _c_int]),
    "hot_get_once": (_c_int, [_vp, _ip, _ip]),
    "hot_autotune": (_c_int, [_vp, _c_int, _ip, _ip, _ip, _dp]),
    "hot_field": (_c_int, [_vp, _vp, _vp]),
    "hot_superposition": (_c_int, [_vp, _vp]),
    "hot_field_adjoint": (_c_int, [_vp, _vp, _vp, _vp]),
    "hot_intensity_loss": (_c_int, [_vp, _vp, _c_double, _vp, _vp]),
    "hot_kernel_launches": (ctypes.c_longlong, [_vp]),
    "hot_use_graphs": (_c_int, [_vp, _c_int]),
    "hot_use_persistent": (_c_int, [_vp, _c_int]),
    "hot_set_trace": (_c_int, [_vp, _c_int]),
    "hot_get_trace": (_c_int, [_vp, _vp, _vp, _c_int]),
    "hot_get_state": (_c_int, [_vp, _vp, _vp]),
    "hot_set_state": (_c_int, [_vp, _vp, _vp]),
    "hot_get_phasors": (_c_int, [_vp, _vp]),
    "hot_set_phasors": (_c_int, [_vp, _vp]),
    "hot_set_wait_limit": (_c_int, [_vp, _c_double]),
    "hot_profile": (_c_int, [_vp, _c_int]),
    "hot_profile_read": (_c_int, [_vp, _vp, _vp]),
    "hot_destroy": (None, [_vp]),
    "hot_last_error": (ctypes.c_char_p, []),
    "hot_sfu_rate": (_c_int, [_c_int, _dp, ctypes.POINTER(_c_int)]),
    "hot_tc_gemm": (_c_int, [_c_int, _c_int, _c_int, _vp, _vp, _vp, _c_int, _c_int, _vp]),
    "hot_tc_shape": (_c_int, [_c_int, _c_int, _c_int, _c_int, _vp]),
    "hot_field_noalloc": (_c_int, [_c_int, _c_int, _c_double, _c_double, _c_double, _c_int, _vp, _vp, _c_int,
                                   _vp, _vp, _vp]),
}
for _name, (_res, _args) in SIGNATURES.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


class HotError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib.hot_last_error().decode(errors="replace")
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")


def _ok(rc: int, where: str) -> int:
    if rc != HOT_OK:
        raise HotError(rc, where)
    return rc


def _host_ptr(a: np.ndarray, dtype) -> tuple:
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(_vp)


def _is_device(x) -> bool:
    return hasattr(x, "data_ptr") and getattr(x, "is_cuda", False)


# ---- C-named wrappers -------------------------------------------------------------

def hot_last_error() -> str:
    return lib.hot_last_error().decode(errors="replace")


def hot_create(width: int, height: int, pitch_m: float, wavelength_m: float, focal_m: float,
               cuda_stream: int | None = None) -> int:
    h = _vp()
    _ok(lib.hot_create(ctypes.byref(h), int(width), int(height), float(pitch_m), float(wavelength_m),
                       float(focal_m), _vp(cuda_stream or 0)), "hot_create")
    return h.value


def hot_set_traps(ctx: int, xyz_m, w0=None) -> None:
    xyz, p = _host_ptr(np.asarray(xyz_m).reshape(-1, 3), np.float64)
    wp = None
    if w0 is not None:
        w0, wp = _host_ptr(np.asarray(w0).reshape(-1), np.float64)
        assert w0.size == len(xyz)
    _ok(lib.hot_set_traps(_vp(ctx), len(xyz), p, wp), "hot_set_traps")


def hot_set_weights(ctx: int, w) -> None:
    w, p = _host_ptr(np.asarray(w).reshape(-1), np.float64)
    _ok(lib.hot_set_weights(_vp(ctx), p), "hot_set_weights")


def hot_set_phase(ctx: int, phi) -> None:
    """phi: host array (N,) or a CUDA float32 tensor of N elements."""
    if _is_device(phi):
        _ok(lib.hot_set_phase(_vp(ctx), _vp(phi.data_ptr()), 1), "hot_set_phase")
    else:
        a, p = _host_ptr(np.asarray(phi).reshape(-1), np.float32)
        _ok(lib.hot_set_phase(_vp(ctx), p, 0), "hot_set_phase")


def hot_set_precision(ctx: int, precision) -> None:
    """precision: "accurate", "fast", "separable", "tensor" or the HOT_PREC_* value."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    _ok(lib.hot_set_precision(_vp(ctx), int(precision)), "hot_set_precision")


def hot_gsw(ctx: int, iters: int, metrics: bool = True):
    """Runs iters GSW iterations; returns (e, u) if metrics else None (queued only)."""
    if metrics:
        e, u = ctypes.c_double(), ctypes.c_double()
        _ok(lib.hot_gsw(_vp(ctx), int(iters), ctypes.byref(e), ctypes.byref(u)), "hot_gsw")
        return e.value, u.value
    _ok(lib.hot_gsw(_vp(ctx), int(iters), None, None), "hot_gsw")
    return None


def hot_phase_out(ctx: int, dst, fmt: int, n: int | None = None):
    """dst: CUDA tensor (filled in stream order) or None -> returns a new host array of n."""
    if _is_device(dst):
        _ok(lib.hot_phase_out(_vp(ctx), _vp(dst.data_ptr()), int(fmt), 1), "hot_phase_out")
        return dst
    if dst is None:
        dst = np.empty(int(n), dtype=np.float32 if fmt == HOT_FMT_F32 else np.uint8)
    _ok(lib.hot_phase_out(_vp(ctx), dst.ctypes.data_as(_vp), int(fmt), 0), "hot_phase_out")
    return dst


def hot_get_fields(ctx: int, M: int):
    V = np.empty(2 * M)
    w = np.empty(M)
    _ok(lib.hot_get_fields(_vp(ctx), V.ctypes.data_as(_vp), w.ctypes.data_as(_vp)), "hot_get_fields")
    return V[0::2] + 1j * V[1::2], w


def hot_superposition(ctx: int, coef) -> None:
    """phi = arg sum_m coef_m e^{i Delta} becomes the phases (SR for coef = e^{i theta})."""
    c = np.asarray(coef, dtype=np.complex128).reshape(-1)
    a, p = _host_ptr(np.stack([c.real, c.imag], axis=-1).reshape(-1), np.float64)
    _ok(lib.hot_superposition(_vp(ctx), p), "hot_superposition")


def hot_field(ctx: int, phi_dev, V_dev) -> None:
    """Eq. 1 fields of device phases phi_dev (N float32) into V_dev (2M float32, Re/Im)."""
    _ok(lib.hot_field(_vp(ctx), _vp(phi_dev.data_ptr()), _vp(V_dev.data_ptr())), "hot_field")


def hot_field_adjoint(ctx: int, phi_dev, G_dev, grad_dev) -> None:
    """Gradient (N float32) of a real loss of V for upstream G_dev = 2 dL/d conj V (2M float32)."""
    _ok(lib.hot_field_adjoint(_vp(ctx), _vp(phi_dev.data_ptr()), _vp(G_dev.data_ptr()),
                              _vp(grad_dev.data_ptr())), "hot_field_adjoint")


def hot_intensity_loss(ctx: int, phi_dev, beta: float, loss_dev, grad_dev=None) -> None:
    """Loss -sum log I + beta var(I) of the traps' intensities for device phases phi_dev, into
    loss_dev (1 float32), and its gradient into grad_dev (N float32) unless None.  Queued."""
    _ok(lib.hot_intensity_loss(_vp(ctx), _vp(phi_dev.data_ptr()), float(beta), _vp(loss_dev.data_ptr()),
                               _vp(grad_dev.data_ptr() if grad_dev is not None else 0)), "hot_intensity_loss")


def hot_get_metrics(ctx: int):
    e, u = ctypes.c_double(), ctypes.c_double()
    _ok(lib.hot_get_metrics(_vp(ctx), ctypes.byref(e), ctypes.byref(u)), "hot_get_metrics")
    return e.value, u.value


def hot_batch_create(ctxs, cuda_stream: int | None = None) -> int:
    arr = (_vp * len(ctxs))(*[_vp(c) for c in ctxs])
    b = _vp()
    _ok(lib.hot_batch_create(ctypes.byref(b), len(ctxs), ctypes.cast(arr, _vp), _vp(cuda_stream or 0)),
        "hot_batch_create")
    return b.value


def hot_batch_gsw(batch: int, iters: int) -> None:
    _ok(lib.hot_batch_gsw(_vp(batch), int(iters)), "hot_batch_gsw")


def hot_batch_destroy(batch: int) -> None:
    lib.hot_batch_destroy(_vp(batch))


def hot_set_band(ctx: int, total_height: int, y0: int) -> None:
    _ok(lib.hot_set_band(_vp(ctx), int(total_height), int(y0)), "hot_set_band")


def hot_sharded_begin(ctx: int) -> None:
    _ok(lib.hot_sharded_begin(_vp(ctx)), "hot_sharded_begin")


def hot_sharded_step(ctx: int, k: int) -> None:
    _ok(lib.hot_sharded_step(_vp(ctx), int(k)), "hot_sharded_step")


def hot_sharded_sums(ctx: int, k: int):
    """(device address, count) of launch k's partial sums: count int64 values."""
    p, n = _vp(), _c_int()
    _ok(lib.hot_sharded_sums(_vp(ctx), int(k), ctypes.byref(p), ctypes.byref(n)), "hot_sharded_sums")
    return p.value, n.value


def hot_sharded_end(ctx: int, iters: int):
    e, u = ctypes.c_double(), ctypes.c_double()
    _ok(lib.hot_sharded_end(_vp(ctx), int(iters), ctypes.byref(e), ctypes.byref(u)), "hot_sharded_end")
    return e.value, u.value


def hot_set_tiling(ctx: int, rows: int = 0, blocks_per_sm: int = 0, chunk: int = 0) -> None:
    _ok(lib.hot_set_tiling(_vp(ctx), int(rows), int(blocks_per_sm), int(chunk)), "hot_set_tiling")


def hot_get_tiling(ctx: int) -> dict:
    r, b, c = _c_int(), _c_int(), _c_int()
    _ok(lib.hot_get_tiling(_vp(ctx), ctypes.byref(r), ctypes.byref(b), ctypes.byref(c)), "hot_get_tiling")
    return {"rows": r.value, "blocks_per_sm": b.value, "chunk": c.value}


def hot_set_block_merge(ctx: int, merge) -> None:
    """merge: schedule blocks per launched block of the GSW step, 1, 2 or 4 (True: 4, False: 1)."""
    if isinstance(merge, bool):
        merge = 4 if merge else 1
    _ok(lib.hot_set_block_merge(_vp(ctx), int(merge)), "hot_set_block_merge")


def hot_get_block_merge(ctx: int) -> dict:
    req, eff = _c_int(), _c_int()
    _ok(lib.hot_get_block_merge(_vp(ctx), ctypes.byref(req), ctypes.byref(eff)), "hot_get_block_merge")
    return {"requested": req.value, "in_effect": eff.value}


def hot_set_once(ctx: int, on: bool) -> None:
    """The one-exponential GSW step of the accurate and fast modes (M <= 128): on (default) or off."""
    _ok(lib.hot_set_once(_vp(ctx), 1 if on else 0), "hot_set_once")


def hot_get_once(ctx: int) -> dict:
    req, eff = _c_int(), _c_int()
    _ok(lib.hot_get_once(_vp(ctx), ctypes.byref(req), ctypes.byref(eff)), "hot_get_once")
    return {"requested": bool(req.value), "in_effect": bool(eff.value)}


def hot_autotune(ctx: int, iters: int) -> dict:
    r, b, c, us = _c_int(), _c_int(), _c_int(), ctypes.c_double()
    _ok(lib.hot_autotune(_vp(ctx), int(iters), ctypes.byref(r), ctypes.byref(b), ctypes.byref(c),
                         ctypes.byref(us)), "hot_autotune")
    return {"rows": r.value, "blocks_per_sm": b.value, "chunk": c.value, "us_per_iter": us.value,
            "merge": hot_get_block_merge(ctx)["in_effect"], "once": hot_get_once(ctx)["in_effect"]}


def hot_batch_set_tiling(batch: int, rows: int = 0, blocks_per_sm: int = 0, chunk: int = 0,
                         group_pairs: float = 0.0) -> None:
    _ok(lib.hot_batch_set_tiling(_vp(batch), int(rows), int(blocks_per_sm), int(chunk), float(group_pairs)),
        "hot_batch_set_tiling")


def hot_batch_get_tiling(batch: int) -> dict:
    r, b, c, g = _c_int(), _c_int(), _c_int(), _c_int()
    gp = ctypes.c_double()
    _ok(lib.hot_batch_get_tiling(_vp(batch), ctypes.byref(r), ctypes.byref(b), ctypes.byref(c), ctypes.byref(gp),
                                 ctypes.byref(g)), "hot_batch_get_tiling")
    return {"rows": r.value, "blocks_per_sm": b.value, "chunk": c.value, "group_pairs": gp.value,
            "groups": g.value}


def hot_batch_autotune(batch: int, iters: int) -> dict:
    r, b, c, us = _c_int(), _c_int(), _c_int(), ctypes.c_double()
    _ok(lib.hot_batch_autotune(_vp(batch), int(iters), ctypes.byref(r), ctypes.byref(b), ctypes.byref(c),
                               ctypes.byref(us)), "hot_batch_autotune")
    return {"rows": r.value, "blocks_per_sm": b.value, "chunk": c.value, "us_per_iter": us.value}


def hot_batch_latency(batch: int, count: int) -> np.ndarray:
    ms = np.empty(count)
    _ok(lib.hot_batch_latency(_vp(batch), ms.ctypes.data_as(_vp), int(count)), "hot_batch_latency")
    return ms


class Batch:
    """GSW on several Holograms at once (one launch per iteration for all of them)."""

    def __init__(self, holos, stream: int | None = None):
        self.holos = list(holos)
        self.handle = hot_batch_create([h.ctx for h in self.holos], stream)

    def gsw(self, iters: int):
        hot_batch_gsw(self.handle, iters)

    def set_tiling(self, rows: int = 0, blocks_per_sm: int = 0, chunk: int = 0, group_pairs: float = 0.0):
        hot_batch_set_tiling(self.handle, rows, blocks_per_sm, chunk, group_pairs)

    def tiling(self) -> dict:
        return hot_batch_get_tiling(self.handle)

    def autotune(self, iters: int) -> dict:
        return hot_batch_autotune(self.handle, iters)

    def latency(self) -> np.ndarray:
        """Per-hologram ms from the start of the last gsw() to that hologram's completion."""
        return hot_batch_latency(self.handle, len(self.holos))

    def metrics(self):
        return [hot_get_metrics(h.ctx) for h in self.holos]

    def close(self):
        if self.handle:
            hot_batch_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def hot_sync(ctx: int) -> None:
    _ok(lib.hot_sync(_vp(ctx)), "hot_sync")


def hot_kernel_launches(ctx: int) -> int:
    return int(lib.hot_kernel_launches(_vp(ctx)))


HOT_KERNEL_STEP, HOT_KERNEL_FORWARD, HOT_KERNEL_FINISH, HOT_KERNEL_OTHER = 0, 1, 2, 3
KERNEL_KINDS = ("step", "forward", "finish", "other")


def hot_use_graphs(ctx: int, enable: bool) -> None:
    _ok(lib.hot_use_graphs(_vp(ctx), int(bool(enable))), "hot_use_graphs")


def hot_set_trace(ctx: int, enable: bool) -> None:
    _ok(lib.hot_set_trace(_vp(ctx), int(bool(enable))), "hot_set_trace")


def hot_get_trace(ctx: int, n: int):
    e, u = np.empty(n), np.empty(n)
    _ok(lib.hot_get_trace(_vp(ctx), e.ctypes.data_as(_vp), u.ctypes.data_as(_vp), int(n)), "hot_get_trace")
    return e, u


def hot_get_state(ctx: int, N: int, M: int):
    phi, w = np.empty(N, dtype=np.float32), np.empty(M, dtype=np.float32)
    _ok(lib.hot_get_state(_vp(ctx), phi.ctypes.data_as(_vp), w.ctypes.data_as(_vp)), "hot_get_state")
    return phi, w


def hot_set_state(ctx: int, phi, w) -> None:
    phi, pp = _host_ptr(np.asarray(phi).reshape(-1), np.float32)
    w, wp = _host_ptr(np.asarray(w).reshape(-1), np.float32)
    _ok(lib.hot_set_state(_vp(ctx), pp, wp), "hot_set_state")


def hot_get_phasors(ctx: int, N: int):
    """The unit phasors the last one-exponential step left for the current phases (float32 [N][2]),
    or None when there are none (HOT_ESTATE)."""
    u = np.empty(2 * N, dtype=np.float32)
    rc = lib.hot_get_phasors(_vp(ctx), u.ctypes.data_as(_vp))
    if rc == HOT_ESTATE:
        return None
    _ok(rc, "hot_get_phasors")
    return u


def hot_set_phasors(ctx: int, u) -> None:
    u, up = _host_ptr(np.asarray(u).reshape(-1), np.float32)
    _ok(lib.hot_set_phasors(_vp(ctx), up), "hot_set_phasors")


def hot_use_persistent(ctx: int, enable: bool) -> None:
    _ok(lib.hot_use_persistent(_vp(ctx), int(bool(enable))), "hot_use_persistent")


def hot_set_wait_limit(ctx: int, seconds: float) -> None:
    _ok(lib.hot_set_wait_limit(_vp(ctx), float(seconds)), "hot_set_wait_limit")


def hot_profile(ctx: int, enable: bool) -> None:
    _ok(lib.hot_profile(_vp(ctx), int(bool(enable))), "hot_profile")


def hot_profile_read(ctx: int) -> dict:
    """{kind: (total_ms, launches)} since the last read (synchronises)."""
    ms = np.zeros(4)
    n = np.zeros(4, dtype=np.int64)
    _ok(lib.hot_profile_read(_vp(ctx), ms.ctypes.data_as(_vp), n.ctypes.data_as(_vp)), "hot_profile_read")
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_KINDS)}


def hot_destroy(ctx: int) -> None:
    lib.hot_destroy(_vp(ctx))


def hot_sfu_rate(op: int = 0):
    """(lane results per clock per SM, SM count) for op 0 = sin+cos of one argument,
    1 = sin alone, 2 = ex2, 3 = FP32 FMA (measured on the current device)."""
    r, n = ctypes.c_double(), _c_int()
    _ok(lib.hot_sfu_rate(int(op), ctypes.byref(r), ctypes.byref(n)), "hot_sfu_rate")
    return r.value, n.value


HOT_TC_TF32, HOT_TC_FP16 = 0, 1
TC_SHAPE_KEYS = ("bn_back", "bn_fwd", "fwd_splits", "fwd_slices_per_split", "Kb", "Kf", "rows_h", "rows_b", "rows_f")


def hot_tc_shape(width: int, height: int, M: int, sms: int) -> dict:
    """Launch shapes of the tensor mode (host computation only)."""
    v = np.zeros(len(TC_SHAPE_KEYS), dtype=np.int32)
    _ok(lib.hot_tc_shape(int(width), int(height), int(M), int(sms), v.ctypes.data_as(_vp)), "hot_tc_shape")
    return {k: int(x) for k, x in zip(TC_SHAPE_KEYS, v)}


def hot_tc_gemm(A, B, C, tile_n: int = 64, operands: int = HOT_TC_TF32, cuda_stream: int | None = None) -> None:
    """C = A B^T on the tensor cores, operands split in two TF32 or FP16 parts: A (rows, K),
    B (cols, K), C (rows, cols) are contiguous float32 CUDA tensors.  Synchronises."""
    rows, K = A.shape
    cols = B.shape[0]
    if B.shape[1] != K or tuple(C.shape) != (rows, cols):
        raise ValueError("hot_tc_gemm: shapes do not match")
    _ok(lib.hot_tc_gemm(int(rows), int(cols), int(K), _vp(A.data_ptr()), _vp(B.data_ptr()), _vp(C.data_ptr()),
                        int(tile_n), int(operands), _vp(cuda_stream or 0)), "hot_tc_gemm")


HOT_NOALLOC_SCRATCH_BYTES = 16 << 20


def hot_field_noalloc(width: int, height: int, pitch_m: float, wavelength_m: float, focal_m: float,
                      xyz_dev, phi_dev, precision, V_dev, eu_dev=None, cuda_stream: int | None = None) -> None:
    """Allocation-free trap fields: all arguments but the sizes are CUDA tensors (device
    memory); xyz_dev (M, 3) float64, phi_dev (N,) float32, V_dev (2M,) float64 output,
    eu_dev (2,) float64 output or None.  Queued on cuda_stream."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    M = int(xyz_dev.numel() // 3)
    _ok(lib.hot_field_noalloc(int(width), int(height), float(pitch_m), float(wavelength_m), float(focal_m), M,
                              _vp(xyz_dev.data_ptr()), _vp(phi_dev.data_ptr()), int(precision),
                              _vp(V_dev.data_ptr()), _vp(eu_dev.data_ptr() if eu_dev is not None else 0),
                              _vp(cuda_stream or 0)), "hot_field_noalloc")


# ---- convenience class -------------------------------------------------------------

class _DeviceArray:
    """A device buffer owned by the library, exposed through __cuda_array_interface__."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 2, "strides": None}


class Hologram:
    """One GSW context: a W x H SLM with the given optics (metres)."""

    def __init__(self, W: int, H: int, pitch: float, wavelength: float, focal: float,
                 stream: int | None = None, precision: str = "accurate"):
        self.W, self.H, self.M = int(W), int(H), 0
        self.ctx = hot_create(W, H, pitch, wavelength, focal, stream)
        hot_set_precision(self.ctx, precision)

    @classmethod
    def from_workload(cls, wl, stream: int | None = None):
        h = cls(wl.W, wl.H, wl.pitch, wl.wavelength, wl.focal, stream, wl.precision)
        h.set_traps(wl.xyz, wl.w0)
        h.set_phase(wl.phi0)
        return h

    @property
    def N(self) -> int:
        return self.W * self.H

    def set_traps(self, xyz, w0=None):
        hot_set_traps(self.ctx, xyz, w0)
        self.M = int(np.asarray(xyz).size // 3)

    def set_weights(self, w):
        hot_set_weights(self.ctx, w)

    def set_phase(self, phi):
        hot_set_phase(self.ctx, phi)

    def superposition(self, coef):
        hot_superposition(self.ctx, coef)

    def set_precision(self, precision):
        hot_set_precision(self.ctx, precision)

    def gsw(self, iters: int, metrics: bool = True):
        return hot_gsw(self.ctx, iters, metrics)

    def phase(self, fmt: str = "f32", out=None):
        f = HOT_FMT_F32 if fmt == "f32" else HOT_FMT_U8
        return hot_phase_out(self.ctx, out, f, self.N)

    def fields(self):
        return hot_get_fields(self.ctx, self.M)

    def metrics(self):
        return hot_get_metrics(self.ctx)

    def sync(self):
        hot_sync(self.ctx)

    def use_graphs(self, enable: bool = True):
        hot_use_graphs(self.ctx, enable)

    def set_tiling(self, rows: int = 0, blocks_per_sm: int = 0, chunk: int = 0):
        hot_set_tiling(self.ctx, rows, blocks_per_sm, chunk)

    def set_block_merge(self, merge=4):
        hot_set_block_merge(self.ctx, merge)

    def set_once(self, on: bool = True):
        hot_set_once(self.ctx, on)

    def use_persistent(self, enable: bool = True):
        hot_use_persistent(self.ctx, enable)

    def set_trace(self, enable: bool = True):
        hot_set_trace(self.ctx, enable)

    def trace(self, iters: int):
        """(e, u) arrays of the last traced gsw(iters): iters + 1 values, F(phi^0) .. F(phi^iters)."""
        return hot_get_trace(self.ctx, iters + 1)

    def get_state(self):
        """(phi, w, u) host copies -- phases, weights and the unit phasors the last one-exponential
        step left for them (None otherwise): resume elsewhere with set_state, bit for bit."""
        phi, w = hot_get_state(self.ctx, self.N, self.M)
        return phi, w, hot_get_phasors(self.ctx, self.N)

    def set_state(self, phi, w, u=None):
        hot_set_state(self.ctx, phi, w)
        if u is not None:
            hot_set_phasors(self.ctx, u)

    def set_wait_limit(self, seconds: float):
        hot_set_wait_limit(self.ctx, seconds)

    def set_band(self, total_height: int, y0: int):
        """This context holds rows y0 .. y0+H-1 of a W x total_height hologram."""
        hot_set_band(self.ctx, total_height, y0)

    # the sharded launch sequence (see paper_0907_4027_gb300.sharded)
    def sharded_begin(self):
        hot_sharded_begin(self.ctx)

    def sharded_step(self, k: int):
        hot_sharded_step(self.ctx, k)

    def sharded_sums(self, k: int):
        """Launch k's partial sums as a zero-copy torch int64 tensor on the device."""
        import torch
        ptr, n = hot_sharded_sums(self.ctx, k)
        return torch.as_tensor(_DeviceArray(ptr, n, "<i8"), device="cuda")

    def sharded_end(self, iters: int):
        return hot_sharded_end(self.ctx, iters)

    def tiling(self) -> dict:
        return dict(hot_get_tiling(self.ctx), merge=hot_get_block_merge(self.ctx)["in_effect"],
                    once=hot_get_once(self.ctx)["in_effect"])

    def autotune(self, iters: int) -> dict:
        """Picks the fastest tiling for hot_gsw(iters); phases and weights are kept."""
        return hot_autotune(self.ctx, iters)

    def profile(self, enable: bool = True):
        hot_profile(self.ctx, enable)

    def profile_read(self) -> dict:
        return hot_profile_read(self.ctx)

    @property
    def launches(self) -> int:
        return hot_kernel_launches(self.ctx)

    def close(self):
        if self.ctx:
            hot_destroy(self.ctx)
            self.ctx = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
