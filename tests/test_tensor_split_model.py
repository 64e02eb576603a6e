"""A CPU model of the tensor mode's operand arithmetic on its hardest case (no GPU).

The tensor mode splits every back-projection operand into two FP16 parts (hi = x rounded to
half, lo = the rest rounded to half; P = c_m Y_m(iy) / max|c|, X_m(ix) from FP32 tables) and
sums hi*hi + hi*lo + lo*hi.  Here that split is applied in numpy with exact (FP64) sums, on the
160 x 120, M = 4096 case whose first weight update spreads the weights ~400x: the split alone
must keep |V_m| after one iteration well inside the 1e-4 tolerance.  (It does, at ~1.3e-5; the
GPU's 3.2e-4 on this case therefore comes from the tensor core's accumulation.)  The tables
follow Eq. 2's column and row parts (pinned against the oracle's Delta in test_oracle_pins).
"""
import numpy as np
import pytest

from paper_0907_4027_gb300 import workloads as wl


@pytest.fixture(scope="module")
def oracle():
    import oracle as o
    o.build()
    return o


def f16_split(a):
    hi = a.astype(np.float16).astype(np.float64)
    return hi, (a - hi).astype(np.float16).astype(np.float64)


def complex_split(c):
    rh, rl = f16_split(c.real)
    ih, il = f16_split(c.imag)
    return rh + 1j * ih, rl + 1j * il


def test_fp16_split_alone_keeps_the_4096_trap_case_within_tolerance(oracle):
    w = wl.random_case(160, 120, 4096, seed=31, precision="accurate")
    W, H = w.W, w.H
    p, lam, f = w.pitch, w.wavelength, w.focal
    V0 = oracle.forward(w.geom, w.xyz, w.phi0)
    _, coef = oracle.update_weights(V0, np.ones(w.M))
    ixp, iyp = (np.arange(W) - W // 2) * p, (np.arange(H) - H // 2) * p
    x, y, z = (w.xyz[:, k][:, None] for k in range(3))
    lens = np.pi * z / (lam * f * f)
    X = np.exp(1j * (lens * ixp ** 2 + 2 * np.pi / (lam * f) * x * ixp)).astype(np.complex64)
    Y = np.exp(1j * (lens * iyp ** 2 + 2 * np.pi / (lam * f) * y * iyp)).astype(np.complex64)
    P = coef[None, :] * Y.T.astype(np.complex128) / np.max(np.abs(coef))
    Ph, Pl = complex_split(P)
    Xh, Xl = complex_split(X.astype(np.complex128))
    S = (Ph @ Xh + Ph @ Xl + Pl @ Xh).reshape(-1)
    V1 = oracle.forward(w.geom, w.xyz, np.angle(S))
    r1 = oracle.gsw(w.geom, w.xyz, 1, w.phi0)
    err = np.max(np.abs(np.abs(V1) - np.abs(r1["V"])) / np.abs(r1["V"]))
    assert err < 5e-5, err
