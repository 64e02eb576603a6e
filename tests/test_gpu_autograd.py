"""Differentiable form: hot_field / hot_field_adjoint through the C ABI and the autograd
Function, against the FP64 oracle (forward and adjoint) and FP64 central differences.

Tolerances: fields 1e-4 relative (as the GSW parity tests); the adjoint superposition
|grad_gpu - grad_oracle| <= tol_S * sum_m |G_m| / N (the FP32 rounding bound of the
superposition, tol_S = 2e-6 accurate, 2e-5 fast); loss gradients within 1e-3 of their norm.
"""
import numpy as np
import pytest

import oracle
from paper_0907_4027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

REL_V = 1e-4
TOL_S = {"accurate": 2e-6, "fast": 2e-5, "separable": 4e-6}


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0907_4027_gb300 import _build
    _build.build()
    from paper_0907_4027_gb300 import autograd as ag
    from paper_0907_4027_gb300 import hot
    return torch, hot, ag


def holo_for(hot, torch, w):
    h = hot.Hologram(w.W, w.H, w.pitch, w.wavelength, w.focal, torch.cuda.current_stream().cuda_stream,
                     w.precision)
    h.set_traps(w.xyz)
    return h


def oracle_loss_G(V, beta=10.0):
    """G = 2 dL/d conj V for L = -sum log I + beta var(I), I = |V|^2 (population variance)."""
    I = np.abs(V) ** 2
    dLdI = -1.0 / I + beta * 2.0 / len(I) * (I - I.mean())
    return 2.0 * dLdI * V


def loss_value(V, beta=10.0):
    I = np.abs(V) ** 2
    return float(-np.log(I).sum() + beta * I.var())


@pytest.mark.parametrize("precision", ["accurate", "fast", "separable"])
@pytest.mark.parametrize("W,H,M", [(100, 37, 13), (64, 64, 130), (33, 20, 3)])
def test_field_and_adjoint_match_oracle(env, W, H, M, precision):
    torch, hot, ag = env
    w = wl.random_case(W, H, M, seed=3 * W + M, precision=precision)
    rng = np.random.default_rng(W + H)
    phi = rng.uniform(-np.pi, np.pi, w.N).astype(np.float32)
    G = (rng.normal(size=M) + 1j * rng.normal(size=M)).astype(np.complex64)
    with holo_for(hot, torch, w) as h:
        phi_d = torch.tensor(phi, device="cuda")
        V = torch.empty(2 * M, dtype=torch.float32, device="cuda")
        hot.hot_field(h.ctx, phi_d, V)
        G_d = torch.view_as_real(torch.tensor(G, device="cuda")).reshape(-1).contiguous()
        grad = torch.empty_like(phi_d)
        hot.hot_field_adjoint(h.ctx, phi_d, G_d, grad)
        torch.cuda.synchronize()
        v = V.cpu().numpy().astype(np.float64)
        Vg = v[0::2] + 1j * v[1::2]
        g = grad.cpu().numpy().astype(np.float64)
    oV = oracle.forward(w.geom, w.xyz, phi.astype(np.float64))
    assert np.max(np.abs(np.abs(Vg) - np.abs(oV)) / np.abs(oV)) < REL_V
    og = oracle.adjoint(w.geom, w.xyz, phi.astype(np.float64), G.astype(np.complex128))
    bound = TOL_S[precision] * np.sum(np.abs(G)) / w.N
    assert np.max(np.abs(g - og)) <= bound, (np.max(np.abs(g - og)), bound)


def test_autograd_loss_gradient_matches_oracle(env):
    torch, hot, ag = env
    w = wl.random_case(96, 80, 12, seed=9, precision="accurate")
    with holo_for(hot, torch, w) as h:
        phi = torch.tensor(w.phi0, dtype=torch.float32, device="cuda", requires_grad=True)
        V = ag.trap_fields(h, phi)
        L = ag.trap_intensity_loss(V)
        L.backward()
        g = phi.grad.cpu().numpy().astype(np.float64)
        Lg = float(L.item())
    phi64 = w.phi0.astype(np.float32).astype(np.float64)
    oV = oracle.forward(w.geom, w.xyz, phi64)
    og = oracle.adjoint(w.geom, w.xyz, phi64, oracle_loss_G(oV))
    assert abs(Lg - loss_value(oV)) < 1e-4 * abs(loss_value(oV))
    assert np.linalg.norm(g - og) < 1e-3 * np.linalg.norm(og)


@pytest.mark.slow
def test_gradient_against_central_differences_1024(env):
    """diff256_1024 (1024 x 1024 px, 256 traps): autograd gradient of
    L = -sum log I + 10 var(I) against FP64 central differences (h = 1e-3 rad) on 32 seeded
    pixels.  The differences use the exact single-pixel update of Eq. 1,
    V(phi + h e_j) = V + (1/N)(e^{i(phi_j + h)} - e^{i phi_j}) e^{-i Delta_j^m}, in FP64."""
    torch, hot, ag = env
    w = wl.diff256_1024()
    with holo_for(hot, torch, w) as h:
        phi = torch.tensor(w.phi0, dtype=torch.float32, device="cuda", requires_grad=True)
        L = ag.trap_intensity_loss(ag.trap_fields(h, phi))
        L.backward()
        g = phi.grad.cpu().numpy().astype(np.float64)
    phi64 = w.phi0.astype(np.float32).astype(np.float64)
    V = oracle.forward(w.geom, w.xyz, phi64)
    pix = np.random.default_rng(0).choice(w.N, 32, replace=False)
    hstep = 1e-3
    fd = []
    for j in pix:
        ix, iy = int(j % w.W), int(j // w.W)
        d = np.array([oracle.delta(w.geom, t, ix, iy) for t in w.xyz])
        base = np.exp(1j * phi64[j])
        Lp = loss_value(V + (np.exp(1j * (phi64[j] + hstep)) - base) * np.exp(-1j * d) / w.N)
        Lm = loss_value(V + (np.exp(1j * (phi64[j] - hstep)) - base) * np.exp(-1j * d) / w.N)
        fd.append((Lp - Lm) / (2 * hstep))
    fd = np.array(fd)
    assert np.linalg.norm(g[pix] - fd) < 2e-3 * np.linalg.norm(fd), (g[pix][:4], fd[:4])


def test_adam_improves_uniformity(env):
    """A few Adam steps on the phases with the trap-intensity loss raise the uniformity and
    lower the loss (the differentiable alternative to the GSW weight update)."""
    torch, hot, ag = env
    w = wl.random_case(128, 128, 16, seed=4, xy_um=40, z_um=8, precision="fast")
    with holo_for(hot, torch, w) as h:
        phi = torch.tensor(w.phi0, dtype=torch.float32, device="cuda", requires_grad=True)
        opt = torch.optim.Adam([phi], lr=1e-2)
        losses, us = [], []
        for it in range(60):
            opt.zero_grad()
            V = ag.trap_fields(h, phi)
            L = ag.trap_intensity_loss(V)
            L.backward()
            opt.step()
            I = (V.abs() ** 2).detach()
            losses.append(L.item())
            us.append(float(1 - (I.max() - I.min()) / (I.max() + I.min())))
    assert losses[-1] < losses[0] and us[-1] > us[0] + 0.2, (losses[0], losses[-1], us[0], us[-1])


@pytest.mark.parametrize("precision", ["accurate", "fast", "separable"])
def test_library_loss_and_gradient_match_oracle(env, precision):
    """hot_intensity_loss: the loss -sum log I + 10 var(I) and its gradient from one library call,
    against the FP64 oracle's loss and gradient (forward field, the derivative of the loss, the
    adjoint), and the autograd Function built on it against the PyTorch-loss path."""
    torch, hot, ag = env
    w = wl.random_case(96, 80, 12, seed=9, precision=precision)
    with holo_for(hot, torch, w) as h:
        phi = torch.tensor(w.phi0, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        grad = torch.empty_like(phi)
        hot.hot_intensity_loss(h.ctx, phi, 10.0, loss, grad)
        L = float(loss.item())
        g = grad.cpu().numpy().astype(np.float64)
        p1 = phi.clone().requires_grad_(True)
        ag.intensity_loss(h, p1).backward()
        p2 = phi.clone().requires_grad_(True)
        ag.trap_intensity_loss(ag.trap_fields(h, p2)).backward()
        g1, g2 = p1.grad.cpu().numpy(), p2.grad.cpu().numpy()
        hot.hot_intensity_loss(h.ctx, phi, 10.0, loss)           # the loss alone
        assert float(loss.item()) == L
    phi64 = w.phi0.astype(np.float32).astype(np.float64)
    oV = oracle.forward(w.geom, w.xyz, phi64)
    og = oracle.adjoint(w.geom, w.xyz, phi64, oracle_loss_G(oV))
    assert abs(L - loss_value(oV)) < 1e-4 * abs(loss_value(oV))
    assert np.linalg.norm(g - og) < 1e-3 * np.linalg.norm(og)
    assert np.array_equal(g1, g.astype(np.float32))
    assert np.linalg.norm(g1 - g2) < 1e-3 * np.linalg.norm(g2)
