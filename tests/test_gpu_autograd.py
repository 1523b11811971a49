"""Differentiation through the library (torch.autograd with hand-written
backward passes): gradients with respect to spinors and to the fundamental
links (su(N) components at the current field), checked against the oracle's
force and against central finite differences along random su(N) directions.

The 16^3 x 32 SU(3) sextet workload (FP64): S_f = phi^dag (D^dag D)^{-1} phi,
8 random su(3) directions, epsilon = 1e-5, relative agreement 1e-7."""
import numpy as np
import pytest
import torch

from tests import _helpers as H
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hr():
    from paper_2503_06721_gb300 import build, hr
    build.build()
    hr.load()
    return hr


def _omega_coords(T, omega):
    """su(N) coordinates omega^a = 2 Tr(T^a omega) of Hermitian matrices omega[..., N, N]."""
    return 2 * np.einsum("aij,...ji->...a", T, omega).real


@pytest.mark.parametrize("sys", [2, 3], ids=["full", "eo"])
def test_action_gradient_finite_differences(hr, oracle_mod, sys):
    from paper_2503_06721_gb300 import synth, torch_ops
    wl = synth.WORKLOADS["su3_sym_32x16x16x16"]
    lat = hr.Lattice(wl.N, wl.rep, wl.dims, wl.bc, wl.m0)
    U = wl.links(device="cuda")
    g = hr.Gauge(lat, U, precs=("f64",))
    ns = lat.volume if sys == hr.FULL else lat.volume // 2
    phi = synth.gaussian_spinor(ns, lat.D, 31, device="cuda")
    omega = torch_ops.zero_omega(g)
    tol = 1e-13
    S = torch_ops.fermion_action(g, phi, omega, sys=sys, tol=tol)
    (grad,) = torch.autograd.grad(S, omega)
    grad = grad.cpu().numpy()
    T = hr.generators(wl.N)
    eps = 1e-5
    for k in range(8):
        w = synth.gaussian_hermitian(lat.volume * 4, wl.N, 100 + k, synth.STREAM_DIRECTION)
        w = w.reshape(lat.volume, 4, wl.N, wl.N)
        dS = float(np.sum(grad * _omega_coords(T, w.numpy())))
        Sd = []
        for sgn in (+1, -1):
            Up = synth.expm_small(1j * sgn * eps * w.to("cuda")) @ U
            g.update(Up)
            Sd.append(float(torch_ops.fermion_action(g, phi, None, sys=sys, tol=tol)))
        g.update(U)
        fd = (Sd[0] - Sd[1]) / (2 * eps)
        assert abs(fd - dS) <= 1e-7 * abs(fd), (k, fd, dS)
    g.close()


def test_action_gradient_vs_oracle_force(hr, oracle_mod):
    """Autograd link gradient of S_f equals the oracle's force on X = A^{-1} phi."""
    from paper_2503_06721_gb300 import synth, torch_ops
    dims, N, rep = (4, 4, 4, 6), 3, "SYM"
    lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), 0.05)
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), 0.05)
    UF = H.links(dims, N, 0.5, seed=61)
    g = hr.Gauge(lat, G.to_gpu(UF), precs=("f64",))
    phi = H.spinor(lat.volume, N * (N + 1) // 2, 63)
    phi_g = G.to_gpu(G.eo_full(oracle_mod, L, phi)).requires_grad_(True)
    omega = torch_ops.zero_omega(g)
    S = torch_ops.fermion_action(g, phi_g, omega, sys=hr.FULL, tol=1e-13)
    gphi, gw = torch.autograd.grad(S, (phi_g, omega))
    UR = oracle_mod.represent_field(L, UF)
    X, ok, it, rr = oracle_mod.cg(L, UR, 0, phi, tol=1e-13)
    Fo = oracle_mod.force(L, UR, X, oracle_mod.dirac_full(L, UR, X))
    np.testing.assert_allclose(gw.cpu().numpy(), Fo, atol=1e-9 * np.abs(Fo).max())
    # grad_phi = 2 A^{-1} phi (PyTorch convention for a real loss)
    np.testing.assert_allclose(G.from_eo_full(oracle_mod, L, gphi.cpu().numpy()), 2 * X,
                               atol=1e-9 * np.abs(X).max())
    s_val = float(S.detach())
    assert abs(s_val - np.vdot(phi.ravel(), X.ravel()).real) < 1e-10 * abs(s_val)


def test_dirac_and_solve_backward(hr, oracle_mod):
    """Backward of D psi and of x = A^{-1} b against autograd-free references:
    loss = Re <c, f(psi)>  -> grad_psi = f^dag-applied c; link gradient by FD."""
    from paper_2503_06721_gb300 import synth, torch_ops
    dims, N, rep = (4, 2, 4, 6), 2, "ADJ"
    lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), 0.3)
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), 0.3)
    UF = H.links(dims, N, 0.6, seed=71)
    Ug = G.to_gpu(UF)
    g = hr.Gauge(lat, Ug, precs=("f64",))
    V = lat.volume
    psi = G.to_gpu(H.spinor(V, lat.D, 73)).requires_grad_(True)
    c = G.to_gpu(H.spinor(V, lat.D, 75))
    T = hr.generators(N)
    w = synth.gaussian_hermitian(V * 4, N, 77, synth.STREAM_DIRECTION).reshape(V, 4, N, N)
    wa = _omega_coords(T, w.numpy())
    for fn in ("dirac", "solve"):
        omega = torch_ops.zero_omega(g)
        f = getattr(torch_ops, fn)
        kw = {"tol": 1e-13} if fn == "solve" else {}
        y = f(g, psi, omega, sys=hr.FULL, **kw)
        loss = torch.vdot(c.reshape(-1), y.reshape(-1)).real
        gpsi, gw = torch.autograd.grad(loss, (psi, omega))
        # grad_psi: Re<c, M psi> = Re<M^dag c, psi>; M = D or A^{-1} (A Hermitian)
        if fn == "dirac":
            want = g.apply(hr.FULL, hr.F64, c, dagger=True)
        else:
            want, _, _ = g.cg_solve(hr.FULL, c, tol=1e-13)
        assert G.rel(gpsi.detach().cpu().numpy(), want.cpu().numpy()) < 1e-9
        # link gradient vs central differences of the loss
        eps = 1e-5
        vals = []
        for sgn in (+1, -1):
            g.update(synth.expm_small(1j * sgn * eps * w.to("cuda")) @ Ug)
            yd = f(g, psi.detach(), None, sys=hr.FULL, **kw)
            vals.append(float(torch.vdot(c.reshape(-1), yd.reshape(-1)).real))
        g.update(Ug)
        fd = (vals[0] - vals[1]) / (2 * eps)
        dl = float(np.sum(gw.cpu().numpy() * wa))
        assert abs(fd - dl) <= 1e-7 * abs(fd), (fn, fd, dl)
