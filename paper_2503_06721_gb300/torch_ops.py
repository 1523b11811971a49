"""torch.autograd wrappers around the library (Sec. 2.5, HMC force).

The gauge field enters through a Lie-algebra displacement omega[V, 4, N*N-1]
at the current links: U(x,mu) -> exp(i sum_a omega^a T^a) U(x,mu), evaluated at
omega = 0.  Passing a zero omega with requires_grad=True makes autograd return
the su(N) derivative of the loss with respect to every fundamental link,
which is exactly what the force kernel computes.  All backward passes are
hand-written:

  y = D psi                 grad_psi = D^dag g,       grad_omega = -1/2 F(psi, g)
  x = A^{-1} b, A = D^dag D  lam = A^{-1} g (a second solve, no stored iterations)
                            grad_b = lam,             grad_omega = 1/2 [F(lam, Dx) + F(x, D lam)]
  S = <phi, A^{-1} phi>     grad_phi = 2 A^{-1} phi,  grad_omega = F(X, D X), X = A^{-1} phi
                            (computed with the solve, hr_cg_solve_force)

where F(X, Y) = d/de [-2 Re <Y, D X>] (hr_dirac_force) and D is D_m for the
FULL system or Dhat for the even/odd one.  Complex gradients follow PyTorch's
convention: for a real loss L, dL = Re <grad, dz>.
"""
from __future__ import annotations

import torch

from . import hr


def _check_zero(omega):
    if omega is not None and bool((omega != 0).any()):
        raise ValueError("omega is the displacement at the current links and must be zero; "
                         "move the links with Gauge.update instead")


def _D(gauge, sys, v, dagger=False):
    return gauge.apply(sys, hr.F64, v, dagger=dagger)


class _DiracFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi, omega, gauge, sys, dagger):
        _check_zero(omega)
        ctx.gauge, ctx.sys, ctx.dagger = gauge, sys, dagger
        ctx.save_for_backward(psi)
        return _D(gauge, sys, psi, dagger)

    @staticmethod
    def backward(ctx, g):
        (psi,) = ctx.saved_tensors
        g = g.contiguous()
        gauge, sys, dagger = ctx.gauge, ctx.sys, ctx.dagger
        grad_psi = _D(gauge, sys, g, not dagger) if ctx.needs_input_grad[0] else None
        grad_omega = None
        if ctx.needs_input_grad[1]:
            # Re<g, dD psi> = -1/2 F(psi, g);  Re<g, dD^dag psi> = Re<psi, dD g> = -1/2 F(g, psi)
            X, Y = (g, psi) if dagger else (psi, g)
            grad_omega = gauge.force(sys, X.contiguous(), Y.contiguous(), coeff=-0.5)
        return grad_psi, grad_omega, None, None, None


class _SolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, omega, gauge, sys, tol, inner):
        _check_zero(omega)
        x, res, st = gauge.cg_solve(sys, b.contiguous(), tol=tol, inner=inner)
        ctx.gauge, ctx.sys, ctx.tol, ctx.inner = gauge, sys, tol, inner
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        gauge, sys = ctx.gauge, ctx.sys
        lam, _, _ = gauge.cg_solve(sys, g.contiguous(), tol=ctx.tol, inner=ctx.inner)
        grad_omega = None
        if ctx.needs_input_grad[1]:
            F = gauge.force(sys, lam, _D(gauge, sys, x), coeff=0.5)
            grad_omega = gauge.force(sys, x, _D(gauge, sys, lam), coeff=0.5, F=F)
        return lam, grad_omega, None, None, None, None


class _ActionFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, omega, gauge, sys, tol, inner):
        _check_zero(omega)
        ctx.gauge, ctx.sys = gauge, sys
        F = None
        if ctx.needs_input_grad[1]:
            # the force needs D X and its neighbours, which the solve's final
            # true residual already applied: solve and force in one call
            X, F, _, res, st = gauge.cg_solve_force(sys, phi.contiguous(), tol=tol, inner=inner, coeff=1.0)
        else:
            X, res, st = gauge.cg_solve(sys, phi.contiguous(), tol=tol, inner=inner)
        ctx.force = F
        ctx.save_for_backward(X)
        S = torch.vdot(phi.reshape(-1), X.reshape(-1)).real
        return S

    @staticmethod
    def backward(ctx, gS):
        (X,) = ctx.saved_tensors
        grad_phi = 2.0 * gS * X if ctx.needs_input_grad[0] else None
        grad_omega = ctx.force * gS if ctx.needs_input_grad[1] else None
        return grad_phi, grad_omega, None, None, None, None


def zero_omega(gauge, requires_grad=True, device="cuda"):
    lat = gauge.lat
    return torch.zeros((lat.volume, 4, lat.N * lat.N - 1), dtype=torch.float64, device=device,
                       requires_grad=requires_grad)


def dirac(gauge, psi, omega=None, sys=hr.FULL, dagger=False):
    """D_m psi (sys=FULL) or Dhat psi (sys=EO_PRECOND), FP64, differentiable."""
    return _DiracFn.apply(psi, omega, gauge, sys, dagger)


def solve(gauge, b, omega=None, sys=hr.FULL, tol=1e-12, inner=hr.F64):
    """x = (D^dag D)^{-1} b (or Dhat^dag Dhat), differentiable."""
    return _SolveFn.apply(b, omega, gauge, sys, tol, inner)


def fermion_action(gauge, phi, omega=None, sys=hr.FULL, tol=1e-12, inner=hr.F64):
    """S_f = phi^dag (D^dag D)^{-1} phi, differentiable in phi and omega."""
    return _ActionFn.apply(phi, omega, gauge, sys, tol, inner)
