"""Rational approximations for the RHMC (Sec. 4.3.2).

The RHMC replaces the fermion determinant's power x^(-alpha) by a rational
function in partial fractions, r(x) = a0 + sum_k a_k / (x + b_k), whose poles
b_k become the shifts of one multi-shift inversion.  The paper computes its
coefficients with the Remez algorithm and stores them in a table; here they
are computed when needed.

For alpha = 1/2 (one flavour, det Q = det (Q^2)^(1/2)) the best uniform
relative approximation of degree (n, n) on [lo, hi] is known in closed form
(Zolotarev): with b = hi / lo, kappa'^2 = 1 - 1/b, K' = K(kappa') and

    c_l = sn^2(l K' / (2n+1); kappa') / (1 - sn^2(l K' / (2n+1); kappa')),

    1/sqrt(y) ~ d0 prod_{l=1..n} (y + c_{2l}) / (y + c_{2l-1})   on [1, b],

with d0 fixed so that the relative error 1 - sqrt(y) r(y) takes its extreme
values +D and -D equally; the error then alternates 2n + 2 times, which by
Chebyshev's alternation theorem characterises the unique best
approximation.  Substituting y = x / lo gives the poles b_l = lo c_{2l-1} of
r on [lo, hi].

This is host-side set-up (numpy / scipy); nothing here runs on the GPU.  In
double precision the evaluated error stops falling near 1e-13 (degree 20 and
above on [1e-4, 1]); max_rel_err is the spread of the evaluated factored
form over its sample points, so near that floor it reports the floor
rather than the exact-arithmetic error.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class RationalApprox:
    """r(x) = a0 + sum_k residues[k] / (x + poles[k]) ~ x^(-alpha) on [lo, hi]."""
    alpha: float
    lo: float
    hi: float
    a0: float
    residues: tuple
    poles: tuple
    max_rel_err: float

    def __call__(self, x):
        x = np.asarray(x, dtype=np.float64)
        out = np.full(x.shape, self.a0)
        for a, b in zip(self.residues, self.poles):
            out = out + a / (x + b)
        return out

    def rel_error(self, x):
        """1 - r(x) / x^(-alpha)."""
        x = np.asarray(x, dtype=np.float64)
        return 1.0 - self(x) * x ** self.alpha


def _zolotarev_factors(n: int, b: float):
    from scipy.special import ellipj, ellipk
    m = 1.0 - 1.0 / b                     # parameter kappa'^2 of the elliptic functions
    K = ellipk(m)
    sn = ellipj(np.arange(1, 2 * n + 1) * K / (2 * n + 1), m)[0]
    c = sn * sn / (1.0 - sn * sn)
    return c[1::2], c[0::2]               # numerator roots c_{2l}, poles c_{2l-1}


def zolotarev_inv_sqrt(n: int, lo: float, hi: float, samples: int = 20001) -> RationalApprox:
    """Best degree-(n, n) relative approximation of x^(-1/2) on [lo, hi]."""
    if not (n >= 1 and 0 < lo < hi):
        raise ValueError("need n >= 1 and 0 < lo < hi")
    b = hi / lo
    num, den = _zolotarev_factors(n, b)
    # d0 from the extreme values of sqrt(y) prod (y + c_2l)/(y + c_2l-1) on [1, b]
    y = np.exp(np.linspace(0.0, np.log(b), samples))
    f = np.sqrt(y) * np.prod((y[:, None] + num) / (y[:, None] + den), axis=1)
    d0 = 2.0 / (f.max() + f.min())
    delta = (f.max() - f.min()) / (f.max() + f.min())
    # partial fractions in x = lo y:  prod (x + lo c_2l) / (x + lo c_2l-1)
    zeros, poles = lo * num, lo * den
    scale = d0 / np.sqrt(lo)
    residues = []
    for k, p in enumerate(poles):
        r = scale * np.prod(zeros - p)
        others = np.delete(poles, k)
        r /= np.prod(others - p)
        residues.append(float(r))
    return RationalApprox(alpha=0.5, lo=float(lo), hi=float(hi), a0=float(scale),
                          residues=tuple(residues), poles=tuple(float(p) for p in poles),
                          max_rel_err=float(delta))


def degree_for(lo: float, hi: float, tol: float, n_max: int = 40) -> int:
    """Smallest Zolotarev degree whose relative error on [lo, hi] is <= tol."""
    for n in range(1, n_max + 1):
        if zolotarev_inv_sqrt(n, lo, hi).max_rel_err <= tol:
            return n
    raise ValueError(f"no degree <= {n_max} reaches {tol} on [{lo}, {hi}]")
