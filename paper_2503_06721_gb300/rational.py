"""Rational approximations for the RHMC (Sec. 4.3.2), through the C ABI.

The RHMC replaces the fermion determinant's power x^(-alpha) by a rational
function in partial fractions, r(x) = a0 + sum_k a_k / (x + b_k), whose poles
b_k become the shifts of one multi-shift inversion.  The paper computes the
coefficients with the Remez algorithm and stores them in a table; here
hr_rational_approx (libhr, a Remez exchange) computes them when needed.  This
module only marshals: approx() returns the library's coefficients as a
RationalApprox, degree_for() asks the library for increasing degrees.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class RationalApprox:
    """r(x) = a0 + sum_k residues[k] / (x + poles[k]) ~ x^(-alpha) on [lo, hi],
    with max |r(x) x^alpha - 1| = max_rel_err."""
    alpha: float
    lo: float
    hi: float
    a0: float
    residues: tuple
    poles: tuple
    max_rel_err: float


def approx(alpha: float, n: int, lo: float, hi: float) -> RationalApprox:
    """The best degree-(n, n) relative approximation of x^(-alpha) on [lo, hi]
    (hr_rational_approx): alpha = 1/2 for the one-flavour action and force,
    alpha = -1/4 for its heat bath."""
    from paper_2503_06721_gb300 import hr
    a0, res, poles, err = hr.rational_approx(alpha, n, lo, hi)
    return RationalApprox(alpha=float(alpha), lo=float(lo), hi=float(hi), a0=a0, residues=res, poles=poles,
                          max_rel_err=err)


def degree_for(alpha: float, lo: float, hi: float, tol: float, n_max: int = 40) -> int:
    """Smallest degree whose relative error on [lo, hi] is <= tol."""
    for n in range(1, n_max + 1):
        if approx(alpha, n, lo, hi).max_rel_err <= tol:
            return n
    raise ValueError(f"no degree <= {n_max} reaches {tol} on [{lo}, {hi}]")
