"""Pins of the RHMC's rational approximation (Sec. 4.3.2), host-side set-up:
the Zolotarev coefficients must give the unique best relative approximation of
x^(-1/2) (Chebyshev's alternation theorem: the error takes its extreme value
with alternating signs at 2n + 2 points), and applied to a matrix through the
oracle's shifted solves they must approximate A^(-1/2) b within that error
(checked against a dense eigendecomposition)."""
import numpy as np
import pytest

from paper_2503_06721_gb300 import rational
from tests import _helpers as H


def _extrema(e):
    d = np.sign(np.diff(e))
    idx = np.where(np.diff(d) != 0)[0] + 1
    return np.concatenate([[0], idx, [len(e) - 1]])


@pytest.mark.parametrize("n,lo,hi", [(3, 1e-2, 1.0), (6, 1e-4, 10.0), (8, 0.05, 900.0)])
def test_equioscillation(n, lo, hi):
    ra = rational.zolotarev_inv_sqrt(n, lo, hi)
    assert len(ra.poles) == n and all(p > 0 for p in ra.poles)
    x = np.exp(np.linspace(np.log(lo), np.log(hi), 400001))
    e = ra.rel_error(x)
    D = np.abs(e).max()
    assert abs(D - ra.max_rel_err) <= 1e-3 * D
    pts = _extrema(e)
    assert len(pts) == 2 * n + 2, len(pts)
    vals = e[pts] / D
    # alternating signs, equal magnitudes
    assert np.all(np.abs(np.abs(vals) - 1) < 2e-3), vals
    assert np.all(vals[1:] * vals[:-1] < 0)
    # both interval ends are extreme points of the best approximation
    assert abs(abs(e[0]) - D) < 2e-3 * D and abs(abs(e[-1]) - D) < 2e-3 * D


def test_error_falls_with_degree():
    errs = [rational.zolotarev_inv_sqrt(n, 1e-3, 1.0).max_rel_err for n in range(2, 12)]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    # Zolotarev's error falls geometrically in n (rate set by the interval)
    ratios = np.array(errs[1:]) / np.array(errs[:-1])
    assert ratios.max() < 0.25 and ratios.std() < 0.1 * ratios.mean()
    n = rational.degree_for(1e-3, 1.0, 1e-7)
    assert rational.zolotarev_inv_sqrt(n, 1e-3, 1.0).max_rel_err <= 1e-7
    assert rational.zolotarev_inv_sqrt(n - 1, 1e-3, 1.0).max_rel_err > 1e-7


def test_partial_fractions_match_product():
    """a0 + sum a_k/(x + b_k) is the same function as the factored form."""
    n, lo, hi = 5, 0.01, 3.0
    ra = rational.zolotarev_inv_sqrt(n, lo, hi)
    num, den = rational._zolotarev_factors(n, hi / lo)
    x = np.exp(np.linspace(np.log(lo / 10), np.log(hi * 10), 101))
    prod = ra.a0 * np.prod((x[:, None] + lo * num) / (x[:, None] + lo * den), axis=1)
    np.testing.assert_allclose(ra(x), prod, rtol=1e-12)


def test_matrix_inverse_square_root(oracle_mod):
    """r(A) b = a0 b + sum_k a_k (A + b_k)^-1 b ~ A^(-1/2) b for A = Dhat^dag Dhat
    on a 2^4 lattice: |r(A) b - A^(-1/2) b| <= D |A^(-1/2) b| when the spectrum of
    A lies in [lo, hi] (the relative bound holds eigenvalue by eigenvalue)."""
    N, rep = 2, "ADJ"
    dims = (2, 2, 2, 2)
    V = 16
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), -0.2)
    D = oracle_mod.rep_dim(N, rep)
    UR = oracle_mod.represent_field(L, H.links(dims, N, 1.0, seed=79))
    nh = V // 2 * 4 * D
    B = np.zeros((nh, nh), np.complex128)
    e = np.zeros(nh, np.complex128)
    for j in range(nh):
        e[:] = 0
        e[j] = 1
        B[:, j] = oracle_mod.dhat(L, UR, e.reshape(V // 2, 4, D)).ravel()
    A = B.conj().T @ B
    lam, Q = np.linalg.eigh(A)
    lo, hi = 0.9 * lam[0], 1.1 * lam[-1]
    ra = rational.zolotarev_inv_sqrt(10, lo, hi)
    b = H.spinor(V // 2, D, 83)
    exact = (Q @ ((Q.conj().T @ b.ravel()) / np.sqrt(lam))).reshape(b.shape)
    xs, ok, its, res = oracle_mod.cg_multishift(L, UR, 1, b, ra.poles, tol=1e-14, max_iter=10000)
    assert all(ok)
    approx = ra.a0 * b + sum(a * x for a, x in zip(ra.residues, xs))
    err = np.linalg.norm(approx - exact) / np.linalg.norm(exact)
    assert err <= ra.max_rel_err * 1.001 + 1e-12, (err, ra.max_rel_err)
    # and the bound is nearly attained by the eigen-components' errors
    assert err >= 1e-3 * ra.max_rel_err
