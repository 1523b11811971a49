"""Pins of the RHMC's rational approximation (Sec. 4.3.2), host-side set-up
through the C ABI (hr_rational_approx, a Remez exchange; no GPU work):

  * Chebyshev's alternation theorem characterises the unique best relative
    approximation of degree (n, n): its error takes its extreme value with
    alternating signs at 2n + 2 points.  Checked on a dense grid for several
    powers, the heat-bath power x^(1/4) and the action power x^(-1/2) among
    them;
  * for x^(-1/2) the best approximation is known in closed form (Zolotarev,
    through Jacobi elliptic functions, written here from scipy's sn and K):
    the library's poles, residues and error must be Zolotarev's;
  * applied to a matrix through the oracle's shifted solves, r(A) b must
    approximate A^(-alpha) b within the error bound (dense
    eigendecomposition), and the heat bath phi = r_{-1/4}(A) eta must give
    phi^dag r_{1/2}(A) phi = eta^dag eta within the two bounds."""
import numpy as np
import pytest

from tests import _helpers as H


@pytest.fixture(scope="module")
def rational():
    from paper_2503_06721_gb300 import build, hr, rational
    build.build()
    hr.load()
    return rational


def _eval(ra, x):
    x = np.asarray(x, dtype=np.float64)
    out = np.full(x.shape, ra.a0)
    for a, b in zip(ra.residues, ra.poles):
        out = out + a / (x + b)
    return out


def _rel_error(ra, x):
    return _eval(ra, x) * x ** ra.alpha - 1.0


def _extrema(e, gap=50):
    """local extrema of a sampled error curve (ends included); candidates
    closer than `gap` samples (rounding noise at a flat extremum) count once"""
    d = np.sign(np.diff(e))
    idx = np.where(np.diff(d) != 0)[0] + 1
    out = [0]
    for i in idx:
        if i - out[-1] < gap and out[-1] != 0:
            if abs(e[i]) > abs(e[out[-1]]):
                out[-1] = i
        else:
            out.append(i)
    if len(e) - 1 - out[-1] < gap:
        out[-1] = len(e) - 1
    else:
        out.append(len(e) - 1)
    return np.array(out)


def _zolotarev(n, lo, hi):
    """Zolotarev's best relative approximation of x^(-1/2) on [lo, hi]:
    with b = hi/lo, m = 1 - 1/b and c_l = sn^2(l K(m)/(2n+1); m) /
    (1 - sn^2(...)), 1/sqrt(y) ~ d prod (y + c_2l)/(y + c_2l-1) on [1, b], d
    levelling the relative error; returns (a0, residues, poles) in x = lo y."""
    from scipy.special import ellipj, ellipk
    b = hi / lo
    m = 1.0 - 1.0 / b
    sn = ellipj(np.arange(1, 2 * n + 1) * ellipk(m) / (2 * n + 1), m)[0]
    c = sn * sn / (1.0 - sn * sn)
    num, den = c[1::2], c[0::2]
    y = np.exp(np.linspace(0.0, np.log(b), 20001))
    f = np.sqrt(y) * np.prod((y[:, None] + num) / (y[:, None] + den), axis=1)
    d0 = 2.0 / (f.max() + f.min())
    zeros, poles = lo * num, lo * den
    scale = d0 / np.sqrt(lo)
    res = [scale * np.prod(zeros - p) / np.prod(np.delete(poles, k) - p) for k, p in enumerate(poles)]
    return scale, np.array(res), poles


POWERS = [(0.5, 3, 1e-2, 1.0), (0.5, 8, 0.05, 900.0), (0.25, 6, 1e-4, 10.0), (-0.25, 6, 1e-4, 10.0),
          (-0.25, 12, 1e-3, 881.5), (0.125, 10, 1e-5, 1e2), (0.75, 8, 1e-3, 1e2), (-0.5, 5, 0.1, 10.0)]


@pytest.mark.parametrize("alpha,n,lo,hi", POWERS)
def test_equioscillation(rational, alpha, n, lo, hi):
    ra = rational.approx(alpha, n, lo, hi)
    assert len(ra.poles) == n and all(p > 0 for p in ra.poles)
    assert list(ra.poles) == sorted(ra.poles)
    x = np.exp(np.linspace(np.log(lo), np.log(hi), 400001))
    e = _rel_error(ra, x)
    D = np.abs(e).max()
    assert abs(D - ra.max_rel_err) <= 1e-3 * D
    pts = _extrema(e)
    assert len(pts) == 2 * n + 2, len(pts)
    vals = e[pts] / D
    assert np.all(np.abs(np.abs(vals) - 1) < 2e-3), vals   # equal magnitudes
    assert np.all(vals[1:] * vals[:-1] < 0)                 # alternating signs
    assert abs(abs(e[0]) - D) < 2e-3 * D and abs(abs(e[-1]) - D) < 2e-3 * D


@pytest.mark.parametrize("n,lo,hi", [(3, 1e-2, 1.0), (6, 1e-4, 10.0), (10, 0.1, 881.5), (14, 1e-5, 1.0)])
def test_inverse_sqrt_is_zolotarev(rational, n, lo, hi):
    ra = rational.approx(0.5, n, lo, hi)
    a0, res, poles = _zolotarev(n, lo, hi)
    np.testing.assert_allclose(ra.poles, poles, rtol=1e-6)
    np.testing.assert_allclose(ra.residues, res, rtol=1e-5)
    assert abs(ra.a0 - a0) <= 1e-6 * a0
    x = np.exp(np.linspace(np.log(lo), np.log(hi), 200001))
    zol = a0 + sum(r / (x + p) for r, p in zip(res, poles))
    dz = np.abs(zol * np.sqrt(x) - 1).max()
    assert abs(ra.max_rel_err - dz) <= 1e-3 * dz + 1e-13


def test_error_falls_with_degree(rational):
    errs = [rational.approx(-0.25, n, 1e-3, 1.0).max_rel_err for n in range(2, 12)]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    ratios = np.array(errs[1:]) / np.array(errs[:-1])
    assert ratios.max() < 0.25 and ratios.std() < 0.1 * ratios.mean()
    n = rational.degree_for(0.5, 1e-3, 1.0, 1e-7)
    assert rational.approx(0.5, n, 1e-3, 1.0).max_rel_err <= 1e-7
    assert rational.approx(0.5, n - 1, 1e-3, 1.0).max_rel_err > 1e-7


def test_below_fp64_floor_not_converged(rational):
    """a degree whose best error lies far below FP64 rounding is refused"""
    from paper_2503_06721_gb300 import hr
    with pytest.raises(hr.HrError) as e:
        hr.rational_approx(0.5, 12, 70.0, 430.0)
    assert e.value.status == -4


def test_rejects_bad_arguments(rational):
    from paper_2503_06721_gb300 import hr
    for args in ((0.0, 4, 0.1, 1.0), (1.0, 4, 0.1, 1.0), (0.5, 0, 0.1, 1.0), (0.5, 65, 0.1, 1.0),
                 (0.5, 4, 0.0, 1.0), (0.5, 4, 2.0, 1.0)):
        with pytest.raises(hr.HrError) as e:
            hr.rational_approx(*args)
        assert e.value.status == -1


def _dense_system(oracle_mod):
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
    return L, UR, D, V, lam, Q


def _apply(oracle_mod, L, UR, ra, b):
    xs, ok, its, res = oracle_mod.cg_multishift(L, UR, 1, b, ra.poles, tol=1e-14, max_iter=10000)
    assert all(ok)
    return ra.a0 * b + sum(a * x for a, x in zip(ra.residues, xs))


@pytest.mark.parametrize("alpha,n", [(0.5, 10), (-0.25, 10), (0.25, 8)])
def test_matrix_power(rational, oracle_mod, alpha, n):
    """r(A) b ~ A^(-alpha) b for A = Dhat^dag Dhat on a 2^4 lattice:
    |r(A) b - A^(-alpha) b| <= D |A^(-alpha) b| when the spectrum of A lies in
    [lo, hi] (the relative bound holds eigenvalue by eigenvalue)."""
    L, UR, D, V, lam, Q = _dense_system(oracle_mod)
    lo, hi = 0.9 * lam[0], 1.1 * lam[-1]
    # the spectrum spans a factor 6: a degree above ~6 has an error below the
    # FP64 floor, which the exchange cannot level (HR_ERR_NOT_CONVERGED)
    n = min(n, rational.degree_for(alpha, lo, hi, 1e-11))
    ra = rational.approx(alpha, n, lo, hi)
    b = H.spinor(V // 2, D, 83)
    exact = (Q @ ((Q.conj().T @ b.ravel()) * lam ** (-alpha))).reshape(b.shape)
    err = np.linalg.norm(_apply(oracle_mod, L, UR, ra, b) - exact) / np.linalg.norm(exact)
    assert err <= ra.max_rel_err * 1.001 + 1e-12, (err, ra.max_rel_err)
    assert err >= 1e-3 * ra.max_rel_err


def test_heat_bath_consistency(rational, oracle_mod):
    """One-flavour RHMC: phi = r_{-1/4}(A) eta ~ A^(1/4) eta makes
    phi^dag r_{1/2}(A) phi ~ eta^dag eta, within the two relative errors."""
    L, UR, D, V, lam, Q = _dense_system(oracle_mod)
    lo, hi = 0.9 * lam[0], 1.1 * lam[-1]
    hb = rational.approx(-0.25, 4, lo, hi)
    ac = rational.approx(0.5, 4, lo, hi)
    eta = H.spinor(V // 2, D, 89)
    phi = _apply(oracle_mod, L, UR, hb, eta)
    S = np.vdot(phi.ravel(), _apply(oracle_mod, L, UR, ac, phi).ravel()).real
    ee = np.vdot(eta.ravel(), eta.ravel()).real
    assert abs(S / ee - 1) <= 2 * hb.max_rel_err + ac.max_rel_err + 1e-12, (S / ee - 1)
