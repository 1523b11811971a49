"""GPU parity of the multi-shift CG (Sec. 4.1.2, Sec. 4.3.2) with the oracle's
definition: one shifted CG solve (A + sigma_k) x_k = b per shift.

What is unique is checked: the oracle recomputes the true residual of every
GPU solution, which must meet the tolerance, and each GPU solution agrees with
the oracle's shifted CG solution within the conditioning bound of the two
residuals.  In exact arithmetic the multi-shift iterates of shift k are the CG
iterates of system k (same Krylov space, same minimisation), so the FP64
iteration count of every shift matches the oracle's shifted CG."""
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


def _shifted_apply(oracle_mod, L, UR, sys, x, sigma):
    if sys == 2:   # FULL, library layout
        full = G.from_eo_full(oracle_mod, L, x)
        y = oracle_mod.dirac_full(L, UR, oracle_mod.dirac_full(L, UR, full), dagger=True)
        return G.eo_full(oracle_mod, L, y) + sigma * x
    return oracle_mod.dhat(L, UR, oracle_mod.dhat(L, UR, x), dagger=True) + sigma * x


def _oracle_solve(oracle_mod, L, UR, sys, b, sigma, tol):
    if sys == 2:
        xo, ok, it, rr = oracle_mod.cg(L, UR, 0, G.from_eo_full(oracle_mod, L, b), tol=tol, sigma=sigma)
        return G.eo_full(oracle_mod, L, xo), ok, it
    xo, ok, it, rr = oracle_mod.cg(L, UR, 1, b, tol=tol, sigma=sigma)
    return xo, ok, it


# the 8^4 SU(2) adjoint correctness configuration (m0 = -0.2, links exp(i 0.3 H))
# and an SU(3) sextet lattice with a ragged vector length
CASES = {
    "su2_adj_8x8x8x8": dict(N=2, rep="ADJ", dims=(8, 8, 8, 8), m0=-0.2, eps=0.3, seed=2503067211),
    "su3_sym_10x6x6x4": dict(N=3, rep="SYM", dims=(10, 6, 6, 4), m0=-0.3, eps=0.4, seed=2503067212),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, hr, oracle_mod):
    c = CASES[request.param]
    lat = hr.Lattice(c["N"], c["rep"], c["dims"], (-1, 1, 1, 1), c["m0"])
    L = oracle_mod.lat(c["N"], c["rep"], c["dims"], (-1, 1, 1, 1), c["m0"])
    from paper_2503_06721_gb300 import synth
    UF = synth.random_links(lat.volume, c["N"], c["eps"], c["seed"]).numpy()
    UR = oracle_mod.represent_field(L, UF)
    g = hr.Gauge(lat, G.to_gpu(UF), precs=("f64", "f32"))
    yield lat, L, UR, g
    g.close()


# shifts in no particular order, with a repeated value and a large one
SHIFTS = [0.02, 0.0, 0.3, 0.0, 5.0]


@pytest.mark.parametrize("sys", [3, 2], ids=["eo", "full"])
@pytest.mark.parametrize("inner", [0, 1], ids=["f64", "f32"])
def test_multishift_parity(hr, oracle_mod, case, sys, inner):
    lat, L, UR, g = case
    ns = lat.nsites(sys if sys == hr.FULL else hr.EVEN)
    nrhs = 2
    b = H.spinor(ns, lat.D, 61, nrhs=nrhs)
    tol = 1e-10
    x, res, st = g.cg_solve_multishift(sys, G.to_gpu(b), SHIFTS, nrhs=nrhs, tol=tol, inner=inner,
                                       inner_tol=1e-5)
    assert st == 0, res
    xs = x.cpu().numpy()
    assert xs.shape == (len(SHIFTS), nrhs, ns, 4, lat.D)
    for k, sigma in enumerate(SHIFTS):
        for j in range(nrhs):
            r = b[j] - _shifted_apply(oracle_mod, L, UR, sys, xs[k, j], sigma)
            true_rel = np.linalg.norm(r) / np.linalg.norm(b[j])
            assert true_rel <= tol * 1.001, (k, j, true_rel)
            assert res[k][j]["status"] == "HR_OK"
            assert abs(res[k][j]["true_rel_residual"] - true_rel) <= 0.05 * true_rel + 1e-15
            xo, ok, it = _oracle_solve(oracle_mod, L, UR, sys, b[j], sigma, 1e-12)
            assert ok
            assert np.linalg.norm(xs[k, j] - xo) / np.linalg.norm(xo) < 1e-6
            if inner == 0:
                _, _, it = _oracle_solve(oracle_mod, L, UR, sys, b[j], sigma, tol)
                # (plus at most a short FP64 correction when the iterated
                # residual met the tolerance and the true one just missed it)
                assert abs(res[k][j]["iters"] - it) <= 0.05 * it + 4, (k, res[k][j], it)
    # equal shifts give identical solutions; a larger shift never takes more iterations
    np.testing.assert_array_equal(xs[1], xs[3])
    its = [res[k][0]["iters"] for k in range(len(SHIFTS))]
    if inner == 0:
        assert its[1] >= its[0] >= its[2] >= its[4]


def test_single_shift_matches_cg(hr, oracle_mod, case):
    """nshift = 1 with shift 0 is plain CG on A: same solution within tolerance."""
    lat, L, UR, g = case
    b = G.to_gpu(H.spinor(lat.nsites(hr.EVEN), lat.D, 67))
    x1, res1, st1 = g.cg_solve_multishift(hr.EO_PRECOND, b, [0.0], tol=1e-11)
    x2, res2, st2 = g.cg_solve(hr.EO_PRECOND, b, tol=1e-11)
    assert st1 == 0 and st2 == 0
    assert abs(res1[0][0]["iters"] - res2[0]["iters"]) <= 2
    d = torch.linalg.vector_norm(x1[0] - x2) / torch.linalg.vector_norm(x2)
    assert d.item() < 1e-8


def test_multishift_zero_rhs_and_limits(hr, oracle_mod, case):
    lat, L, UR, g = case
    ns = lat.nsites(hr.EVEN)
    b = H.spinor(ns, lat.D, 71, nrhs=2)
    b[0] = 0.0   # an all-zero source: every shift's solution is 0, exactly
    x, res, st = g.cg_solve_multishift(hr.EO_PRECOND, G.to_gpu(b), [0.1, 0.0], nrhs=2, inner=hr.F32)
    assert st == 0
    xs = x.cpu().numpy()
    assert np.abs(xs[:, 0]).max() == 0
    assert all(res[k][0]["true_rel_residual"] == 0 for k in range(2))
    # a cap of 3 iterations leaves every shift above the tolerance
    x, res, st = g.cg_solve_multishift(hr.EO_PRECOND, G.to_gpu(b[1]), [0.0, 0.5], max_iter=3, check=False)
    assert st == -4 and res[0][0]["status"] == "HR_ERR_NOT_CONVERGED"
    # a non-finite source is reported, not iterated on
    bn = b[1].copy()
    bn[3, 2, 0] = np.nan
    x, res, st = g.cg_solve_multishift(hr.EO_PRECOND, G.to_gpu(bn), [0.0, 0.5], check=False)
    assert st == -5


def test_multishift_bad_arguments(hr, case):
    lat, L, UR, g = case
    b = G.to_gpu(H.spinor(lat.nsites(hr.EVEN), lat.D, 73))
    for shifts, inner in (([-0.1, 0.0], hr.F64), ([float("nan")], hr.F64), ([0.0], hr.F16),
                          ([0.0] * 65, hr.F64)):
        with pytest.raises(hr.HrError):
            g.cg_solve_multishift(hr.EO_PRECOND, b, shifts, inner=inner)


def test_field_lincomb(hr, case):
    """y = a0 b + sum_k a_k x_k against numpy, every parity, aliasing y = b."""
    lat, L, UR, g = case
    for par in (hr.EVEN, hr.FULL):
        ns = lat.nsites(par)
        b = H.spinor(ns, lat.D, 89, nrhs=2)
        x = np.stack([H.spinor(ns, lat.D, 90 + k, nrhs=2) for k in range(3)])
        a = [0.5, -1.25, 3.0]
        want = 0.75 * b + sum(c * xk for c, xk in zip(a, x))
        y = hr.field_lincomb(lat, par, 0.75, G.to_gpu(b), a, G.to_gpu(x), nrhs=2)
        np.testing.assert_allclose(y.cpu().numpy(), want, rtol=0, atol=1e-14 * np.abs(want).max())
        bd = G.to_gpu(b)
        hr.field_lincomb(lat, par, 0.75, bd, a, G.to_gpu(x), y=bd, nrhs=2)
        np.testing.assert_allclose(bd.cpu().numpy(), want, rtol=0, atol=1e-14 * np.abs(want).max())
    # no terms: y = a0 b
    b = H.spinor(lat.nsites(hr.EVEN), lat.D, 97)
    y = hr.field_lincomb(lat, hr.EVEN, -2.0, G.to_gpu(b), [], None)
    np.testing.assert_array_equal(y.cpu().numpy(), -2.0 * b)


@pytest.mark.parametrize("inner", [0, 1], ids=["f64", "f32"])
def test_rational_apply(hr, oracle_mod, case, inner):
    """The RHMC's r(A) b with Zolotarev poles and residues (Sec. 4.3.2) against
    the oracle's definition a0 b + sum_k a_k (A + b_k)^-1 b (one shifted CG per
    pole)."""
    from paper_2503_06721_gb300 import rational
    lat, L, UR, g = case
    m4 = 4 + L.m0
    ra = rational.approx(0.5, 8, 1e-3, (m4 * m4 + 16) ** 2)
    b = H.spinor(lat.nsites(hr.EVEN), lat.D, 101)
    y, x, res = hr.rational_apply(g, hr.EO_PRECOND, G.to_gpu(b), ra, tol=1e-11, inner=inner)
    assert all(r[0]["status"] == "HR_OK" for r in res)
    xo, ok, its, rr = oracle_mod.cg_multishift(L, UR, 1, b, ra.poles, tol=1e-12)
    assert all(ok)
    want = ra.a0 * b + sum(a * xk for a, xk in zip(ra.residues, xo))
    got = y.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-9


def test_solver_counters_left_clean(hr, oracle_mod, case):
    """A solve leaves the handle's reduction tickets at zero: a CG with one
    right-hand side, then a 2-shift solve, then a 10-shift solve (whose systems
    4 and 8 reduce on the tickets the earlier graphs counted loop bodies in)
    must all agree with the oracle."""
    lat, L, UR, g = case
    b = H.spinor(lat.nsites(hr.EVEN), lat.D, 103)
    bd = G.to_gpu(b)
    g.cg_solve(hr.EO_PRECOND, bd, tol=1e-10)
    g.cg_solve_multishift(hr.EO_PRECOND, bd, [0.0, 0.5], tol=1e-10)
    shifts = [0.01 * 2 ** k for k in range(10)]
    x, res, st = g.cg_solve_multishift(hr.EO_PRECOND, bd, shifts, tol=1e-10)
    assert st == 0
    xs = x.cpu().numpy()
    for k, s in enumerate(shifts):
        r = b - _shifted_apply(oracle_mod, L, UR, 3, xs[k], s)
        true_rel = np.linalg.norm(r) / np.linalg.norm(b)
        assert true_rel <= 1e-10 * 1.001, (k, true_rel)
        assert abs(res[k][0]["true_rel_residual"] - true_rel) <= 0.05 * true_rel + 1e-15, (k, res[k][0])


@pytest.mark.parametrize("inner", [0, 1], ids=["f64", "f32"])
def test_rhmc_heat_bath_against_dense_powers(hr, oracle_mod, inner):
    """One-flavour RHMC on the GPU (Sec. 4.3.2): the heat bath phi =
    r_{-1/4}(A) eta and the action phi^dag r_{1/2}(A) phi, each a multi-shift
    solve plus hr_field_lincomb with hr_rational_approx's coefficients, against
    A^(1/4) eta and eta^dag eta from the oracle's dense 2^4 matrix
    (A = Dhat^dag Dhat, eigendecomposition): both within the approximations'
    relative errors (plus the solves' 1e-12 tolerance)."""
    from paper_2503_06721_gb300 import rational
    N, rep, dims, m0 = 2, "ADJ", (2, 2, 2, 2), -0.2
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), m0)
    lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), m0)
    UF = H.links(dims, N, 1.0, seed=79)
    UR = oracle_mod.represent_field(L, UF)
    D, V = lat.D, lat.volume
    nh = V // 2 * 4 * D
    B = np.zeros((nh, nh), np.complex128)
    e = np.zeros(nh, np.complex128)
    for j in range(nh):
        e[:] = 0
        e[j] = 1
        B[:, j] = oracle_mod.dhat(L, UR, e.reshape(V // 2, 4, D)).ravel()
    lam, Q = np.linalg.eigh(B.conj().T @ B)
    lo, hi = 0.9 * lam[0], 1.1 * lam[-1]
    hb = rational.approx(-0.25, 4, lo, hi)
    ac = rational.approx(0.5, 4, lo, hi)
    g = hr.Gauge(lat, G.to_gpu(UF), precs=("f64", "f32"))
    eta = H.spinor(V // 2, D, 89)
    phi, _, res = hr.rational_apply(g, hr.EO_PRECOND, G.to_gpu(eta), hb, tol=1e-12, inner=inner)
    assert all(r[0]["status"] == "HR_OK" for r in res)
    exact = (Q @ ((Q.conj().T @ eta.ravel()) * lam ** 0.25)).reshape(eta.shape)
    err = np.linalg.norm(phi.cpu().numpy() - exact) / np.linalg.norm(exact)
    assert err <= hb.max_rel_err * 1.001 + 1e-10, (err, hb.max_rel_err)
    y, _, res = hr.rational_apply(g, hr.EO_PRECOND, phi, ac, tol=1e-12, inner=inner)
    S = hr.field_dot(lat, hr.EVEN, hr.F64, phi, y)[0].real
    ee = float(np.vdot(eta.ravel(), eta.ravel()).real)
    assert abs(S / ee - 1) <= 2 * hb.max_rel_err + ac.max_rel_err + 1e-10, S / ee - 1
    g.close()
