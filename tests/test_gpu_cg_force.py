"""GPU parity of the CG solver (plain FP64 and FP64 defect correction around
FP32 / F16 / BF16 inner solves) and of the fermion force, against the oracle.

Solver checks use what is unique: the oracle recomputes the true residual
|b - A x_gpu| / |b| of the GPU solution, which must meet the requested
tolerance, and the GPU solution must agree with the oracle's own CG solution
within the conditioning bound of the two residuals."""
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


def _normal_apply(oracle_mod, L, UR, sys, x):
    if sys == 2:   # FULL, library layout
        full = G.from_eo_full(oracle_mod, L, x)
        y = oracle_mod.dirac_full(L, UR, oracle_mod.dirac_full(L, UR, full), dagger=True)
        return G.eo_full(oracle_mod, L, y)
    return oracle_mod.dhat(L, UR, oracle_mod.dhat(L, UR, x), dagger=True)


# the 8^4 SU(2) adjoint correctness configuration: m0 = -0.2, links exp(i 0.3 H),
# antiperiodic in time
CFG1 = dict(N=2, rep="ADJ", dims=(8, 8, 8, 8), m0=-0.2, eps=0.3, seed=2503067211)


@pytest.fixture(scope="module")
def cfg1(hr, oracle_mod):
    c = CFG1
    lat = hr.Lattice(c["N"], c["rep"], c["dims"], (-1, 1, 1, 1), c["m0"])
    L = oracle_mod.lat(c["N"], c["rep"], c["dims"], (-1, 1, 1, 1), c["m0"])
    from paper_2503_06721_gb300 import synth
    UF = synth.random_links(lat.volume, c["N"], c["eps"], c["seed"]).numpy()
    UR = oracle_mod.represent_field(L, UF)
    g = hr.Gauge(lat, G.to_gpu(UF), precs=("f64", "f32", "f16", "bf16"), stored=True, rebuild=True)
    return lat, L, UF, UR, g


@pytest.mark.parametrize("sys", [3, 2], ids=["eo", "full"])
@pytest.mark.parametrize("inner", [0, 1, 2, 3], ids=["f64", "f32", "f16", "bf16"])
def test_cg_cfg1(hr, oracle_mod, cfg1, sys, inner):
    lat, L, UF, UR, g = cfg1
    ns = lat.nsites(sys if sys == hr.FULL else hr.EVEN)
    b = H.spinor(ns, lat.D, 17)
    tol = 1e-10
    x, res, st = g.cg_solve(sys, G.to_gpu(b), tol=tol, max_iter=5000, inner=inner, inner_tol=1e-4)
    assert st == 0, res
    xs = x.cpu().numpy()
    r = b - _normal_apply(oracle_mod, L, UR, sys, xs)
    true_rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert true_rel <= tol * 1.001, true_rel
    assert abs(res[0]["true_rel_residual"] - true_rel) <= 0.05 * true_rel + 1e-15
    # oracle solution for the same system (Hestenes-Stiefel CG, Neumaier sums)
    if sys == hr.FULL:
        bo = G.from_eo_full(oracle_mod, L, b)
        xo, ok, it, rr = oracle_mod.cg(L, UR, 0, bo, tol=1e-12)
        xo = G.eo_full(oracle_mod, L, xo)
    else:
        xo, ok, it, rr = oracle_mod.cg(L, UR, 1, b, tol=1e-12)
    assert ok
    assert np.linalg.norm(xs - xo) / np.linalg.norm(xo) < 1e-6
    if inner == 0:
        # plain FP64 CG takes about as many iterations as the oracle's at the same tolerance
        if sys == hr.FULL:
            _, _, it, _ = oracle_mod.cg(L, UR, 0, G.from_eo_full(oracle_mod, L, b), tol=tol)
        else:
            _, _, it, _ = oracle_mod.cg(L, UR, 1, b, tol=tol)
        assert abs(res[0]["iters"] - it) <= 0.05 * it + 2


def test_cfg1_one_apply_and_50_iterations(hr, oracle_mod, cfg1):
    """The correctness configuration as stated: one D_w apply plus 50 CG
    iterations on D^dag D; the 50-iteration iterate matches the oracle's."""
    lat, L, UF, UR, g = cfg1
    V = lat.volume
    psi = H.spinor(V, lat.D, 19)
    y = g.apply(hr.FULL, hr.F64, G.to_gpu(G.eo_full(oracle_mod, L, psi)))
    want = G.eo_full(oracle_mod, L, oracle_mod.dirac_full(L, UR, psi))
    assert G.rel(y.cpu().numpy(), want) <= 1e-13
    b = G.eo_full(oracle_mod, L, psi)
    x, res, st = g.cg_solve(hr.FULL, G.to_gpu(b), tol=1e-30, max_iter=50, check=False)
    assert res[0]["iters"] == 50 and st == -4
    xo, ok, it, rr = oracle_mod.cg(L, UR, 0, G.from_eo_full(oracle_mod, L, b), tol=1e-30, max_iter=50)
    assert it == 50
    assert G.rel(x.cpu().numpy(), G.eo_full(oracle_mod, L, xo)) < 1e-9


def test_cg_multi_rhs_and_zero_rhs(hr, oracle_mod, cfg1):
    lat, L, UF, UR, g = cfg1
    b = H.spinor(lat.volume // 2, lat.D, 23, nrhs=3)
    b[1] = 0.0   # an all-zero right-hand side converges at once with x = 0
    x, res, st = g.cg_solve(hr.EO_PRECOND, G.to_gpu(b), nrhs=3, tol=1e-10, inner=hr.F32)
    assert st == 0
    xs = x.cpu().numpy()
    assert np.abs(xs[1]).max() == 0
    for k in (0, 2):
        r = b[k] - _normal_apply(oracle_mod, L, UR, 3, xs[k])
        assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1e-10 * 1.001


def test_cg_not_converged_and_nonfinite(hr, oracle_mod, cfg1):
    lat, L, UF, UR, g = cfg1
    b = H.spinor(lat.volume // 2, lat.D, 29)
    x, res, st = g.cg_solve(hr.EO_PRECOND, G.to_gpu(b), tol=1e-10, max_iter=3, check=False)
    assert st == -4 and res[0]["status"] == "HR_ERR_NOT_CONVERGED"
    b[5, 1, 0] = np.nan
    x, res, st = g.cg_solve(hr.EO_PRECOND, G.to_gpu(b), tol=1e-10, check=False)
    assert st == -5


@pytest.mark.parametrize("N,rep", [(3, "SYM"), (2, "ADJ"), (4, "ASYM"), (3, "FUND"), (4, "ASYM_REAL")])
def test_force_parity(hr, oracle_mod, N, rep):
    dims = (4, 4, 2, 6)
    lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), -0.1)
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), -0.1)
    UF = H.links(dims, N, 0.6, seed=37)
    UR = oracle_mod.represent_field(L, UF)
    g = hr.Gauge(lat, G.to_gpu(UF), precs=("f64",))
    V = lat.volume
    X = H.spinor(V, lat.D, 41)
    Y = H.spinor(V, lat.D, 43)
    Fo = oracle_mod.force(L, UR, X, Y)
    F = g.force(hr.FULL, G.to_gpu(G.eo_full(oracle_mod, L, X)), G.to_gpu(G.eo_full(oracle_mod, L, Y)),
                coeff=1.0)
    np.testing.assert_allclose(F.cpu().numpy(), Fo, atol=1e-12 * np.abs(Fo).max())
    # even/odd system: S = -2 Re <Y_e, Dhat X_e>  ->  minus the full formula on
    # X' = (X_e, D_oe X_e), Y' = (Y_e, (D^dag)_oe Y_e)
    Xe, Ye = X[: V // 2], Y[: V // 2]
    Xp = oracle_mod.merge(L, Xe, oracle_mod.hop_parity(L, UR, 1, Xe))
    Yp = oracle_mod.merge(L, Ye, oracle_mod.hop_parity(L, UR, 1, Ye, dagger=True))
    Fo = -oracle_mod.force(L, UR, Xp, Yp)
    F = g.force(hr.EO_PRECOND, G.to_gpu(Xe), G.to_gpu(Ye), coeff=2.0)
    np.testing.assert_allclose(F.cpu().numpy(), 2.0 * Fo, atol=1e-12 * np.abs(Fo).max())


@pytest.mark.parametrize("N,rep", [(3, "SYM"), (2, "ADJ"), (3, "ADJ"), (4, "ASYM"), (3, "FUND"), (4, "ASYM_REAL")])
def test_force_parity_df64(hr, oracle_mod, N, rep):
    """The float-float force (hr_dirac_force_prec, HR_DF64: about 48
    significant bits on the DF64 links) against the oracle's FP64 force: every
    component within 1e-12 of max |F|, the FP64 kernel's own bar; and it
    refuses a handle without DF64 links."""
    dims = (4, 4, 2, 6)
    lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), -0.1)
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), -0.1)
    UF = H.links(dims, N, 0.6, seed=37)
    UR = oracle_mod.represent_field(L, UF)
    g = hr.Gauge(lat, G.to_gpu(UF), precs=("f64", "df64"))
    V = lat.volume
    X = H.spinor(V, lat.D, 41)
    Y = H.spinor(V, lat.D, 43)
    Fo = oracle_mod.force(L, UR, X, Y)
    F = g.force(hr.FULL, G.to_gpu(G.eo_full(oracle_mod, L, X)), G.to_gpu(G.eo_full(oracle_mod, L, Y)),
                coeff=1.0, arith=hr.DF64)
    e_full = np.abs(F.cpu().numpy() - Fo).max() / np.abs(Fo).max()
    assert e_full <= 1e-12, e_full
    Xe, Ye = X[: V // 2], Y[: V // 2]
    Xp = oracle_mod.merge(L, Xe, oracle_mod.hop_parity(L, UR, 1, Xe))
    Yp = oracle_mod.merge(L, Ye, oracle_mod.hop_parity(L, UR, 1, Ye, dagger=True))
    Fo = -oracle_mod.force(L, UR, Xp, Yp)
    F = g.force(hr.EO_PRECOND, G.to_gpu(Xe), G.to_gpu(Ye), coeff=2.0, arith=hr.DF64)
    e_eo = np.abs(F.cpu().numpy() - 2.0 * Fo).max() / np.abs(2.0 * Fo).max()
    assert e_eo <= 1e-12, e_eo
    G.report("force_df64", N=N, rep=rep, full=e_full, eo=e_eo)
    g64 = hr.Gauge(lat, G.to_gpu(UF), precs=("f64",))
    with pytest.raises(hr.HrError) as e:
        g64.force(hr.FULL, G.to_gpu(G.eo_full(oracle_mod, L, X)), G.to_gpu(G.eo_full(oracle_mod, L, Y)),
                  arith=hr.DF64)
    assert e.value.status == -1
    g.close()
    g64.close()


@pytest.mark.parametrize("N,rep", [(3, "SYM"), (3, "ADJ"), (4, "ASYM_REAL")])
def test_cg_solve_force_fused_df64(hr, oracle_mod, N, rep):
    """With float-float residuals the fused solve + force runs the float-float
    force: bit for bit hr_cg_solve + Y = Dhat x + hr_dirac_force_prec(DF64),
    and within 1e-12 of max |F| of the FP64 force of the same x."""
    dims = (8, 4, 4, 6)
    lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), -0.2)
    UF = H.links(dims, N, 0.5, seed=31)
    g = hr.Gauge(lat, G.to_gpu(UF), precs=("f64", "f32", "df64"))
    b = G.to_gpu(H.spinor(lat.nsites(hr.EVEN), lat.D, 23))
    x1, F1, Y1, res, st = g.cg_solve_force(hr.EO_PRECOND, b, tol=1e-10, inner=hr.F32, inner_tol=1e-4,
                                           residual=hr.DF64, coeff=0.7, want_y=True)
    assert st == 0 and res[0]["true_rel_residual"] <= 1e-10
    x2, res2, st2 = g.cg_solve(hr.EO_PRECOND, b, tol=1e-10, inner=hr.F32, inner_tol=1e-4, residual=hr.DF64)
    assert st2 == 0
    Y2 = g.apply(hr.EO_PRECOND, hr.F64, x2)
    F2 = g.force(hr.EO_PRECOND, x2, Y2, coeff=0.7, arith=hr.DF64)
    F3 = g.force(hr.EO_PRECOND, x2, Y2, coeff=0.7)
    torch.cuda.synchronize()
    assert torch.equal(x1, x2)
    assert torch.equal(Y1, Y2)
    assert torch.equal(F1, F2)
    assert ((F1 - F3).abs().max() / F3.abs().max()).item() <= 1e-12
    g.close()


@pytest.mark.parametrize("N,rep", [(3, "SYM"), (3, "ADJ"), (4, "FUND")])
@pytest.mark.parametrize("sys", [3, 2], ids=["eo", "full"])
@pytest.mark.parametrize("inner", [0, 1], ids=["f64", "f32"])
def test_cg_solve_force_fused(hr, oracle_mod, N, rep, sys, inner):
    """hr_cg_solve_force equals hr_cg_solve + Y = D x + hr_dirac_force bit for
    bit: it applies the same FP64 kernels to the same x, it only keeps the
    operator applications of the final true residual instead of redoing them."""
    dims = (8, 4, 4, 6)
    lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), -0.2)
    UF = H.links(dims, N, 0.5, seed=31)
    g = hr.Gauge(lat, G.to_gpu(UF), precs=("f64", "f32"))
    ns = lat.nsites(sys if sys == hr.FULL else hr.EVEN)
    b = G.to_gpu(H.spinor(ns, lat.D, 23))
    x1, F1, Y1, res, st = g.cg_solve_force(sys, b, tol=1e-10, inner=inner, inner_tol=1e-4, coeff=0.7,
                                           want_y=True)
    assert st == 0 and res[0]["true_rel_residual"] <= 1e-10
    x2, res2, st2 = g.cg_solve(sys, b, tol=1e-10, inner=inner, inner_tol=1e-4)
    assert st2 == 0
    Y2 = g.apply(sys, hr.F64, x2)
    F2 = g.force(sys, x2, Y2, coeff=0.7)
    torch.cuda.synchronize()
    assert torch.equal(x1, x2)
    assert torch.equal(Y1, Y2)
    assert torch.equal(F1, F2)
    g.close()
