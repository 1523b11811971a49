"""GPU parity of the clover and exponential-clover diagonal (Sec. 5.1.2,
Sec. 5.1.3) with the oracle: D_m and Dhat = C_ee - D_eo C_oo^-1 D_oe with
the clover term, in FP64 and FP32, plain and dagger, on lattices that span
several 32-site tiles and end in a ragged tail; solves with the clover term
(CG and multi-shift, FP64 and FP32 inner) against the oracle's CG; the term
follows hr_gauge_update; and the entry points without a clover force refuse."""
import numpy as np
import pytest
import torch

from tests import _helpers as H
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

CSW = 1.3


@pytest.fixture(scope="module")
def hr():
    from paper_2503_06721_gb300 import build, hr
    build.build()
    hr.load()
    return hr


def _case(hr, oracle_mod, N, rep, dims=(4, 4, 2, 6), m0=-0.1, eps=0.6, seed=223, mode=1):
    lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), m0)
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), m0)
    U = H.links(dims, N, eps, seed=seed)
    UR = oracle_mod.represent_field(L, U)
    C = oracle_mod.clover_term(L, UR, CSW, exponential=(mode == 2))
    Ud = G.to_gpu(U)
    g = hr.Gauge(lat, Ud, precs=("f64", "f32"))
    g.set_clover(Ud, CSW, mode)
    return lat, L, U, UR, C, g, Ud


@pytest.mark.parametrize("mode", [1, 2], ids=["clover", "expclover"])
@pytest.mark.parametrize("N,rep", [(2, "ADJ"), (3, "SYM"), (3, "FUND"), (4, "ASYM"), (2, "FUND"), (4, "ASYM_REAL")])
def test_clover_operator_parity(hr, oracle_mod, N, rep, mode):
    lat, L, U, UR, C, g, Ud = _case(hr, oracle_mod, N, rep, mode=mode)
    V, D = lat.volume, lat.D
    psi = H.spinor(V, D, 227)
    xe = H.spinor(V // 2, D, 229)
    for prec in (hr.F64, hr.F32):
        tol = G.TOL[prec]
        for dag in (False, True):
            src = G.eo_full(oracle_mod, L, psi)
            x_in = G.prec_fields(hr, lat, hr.FULL, G.to_gpu(src), prec)
            y = g.apply(hr.FULL, prec, x_in, dagger=dag)
            xin64 = G.from_eo_full(oracle_mod, L, G.back_to_f64(hr, lat, hr.FULL, x_in, prec).cpu().numpy())
            want = G.eo_full(oracle_mod, L, oracle_mod.dirac_full_clover(L, UR, C, xin64, dagger=dag))
            got = G.back_to_f64(hr, lat, hr.FULL, y, prec).cpu().numpy()
            assert G.rel(got, want) <= tol, (prec, dag, G.rel(got, want))
            xi = G.prec_fields(hr, lat, hr.EVEN, G.to_gpu(xe), prec)
            y = g.apply(hr.EO_PRECOND, prec, xi, dagger=dag)
            xi64 = G.back_to_f64(hr, lat, hr.EVEN, xi, prec).cpu().numpy()
            want = oracle_mod.dhat_clover(L, UR, C, xi64, dagger=dag)
            got = G.back_to_f64(hr, lat, hr.EVEN, y, prec).cpu().numpy()
            assert G.rel(got, want) <= tol * 4, (prec, dag, G.rel(got, want))
    g.close()


def _shifted_apply(oracle_mod, L, UR, C, sys, x, sigma=0.0):
    if sys == 2:
        full = G.from_eo_full(oracle_mod, L, x)
        y = oracle_mod.dirac_full_clover(L, UR, C, oracle_mod.dirac_full_clover(L, UR, C, full), dagger=True)
        return G.eo_full(oracle_mod, L, y) + sigma * x
    return oracle_mod.dhat_clover(L, UR, C, oracle_mod.dhat_clover(L, UR, C, x), dagger=True) + sigma * x


@pytest.mark.parametrize("mode", [1, 2], ids=["clover", "expclover"])
@pytest.mark.parametrize("sys", [3, 2], ids=["eo", "full"])
@pytest.mark.parametrize("inner", [0, 1], ids=["f64", "f32"])
def test_clover_solves(hr, oracle_mod, sys, inner, mode):
    lat, L, U, UR, C, g, Ud = _case(hr, oracle_mod, 3, "SYM", dims=(8, 4, 4, 6), mode=mode)
    ns = lat.nsites(sys if sys == hr.FULL else hr.EVEN)
    b = H.spinor(ns, lat.D, 233, nrhs=2)
    tol = 1e-10
    x, res, st = g.cg_solve(sys, G.to_gpu(b), nrhs=2, tol=tol, inner=inner, inner_tol=1e-5)
    assert st == 0, res
    xs = x.cpu().numpy()
    for j in range(2):
        r = b[j] - _shifted_apply(oracle_mod, L, UR, C, sys, xs[j])
        assert np.linalg.norm(r) / np.linalg.norm(b[j]) <= tol * 1.001
        A = lambda v: _shifted_apply(oracle_mod, L, UR, C, sys, v)
        xo, ok, it, rel = oracle_mod.cg_apply(A, b[j], tol=1e-12)
        assert ok
        assert np.linalg.norm(xs[j] - xo) / np.linalg.norm(xo) < 1e-6
    # multi-shift with the clover term
    shifts = [0.05, 0.0, 1.0]
    xm, resm, st = g.cg_solve_multishift(sys, G.to_gpu(b[0]), shifts, tol=tol, inner=inner)
    assert st == 0
    for k, sgm in enumerate(shifts):
        r = b[0] - _shifted_apply(oracle_mod, L, UR, C, sys, xm[k].cpu().numpy(), sgm)
        assert np.linalg.norm(r) / np.linalg.norm(b[0]) <= tol * 1.001
    g.close()


def test_clover_follows_update_and_removal(hr, oracle_mod):
    lat, L, U, UR, C, g, Ud = _case(hr, oracle_mod, 2, "ADJ")
    U2 = H.links(lat.dims, 2, 0.9, seed=239)
    g.update(G.to_gpu(U2))
    UR2 = oracle_mod.represent_field(L, U2)
    C2 = oracle_mod.clover_term(L, UR2, CSW)
    psi = H.spinor(lat.volume, lat.D, 241)
    y = g.apply(hr.FULL, hr.F64, G.to_gpu(G.eo_full(oracle_mod, L, psi)))
    want = G.eo_full(oracle_mod, L, oracle_mod.dirac_full_clover(L, UR2, C2, psi))
    assert G.rel(y.cpu().numpy(), want) <= 1e-13
    # removing the term restores the plain Wilson operator
    g.set_clover(None, 0.0, hr.CLOVER_NONE)
    y = g.apply(hr.FULL, hr.F64, G.to_gpu(G.eo_full(oracle_mod, L, psi)))
    want = G.eo_full(oracle_mod, L, oracle_mod.dirac_full(L, UR2, psi))
    assert G.rel(y.cpu().numpy(), want) <= 1e-13
    g.close()


def test_clover_refusals(hr, oracle_mod):
    lat, L, U, UR, C, g, Ud = _case(hr, oracle_mod, 3, "FUND")
    b = G.to_gpu(H.spinor(lat.nsites(hr.EVEN), lat.D, 251))
    with pytest.raises(hr.HrError):
        g.cg_solve_force(hr.EO_PRECOND, b)
    with pytest.raises(hr.HrError):
        g.force(hr.EO_PRECOND, b, b)
    with pytest.raises(hr.HrError):
        hr.cg_solve_batched([g], hr.EO_PRECOND, [b], [torch.zeros_like(b)], [1])
    g.close()
