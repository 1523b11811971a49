"""GPU parity of the pairs run by the colour-parallel hopping kernel (one
thread per colour row of a site, Sec. 8.2): the fundamental of SU(5), SU(6),
SU(8) and the SU(4) adjoint (D_R = 15, real links) and symmetric (D_R = 10)
representations,
with the oracle: every parity selector, plain and dagger, FP64 and FP32, on a
lattice that spans several 32-site tiles and ends in a ragged tail; solves
(which run on the multi-shift engine for these pairs); the fermion force; and
the refusals of what the kernel does not provide."""
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


COLOUR_PAIRS = [(5, "FUND"), (6, "FUND"), (8, "FUND"), (4, "ADJ"), (4, "SYM")]


def _case(hr, oracle_mod, N, dims=(4, 4, 2, 6), m0=-0.1, eps=0.6, seed=257, precs=("f64", "f32"), rep="FUND"):
    lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), m0)
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), m0)
    U = H.links(dims, N, eps, seed=seed)
    UR = oracle_mod.represent_field(L, U)
    g = hr.Gauge(lat, G.to_gpu(U), precs=precs)
    return lat, L, U, UR, g


@pytest.mark.parametrize("N,rep", COLOUR_PAIRS)
def test_largen_operator_parity(hr, oracle_mod, N, rep):
    lat, L, U, UR, g = _case(hr, oracle_mod, N, rep=rep)
    V, D = lat.volume, lat.D
    psi = H.spinor(V, D, 263)
    half = H.spinor(V // 2, D, 269)
    for prec in (hr.F64, hr.F32):
        tol = G.TOL[prec]
        for dag in (False, True):
            for par in (hr.EVEN, hr.ODD):
                xi = G.prec_fields(hr, lat, 1 - par, G.to_gpu(half), prec)
                y = g.apply(par, prec, xi, dagger=dag)
                x64 = G.back_to_f64(hr, lat, 1 - par, xi, prec).cpu().numpy()
                want = oracle_mod.hop_parity(L, UR, 0 if par == hr.EVEN else 1, x64, dagger=dag)
                got = G.back_to_f64(hr, lat, par, y, prec).cpu().numpy()
                assert G.rel(got, want) <= tol, (prec, dag, par, G.rel(got, want))
            src = G.eo_full(oracle_mod, L, psi)
            xf = G.prec_fields(hr, lat, hr.FULL, G.to_gpu(src), prec)
            y = g.apply(hr.FULL, prec, xf, dagger=dag)
            x64 = G.from_eo_full(oracle_mod, L, G.back_to_f64(hr, lat, hr.FULL, xf, prec).cpu().numpy())
            want = G.eo_full(oracle_mod, L, oracle_mod.dirac_full(L, UR, x64, dagger=dag))
            got = G.back_to_f64(hr, lat, hr.FULL, y, prec).cpu().numpy()
            assert G.rel(got, want) <= tol
            xe = G.prec_fields(hr, lat, hr.EVEN, G.to_gpu(half), prec)
            y = g.apply(hr.EO_PRECOND, prec, xe, dagger=dag)
            x64 = G.back_to_f64(hr, lat, hr.EVEN, xe, prec).cpu().numpy()
            want = oracle_mod.dhat(L, UR, x64, dagger=dag)
            got = G.back_to_f64(hr, lat, hr.EVEN, y, prec).cpu().numpy()
            assert G.rel(got, want) <= tol
    # several right-hand sides in one launch
    b = H.spinor(V // 2, D, 271, nrhs=3)
    y = g.apply(hr.EVEN, hr.F64, G.to_gpu(b), nrhs=3).cpu().numpy()
    for k in range(3):
        assert G.rel(y[k], oracle_mod.hop_parity(L, UR, 0, b[k])) <= 1e-13
    g.close()


@pytest.mark.parametrize("sys", [3, 2], ids=["eo", "full"])
@pytest.mark.parametrize("inner", [0, 1], ids=["f64", "f32"])
@pytest.mark.parametrize("N,rep", [(5, "FUND"), (4, "ADJ")])
def test_largen_solve(hr, oracle_mod, sys, inner, N, rep):
    lat, L, U, UR, g = _case(hr, oracle_mod, N, dims=(8, 4, 4, 4), m0=0.1, rep=rep)
    ns = lat.nsites(sys if sys == hr.FULL else hr.EVEN)
    b = H.spinor(ns, lat.D, 277)
    tol = 1e-10
    x, res, st = g.cg_solve(sys, G.to_gpu(b), tol=tol, inner=inner, inner_tol=1e-5)
    assert st == 0, res
    xs = x.cpu().numpy()
    if sys == hr.FULL:
        full = G.from_eo_full(oracle_mod, L, xs)
        Ax = G.eo_full(oracle_mod, L, oracle_mod.dirac_full(L, UR, oracle_mod.dirac_full(L, UR, full), dagger=True))
        xo, ok, it, rr = oracle_mod.cg(L, UR, 0, G.from_eo_full(oracle_mod, L, b), tol=1e-12)
        xo = G.eo_full(oracle_mod, L, xo)
    else:
        Ax = oracle_mod.dhat(L, UR, oracle_mod.dhat(L, UR, xs), dagger=True)
        xo, ok, it, rr = oracle_mod.cg(L, UR, 1, b, tol=1e-12)
    assert np.linalg.norm(b - Ax) / np.linalg.norm(b) <= tol * 1.001
    assert ok and np.linalg.norm(xs - xo) / np.linalg.norm(xo) < 1e-6
    g.close()


@pytest.mark.parametrize("N,rep", [(5, "FUND"), (8, "FUND"), (4, "ADJ"), (4, "SYM")])
def test_largen_force(hr, oracle_mod, N, rep):
    lat, L, U, UR, g = _case(hr, oracle_mod, N, precs=("f64",), rep=rep)
    V = lat.volume
    X = H.spinor(V, lat.D, 281)
    Y = H.spinor(V, lat.D, 283)
    Fo = oracle_mod.force(L, UR, X, Y)
    F = g.force(hr.FULL, G.to_gpu(G.eo_full(oracle_mod, L, X)), G.to_gpu(G.eo_full(oracle_mod, L, Y)))
    np.testing.assert_allclose(F.cpu().numpy(), Fo, atol=1e-12 * np.abs(Fo).max())
    g.close()


def test_largen_refusals(hr, oracle_mod):
    lat, L, U, UR, g = _case(hr, oracle_mod, 6, precs=("f64", "f16"))
    b = G.to_gpu(H.spinor(lat.nsites(hr.EVEN), lat.D, 293))
    bh = hr.field_convert(lat, hr.EVEN, b, hr.F64, hr.F16)
    with pytest.raises(hr.HrError):
        g.apply(hr.EVEN, hr.F16, bh)
    with pytest.raises(hr.HrError):
        g.cg_solve_force(hr.EO_PRECOND, b)
    g.close()
