"""GPU parity of the float-float (DF64) operator against the FP64 oracle and
of the defect-correction solver that forms its true residuals with it.

DF64 stores every FP64 value as an exact pair of floats and computes in
float-float arithmetic (about 48 significant bits), so it is held to the FP64
bar: every selector and its adjoint in every compiled (N, representation)
pair, on a lattice whose half volume ends in a ragged tile."""
import numpy as np
import pytest
import torch

from tests import _helpers as H
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

DIMS = (6, 4, 2, 6)   # V/2 = 144 = 4.5 tiles of 32


@pytest.fixture(scope="module")
def hr():
    from paper_2503_06721_gb300 import build, hr
    build.build()
    hr.load()
    return hr


def _oracle_apply(oracle_mod, L, UR, par, x_host, dagger):
    if par in (0, 1):
        return oracle_mod.hop_parity(L, UR, par, x_host, dagger)
    if par == 2:
        full = G.from_eo_full(oracle_mod, L, x_host)
        return G.eo_full(oracle_mod, L, oracle_mod.dirac_full(L, UR, full, dagger))
    return oracle_mod.dhat(L, UR, x_host, dagger)


@pytest.mark.parametrize("N,rep", G.PAIRS)
def test_df64_operator_parity(hr, oracle_mod, N, rep):
    dims, bc, m0 = DIMS, (-1, 1, 1, -1), -0.23
    lat = hr.Lattice(N, rep, dims, bc, m0)
    L = oracle_mod.lat(N, rep, dims, bc, m0)
    UF = H.links(dims, N, 0.7, seed=5)
    UR = oracle_mod.represent_field(L, UF)
    g = hr.Gauge(lat, G.to_gpu(UF), precs=("f64", "df64"))
    psi = H.spinor(lat.volume, lat.D, 7)
    for par in (hr.EVEN, hr.ODD, hr.FULL, hr.EO_PRECOND):
        src = psi if par == hr.FULL else psi[: lat.volume // 2]
        in_par = hr.FULL if par == hr.FULL else hr.EVEN
        x = G.to_gpu(src)
        xd = hr.field_convert(lat, in_par, x, hr.F64, hr.DF64)
        # the library's (hi, lo) split equals the host's float-float storage
        xin, back = G.kernel_input(src, hr.DF64)
        assert torch.equal(xd, xin)
        assert np.abs(back - src).max() <= 2.0 ** -47 * np.abs(src).max()
        for dagger in (False, True):
            y = g.apply(par, hr.DF64, xin, dagger=dagger)
            got = G.kernel_output(y, hr.DF64, lat.nsites(in_par), lat.D)[0]
            want = _oracle_apply(oracle_mod, L, UR, par, back, dagger)
            err = G.rel(got, want)
            assert err <= G.TOL[hr.DF64], (par, dagger, err)
    g.close()


def test_df64_needs_stored_links(hr, oracle_mod):
    lat = hr.Lattice(3, "SYM", DIMS)
    UF = H.links(DIMS, 3, 0.5, seed=3)
    g = hr.Gauge(lat, G.to_gpu(UF), precs=("f64", "f32", "df64"), stored=True, rebuild=True)
    xd = hr.field_convert(lat, hr.EVEN, G.to_gpu(H.spinor(lat.volume // 2, lat.D, 2)), hr.F64, hr.DF64)
    g.set_link_mode(hr.LINKS_REBUILD)
    with pytest.raises(hr.HrError):
        g.apply(hr.EVEN, hr.DF64, xd)
    b = G.to_gpu(H.spinor(lat.volume // 2, lat.D, 4))
    with pytest.raises(hr.HrError) as e:
        g.cg_solve(hr.EO_PRECOND, b, inner=hr.F32, residual=hr.DF64)
    assert e.value.status == -1
    g.close()


@pytest.mark.parametrize("inner", [1, 2], ids=["f32", "f16"])
def test_cg_df64_residuals(hr, oracle_mod, inner):
    """Mixed CG whose outer true residuals are formed in float-float: the
    oracle's own true residual of the returned x meets the tolerance, the
    reported residual is the FP64 one, and x agrees with the solve that uses
    FP64 residuals throughout."""
    from paper_2503_06721_gb300 import synth
    N, rep, dims, m0 = 3, "SYM", (8, 8, 8, 8), -0.3
    lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), m0)
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), m0)
    UF = synth.random_links(lat.volume, N, 0.4, 77).numpy()
    UR = oracle_mod.represent_field(L, UF)
    g = hr.Gauge(lat, G.to_gpu(UF), precs=("f64", "f32", "f16", "df64"))
    b = H.spinor(lat.volume // 2, lat.D, 19)
    tol = 1e-10
    x, res, st = g.cg_solve(hr.EO_PRECOND, G.to_gpu(b), tol=tol, inner=inner, inner_tol=1e-4,
                            residual=hr.DF64)
    assert st == 0, res
    xs = x.cpu().numpy()
    r = b - oracle_mod.dhat(L, UR, oracle_mod.dhat(L, UR, xs), dagger=True)
    true_rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert true_rel <= tol * 1.001, true_rel
    assert abs(res[0]["true_rel_residual"] - true_rel) <= 0.05 * true_rel + 1e-15
    x64, res64, st64 = g.cg_solve(hr.EO_PRECOND, G.to_gpu(b), tol=tol, inner=inner, inner_tol=1e-4)
    assert st64 == 0
    assert np.linalg.norm(xs - x64.cpu().numpy()) / np.linalg.norm(xs) < 1e-8
    assert abs(res[0]["outer_iters"] - res64[0]["outer_iters"]) <= 1
    g.close()
