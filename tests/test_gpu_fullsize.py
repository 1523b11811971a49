"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times: sampled output sites are recomputed one by one by the
oracle from gathered links and neighbour spinors, and whole-lattice
identities (gamma5-hermiticity of Dhat, the solver's true residual) are
checked with the library's own compensated dot products."""
import gc

import numpy as np
import pytest
import torch

from tests import gpu_common as G

pytestmark = pytest.mark.gpu

NSAMPLE = 4096


@pytest.fixture(scope="module")
def hr():
    from paper_2503_06721_gb300 import build, hr
    build.build()
    hr.load()
    return hr


def _free():
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _sampled_check(hr, oracle_mod, wl, U, x_in, y_out, parity, dagger, tol, seed=0, link_prec=0,
                   half_prec=None, scales=None, label=None):
    """compare y_out (half field of `parity`, any precision promoted to FP64)
    with the oracle at NSAMPLE random sites; x_in is the input half field.
    link_prec != 0: the oracle uses the represented links rounded as the
    kernel stores them in that precision.  half_prec (F16/BF16) with the
    output's site scales: the tight per-component half-precision bound."""
    T, X, Y, Z = wl.dims
    V = T * X * Y * Z
    dev = U.device
    gen = torch.Generator(device="cpu").manual_seed(seed)
    i = torch.randint(0, V // 2, (NSAMPLE,), generator=gen).to(dev)
    # the site of parity `parity` with half index i is 2i or 2i+1
    lex = 2 * i

    def coords(l):
        z = l % Z
        y = (l // Z) % Y
        x = (l // (Y * Z)) % X
        t = l // (X * Y * Z)
        return torch.stack([t, x, y, z], -1)

    c = coords(lex)
    lex = torch.where((c.sum(-1) & 1) == parity, lex, lex + 1)
    c = coords(lex)
    dims = torch.tensor(wl.dims, device=dev)
    Ul = torch.empty((NSAMPLE, 8, wl.N, wl.N), dtype=torch.complex128, device=dev)
    ps = torch.empty((NSAMPLE, 8) + tuple(x_in.shape[1:]), dtype=torch.complex128, device=dev)
    for k in range(8):
        mu, d = k & 3, (1 if k < 4 else -1)
        cn = c.clone()
        cn[:, mu] = (cn[:, mu] + d) % dims[mu]
        nb = ((cn[:, 0] * X + cn[:, 1]) * Y + cn[:, 2]) * Z + cn[:, 3]
        owner = lex if k < 4 else nb
        Ul[:, k] = U[owner, mu]
        ps[:, k] = x_in[nb // 2].to(torch.complex128)
    L = oracle_mod.lat(wl.N, wl.rep, wl.dims, wl.bc, wl.m0)
    if link_prec:
        from oracle import storage as OS
        R = oracle_mod.represent_links(wl.N, wl.rep, Ul.cpu().numpy())
        R = OS.round_links(R, link_prec, real=(wl.rep in G.REAL_REPS))
        ref = oracle_mod.hop_local(L, c.cpu().numpy(), R, ps.cpu().numpy(), dagger, represented=True)
    else:
        ref = oracle_mod.hop_local(L, c.cpu().numpy(), Ul.cpu().numpy(), ps.cpu().numpy(), dagger)
    got = y_out[i].to(torch.complex128).cpu().numpy()
    err = G.rel(got, ref)
    if half_prec is not None:
        exc = G.scaled_excess(got, np.asarray(scales)[i.cpu().numpy()], ref, half_prec)
        G.report(label or f"sampled/{wl.name}/{half_prec}", rel=err, excess=exc)
        assert exc <= 1.0, (exc, err)
    else:
        G.report(label or f"sampled/{wl.name}", rel=err)
        assert err <= tol, err
    return err


def _dhat_hermiticity(hr, lat, g, prec, dt, seed):
    """<phi, Dhat psi> = <Dhat^dag phi, psi> on the whole lattice (any size)."""
    from paper_2503_06721_gb300 import synth
    vh = lat.volume // 2
    phi = synth.gaussian_spinor(vh, lat.D, seed, device="cuda").to(dt)
    psi = synth.gaussian_spinor(vh, lat.D, seed + 1, device="cuda").to(dt)
    a = hr.field_dot(lat, hr.EVEN, prec, phi, g.apply(hr.EO_PRECOND, prec, psi))[0]
    b = hr.field_dot(lat, hr.EVEN, prec, g.apply(hr.EO_PRECOND, prec, phi, dagger=True), psi)[0]
    return abs(a - b) / abs(a)


def test_sym_32x32x32x64_deo(hr, oracle_mod):
    """SU(3) sextet 32^3 x 64: D_eo and D_oe (and adjoints) in FP64 and FP32."""
    from paper_2503_06721_gb300 import synth
    wl = synth.WORKLOADS["su3_sym_64x32x32x32"]
    lat = hr.Lattice(wl.N, wl.rep, wl.dims, wl.bc, wl.m0)
    U = wl.links(device="cuda")
    g = hr.Gauge(lat, U, precs=("f64", "f32"), stored=True)
    g.tune(hr.F32)   # the benchmark's kernel variants
    x = synth.gaussian_spinor(lat.volume // 2, lat.D, 5, device="cuda")
    for prec, dt in ((hr.F64, torch.complex128), (hr.F32, torch.complex64)):
        xin = x.to(dt)
        for parity, dagger in ((0, False), (1, True)):
            y = g.apply(parity, prec, xin, dagger=dagger)
            _sampled_check(hr, oracle_mod, wl, U, xin, y, parity, dagger, G.TOL[prec], seed=parity)
        rel = _dhat_hermiticity(hr, lat, g, prec, dt, 11)
        assert rel < (1e-12 if prec == hr.F64 else 1e-5), rel
    g.close()
    del U, x
    _free()


def test_adj_64x64x64x128_stored_and_rebuilt(hr, oracle_mod):
    """SU(3) adjoint 64^3 x 128 (FP32 spinors): D_eo with stored 8x8 links and
    with links rebuilt in the kernel from the stored fundamental 3x3 links."""
    from paper_2503_06721_gb300 import synth
    wl = synth.WORKLOADS["su3_adj_128x64x64x64"]
    lat = hr.Lattice(wl.N, wl.rep, wl.dims, wl.bc, wl.m0)
    U = wl.links(device="cuda")
    g = hr.Gauge(lat, U, precs=("f32",), stored=True, rebuild=True)
    x = synth.gaussian_spinor(lat.volume // 2, lat.D, 7, device="cuda").to(torch.complex64)
    for mode in (hr.LINKS_STORED, hr.LINKS_REBUILD):
        g.set_link_mode(mode)
        g.tune(hr.F32)
        y = g.apply(hr.EVEN, hr.F32, x)
        _sampled_check(hr, oracle_mod, wl, U, x, y, 0, False, G.TOL[hr.F32], seed=mode)
        del y
    g.close()
    del U, x
    _free()


@pytest.mark.parametrize("name", ["su4_fund_48x24x24x24", "su4_asym_48x24x24x24"])
def test_su4_24x24x24x48_deo(hr, oracle_mod, name):
    from paper_2503_06721_gb300 import synth
    wl = synth.WORKLOADS[name]
    lat = hr.Lattice(wl.N, wl.rep, wl.dims, wl.bc, wl.m0)
    U = wl.links(device="cuda")
    g = hr.Gauge(lat, U, precs=("f32", "f16"), stored=True)
    g.tune(hr.F32)
    g.tune(hr.F16)
    x = synth.gaussian_spinor(lat.volume // 2, lat.D, 9, device="cuda")
    y = g.apply(hr.EVEN, hr.F32, x.to(torch.complex64))
    _sampled_check(hr, oracle_mod, wl, U, x.to(torch.complex64), y, 0, False, G.TOL[hr.F32], link_prec=hr.F32)
    # F16: the input stored on the host, the oracle on the kernel's rounded links
    xh, x16 = G.kernel_input(x.cpu().numpy(), hr.F16)
    yh = g.apply(hr.EVEN, hr.F16, xh)
    y16, sc = G.kernel_output(yh, hr.F16, lat.volume // 2, lat.D)
    _sampled_check(hr, oracle_mod, wl, U, G.to_gpu(x16), G.to_gpu(y16), 0, False, None, link_prec=hr.F16,
                   half_prec=hr.F16, scales=sc)
    g.close()
    del U, x
    _free()


def test_sym_32x32x32x64_mixed_cg(hr, oracle_mod):
    """The benchmark's solve, in its launch configuration (stored and
    fundamental links, link mode and kernel variants chosen by the tuner,
    fused solve + force): mixed-precision (FP32 inner) CG on Dhat^dag Dhat
    reaches 1e-10; the true residual is recomputed in FP64 by the library and
    cross-checked at sampled sites of Dhat x by the oracle's hopping term; the
    FP32 operator in the solver's link mode matches the oracle at sampled
    sites; the fused force equals solve + apply + force."""
    from paper_2503_06721_gb300 import synth
    wl = synth.WORKLOADS["su3_sym_64x32x32x32"]
    lat = hr.Lattice(wl.N, wl.rep, wl.dims, wl.bc, wl.m0)
    U = wl.links(device="cuda")
    g = hr.Gauge(lat, U, precs=("f64", "f32"), stored=True, rebuild=True)
    g.set_link_mode(hr.LINKS_AUTO)
    g.tune(hr.F32)
    g.tune(hr.F64)
    b = synth.gaussian_spinor(lat.volume // 2, lat.D, 13, device="cuda")
    x, F, Y, res, st = g.cg_solve_force(hr.EO_PRECOND, b, tol=1e-10, inner=hr.F32, inner_tol=1e-5,
                                        coeff=-1.0, want_y=True)
    assert st == 0 and res[0]["true_rel_residual"] <= 1e-10
    if g.link_mode(hr.F64) == hr.LINKS_STORED:
        F2 = g.force(hr.EO_PRECOND, x, g.apply(hr.EO_PRECOND, hr.F64, x), coeff=-1.0)
        assert torch.equal(F, F2)
        del F2
    del F, Y
    x32 = x.to(torch.complex64)
    y32 = g.apply(hr.EVEN, hr.F32, x32)
    _sampled_check(hr, oracle_mod, wl, U, x32, y32, 0, False, G.TOL[hr.F32], seed=4)
    del x32, y32
    # independent residual: A x - b with A applied hop by hop and |.| by field_dot
    t = g.apply(hr.EO_PRECOND, hr.F64, x)
    Ax = g.apply(hr.EO_PRECOND, hr.F64, t, dagger=True)
    r = Ax - b
    rr = hr.field_dot(lat, hr.EVEN, hr.F64, r, r)[0].real
    bb = hr.field_dot(lat, hr.EVEN, hr.F64, b, b)[0].real
    assert (rr / bb) ** 0.5 <= 1.01e-10
    # the odd intermediate of Dhat x at sampled sites
    xo = g.apply(hr.ODD, hr.F64, x)
    _sampled_check(hr, oracle_mod, wl, U, x, xo, 1, False, G.TOL[hr.F64], seed=3)
    g.close()
    _free()


def test_adj_64x64x64x128_mixed_cg(hr, oracle_mod):
    """SU(3) adjoint 64^3 x 128, m0 = -0.35, links exp(i 0.5 H): the
    mixed-precision solve of Dhat^dag Dhat x = b to a true residual of 1e-10
    with FP32 inner iterations on links rebuilt in the kernel from the stored
    fundamental 3 x 3 links (FP32 and, for the FP64 true residuals, FP64).
    Stored 8 x 8 FP64 links are not kept: duplicated per parity they would take
    137 GB beside the 58 GB of fundamental records.  The solution is checked
    by an independent FP64 residual b - Dhat^dag Dhat x (library operator and
    compensated dot products) and the FP64 operator it uses is checked against
    the oracle at 4096 sampled sites of D_oe x and of D_eo D_oe x."""
    from paper_2503_06721_gb300 import synth
    wl = synth.WORKLOADS["su3_adj_128x64x64x64"]
    lat = hr.Lattice(wl.N, wl.rep, wl.dims, wl.bc, wl.m0)
    U = wl.links(device="cuda")
    g = hr.Gauge(lat, U, precs=("f64", "f32"), stored=False, rebuild=True)
    b = synth.gaussian_spinor(lat.volume // 2, lat.D, 17, device="cuda")
    x, res, st = g.cg_solve(hr.EO_PRECOND, b, tol=1e-10, inner=hr.F32, inner_tol=1e-5)
    G.report("cg/su3_adj_128x64x64x64", iters=res[0]["iters"], outer=res[0]["outer_iters"],
             true_rel_residual=res[0]["true_rel_residual"])
    assert st == 0 and res[0]["true_rel_residual"] <= 1e-10, res
    xo = g.apply(hr.ODD, hr.F64, x)
    _sampled_check(hr, oracle_mod, wl, U, x, xo, 1, False, G.TOL[hr.F64], seed=21,
                   label="sampled/su3_adj_128x64x64x64/f64_rebuild/D_oe")
    xe = g.apply(hr.EVEN, hr.F64, xo)
    _sampled_check(hr, oracle_mod, wl, U, xo, xe, 0, False, G.TOL[hr.F64], seed=22,
                   label="sampled/su3_adj_128x64x64x64/f64_rebuild/D_eo")
    del xo, xe
    t = g.apply(hr.EO_PRECOND, hr.F64, x)
    r = g.apply(hr.EO_PRECOND, hr.F64, t, dagger=True)
    del t
    r -= b
    rr = hr.field_dot(lat, hr.EVEN, hr.F64, r, r)[0].real
    bb = hr.field_dot(lat, hr.EVEN, hr.F64, b, b)[0].real
    assert (rr / bb) ** 0.5 <= 1.01e-10, (rr / bb) ** 0.5
    g.close()
    del U, x, b, r
    _free()
