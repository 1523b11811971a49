"""GPU parity of the Wilson-Dirac operator against the FP64 oracle, through
the C ABI: represent (stored and in-kernel rebuilt links), D_eo / D_oe, the
full D_m, the even/odd preconditioned Dhat and all their adjoints, in every
compiled (N, representation) pair and storage precision, on lattices whose
half volume spans several 32-site tiles and ends in a ragged tail."""
import numpy as np
import pytest
import torch

from tests import _helpers as H
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

DIMS = (6, 4, 2, 6)   # V = 288, V/2 = 144 = 4.5 tiles of 32


@pytest.fixture(scope="module")
def hr():
    from paper_2503_06721_gb300 import build, hr
    build.build()
    hr.load()
    return hr


def _setup(hr, oracle_mod, N, rep, dims=DIMS, m0=-0.23, eps=0.7, bc=(-1, 1, 1, -1), seed=5,
           precs=("f64", "f32", "f16", "bf16")):
    lat = hr.Lattice(N, rep, dims, bc, m0)
    L = oracle_mod.lat(N, rep, dims, bc, m0)
    UF = H.links(dims, N, eps, seed=seed)
    g = hr.Gauge(lat, G.to_gpu(UF), precs=precs, stored=True, rebuild=True)
    UR = oracle_mod.represent_field(L, UF)
    return lat, L, UF, UR, g


def _oracle_apply(oracle_mod, L, UR, par, x_host, dagger):
    """oracle for each hr_parity selector, on library-layout host fields."""
    if par in (0, 1):
        return oracle_mod.hop_parity(L, UR, par, x_host, dagger)
    if par == 2:
        full = G.from_eo_full(oracle_mod, L, x_host)
        return G.eo_full(oracle_mod, L, oracle_mod.dirac_full(L, UR, full, dagger))
    return oracle_mod.dhat(L, UR, x_host, dagger)


def _kernel_links(oracle_mod, L, UF, UR, rep, prec, mode):
    """the links the kernel reads, rounded on the host from the same FP64
    input: stored mode rounds U_R entry by entry (real parts only for the
    real adjoint); rebuild mode rounds U_F and the kernel represents that."""
    from oracle import storage as OS
    if mode == 0:
        return OS.round_links(UR, prec, real=(rep in G.REAL_REPS))
    return oracle_mod.represent_field(L, OS.round_links(UF, prec))


@pytest.mark.parametrize("N,rep", G.PAIRS)
@pytest.mark.parametrize("prec", [0, 1, 2, 3], ids=["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("mode", [0, 1], ids=["stored", "rebuild"])
def test_operator_parity(hr, oracle_mod, N, rep, prec, mode):
    """Every block, plain and adjoint.  The oracle runs on the kernel's own
    rounded inputs (host-rounded links and spinors, promoted to FP64), so the
    comparison isolates the kernel's arithmetic: FP64 and FP32 at the parity
    bars; F16/BF16 component by component within half a code spacing of the
    output site's scale plus FP32 arithmetic (and, for Dhat, the possible
    rounding flips of its stored intermediate)."""
    from oracle import storage as OS
    lat, L, UF, UR, g = _setup(hr, oracle_mod, N, rep)
    g.set_link_mode(mode)
    URk = _kernel_links(oracle_mod, L, UF, UR, rep, prec, mode)
    D = lat.D
    V = lat.volume
    psi = H.spinor(V, D, 7)
    half = psi[: V // 2]
    m4 = 4.0 + lat.m0
    for par in (hr.EVEN, hr.ODD, hr.FULL, hr.EO_PRECOND):
        in_par = hr.FULL if par == hr.FULL else hr.EVEN
        ns = lat.nsites(in_par)
        xin, xh = G.kernel_input(psi if par == hr.FULL else half, prec)
        for dagger in (False, True):
            y = g.apply(par, prec, xin, dagger=dagger)
            torch.cuda.synchronize()
            got, sc = G.kernel_output(y, prec, ns, D)
            allow = None
            if prec in (hr.F16, hr.BF16) and par == hr.EO_PRECOND:
                # the kernel stores mid = D_oe x in the field's precision
                mid = oracle_mod.hop_parity(L, URk, 1, xh, dagger)
                want = m4 * m4 * xh - oracle_mod.hop_parity(L, URk, 0, OS.stored_spinor(mid, prec), dagger)
                allow = G.rounding_allowance(oracle_mod, L, mid, 1, prec)
            else:
                want = _oracle_apply(oracle_mod, L, URk, par, xh, dagger)
            err = G.rel(got, want)
            if prec in (hr.F16, hr.BF16):
                exc = G.scaled_excess(got, sc, want, prec, allow)
                G.report(f"op/{N}{rep}/{prec}/{mode}/{par}/{int(dagger)}", rel=err, excess=exc)
                assert exc <= 1.0, (par, dagger, exc, err)
            else:
                G.report(f"op/{N}{rep}/{prec}/{mode}/{par}/{int(dagger)}", rel=err)
                assert err <= G.TOL[prec], (par, dagger, err)
    g.close()


@pytest.mark.parametrize("prec", [2, 3], ids=["f16", "bf16"])
@pytest.mark.parametrize("D_pair", [(3, "SYM"), (2, "FUND")])
def test_field_convert_equals_host_storage(hr, oracle_mod, prec, D_pair):
    """hr_field_convert F64 -> F16/BF16 writes exactly the bytes of the host
    storage model (per-site FP32 scale, codes rounded to nearest even), and
    F16/BF16 -> F64 returns fl32(s * code) for every component."""
    N, rep = D_pair
    lat = hr.Lattice(N, rep, DIMS)
    nrhs = 2
    a = H.spinor(lat.volume // 2, lat.D, 21, nrhs=nrhs) * np.exp(np.linspace(-3, 3, lat.volume // 2))[None, :, None, None]
    a[0, 5] = 0.0   # an all-zero site: scale 0, codes 0
    dev = hr.field_convert(lat, hr.EVEN, G.to_gpu(a), hr.F64, prec, nrhs)
    from oracle import storage as OS
    codes, scales = OS.quantize_spinor(a, prec)
    got_codes, got_scales = G.unpack_scaled(dev.cpu().numpy(), prec, nrhs, lat.volume // 2, lat.D)
    np.testing.assert_array_equal(got_scales, scales)
    np.testing.assert_array_equal(got_codes, codes)
    back = G.back_to_f64(hr, lat, hr.EVEN, dev, prec, nrhs).cpu().numpy()
    want = OS.round_complex(OS.dequantize(codes, scales), "f32")
    np.testing.assert_array_equal(back, want)


def _conversion_values(n, seed):
    """FP64 values that exercise every branch of an FP64 -> FP32 rounding:
    magnitudes 2^-100 .. 2^100 (including results below the FP32 normal
    range), exact ties at the last kept bit (both parities of that bit),
    values whose rounding carries into the exponent, and signed zeros."""
    rng = np.random.default_rng(seed)
    v = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-100, 100, n)) * rng.choice([-1.0, 1.0], n)
    k = rng.integers(0, 2 ** 22, 512)
    e = rng.integers(-30, 30, 512)
    v[:512] = np.ldexp(1.0 + (2 * k + 1) * 2.0 ** -24, e)        # ties, kept bit even or odd
    v[512:1024] = -np.ldexp(1.0 + (2 * k + 1) * 2.0 ** -24, e)
    v[1024:1536] = np.ldexp(2.0 - 2.0 ** -30, e)                  # rounds up to 2^(e+1)
    v[1536:1544] = [0.0, -0.0, 1.0, -1.0, 2.0 ** -126, -2.0 ** -127, 2.0 ** -149, 3.0e38]
    return v


@pytest.mark.parametrize("prec", [1, 4], ids=["f32", "df64"])
def test_field_convert_bits_equal_host_rounding(hr, prec):
    """hr_field_convert F64 -> F32 rounds every part to the nearest FP32
    number (ties to even) and F64 -> DF64 splits it into hi = fl32(v), lo =
    fl32(v - hi), bit for bit as the host storage model does; the conversions
    back to F64 return the stored values exactly."""
    from oracle import storage as OS
    lat = hr.Lattice(3, "SYM", DIMS)
    ns, D = lat.volume // 2, lat.D
    n = ns * 4 * D
    v = _conversion_values(2 * n, 91 + prec)
    a = (v[:n] + 1j * v[n:]).reshape(ns, 4, D)
    dev = hr.field_convert(lat, hr.EVEN, G.to_gpu(a), hr.F64, prec)
    torch.cuda.synchronize()
    got = dev.cpu().numpy()
    bits = lambda x: np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    if prec == hr.F32:
        for g_, x in ((got.real, a.real), (got.imag, a.imag)):
            assert np.array_equal(bits(g_), bits(OS.round_binary(x, "f32")))
        want = OS.round_complex(a, "f32")
    else:
        rh, rl = OS.split_df64(a.real)
        ih, il = OS.split_df64(a.imag)
        assert np.array_equal(bits(got), bits(np.stack([rh, rl, ih, il], -1)))
        want = (rh + rl) + 1j * (ih + il)
    back = hr.field_convert(lat, hr.EVEN, dev, prec, hr.F64, dst=torch.empty_like(G.to_gpu(a)))
    back = np.ascontiguousarray(back.cpu().numpy())
    assert np.array_equal(back.view(np.uint64), np.ascontiguousarray(want, dtype=np.complex128).view(np.uint64))


@pytest.mark.parametrize("mode", [0, 1], ids=["stored", "rebuild"])
def test_asym_real_equivalent_to_asym(hr, oracle_mod, mode):
    """The library's SU(4) 2AS operator in the real basis (real links, 144 B per
    FP32 link) is the complex-basis one in rotated colour coordinates:
    D_real (W^dag psi) = W^dag (D_2AS psi) with the fixed unitary W, for every
    block and the adjoint, FP64 and FP32."""
    W = np.einsum("mij,nij->mn", oracle_mod.rep_basis(4, "ASYM").conj(),
                  oracle_mod.rep_basis(4, "ASYM_REAL"))
    dims, bc, m0 = DIMS, (-1, 1, 1, -1), -0.23
    UF = H.links(dims, 4, 0.7, seed=5)
    lat_c, lat_r = hr.Lattice(4, "ASYM", dims, bc, m0), hr.Lattice(4, "ASYM_REAL", dims, bc, m0)
    g_c = hr.Gauge(lat_c, G.to_gpu(UF), precs=("f64", "f32"), stored=True, rebuild=True)
    g_r = hr.Gauge(lat_r, G.to_gpu(UF), precs=("f64", "f32"), stored=True, rebuild=True)
    g_c.set_link_mode(mode)
    g_r.set_link_mode(mode)
    psi = H.spinor(lat_c.volume, 6, 31)
    rot = lambda x: x @ W.conj()
    for prec, dt in ((hr.F64, torch.complex128), (hr.F32, torch.complex64)):
        for par in (hr.EVEN, hr.ODD, hr.FULL, hr.EO_PRECOND):
            x = psi if par == hr.FULL else psi[: lat_c.volume // 2]
            for dagger in (False, True):
                yc = g_c.apply(par, prec, G.to_gpu(x, dt), dagger=dagger).to(torch.complex128).cpu().numpy()
                yr = g_r.apply(par, prec, G.to_gpu(rot(x), dt), dagger=dagger).to(torch.complex128).cpu().numpy()
                assert G.rel(yr, rot(yc)) <= 2 * G.TOL[prec], (prec, par, dagger)
    g_c.close()
    g_r.close()


def test_rebuild_equals_stored_f64(hr, oracle_mod):
    lat, L, UF, UR, g = _setup(hr, oracle_mod, 3, "ADJ", dims=(4, 4, 4, 8))
    x = G.to_gpu(H.spinor(lat.volume // 2, lat.D, 9))
    a = g.apply(hr.EVEN, hr.F64, x)
    g.set_link_mode(hr.LINKS_REBUILD)
    b = g.apply(hr.EVEN, hr.F64, x)
    assert G.rel(b.cpu().numpy(), a.cpu().numpy()) < 1e-14


def test_free_field_plane_wave_gpu(hr, oracle_mod):
    """U = 1: D psi = [m + sum(1 - cos p) + i sum gamma sin p] psi on the GPU too."""
    dims = (8, 4, 4, 6)
    N, rep, m0 = 3, "SYM", -0.37
    lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), m0)
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), m0)
    g = hr.Gauge(lat, G.to_gpu(H.unit_links(dims, N)), precs=("f64",))
    x = H.coords(dims)
    p = np.array([3 * np.pi / 8, 2 * np.pi / 4, 0.0, 2 * np.pi / 6])
    gam = [oracle_mod.gamma(mu) for mu in range(4)]
    chi = (np.arange(24).reshape(4, 6) + 1j * np.arange(24)[::-1].reshape(4, 6)) / 10
    psi = np.exp(1j * x @ p)[:, None, None] * chi[None]
    Dp = (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(gam[mu] * np.sin(p[mu]) for mu in range(4))
    want = np.exp(1j * x @ p)[:, None, None] * (Dp @ chi)[None]
    y = g.apply(hr.FULL, hr.F64, G.to_gpu(G.eo_full(oracle_mod, L, psi)))
    got = G.from_eo_full(oracle_mod, L, y.cpu().numpy())
    assert np.abs(got - want).max() < 1e-13


def test_multi_rhs_apply(hr, oracle_mod):
    lat, L, UF, UR, g = _setup(hr, oracle_mod, 4, "ASYM", precs=("f64", "f32"))
    nrhs = 3
    xs = H.spinor(lat.volume // 2, lat.D, 11, nrhs=nrhs)
    for prec, dt in ((hr.F64, torch.complex128), (hr.F32, torch.complex64)):
        x = G.to_gpu(xs, dt)
        y = g.apply(hr.EO_PRECOND, prec, x, nrhs=nrhs).to(torch.complex128).cpu().numpy()
        for k in range(nrhs):
            xin = xs[k].astype(np.complex64 if prec == hr.F32 else np.complex128).astype(np.complex128)
            assert G.rel(y[k], oracle_mod.dhat(L, UR, xin)) <= G.TOL[prec]


def test_field_dot_and_convert(hr, oracle_mod):
    lat = hr.Lattice(3, "SYM", DIMS)
    a = H.spinor(lat.volume // 2, lat.D, 13, nrhs=2)
    ga = G.to_gpu(a)
    d = hr.field_dot(lat, hr.EVEN, hr.F64, ga, ga.flip(0).contiguous(), nrhs=2)
    for k in range(2):
        want = np.vdot(a[k].ravel(), a[1 - k].ravel())
        assert abs(d[k] - want) <= 1e-13 * abs(want)
    # F16 round trip keeps every component within half an ulp of its site scale
    h = hr.field_convert(lat, hr.EVEN, ga, hr.F64, hr.F16, 2)
    back = G.back_to_f64(hr, lat, hr.EVEN, h, hr.F16, 2).cpu().numpy()
    scale = np.abs(np.stack([a.real, a.imag])).max(axis=(0, 3, 4))
    err = np.maximum(np.abs(back.real - a.real), np.abs(back.imag - a.imag)).max(axis=(2, 3))
    assert (err <= scale * 2.0 ** -11 * 1.0001).all()


def test_invalid_precision_rejected(hr, oracle_mod):
    lat, L, UF, UR, g = _setup(hr, oracle_mod, 3, "SYM", precs=("f64",))
    x = G.to_gpu(H.spinor(lat.volume // 2, lat.D, 3)).to(torch.complex64)
    with pytest.raises(hr.HrError) as e:
        g.apply(hr.EVEN, hr.F32, x)
    assert e.value.status == -1
