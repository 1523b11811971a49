"""The hopping-kernel variants (direct, shared-memory staged, staged at a
tighter register budget, staged with staged links) and the autotuner that
picks among them.

Every variant must produce the same bits as the direct kernel in every
epilogue: the plain store (D_eo, D_oe, D_m, Dhat and their adjoints), the
store with |out|^2, and the fused CG update, checked here through whole
operator applications and whole mixed-precision solves, including a block of
right-hand sides and in-kernel rebuilt links.  The parity of the direct
kernel with the oracle is covered in test_gpu_dirac.py and
test_gpu_cg_force.py."""
import numpy as np
import pytest
import torch

from tests import _helpers as H
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

DIMS = (6, 4, 2, 6)   # V/2 = 144: four full warps and a ragged one
CASES = [(3, "ADJ"), (3, "SYM"), (4, "FUND"), (2, "ADJ")]


@pytest.fixture(scope="module")
def hr():
    from paper_2503_06721_gb300 import build, hr
    build.build()
    hr.load()
    return hr


def _gauge(hr, N, rep, dims=DIMS, m0=-0.23, rebuild=False):
    lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), m0)
    UF = H.links(dims, N, 0.6, seed=21)
    g = hr.Gauge(lat, G.to_gpu(UF), precs=("f64", "f32", "f16", "bf16"), stored=True, rebuild=rebuild)
    return lat, g


def _variants(lat, nrhs=1):
    v = [0, 1, 3] if lat.D <= 4 else [0, 1, 2, 3]
    return v + [4] if nrhs > 1 else v


def _written_bytes(hr, lat, par, prec, y):
    """the bytes an application writes: the data and, for F16/BF16, the
    per-site scales (not the alignment padding between and after them)"""
    raw = y.view(torch.uint8).reshape(-1).cpu().numpy()
    if prec in (hr.F32, hr.F64):
        return raw.copy()
    ns = lat.nsites(par)
    data = ns * 4 * lat.D * 4
    off = (data + 255) // 256 * 256
    return np.concatenate([raw[:data], raw[off:off + 4 * ns]])


@pytest.mark.parametrize("N,rep", CASES)
@pytest.mark.parametrize("prec", [1, 2, 3], ids=["f32", "f16", "bf16"])
def test_variants_bitwise_apply(hr, N, rep, prec):
    lat, g = _gauge(hr, N, rep)
    psi = H.spinor(lat.volume, lat.D, 5)
    out = {}
    for v in _variants(lat):
        g.set_tuning(autotune=False, variant=v)
        res = []
        for par in (hr.EVEN, hr.ODD, hr.FULL, hr.EO_PRECOND):
            in_par = hr.FULL if par == hr.FULL else hr.EVEN
            x = G.to_gpu(psi if par == hr.FULL else psi[: lat.volume // 2])
            xin = G.prec_fields(hr, lat, in_par, x, prec)
            for dagger in (False, True):
                y = g.apply(par, prec, xin, dagger=dagger)
                res.append(_written_bytes(hr, lat, in_par, prec, y))
        out[v] = res
    for v in out:
        for a, b in zip(out[0], out[v]):
            assert np.array_equal(a, b), v
    g.close()


@pytest.mark.parametrize("N,rep", CASES)
@pytest.mark.parametrize("rebuild", [False, True], ids=["stored", "rebuild"])
def test_variants_bitwise_solve(hr, N, rep, rebuild):
    lat, g = _gauge(hr, N, rep, dims=(8, 4, 4, 6), rebuild=rebuild)
    if rebuild:
        g.set_link_mode(hr.LINKS_REBUILD)
    nrhs = 3
    b = G.to_gpu(H.spinor(lat.volume // 2, lat.D, 8, nrhs=nrhs))
    runs = {}
    for v in _variants(lat, nrhs):
        g.set_tuning(autotune=False, variant=v)
        x, res, st = g.cg_solve(hr.EO_PRECOND, b, nrhs=nrhs, tol=1e-10, inner=hr.F32, inner_tol=1e-4)
        assert st == 0
        runs[v] = (x.cpu().numpy(), [r["iters"] for r in res], [r["outer_iters"] for r in res])
    for v in runs:
        assert np.array_equal(runs[0][0], runs[v][0]), v
        assert runs[0][1] == runs[v][1] and runs[0][2] == runs[v][2]
    g.close()


def test_tune_records_a_compiled_variant(hr):
    lat, g = _gauge(hr, 3, "ADJ", dims=(8, 8, 8, 8))
    g.set_tuning(autotune=True, variant=-1)
    for prec in (hr.F32, hr.F16):
        for nrhs in (1, 4):
            g.tune(prec, nrhs=nrhs)
            for epi in (hr.EPI_STORE, hr.EPI_STORE_NORM, hr.EPI_CG_UPDATE):
                assert g.hop_variant(prec, epi, nrhs) in _variants(lat, nrhs)
    # FP64 has the direct kernel only; tuning it is a no-op
    g.tune(hr.F64)
    assert g.hop_variant(hr.F64, hr.EPI_CG_UPDATE, 1) == hr.HOP_DIRECT
    # results after tuning equal the direct kernel's
    x = G.to_gpu(H.spinor(lat.volume // 2, lat.D, 3)).to(torch.complex64)
    y_tuned = g.apply(hr.EO_PRECOND, hr.F32, x).cpu().numpy()
    g.set_tuning(autotune=False, variant=hr.HOP_DIRECT)
    y_direct = g.apply(hr.EO_PRECOND, hr.F32, x).cpu().numpy()
    assert np.array_equal(y_tuned, y_direct)
    g.close()


def test_tuning_arguments_checked(hr):
    lat, g = _gauge(hr, 3, "SYM")
    for bad in ((2, -1), (1, 5), (1, -2)):
        with pytest.raises(hr.HrError) as e:
            g.set_tuning(*bad)
        assert e.value.status == -1
    g2 = hr.Gauge(lat, G.to_gpu(H.links(DIMS, 3, 0.6, seed=1)), precs=("f64",))
    with pytest.raises(hr.HrError):
        g2.tune(hr.F32)
    assert g2.hop_variant(hr.F64, 7, 1) == -1
    g.close()
    g2.close()


def test_auto_link_mode(hr, oracle_mod):
    """LINKS_AUTO: the tuner keeps, per precision, the faster of stored and
    rebuilt links (the 16-bit precisions always their stored links); solves
    in that mode still meet their tolerance, and the mode needs both
    storages."""
    lat, g = _gauge(hr, 3, "SYM", dims=(8, 8, 8, 8), rebuild=True)
    g.set_link_mode(hr.LINKS_AUTO)
    assert g.link_mode(hr.F32) == hr.LINKS_STORED   # until tuned
    g.tune(hr.F32)
    assert g.link_mode(hr.F32) in (hr.LINKS_STORED, hr.LINKS_REBUILD)
    for half in (hr.F16, hr.BF16):
        g.tune(half)
        assert g.link_mode(half) == hr.LINKS_STORED
    b = H.spinor(lat.volume // 2, lat.D, 12)
    x, res, st = g.cg_solve(hr.EO_PRECOND, G.to_gpu(b), tol=1e-10, inner=hr.F32, inner_tol=1e-4)
    assert st == 0 and res[0]["true_rel_residual"] <= 1e-10
    L = oracle_mod.lat(3, "SYM", (8, 8, 8, 8), (-1, 1, 1, 1), -0.23)
    UR = oracle_mod.represent_field(L, H.links((8, 8, 8, 8), 3, 0.6, seed=21))
    r = b - oracle_mod.dhat(L, UR, oracle_mod.dhat(L, UR, x.cpu().numpy()), dagger=True)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.001e-10
    g.close()
    lat2, g2 = _gauge(hr, 3, "SYM")
    with pytest.raises(hr.HrError):
        g2.set_link_mode(hr.LINKS_AUTO)
    g2.close()


@pytest.mark.parametrize("N,rep", [(3, "SYM"), (4, "FUND"), (3, "ADJ")])
@pytest.mark.parametrize("prec", [1, 2], ids=["f32", "f16"])
def test_variants_bitwise_multi_rhs_apply(hr, N, rep, prec):
    """A block of 5 right-hand sides (one full group of 4 and a ragged group)
    through every selector: all variants, the multi-RHS one included, give
    the bits of the direct kernel."""
    lat, g = _gauge(hr, N, rep)
    nrhs = 5
    psi = H.spinor(lat.volume, lat.D, 6, nrhs=nrhs)
    out = {}
    for v in _variants(lat, nrhs):
        g.set_tuning(autotune=False, variant=v)
        res = []
        for par in (hr.EVEN, hr.ODD, hr.FULL, hr.EO_PRECOND):
            in_par = hr.FULL if par == hr.FULL else hr.EVEN
            x = G.to_gpu(psi if par == hr.FULL else psi[:, : lat.volume // 2])
            xin = G.prec_fields(hr, lat, in_par, x, prec, nrhs)
            for dagger in (False, True):
                y = g.apply(par, prec, xin, nrhs=nrhs, dagger=dagger)
                if prec == hr.F32:
                    res.append(y.view(torch.uint8).cpu().numpy().copy())
                else:
                    res.append(G.back_to_f64(hr, lat, in_par, y, prec, nrhs).cpu().numpy())
        out[v] = res
    for v in out:
        for a, b in zip(out[0], out[v]):
            assert np.array_equal(a, b), v
    g.close()


@pytest.mark.parametrize("dims", [(2, 2, 2, 4), (4, 2, 2, 2), (2, 4, 6, 2)], ids=["vh16", "vh16b", "vh48"])
def test_variants_on_lattices_smaller_than_a_block(hr, oracle_mod, dims):
    """Lattices whose half volume is below one warp or one block: every
    variant (whole warps past the end, a single partial tile) matches the
    oracle and the direct kernel, for one and for three right-hand sides."""
    N, rep = 3, "SYM"
    lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), -0.3)
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), -0.3)
    UF = H.links(dims, N, 0.6, seed=8)
    UR = oracle_mod.represent_field(L, UF)
    g = hr.Gauge(lat, G.to_gpu(UF), precs=("f64", "f32"))
    vh = lat.volume // 2
    for nrhs in (1, 3):
        xs = H.spinor(vh, lat.D, 4, nrhs=nrhs)
        x = G.to_gpu(xs, torch.complex64)
        outs = {}
        for v in _variants(lat, nrhs):
            g.set_tuning(autotune=False, variant=v)
            outs[v] = g.apply(hr.EO_PRECOND, hr.F32, x, nrhs=nrhs).cpu().numpy()
        for v in outs:
            assert np.array_equal(outs[0], outs[v]), v
        ref = [oracle_mod.dhat(L, UR, (xs if nrhs == 1 else xs[k]).astype(np.complex64).astype(np.complex128))
               for k in range(nrhs)]
        got = outs[0] if nrhs > 1 else outs[0][None]
        for k in range(nrhs):
            assert G.rel(got[k].astype(np.complex128), ref[k]) <= G.TOL[hr.F32]
        g.set_tuning(autotune=True, variant=-1)
        b = G.to_gpu(xs if nrhs == 1 else xs)
        xsol, res, st = g.cg_solve(hr.EO_PRECOND, b, nrhs=nrhs, tol=1e-10, inner=hr.F32, inner_tol=1e-4)
        assert st == 0 and all(r["true_rel_residual"] <= 1e-10 for r in res)
    g.close()
