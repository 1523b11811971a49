"""Batched solves: many right-hand sides and uneven lattice/mass instances
solved together (one CUDA graph per inner solve), FP32 inner / FP64
refinement to 1e-10.  Every solution is checked through an independent
residual: the oracle's operator on small lattices, the library's own FP64
operator and compensated dot products at full size."""
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


def point_sources(D, nsites):
    """12 point sources at the origin: 4 spins x 3 colour subsets {c : c mod 3 = k}."""
    b = np.zeros((12, nsites, 4, D), np.complex128)
    for s in range(4):
        for k in range(3):
            for c in range(D):
                if c % 3 == k:
                    b[3 * s + k, 0, s, c] = 1.0
    return b


def test_batched_small_vs_oracle(hr, oracle_mod):
    """uneven instances and rhs counts; each solution checked by the oracle."""
    N, rep = 4, "FUND"
    inst = [((4, 4, 4, 4), -0.1, 3), ((6, 4, 4, 6), -0.25, 12), ((8, 2, 4, 4), -0.4, 1)]
    gauges, bs, xs, Ls, URs, nr = [], [], [], [], [], []
    for i, (dims, m0, n) in enumerate(inst):
        lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), m0)
        L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), m0)
        UF = H.links(dims, N, 0.4, seed=200 + i)
        gauges.append(hr.Gauge(lat, G.to_gpu(UF), precs=("f64", "f32")))
        vh = lat.volume // 2
        b = point_sources(lat.D, vh) if n == 12 else H.spinor(vh, lat.D, 300 + i, nrhs=n)
        b = b.reshape(n, vh, 4, lat.D)
        bs.append(G.to_gpu(b))
        xs.append(torch.zeros_like(bs[-1]))
        Ls.append(L)
        URs.append(oracle_mod.represent_field(L, UF))
        nr.append(n)
    res, st = hr.cg_solve_batched(gauges, hr.EO_PRECOND, bs, xs, nr, tol=1e-10, inner=hr.F32)
    assert st == 0, res
    k = 0
    for i in range(len(inst)):
        x = xs[i].cpu().numpy()
        b = bs[i].cpu().numpy()
        for j in range(nr[i]):
            r = b[j] - oracle_mod.dhat(Ls[i], URs[i], oracle_mod.dhat(Ls[i], URs[i], x[j]), dagger=True)
            rel = np.linalg.norm(r) / np.linalg.norm(b[j])
            assert rel <= 1.001e-10, (i, j, rel)
            assert res[k]["status"] == "HR_OK"
            k += 1


def test_batched_equals_separate(hr, oracle_mod):
    """the batched solve gives the same solutions as separate solves (FP64 CG)."""
    N, rep = 3, "SYM"
    dims_list = [(4, 4, 2, 6), (6, 2, 4, 4)]
    gauges, bs, xs = [], [], []
    for i, dims in enumerate(dims_list):
        lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), -0.2)
        gauges.append(hr.Gauge(lat, G.to_gpu(H.links(dims, N, 0.5, seed=400 + i)), precs=("f64",)))
        bs.append(G.to_gpu(H.spinor(lat.volume // 2, lat.D, 500 + i, nrhs=2)))
        xs.append(torch.zeros_like(bs[-1]))
    res, st = hr.cg_solve_batched(gauges, hr.EO_PRECOND, bs, xs, [2, 2], tol=1e-11, inner=hr.F64)
    assert st == 0
    for g, b, x in zip(gauges, bs, xs):
        xs1, r1, st1 = g.cg_solve(hr.EO_PRECOND, b, nrhs=2, tol=1e-11)
        assert G.rel(x.cpu().numpy().reshape(-1, 4, g.lat.D), xs1.cpu().numpy().reshape(-1, 4, g.lat.D)) < 1e-9


@pytest.mark.parametrize("rep", ["FUND", "ASYM", "ASYM_REAL"])
def test_batched_full_size_su4(hr, oracle_mod, rep):
    """SU(4) 24^3 x 48 with 12 point sources, plus 8^4, 12^4, 16^3 x 32 instances at
    m0 = -0.1, -0.25, -0.4, one batched FP32-inner / FP64-refined solve to 1e-10."""
    from paper_2503_06721_gb300 import synth
    wl = synth.WORKLOADS[f"su4_{rep.lower()}_48x24x24x24"]
    specs = [(wl.dims, wl.m0, 12)] + [(d, m, 4) for d, m in synth.UNEVEN_INSTANCES]
    gauges, bs, xs, nr = [], [], [], []
    for i, (dims, m0, n) in enumerate(specs):
        lat = hr.Lattice(wl.N, rep, dims, wl.bc, m0)
        V = lat.volume
        U = synth.random_links(V, wl.N, wl.eps, wl.seed + i, device="cuda")
        gauges.append(hr.Gauge(lat, U, precs=("f64", "f32")))
        if n == 12:
            b = torch.as_tensor(point_sources(lat.D, V // 2)).to("cuda")
        else:
            b = synth.gaussian_spinor(V // 2, lat.D, 600 + i, device="cuda", nrhs=n)
        bs.append(b.contiguous())
        xs.append(torch.zeros_like(bs[-1]))
        nr.append(n)
    res, st = hr.cg_solve_batched(gauges, hr.EO_PRECOND, bs, xs, nr, tol=1e-10, inner=hr.F32)
    assert st == 0, res
    for g, b, x, n in zip(gauges, bs, xs, nr):
        lat = g.lat
        t = g.apply(hr.EO_PRECOND, hr.F64, x, nrhs=n)
        Ax = g.apply(hr.EO_PRECOND, hr.F64, t, nrhs=n, dagger=True)
        r = (Ax - b).contiguous()
        rr = hr.field_dot(lat, hr.EVEN, hr.F64, r, r, nrhs=n)
        bb = hr.field_dot(lat, hr.EVEN, hr.F64, b, b, nrhs=n)
        for k in range(n):
            assert (rr[k].real / bb[k].real) ** 0.5 <= 1.01e-10
        g.close()
