"""hr_field_dot_static, the dot product for callers that must not allocate
device memory (code running under another allocator that owns the device
memory, or on a path that cannot take cudaMalloc's implicit device
synchronisation), called through the C ABI.  Its result is checked against
hr_field_dot (which allocates its scratch) and against an FP64 dot product
of the stored values computed on the host, on two calls in a row (the fixed
scratch array keeps the previous call's contents).  This file is collected
last so that a failure here stops a -x run only after every other test ran."""
import ctypes

import numpy as np
import pytest
import torch

from tests import gpu_common as G

pytestmark = pytest.mark.gpu

# the fixed launch shape of hr_field_dot_static: at most 1216 blocks of 256
# threads; lattices with more sites per right-hand side make each thread
# take several sites
STATIC_THREADS = 1216 * 256


@pytest.fixture(scope="module")
def hr():
    from paper_2503_06721_gb300 import build, hr
    build.build()
    hr.load()
    return hr


def _dot_static(hr, lat, par, prec, a, b, nrhs):
    d = lat.desc()
    out = (ctypes.c_double * (2 * nrhs))()
    st = hr.load().hr_field_dot_static(ctypes.byref(d), par, prec, ctypes.c_void_p(a.data_ptr()),
                                       ctypes.c_void_p(b.data_ptr()), nrhs, out,
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, [complex(out[2 * k], out[2 * k + 1]) for k in range(nrhs)]


CASES = [
    # SU(3) sextet 32^4, even sites: 524288 sites per right-hand side, more
    # than the fixed grid's threads, so each thread sums up to two sites
    ((3, "SYM", (32, 32, 32, 32)), 0, 2),
    # SU(5) fundamental (D = 5), whole lattice
    ((5, "FUND", (8, 8, 8, 8)), 2, 3),
]


@pytest.mark.parametrize("case", range(len(CASES)), ids=["su3sym_32x32x32x32_capped", "su5fund_8x8x8x8_full"])
@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4], ids=["f64", "f32", "f16", "bf16", "df64"])
def test_static_dot_matches_allocating_dot(hr, prec, case):
    from paper_2503_06721_gb300 import synth
    (N, rep, dims), par, nrhs = CASES[case]
    lat = hr.Lattice(N, rep, dims)
    ns = lat.nsites(par)
    if case == 0:
        assert ns > STATIC_THREADS   # the grid is capped and the grid-stride loop runs
    a64 = synth.gaussian_spinor(ns, lat.D, 1, nrhs=nrhs).numpy()
    b64 = synth.gaussian_spinor(ns, lat.D, 2, nrhs=nrhs).numpy()
    # fields stored on the host in precision prec; av, bv the stored values in FP64
    a, av = G.kernel_input(a64, prec)
    b, bv = G.kernel_input(b64, prec)
    want_alloc = hr.field_dot(lat, par, prec, a, b, nrhs=nrhs)
    want_host = [np.vdot(av[k].ravel(), bv[k].ravel()) for k in range(nrhs)]
    mag = [float(np.abs(av[k]).ravel() @ np.abs(bv[k]).ravel()) for k in range(nrhs)]
    # F16/BF16 values are formed as fl32(scale * code) in the kernels: 2^-24 relative per value
    tol_host = 1e-12 if prec in (0, 1, 4) else 2.0 ** -22
    for call in range(2):   # the array keeps the previous call's contents
        st, got = _dot_static(hr, lat, par, prec, a, b, nrhs)
        assert st == 0, hr.load().hr_last_error()
        for k in range(nrhs):
            assert abs(got[k] - want_alloc[k]) <= 1e-13 * mag[k], (call, k, got[k], want_alloc[k])
            assert abs(got[k] - want_host[k]) <= tol_host * mag[k], (call, k, got[k], want_host[k])


def test_static_dot_rejects_oversize_and_bad_parity(hr):
    lat = hr.Lattice(3, "SYM", (4, 4, 4, 4))
    x = torch.zeros((17, lat.volume // 2, 4, lat.D), dtype=torch.complex128, device="cuda")
    st, _ = _dot_static(hr, lat, hr.EVEN, hr.F64, x, x, 17)
    assert st == -1
    assert b"1..16" in hr.load().hr_last_error()
    st, _ = _dot_static(hr, lat, 7, hr.F64, x, x, 1)
    assert st == -1
