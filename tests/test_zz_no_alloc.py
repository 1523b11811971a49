"""hr_field_dot_static, the dot product for callers that must not allocate
device memory, called through the C ABI and checked against hr_field_dot
(which allocates its scratch) on two calls in a row.  This file is collected
last so a failure here stops a -x run only after every other test ran."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["f64", "f32", "f16"])
def test_static_dot_matches_allocating_dot(hr, prec):
    from paper_2503_06721_gb300 import synth
    # 32^3 x 16 sextet: more sites than the fixed block count covers in one pass
    lat = hr.Lattice(3, "SYM", (16, 32, 32, 32))
    nrhs = 3
    vh = lat.volume // 2
    a64 = synth.gaussian_spinor(vh, lat.D, 1, device="cuda", nrhs=nrhs)
    b64 = synth.gaussian_spinor(vh, lat.D, 2, device="cuda", nrhs=nrhs)
    if prec == hr.F64:
        a, b = a64, b64
    elif prec == hr.F32:
        a, b = a64.to(torch.complex64), b64.to(torch.complex64)
    else:
        a = hr.field_convert(lat, hr.EVEN, a64, hr.F64, prec, nrhs)
        b = hr.field_convert(lat, hr.EVEN, b64, hr.F64, prec, nrhs)
    want = hr.field_dot(lat, hr.EVEN, prec, a, b, nrhs=nrhs)
    for call in range(2):   # the array keeps the previous call's contents
        st, got = _dot_static(hr, lat, hr.EVEN, prec, a, b, nrhs)
        assert st == 0, hr.load().hr_last_error()
        for k in range(nrhs):
            assert abs(got[k] - want[k]) <= 1e-12 * abs(want[k]), (call, k, got[k], want[k])


def test_static_dot_rejects_oversize(hr):
    lat = hr.Lattice(3, "SYM", (4, 4, 4, 4))
    x = torch.zeros((17, lat.volume // 2, 4, lat.D), dtype=torch.complex128, device="cuda")
    st, _ = _dot_static(hr, lat, hr.EVEN, hr.F64, x, x, 17)
    assert st == -1
    assert b"1..16" in hr.load().hr_last_error()
