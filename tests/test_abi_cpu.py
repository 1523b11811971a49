"""CPU-only checks of the C ABI: the shared library loads, exports every
function include/hr.h declares, and reports argument errors without a GPU."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _declared():
    src = (ROOT / "include" / "hr.h").read_text()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hr_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_06721_gb300 import build, hr
    build.build()
    return hr.load()


def test_header_matches_binding():
    from paper_2503_06721_gb300 import hr
    assert _declared() == sorted(hr.EXPORTS)


def test_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_pure_host_calls(lib):
    from paper_2503_06721_gb300 import hr
    assert lib.hr_rep_dim(3, hr.SYM) == 6
    assert lib.hr_rep_dim(3, hr.ADJ) == 8
    assert lib.hr_rep_dim(4, hr.ASYM) == 6
    assert lib.hr_rep_dim(4, hr.ASYM_REAL) == 6
    assert lib.hr_rep_dim(3, hr.ASYM_REAL) == -1
    assert lib.hr_rep_dim(9, hr.FUND) == -1
    assert lib.hr_rep_dim(8, hr.FUND) == 8
    assert b"HR_ERR_INVALID" in lib.hr_status_string(-1)
    lat = hr.Lattice(3, "SYM", (8, 4, 4, 4))
    assert hr.field_bytes(lat, hr.EVEN, hr.F64) == 256 * 4 * 6 * 16
    assert hr.field_bytes(lat, hr.FULL, hr.F32, 2) == 2 * 512 * 4 * 6 * 8
    # F16: data rounded up to 256 B, then one float scale per site (rounded up)
    assert hr.field_bytes(lat, hr.EVEN, hr.F16) == 256 * 4 * 6 * 4 + 1024
    bad = hr.Lattice(3, "SYM", (8, 4, 4, 5))
    assert hr.field_bytes(bad, hr.EVEN, hr.F64) == 0


def test_generators_match_oracle(lib, oracle_mod):
    import numpy as np
    from paper_2503_06721_gb300 import hr
    for N in (2, 3, 4, 5, 6, 8):
        np.testing.assert_allclose(hr.generators(N), oracle_mod.generators(N), atol=1e-16)


def test_argument_errors_without_gpu(lib):
    from paper_2503_06721_gb300 import hr
    out = ctypes.c_void_p(0)
    d = hr.Lattice(3, "SYM", (8, 4, 4, 4)).desc()
    # NULL U_fund is rejected before any CUDA call
    assert lib.hr_represent_gauge(ctypes.byref(d), None, 1, 1, None, ctypes.byref(out)) == -1
    assert b"U_fund" in lib.hr_last_error()
    d.dims[3] = 5
    assert lib.hr_represent_gauge(ctypes.byref(d), ctypes.c_void_p(16), 1, 1, None,
                                  ctypes.byref(out)) == -1
    d.dims[3] = 4
    d.N = 9
    assert lib.hr_represent_gauge(ctypes.byref(d), ctypes.c_void_p(16), 1, 1, None,
                                  ctypes.byref(out)) == -1
    d.N = 5   # SU(5): the fundamental only, stored links only
    assert lib.hr_represent_gauge(ctypes.byref(d), ctypes.c_void_p(16), 1, 1, None,
                                  ctypes.byref(out)) == -7
    d.rep = hr.FUND
    assert lib.hr_represent_gauge(ctypes.byref(d), ctypes.c_void_p(16), 1, 2, None,
                                  ctypes.byref(out)) == -7
    assert b"stored links only" in lib.hr_last_error()
    d.N = 2
    d.rep = hr.ASYM   # the SU(2) antisymmetric (D = 1, a singlet) is not compiled
    assert lib.hr_represent_gauge(ctypes.byref(d), ctypes.c_void_p(16), 1, 1, None,
                                  ctypes.byref(out)) == -7
    assert lib.hr_dirac_apply(None, 0, 0, None, None, 1, None) == -1
    p = hr.CgParams(1e-10, 100, hr.F64, 1e-5, 0)
    r = hr.CgResult()
    assert lib.hr_cg_solve(None, hr.EO_PRECOND, None, None, 1, ctypes.byref(p), ctypes.byref(r),
                           None) == -1
    assert lib.hr_dirac_force(None, hr.FULL, None, None, 1.0, None, None) == -1
    assert lib.hr_dirac_force_prec(None, hr.FULL, None, None, 1.0, None, hr.DF64, None) == -1
