"""Pins of the oracle's reduced-precision storage model (oracle/storage.py):
rounding to FP32, binary16 and bfloat16 against brute-force nearest-number
search over the formats' own bit patterns (ties to even), hand-worked codes
of the per-site scaled spinor storage, and its invariants."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import storage as OS


def _table(fmt):
    """every finite number of a 16-bit format, sorted, with its bit pattern"""
    bits = np.arange(1 << 16, dtype=np.uint32)
    if fmt == "f16":
        vals = bits.astype(np.uint16).view(np.float16).astype(np.float64)
    else:
        with np.errstate(invalid="ignore"):
            vals = (bits << 16).view(np.float32).astype(np.float64)
    ok = np.isfinite(vals) & ~((vals == 0) & (bits >> 15 == 1))   # drop -0
    vals, bits = vals[ok], bits[ok]
    order = np.argsort(vals, kind="stable")
    return vals[order], bits[order]


def _nearest_even(x, vals, bits):
    """brute force: the nearest table entry, ties to the even bit pattern"""
    i = np.clip(np.searchsorted(vals, x), 1, len(vals) - 1)
    lo, hi = vals[i - 1], vals[i]
    dlo, dhi = x - lo, hi - x
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (bits[i] % 2 == 0))
    return np.where(pick_hi, hi, lo)


def _probe_values(vals, rng):
    inside = vals[(np.abs(vals) <= 4.0)]
    mids = 0.5 * (inside[:-1] + inside[1:])           # exact ties
    x = np.concatenate([
        rng.uniform(-2, 2, 20000),
        rng.uniform(-1e-4, 1e-4, 5000),               # binary16 subnormal range
        mids[::7], np.nextafter(mids[::7], np.inf), np.nextafter(mids[::7], -np.inf),
        inside[::11]])
    return x


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_round_binary_16bit_formats_brute_force(fmt):
    vals, bits = _table(fmt)
    x = _probe_values(vals, np.random.default_rng(7))
    got = OS.round_binary(x, fmt)
    want = _nearest_even(x, vals, bits)
    np.testing.assert_array_equal(got, want)


def test_round_binary_f32_nearest_and_ties_even():
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.uniform(-3, 3, 20000), rng.uniform(-1e-39, 1e-39, 2000)])
    r = OS.round_binary(x, "f32")
    r32 = r.astype(np.float32)
    assert (r32.astype(np.float64) == r).all()                 # representable
    up = np.nextafter(r32, np.float32(np.inf)).astype(np.float64)
    dn = np.nextafter(r32, np.float32(-np.inf)).astype(np.float64)
    assert (np.abs(x - r) <= np.abs(x - up)).all() and (np.abs(x - r) <= np.abs(x - dn)).all()
    # exact ties between neighbours go to the even significand
    a = rng.uniform(0.5, 1, 500).astype(np.float32)
    b = np.nextafter(a, np.float32(2))
    t = 0.5 * (a.astype(np.float64) + b.astype(np.float64))
    rt = OS.round_binary(t, "f32").astype(np.float32)
    even = np.where(a.view(np.uint32) % 2 == 0, a, b)
    np.testing.assert_array_equal(rt, even)


def test_round_binary_worked_values():
    # 0.3 in binary16: spacing 2^-12 on [1/4, 1/2); 0.3 * 4096 = 1228.8 -> 1229
    assert OS.round_binary(np.array([0.3]), "f16")[0] == float(Fraction(1229, 4096))
    # 1/3 in bfloat16: spacing 2^-9 on [1/4, 1/2); 512/3 = 170.67 -> 171
    assert OS.round_binary(np.array([1 / 3]), "bf16")[0] == float(Fraction(171, 512))
    # a tie in binary16 at 1 + 2^-11 (between 1 and 1 + 2^-10) goes to the even 1
    assert OS.round_binary(np.array([1 + 2.0 ** -11]), "f16")[0] == 1.0
    assert OS.round_binary(np.array([1 + 3 * 2.0 ** -11]), "f16")[0] == 1 + 2 * 2.0 ** -10
    # smallest binary16 subnormal 2^-24; half of it is a tie that goes to 0
    assert OS.round_binary(np.array([2.0 ** -25]), "f16")[0] == 0.0
    assert OS.round_binary(np.array([1.5 * 2.0 ** -25]), "f16")[0] == 2.0 ** -24


def test_quantize_spinor_worked_site():
    # one site, D = 1: components (re, im) per spin; largest |component| 2.0
    x = np.array([[[2.0 + 0.3j], [-1.0 + 0.0j], [0.6 - 0.1j], [0.0 + 1.0j]]])
    codes, s = OS.quantize_spinor(x, "f16")
    assert s[0] == 2.0
    # inv = 1/2 exactly; codes = round16(v / 2)
    want = np.array([1.0 + 1j * float(Fraction(1229, 8192)), -0.5, float(Fraction(1229, 4096))
                     - 1j * float(Fraction(1638, 32768)), 0.5j])
    # 0.15 on [1/8, 1/4): spacing 2^-13, 0.15 * 8192 = 1228.8 -> 1229
    # 0.05 on [1/32, 1/16): spacing 2^-15, 0.05 * 32768 = 1638.4 -> 1638
    np.testing.assert_array_equal(codes[0, :, 0], want)
    np.testing.assert_array_equal(OS.dequantize(codes, s), 2.0 * codes)


@pytest.mark.parametrize("fmt,q", [("f16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_quantize_spinor_invariants(fmt, q):
    rng = np.random.default_rng(5)
    x = (rng.normal(size=(3, 50, 4, 6)) + 1j * rng.normal(size=(3, 50, 4, 6))) * \
        np.exp(rng.normal(size=(3, 50, 1, 1)))
    codes, s = OS.quantize_spinor(x, fmt)
    x32 = OS.round_complex(x, "f32")
    # the scale is the largest |component| of the FP32 site, an FP32 number
    np.testing.assert_array_equal(s, np.maximum(np.abs(x32.real), np.abs(x32.imag)).max(axis=(-1, -2)))
    assert (s.astype(np.float32).astype(np.float64) == s).all()
    # codes are numbers of the format in [-1, 1]; the largest is +-1
    for part in (codes.real, codes.imag):
        np.testing.assert_array_equal(OS.round_binary(part, fmt), part)
        assert np.abs(part).max() <= 1.0
    top = np.maximum(np.abs(codes.real), np.abs(codes.imag)).max(axis=(-1, -2))
    np.testing.assert_array_equal(top, 1.0)
    # each stored value is within half a code spacing (at most q/2 below 1) of
    # the FP32 value, relative to the scale
    d = OS.dequantize(codes, s) - x32
    err = np.maximum(np.abs(d.real), np.abs(d.imag)) / s[..., None, None]
    assert err.max() <= 0.5 * q * (1 + 2.0 ** -20)


def test_stored_spinor_and_links_pass_through():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(10, 4, 3)) + 1j * rng.normal(size=(10, 4, 3))
    np.testing.assert_array_equal(OS.stored_spinor(x, 0), x)
    np.testing.assert_array_equal(OS.stored_spinor(x, 1), x.astype(np.complex64).astype(np.complex128))
    U = rng.normal(size=(5, 4, 3, 3)) + 1j * rng.normal(size=(5, 4, 3, 3))
    np.testing.assert_array_equal(OS.round_links(U, 0), U)
    np.testing.assert_array_equal(OS.round_links(U, 3, real=True).imag, 0.0)
    np.testing.assert_array_equal(OS.round_links(U, 3, real=True).real, OS.round_binary(U.real, "bf16"))
