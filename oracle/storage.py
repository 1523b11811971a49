"""Reduced-precision storage model of the oracle (TEST INFRASTRUCTURE ONLY).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this module.  It shares no code with the GPU library.

The paper stores fields in double precision and offers single-precision
fields and operators (Sec. 3.1.1).  The library adds binary16 and bfloat16
spinor storage with one scale per site.  This module writes out, from the
IEEE 754 definitions, what a number looks like after it has been stored in
such a format, so that the oracle can be run on exactly the rounded inputs a
kernel reads (promoted to FP64) and the comparison isolates the kernel's own
arithmetic:

  round_binary(x, fmt)  round-to-nearest, ties-to-even, of FP64 values to a
                        binary format with p significand bits and minimum
                        normal exponent emin (FP32: 24, -126; binary16: 11,
                        -14; bfloat16: 8, -126), subnormals included;
  round_links(UR, prec, real)
                        represented (or fundamental) links stored entry by
                        entry in FP32 / binary16 / bfloat16 (unitary links
                        have |entries| <= 1 and need no scale);
  split_df64(x)         float-float storage (hi, lo) of FP64 values;
  quantize_spinor(x, prec)
                        the per-site scaled storage of a spinor field: each
                        value is first rounded to FP32 (the arithmetic type of
                        the reduced-precision kernels), s_x = the largest
                        |component| of site x, inv = fl32(1 / s_x), and each
                        stored code = round(fl32(inv * v)) in the narrow
                        format; the value a kernel reads is s_x * code.

Every step in FP32 is a single rounding of an exactly computed FP64 value:
products of two FP32 numbers are exact in FP64, and a quotient rounded first
to FP64 and then to FP32 equals the correctly rounded FP32 quotient because
53 >= 2 * 24 + 2.
"""
from __future__ import annotations

import numpy as np

# (significand bits including the implicit one, minimum normal exponent)
FORMATS = {"f32": (24, -126), "f16": (11, -14), "bf16": (8, -126)}
# hr_prec numbering of the library's ABI
PREC_NAMES = {1: "f32", 2: "f16", 3: "bf16"}


def _fmt(prec):
    name = PREC_NAMES.get(prec, prec)
    return FORMATS[name]


def round_binary(x, prec):
    """x (float64 array) rounded to the nearest number of the binary format
    (ties to even), returned as float64.  No overflow handling: the stored
    values here are at most 1 in magnitude (codes) or small (spinors)."""
    p, emin = _fmt(prec)
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)                       # x = m 2^e with 1/2 <= |m| < 1
    E = np.maximum(e - 1, emin)              # exponent of the leading bit (clamped: subnormals)
    q = E - (p - 1)                          # exponent of the last significand bit
    return np.ldexp(np.rint(np.ldexp(x, -q)), q)   # exact scalings; rint rounds half to even


def round_complex(z, prec):
    z = np.asarray(z, dtype=np.complex128)
    return round_binary(z.real, prec) + 1j * round_binary(z.imag, prec)


def round_links(UR, prec, real=False):
    """Links as stored in precision prec: every entry rounded once from FP64
    (for the real adjoint representation the imaginary parts are zero and only
    the real parts are stored)."""
    UR = np.asarray(UR, dtype=np.complex128)
    if prec in (0, "f64"):
        return UR.copy()
    if real:
        return round_binary(UR.real, prec) + 0j
    return round_complex(UR, prec)


def quantize_spinor(x, prec):
    """Per-site scaled storage of a spinor field x[..., nsites, 4, D] (FP64).
    Returns (codes, scales): codes complex128 of the same shape, every real
    and imaginary part a number of the narrow format in [-1, 1]; scales
    float64 [..., nsites] (FP32 numbers).  The stored value is
    scales[..., None, None] * codes."""
    x = np.asarray(x, dtype=np.complex128)
    re = round_binary(x.real, "f32")
    im = round_binary(x.imag, "f32")
    s = np.maximum(np.abs(re), np.abs(im)).max(axis=(-1, -2))
    safe = np.where(s > 0, s, 1.0)
    inv = np.where(s > 0, round_binary(1.0 / safe, "f32"), 0.0)[..., None, None]
    cre = round_binary(round_binary(inv * re, "f32"), prec)
    cim = round_binary(round_binary(inv * im, "f32"), prec)
    return cre + 1j * cim, s


def dequantize(codes, scales):
    return np.asarray(scales)[..., None, None] * np.asarray(codes)


def split_df64(x):
    """Float-float storage of FP64 values: hi = fl32(x), lo = fl32(x - hi)
    (x - hi is exact in FP64).  Returns (hi, lo) as float64 arrays; the
    stored value is hi + lo, within 2^-48 |x| of x."""
    x = np.asarray(x, dtype=np.float64)
    hi = round_binary(x, "f32")
    return hi, round_binary(x - hi, "f32")


def stored_spinor(x, prec):
    """The values a kernel reads from a field stored in precision prec,
    promoted to FP64 (FP64 itself is returned unchanged)."""
    if prec in (0, "f64"):
        return np.asarray(x, dtype=np.complex128).copy()
    if prec in (1, "f32"):
        return round_complex(x, "f32")
    if prec in (4, "df64"):
        x = np.asarray(x, dtype=np.complex128)
        return sum(split_df64(x.real)) + 1j * sum(split_df64(x.imag))
    return dequantize(*quantize_spinor(x, prec))
