"""Helpers shared by the GPU parity tests (layout conversion between the
oracle's lexicographic fields and the library's parity-ordered fields, and
host-side packing of the reduced-precision storage so that the oracle reads
exactly what a kernel reads without taking any value from the GPU)."""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from oracle import storage as OS
from tests import _helpers as H

PAIRS = [(2, "FUND"), (2, "ADJ"), (2, "SYM"), (3, "FUND"), (3, "ADJ"), (3, "SYM"), (3, "ASYM"),
         (4, "FUND"), (4, "ASYM"), (4, "ASYM_REAL")]
# representations whose links the library stores as reals
REAL_REPS = ("ADJ", "ASYM_REAL")

# per-site relative tolerance (max_x |d(x)| / rms_x |ref(x)|):
#   FP64 and FP32: the stated parity bar (1e-13 / 1e-5);
#   F16 / BF16: each stored number carries a relative rounding error <= u
#   (u = 2^-11 for binary16, 2^-8 for bfloat16) in the link and in the spinor;
#   an output site sums 8 hops x 2 D products of such numbers with random
#   signs, so its relative error is bounded by about 2u sqrt(16 D) <= 2u * 12
#   for D <= 8.  The bound, not a fitted number, is the tolerance.
#   DF64 (float-float, about 48 bits) is held to the FP64 bar.
TOL = {0: 1e-13, 1: 1e-5, 2: 24 * 2.0 ** -11, 3: 24 * 2.0 ** -8, 4: 1e-13}

# Tight half-precision bound, used where the oracle runs on the kernel's own
# rounded inputs (links and spinors rounded on the host by oracle.storage):
# an output component is the kernel's FP32 value v rounded to a code of the
# narrow format times the site scale s, so |got - want| <= (q/2) s + |v - want|
# with q the spacing of codes in [1/2, 1) (2^-11 binary16, 2^-8 bfloat16),
# and |v - want| is the kernel's FP32 arithmetic on identical inputs, held to
# TAU32 * rms: a fifth of the FP32 parity bar (1e-5), against observed FP32
# errors of about 1e-7 (a few ulp of FP32 over sums of at most 2 D + 12
# rounded terms).
CODE_SPACING = {2: 2.0 ** -11, 3: 2.0 ** -8}
TAU32 = 2e-6


def gpu():
    return torch.device("cuda:0")


def to_gpu(a, dtype=torch.complex128):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device=gpu(), dtype=dtype)


def eo_full(oracle_mod, L, full):
    """lexicographic full field -> library FULL layout (even half, then odd half)."""
    e, o = oracle_mod.split(L, full)
    return np.concatenate([e, o], axis=0)


def from_eo_full(oracle_mod, L, eo):
    vh = eo.shape[0] // 2
    return oracle_mod.merge(L, eo[:vh], eo[vh:])


def prec_fields(hr, lat, parity, x64, prec, nrhs=1):
    """an FP64 device field -> the same field in precision prec (device)."""
    if prec == hr.F64:
        return x64
    if prec == hr.F32:
        return x64.to(torch.complex64)
    return hr.field_convert(lat, parity, x64, hr.F64, prec, nrhs)


def back_to_f64(hr, lat, parity, y, prec, nrhs=1):
    if prec == hr.F64:
        return y
    if prec == hr.F32:
        return y.to(torch.complex128)
    out = torch.empty((lat.nsites(parity), 4, lat.D) if nrhs == 1 else
                      (nrhs, lat.nsites(parity), 4, lat.D), dtype=torch.complex128, device=y.device)
    return hr.field_convert(lat, parity, y, prec, hr.F64, nrhs, dst=out)


def oracle_input(hr, lat, parity, x64, prec, nrhs=1):
    """what the kernel actually reads, promoted to FP64 on the host."""
    return back_to_f64(hr, lat, parity, prec_fields(hr, lat, parity, x64, prec, nrhs), prec,
                       nrhs).cpu().numpy()


def rel(a, b):
    return H.rel_site_norm(a, b)


# ---- reduced-precision storage on the host (layout of include/hr.h) ----

def _align(n, a=256):
    return (n + a - 1) // a * a


def pack_scaled(codes, scales, prec):
    """codes complex128 [nrhs, ns, 4, D] (numbers of the narrow format) and
    scales [nrhs, ns] -> the ABI bytes of an F16/BF16 field (uint8 numpy)."""
    nrhs, ns, _, D = codes.shape
    data_b = ns * 4 * D * 4
    blk = _align(data_b) + _align(ns * 4)
    out = np.zeros(nrhs * blk, np.uint8)
    for k in range(nrhs):
        pairs = np.stack([codes[k].real, codes[k].imag], -1).reshape(-1)
        if prec == 2:
            raw = pairs.astype(np.float16).view(np.uint8)
        else:
            raw = (pairs.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16).view(np.uint8)
        out[k * blk:k * blk + data_b] = raw
        sc = np.asarray(scales[k], np.float32).view(np.uint8)
        out[k * blk + _align(data_b):k * blk + _align(data_b) + ns * 4] = sc
    return out


def unpack_scaled(buf, prec, nrhs, ns, D):
    """ABI bytes of an F16/BF16 field -> (codes complex128, scales float64);
    the stored values are scales[..., None, None] * codes (exact in FP64)."""
    buf = np.asarray(buf, np.uint8)
    data_b = ns * 4 * D * 4
    blk = _align(data_b) + _align(ns * 4)
    codes = np.empty((nrhs, ns, 4, D), np.complex128)
    scales = np.empty((nrhs, ns), np.float64)
    for k in range(nrhs):
        raw = buf[k * blk:k * blk + data_b]
        if prec == 2:
            v = raw.view(np.float16).astype(np.float64)
        else:
            v = (raw.view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        v = v.reshape(ns, 4, D, 2)
        codes[k] = v[..., 0] + 1j * v[..., 1]
        scales[k] = buf[k * blk + _align(data_b):k * blk + _align(data_b) + ns * 4].view(np.float32)
    return codes, scales


def kernel_input(x64, prec):
    """A field in precision prec built on the HOST from the FP64 values x64
    (numpy [ns,4,D] or [nrhs,ns,4,D]): returns (device tensor in the ABI
    layout, the stored values promoted to FP64 as a numpy array of x64's
    shape).  The oracle reads the second; nothing comes from the GPU."""
    x64 = np.asarray(x64, np.complex128)
    if prec == 0:
        return to_gpu(x64), x64.copy()
    if prec == 1:
        xs = OS.round_complex(x64, "f32")
        return to_gpu(xs, torch.complex64), xs
    if prec == 4:
        rh, rl = OS.split_df64(x64.real)
        ih, il = OS.split_df64(x64.imag)
        quad = np.stack([rh, rl, ih, il], -1).astype(np.float32)
        return torch.as_tensor(quad).to(gpu()), (rh + rl) + 1j * (ih + il)
    one = x64.ndim == 3
    xx = x64[None] if one else x64
    codes, scales = OS.quantize_spinor(xx, prec)
    dev = torch.as_tensor(pack_scaled(codes, scales, prec)).to(gpu())
    vals = OS.dequantize(codes, scales)
    return dev, (vals[0] if one else vals)


def kernel_output(y, prec, ns, D, nrhs=1):
    """A device field in precision prec -> (FP64 values numpy, site scales or
    None), decoded on the host without rounding."""
    if prec in (0, 1):
        return y.to(torch.complex128).cpu().numpy(), None
    if prec == 4:
        q = y.cpu().numpy().astype(np.float64)
        return (q[..., 0] + q[..., 1]) + 1j * (q[..., 2] + q[..., 3]), None
    codes, scales = unpack_scaled(y.cpu().numpy(), prec, nrhs, ns, D)
    vals = OS.dequantize(codes, scales)
    if nrhs == 1:
        return vals[0], scales[0]
    return vals, scales


def scaled_excess(got, scales, want, prec, allowance=None):
    """max over components of |got - want| / ((q/2) s_x + allowance_x + TAU32 rms):
    <= 1 passes the tight half-precision bound (see CODE_SPACING)."""
    got = np.asarray(got).reshape(got.shape[0], -1)
    want = np.asarray(want).reshape(want.shape[0], -1)
    rms = np.sqrt((np.abs(want) ** 2).sum(1).mean())
    bound = 0.5 * CODE_SPACING[prec] * np.asarray(scales)[:, None] + TAU32 * rms
    if allowance is not None:
        bound = bound + np.asarray(allowance)[:, None]
    d = np.maximum(np.abs(got.real - want.real), np.abs(got.imag - want.imag))
    return float((d / bound).max())


def rounding_allowance(oracle_mod, L, mid_half, mid_parity, prec, tau=TAU32):
    """Where an intermediate field (half field of parity mid_parity, oracle
    values) is stored in F16/BF16 inside one operator call, a component whose
    code lies within the kernel's FP32 error (tau * rms, in code units tau *
    rms / s_y) of a rounding midpoint may round either way on the GPU.  Returns,
    per site of the other parity, the sum over its 8 neighbours y of the
    largest change such a flip can make, 2 x (code spacing) x s_y per
    ambiguous component: one hop passes a change e of one component to every
    output component with a factor of at most |U_rc| <= 1."""
    p, _ = OS.FORMATS[OS.PREC_NAMES[prec]]
    m = np.asarray(mid_half, np.complex128)
    rms = np.sqrt((np.abs(m) ** 2).sum(axis=(-1, -2)).mean())
    re, im = OS.round_binary(m.real, "f32"), OS.round_binary(m.imag, "f32")
    s = np.maximum(np.abs(re), np.abs(im)).max(axis=(-1, -2))
    safe = np.where(s > 0, s, 1.0)[:, None, None]
    per_site = np.zeros(len(s))
    for part in (re, im):
        c = np.abs(part) / safe
        _, e = np.frexp(np.where(c > 0, c, 1.0))
        spacing = np.ldexp(1.0, e - 1 - (p - 1))
        t = c / spacing
        dist = np.abs(t - np.floor(t) - 0.5) * spacing
        amb = (dist <= tau * rms / safe) & (c > 0)
        per_site += (amb * 2.0 * spacing).reshape(len(s), -1).sum(1) * s
    nb = oracle_mod._neighbours(L)
    par = oracle_mod.parity_of_sites(L)
    lex = np.arange(oracle_mod.volume(L))
    out_lex = lex[par != mid_parity]
    out = np.zeros(len(out_lex))
    for sdir in range(2):
        for mu in range(4):
            out += per_site[nb[sdir, out_lex, mu] // 2]
    res = np.zeros(len(out_lex))
    res[out_lex // 2] = out
    return res


def report(case, **vals):
    """Appends one JSON line of observed errors to $HR_PARITY_REPORT (if set)."""
    path = os.environ.get("HR_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(dict(case=case, **vals)) + "\n")
