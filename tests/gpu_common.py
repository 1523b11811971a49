"""Helpers shared by the GPU parity tests (layout conversion between the
oracle's lexicographic fields and the library's parity-ordered fields)."""
from __future__ import annotations

import numpy as np
import torch

from tests import _helpers as H

PAIRS = [(2, "FUND"), (2, "ADJ"), (2, "SYM"), (3, "FUND"), (3, "ADJ"), (3, "SYM"), (3, "ASYM"),
         (4, "FUND"), (4, "ASYM")]

# per-site relative tolerance (max_x |d(x)| / rms_x |ref(x)|):
#   FP64 and FP32: the stated parity bar (1e-13 / 1e-5);
#   F16 / BF16: each stored number carries a relative rounding error <= u
#   (u = 2^-11 for binary16, 2^-8 for bfloat16) in the link and in the spinor;
#   an output site sums 8 hops x 2 D products of such numbers with random
#   signs, so its relative error is bounded by about 2u sqrt(16 D) <= 2u * 12
#   for D <= 8.  The bound, not a fitted number, is the tolerance.
#   DF64 (float-float, about 48 bits) is held to the FP64 bar.
TOL = {0: 1e-13, 1: 1e-5, 2: 24 * 2.0 ** -11, 3: 24 * 2.0 ** -8, 4: 1e-13}


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
