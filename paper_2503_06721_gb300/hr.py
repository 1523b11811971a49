"""ctypes binding of libhr (include/hr.h): the same names, argument marshalling
only.  Every operation runs in the library's CUDA kernels; if libhr.so is
missing this module raises instead of falling back to anything else.

Tensors are torch CUDA tensors (PyTorch supplies device memory and streams):
  FP64 fields  complex128 [nrhs, nsites, 4, D] (or [nsites, 4, D])
  FP32 fields  complex64  of the same shape
  F16/BF16     uint8 buffers of field_bytes(...) bytes (data + per-site scales)
  DF64 fields  float32 [nrhs, nsites, 4, D, 4] = (re.hi, re.lo, im.hi, im.lo)
  gauge input  complex128 [V, 4, N, N]
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from pathlib import Path

import numpy as np
import torch

_LIB_PATH = Path(__file__).resolve().parent / "_lib" / "libhr.so"

FUND, ADJ, SYM, ASYM, ASYM_REAL = 0, 1, 2, 3, 4
REPS = {"FUND": FUND, "ADJ": ADJ, "SYM": SYM, "ASYM": ASYM, "2AS": ASYM, "ASYM_REAL": ASYM_REAL,
        "2AS_REAL": ASYM_REAL}
F64, F32, F16, BF16, DF64 = 0, 1, 2, 3, 4
PRECS = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16, "df64": DF64}
EVEN, ODD, FULL, EO_PRECOND = 0, 1, 2, 3
HOP_DIRECT, HOP_STAGED, HOP_STAGED_TIGHT, HOP_STAGED_LINKS, HOP_MRHS = 0, 1, 2, 3, 4
EPI_STORE, EPI_STORE_NORM, EPI_CG_UPDATE = 0, 1, 2
LINKS_STORED, LINKS_REBUILD, LINKS_AUTO = 0, 1, 2

STATUS = {0: "HR_OK", -1: "HR_ERR_INVALID", -2: "HR_ERR_CUDA", -3: "HR_ERR_NOMEM",
          -4: "HR_ERR_NOT_CONVERGED", -5: "HR_ERR_NONFINITE", -6: "HR_ERR_TIMEOUT",
          -7: "HR_ERR_UNSUPPORTED"}

# every symbol include/hr.h declares
EXPORTS = ["hr_represent_gauge", "hr_gauge_update", "hr_gauge_set_link_mode", "hr_gauge_destroy",
           "hr_tune", "hr_gauge_set_tuning", "hr_gauge_hop_variant", "hr_gauge_link_mode",
           "hr_field_bytes", "hr_field_convert", "hr_field_dot", "hr_field_dot_static",
           "hr_dirac_apply", "hr_dirac_dagger",
           "hr_cg_solve", "hr_cg_solve_batched", "hr_cg_solve_force", "hr_cg_solve_multishift",
           "hr_field_lincomb", "hr_rational_approx", "hr_dirac_force", "hr_dirac_force_prec", "hr_gauge_action", "hr_gauge_force", "hr_link_update",
           "hr_momenta_energy", "hr_md_trajectory", "hr_hmc_update", "hr_gauge_set_clover", "hr_rep_dim", "hr_generators",
           "hr_status_string", "hr_last_error", "hr_launch_count"]


class HrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class LatticeDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("rep", ctypes.c_int), ("dims", ctypes.c_int * 4),
                ("bc", ctypes.c_int * 4), ("m0", ctypes.c_double)]


class CgParams(ctypes.Structure):
    _fields_ = [("tol_rel", ctypes.c_double), ("max_iter", ctypes.c_int), ("inner", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("use_initial_guess", ctypes.c_int),
                ("residual", ctypes.c_int)]


class CgResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("true_rel_residual", ctypes.c_double), ("status", ctypes.c_int)]


class MdParams(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("tau", ctypes.c_double), ("nsteps", ctypes.c_int),
                ("integrator", ctypes.c_int), ("sys", ctypes.c_int), ("cg", CgParams)]


class MdStats(ctypes.Structure):
    _fields_ = [("force_evals", ctypes.c_int), ("cg_iters", ctypes.c_int),
                ("max_true_rel_residual", ctypes.c_double), ("status", ctypes.c_int)]


class HmcResult(ctypes.Structure):
    _fields_ = [("H0", ctypes.c_double * 3), ("H1", ctypes.c_double * 3), ("dH", ctypes.c_double),
                ("accepted", ctypes.c_int), ("md", MdStats)]


MD_LEAPFROG, MD_OMELYAN2 = 0, 1
CLOVER_NONE, CLOVER_PLAIN, CLOVER_EXP = 0, 1, 2
T_FUND = 0.5


_lib = None


def lib_path() -> Path:
    return _LIB_PATH


def load():
    """Opens libhr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not _LIB_PATH.exists():
        raise RuntimeError(f"{_LIB_PATH} is not built; run paper_2503_06721_gb300.build.build()")
    L = ctypes.CDLL(str(_LIB_PATH))
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    LP = ctypes.POINTER(LatticeDesc)
    sig = {
        "hr_represent_gauge": (I, [LP, P, ctypes.c_uint, ctypes.c_uint, P, ctypes.POINTER(P)]),
        "hr_gauge_update": (I, [P, P, P]),
        "hr_gauge_set_link_mode": (I, [P, I]),
        "hr_gauge_destroy": (I, [P]),
        "hr_tune": (I, [P, I, I, P]),
        "hr_gauge_set_tuning": (I, [P, I, I]),
        "hr_gauge_hop_variant": (I, [P, I, I, I]),
        "hr_gauge_link_mode": (I, [P, I]),
        "hr_field_bytes": (S, [LP, I, I, I]),
        "hr_field_convert": (I, [LP, I, I, P, I, P, I, P]),
        "hr_field_dot": (I, [LP, I, I, P, P, I, ctypes.POINTER(D), P]),
        "hr_field_dot_static": (I, [LP, I, I, P, P, I, ctypes.POINTER(D), P]),
        "hr_dirac_apply": (I, [P, I, I, P, P, I, P]),
        "hr_dirac_dagger": (I, [P, I, I, P, P, I, P]),
        "hr_cg_solve": (I, [P, I, P, P, I, ctypes.POINTER(CgParams), ctypes.POINTER(CgResult), P]),
        "hr_cg_solve_batched": (I, [I, ctypes.POINTER(P), I, ctypes.POINTER(P), ctypes.POINTER(P),
                                    ctypes.POINTER(I), ctypes.POINTER(CgParams),
                                    ctypes.POINTER(CgResult), P]),
        "hr_dirac_force": (I, [P, I, P, P, D, P, P]),
        "hr_dirac_force_prec": (I, [P, I, P, P, D, P, I, P]),
        "hr_cg_solve_multishift": (I, [P, I, P, P, I, ctypes.POINTER(D), I, ctypes.POINTER(CgParams),
                                       ctypes.POINTER(CgResult), P]),
        "hr_field_lincomb": (I, [LP, I, D, P, I, ctypes.POINTER(D), P, P, I, P]),
        "hr_rational_approx": (I, [D, I, D, D, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D),
                                   ctypes.POINTER(D)]),
        "hr_gauge_action": (I, [LP, P, D, ctypes.POINTER(D), P]),
        "hr_gauge_force": (I, [LP, P, D, D, P, P]),
        "hr_link_update": (I, [LP, P, P, D, P]),
        "hr_momenta_energy": (I, [LP, P, ctypes.POINTER(D), P]),
        "hr_md_trajectory": (I, [P, P, P, P, ctypes.POINTER(MdParams), ctypes.POINTER(MdStats), P]),
        "hr_hmc_update": (I, [P, P, P, P, D, ctypes.POINTER(MdParams), ctypes.POINTER(HmcResult), P]),
        "hr_gauge_set_clover": (I, [P, P, D, I, P]),
        "hr_cg_solve_force": (I, [P, I, P, P, ctypes.POINTER(CgParams), ctypes.POINTER(CgResult), P, D, P, P]),
        "hr_rep_dim": (I, [I, I]),
        "hr_generators": (I, [I, ctypes.POINTER(D)]),
        "hr_status_string": (ctypes.c_char_p, [I]),
        "hr_last_error": (ctypes.c_char_p, []),
        "hr_launch_count": (ctypes.c_ulonglong, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise HrError(status, load().hr_last_error().decode())


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def launch_count() -> int:
    return int(load().hr_launch_count())


def rep_dim(N: int, rep) -> int:
    return load().hr_rep_dim(N, REPS.get(rep, rep) if isinstance(rep, str) else rep)


def generators(N: int):
    import numpy as np
    buf = (ctypes.c_double * (2 * (N * N - 1) * N * N))()
    _check(load().hr_generators(N, buf))
    a = np.frombuffer(buf, dtype=np.float64).copy()
    return (a[0::2] + 1j * a[1::2]).reshape(N * N - 1, N, N)


@dataclass
class Lattice:
    N: int
    rep: str
    dims: tuple
    bc: tuple = (-1, 1, 1, 1)
    m0: float = 0.0

    @property
    def D(self) -> int:
        return rep_dim(self.N, self.rep)

    @property
    def volume(self) -> int:
        T, X, Y, Z = self.dims
        return T * X * Y * Z

    def desc(self) -> LatticeDesc:
        d = LatticeDesc()
        d.N = self.N
        d.rep = REPS[self.rep] if isinstance(self.rep, str) else self.rep
        for i in range(4):
            d.dims[i] = self.dims[i]
            d.bc[i] = self.bc[i]
        d.m0 = self.m0
        return d

    def nsites(self, parity: int) -> int:
        return self.volume if parity == FULL else self.volume // 2


def field_bytes(lat: Lattice, parity: int, prec: int, nrhs: int = 1) -> int:
    d = lat.desc()
    return int(load().hr_field_bytes(ctypes.byref(d), parity, prec, nrhs))


def empty_field(lat: Lattice, parity: int, prec: int, nrhs: int = 1, device="cuda"):
    ns = lat.nsites(parity)
    shape = (nrhs, ns, 4, lat.D) if nrhs > 1 else (ns, 4, lat.D)
    if prec == F64:
        return torch.empty(shape, dtype=torch.complex128, device=device)
    if prec == F32:
        return torch.empty(shape, dtype=torch.complex64, device=device)
    if prec == DF64:
        return torch.empty(shape + (4,), dtype=torch.float32, device=device)
    return torch.empty(field_bytes(lat, parity, prec, nrhs), dtype=torch.uint8, device=device)


def field_convert(lat: Lattice, parity: int, src, src_prec: int, dst_prec: int, nrhs: int = 1,
                  dst=None, stream=None):
    if dst is None:
        dst = empty_field(lat, parity, dst_prec, nrhs, src.device)
    d = lat.desc()
    _check(load().hr_field_convert(ctypes.byref(d), parity, src_prec, _ptr(src), dst_prec, _ptr(dst),
                                   nrhs, _stream(stream)))
    return dst


def field_dot(lat: Lattice, parity: int, prec: int, a, b, nrhs: int = 1, stream=None):
    d = lat.desc()
    out = (ctypes.c_double * (2 * nrhs))()
    _check(load().hr_field_dot(ctypes.byref(d), parity, prec, _ptr(a), _ptr(b), nrhs, out,
                               _stream(stream)))
    return [complex(out[2 * k], out[2 * k + 1]) for k in range(nrhs)]


def field_lincomb(lat: Lattice, parity: int, a0: float, b, coeffs, x, y=None, nrhs: int = 1, stream=None):
    """y = a0 b + sum_k coeffs[k] x[k] (FP64 fields; x as cg_solve_multishift returns it)."""
    d = lat.desc()
    n = len(coeffs)
    if y is None:
        y = torch.empty_like(b)
    arr = (ctypes.c_double * max(n, 1))(*[float(c) for c in coeffs])
    _check(load().hr_field_lincomb(ctypes.byref(d), parity, float(a0), _ptr(b), n, arr, _ptr(x), _ptr(y),
                                   nrhs, _stream(stream)))
    return y


def rational_approx(alpha: float, n: int, lo: float, hi: float):
    """(a0, residues, poles, max_rel_err) of the best degree-(n, n) relative
    approximation of x^(-alpha) on [lo, hi] (hr_rational_approx)."""
    a0, err = ctypes.c_double(0.0), ctypes.c_double(0.0)
    res, poles = (ctypes.c_double * n)(), (ctypes.c_double * n)()
    _check(load().hr_rational_approx(float(alpha), int(n), float(lo), float(hi), ctypes.byref(a0), res, poles,
                                     ctypes.byref(err)))
    return a0.value, tuple(res), tuple(poles), err.value


def rational_apply(g, sys: int, b, approx, nrhs: int = 1, tol: float = 1e-10, inner: int = F64,
                   inner_tol: float = 1e-5, stream=None):
    """r(A) b = a0 b + sum_k a_k (A + b_k)^-1 b for a RationalApprox (the RHMC's
    heat-bath and action terms, Sec. 4.3.2): one multi-shift inversion over the
    poles, then one linear-combination kernel.  Returns (y, x_k, results)."""
    x, res, st = g.cg_solve_multishift(sys, b, approx.poles, nrhs=nrhs, tol=tol, inner=inner,
                                       inner_tol=inner_tol, stream=stream)
    par = FULL if sys == FULL else EVEN
    y = field_lincomb(g.lat, par, approx.a0, b, approx.residues, x, nrhs=nrhs, stream=stream)
    return y, x, res


# ---- HMC building blocks (Sec. 2.4, 2.5, 4.2) ----

def gauge_action(lat: Lattice, U_fund, beta: float, stream=None) -> float:
    """S_g = beta sum (1 - Re tr P / N) (hr_gauge_action)."""
    d = lat.desc()
    out = ctypes.c_double(0.0)
    _check(load().hr_gauge_action(ctypes.byref(d), _ptr(U_fund), float(beta), ctypes.byref(out),
                                  _stream(stream)))
    return out.value


def gauge_force(lat: Lattice, U_fund, beta: float, coeff: float = 1.0, F=None, stream=None):
    """F += coeff * dS_g/de^a (hr_gauge_force); F[V, 4, N*N-1] FP64."""
    if F is None:
        F = torch.zeros((lat.volume, 4, lat.N ** 2 - 1), dtype=torch.float64, device=U_fund.device)
    d = lat.desc()
    _check(load().hr_gauge_force(ctypes.byref(d), _ptr(U_fund), float(beta), float(coeff), _ptr(F),
                                 _stream(stream)))
    return F


def link_update(lat: Lattice, U_fund, pi, eps: float, stream=None):
    """U <- exp(i eps pi^a T^a) U in place (hr_link_update)."""
    d = lat.desc()
    _check(load().hr_link_update(ctypes.byref(d), _ptr(U_fund), _ptr(pi), float(eps), _stream(stream)))
    return U_fund


def momenta_energy(lat: Lattice, pi, stream=None) -> float:
    """T_F/2 sum pi^2 (hr_momenta_energy)."""
    d = lat.desc()
    out = ctypes.c_double(0.0)
    _check(load().hr_momenta_energy(ctypes.byref(d), _ptr(pi), ctypes.byref(out), _stream(stream)))
    return out.value


def md_trajectory(g, U_fund, pi, phi, beta: float, tau: float, nsteps: int, integrator: int = MD_OMELYAN2,
                  sys: int = EO_PRECOND, tol: float = 1e-10, inner: int = F64, inner_tol: float = 1e-5,
                  chrono: bool = False, stream=None) -> dict:
    """One MD trajectory in place on (U_fund, pi), g re-represented (hr_md_trajectory)."""
    p = MdParams(float(beta), float(tau), int(nsteps), int(integrator), int(sys),
                 CgParams(tol, 100000, inner, inner_tol, int(chrono), F64))
    st = MdStats()
    _check(load().hr_md_trajectory(g.handle, _ptr(U_fund), _ptr(pi), _ptr(phi), ctypes.byref(p),
                                   ctypes.byref(st), _stream(stream)))
    return dict(force_evals=st.force_evals, cg_iters=st.cg_iters,
                max_true_rel_residual=st.max_true_rel_residual)


def fermion_action(g, sys: int, phi, tol: float = 1e-12, inner: int = F64, stream=None) -> float:
    """S_f = phi^dag A^-1 phi: one solve (hr_cg_solve) and one dot product (hr_field_dot)."""
    x, res, st = g.cg_solve(sys, phi, tol=tol, inner=inner, stream=stream)
    par = FULL if sys == FULL else EVEN
    return field_dot(g.lat, par, F64, phi, x, stream=stream)[0].real


def hamiltonian(g, U_fund, pi, phi, beta: float, sys: int = EO_PRECOND, tol: float = 1e-12, inner: int = F64,
                stream=None):
    """(H_pi, S_g, S_f) of Sec. 2.5 for the links g represents (= U_fund)."""
    Sf = fermion_action(g, sys, phi, tol, inner=inner, stream=stream) if phi is not None else 0.0
    return momenta_energy(g.lat, pi, stream), gauge_action(g.lat, U_fund, beta, stream), Sf


def hmc_trajectory(g, U_fund, pi, eta, beta: float, tau: float, nsteps: int, u_accept: float,
                   integrator: int = MD_OMELYAN2, sys: int = EO_PRECOND, tol: float = 1e-10,
                   inner: int = F64, inner_tol: float = 1e-5, stream=None) -> dict:
    """One HMC update (Sec. 2.5, hr_hmc_update): pseudofermion heat bath phi =
    Dhat^dag eta (D^dag eta for sys = FULL), H before, one MD trajectory, H
    after, and the Metropolis test exp(-dH) > u_accept.  pi (heat-bath
    momenta, pi^a ~ N(0, 1/T_F)), eta (Gaussian, or None for the pure gauge
    theory) and u_accept (uniform in [0, 1)) are the caller's random draws.
    On acceptance U_fund holds the new links; on rejection it is restored.  g
    represents U_fund on return."""
    p = MdParams(float(beta), float(tau), int(nsteps), int(integrator), int(sys),
                 CgParams(tol, 100000, inner, inner_tol, 0, F64))
    r = HmcResult()
    _check(load().hr_hmc_update(g.handle, _ptr(U_fund), _ptr(pi), _ptr(eta), float(u_accept), ctypes.byref(p),
                                ctypes.byref(r), _stream(stream)))
    return dict(dH=r.dH, accepted=bool(r.accepted), H0=tuple(r.H0), H1=tuple(r.H1),
                force_evals=r.md.force_evals, cg_iters=r.md.cg_iters,
                max_true_rel_residual=r.md.max_true_rel_residual)


def _prec_mask(precs) -> int:
    m = 0
    for p in precs:
        m |= 1 << (PRECS[p] if isinstance(p, str) else p)
    return m


class Gauge:
    """Owns an hr_gauge handle built by hr_represent_gauge."""

    def __init__(self, lat: Lattice, U_fund: torch.Tensor, precs=("f64", "f32"),
                 stored: bool = True, rebuild: bool = False, stream=None):
        assert U_fund.is_cuda and U_fund.dtype == torch.complex128
        assert U_fund.numel() == lat.volume * 4 * lat.N * lat.N
        self.lat = lat
        self._desc = lat.desc()
        self.handle = ctypes.c_void_p(0)
        modes = (1 << LINKS_STORED if stored else 0) | (1 << LINKS_REBUILD if rebuild else 0)
        _check(load().hr_represent_gauge(ctypes.byref(self._desc), _ptr(U_fund.contiguous()),
                                         _prec_mask(precs), modes, _stream(stream),
                                         ctypes.byref(self.handle)))

    def update(self, U_fund, stream=None):
        _check(load().hr_gauge_update(self.handle, _ptr(U_fund.contiguous()), _stream(stream)))

    def set_clover(self, U_fund, csw: float, mode: int = CLOVER_PLAIN, stream=None):
        """Adds the clover (or exponential clover) diagonal built from U_fund
        (hr_gauge_set_clover); mode CLOVER_NONE removes it."""
        _check(load().hr_gauge_set_clover(self.handle, _ptr(U_fund.contiguous() if U_fund is not None else None),
                                          float(csw), int(mode), _stream(stream)))

    def set_link_mode(self, mode: int):
        _check(load().hr_gauge_set_link_mode(self.handle, mode))

    def tune(self, prec: int, nrhs: int = 1, stream=None):
        """Times the hopping-kernel variants of every epilogue in precision
        prec and records the fastest (hr_tune)."""
        _check(load().hr_tune(self.handle, prec, nrhs, _stream(stream)))

    def set_tuning(self, autotune: bool = True, variant: int = -1):
        _check(load().hr_gauge_set_tuning(self.handle, int(autotune), variant))

    def hop_variant(self, prec: int, epilogue: int, nrhs: int = 1) -> int:
        return load().hr_gauge_hop_variant(self.handle, prec, epilogue, nrhs)

    def link_mode(self, prec: int) -> int:
        """the link mode (LINKS_STORED or LINKS_REBUILD) launches in prec use now"""
        return load().hr_gauge_link_mode(self.handle, prec)

    def close(self):
        if self.handle and self.handle.value:
            load().hr_gauge_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, parity: int, prec: int, x, out=None, nrhs: int = 1, dagger: bool = False,
              stream=None):
        out_par = EVEN if parity == EO_PRECOND else parity
        if out is None:
            ns = self.lat.nsites(FULL if parity == FULL else EVEN)
            if prec in (F64, F32, DF64):
                out = torch.empty_like(x)
            else:
                out = torch.empty(field_bytes(self.lat, out_par if parity != FULL else FULL, prec, nrhs),
                                  dtype=torch.uint8, device=x.device)
        f = load().hr_dirac_dagger if dagger else load().hr_dirac_apply
        _check(f(self.handle, parity, prec, _ptr(x), _ptr(out), nrhs, _stream(stream)))
        return out

    def cg_solve(self, sys: int, b, x=None, nrhs: int = 1, tol: float = 1e-10,
                 max_iter: int = 10000, inner: int = F64, inner_tol: float = 1e-5,
                 use_initial_guess: bool = False, residual: int = F64, stream=None,
                 check: bool = True):
        if x is None:
            x = torch.zeros_like(b)
        p = CgParams(tol, max_iter, inner, inner_tol, int(use_initial_guess), residual)
        res = (CgResult * nrhs)()
        st = load().hr_cg_solve(self.handle, sys, _ptr(b), _ptr(x), nrhs, ctypes.byref(p), res,
                                _stream(stream))
        if check:
            _check(st)
        out = [dict(iters=r.iters, outer_iters=r.outer_iters, true_rel_residual=r.true_rel_residual,
                    status=STATUS.get(r.status, r.status)) for r in res]
        return x, out, st

    def cg_solve_force(self, sys: int, b, x=None, tol: float = 1e-10, max_iter: int = 10000,
                       inner: int = F64, inner_tol: float = 1e-5, residual: int = F64, coeff: float = 1.0,
                       F=None, want_y: bool = False, stream=None, check: bool = True):
        """x = A^-1 b and F += coeff * force(x, D x) in one call (hr_cg_solve_force)."""
        if x is None:
            x = torch.zeros_like(b)
        if F is None:
            F = torch.zeros((self.lat.volume, 4, self.lat.N ** 2 - 1), dtype=torch.float64,
                            device=b.device)
        Y = torch.empty_like(b) if want_y else None
        p = CgParams(tol, max_iter, inner, inner_tol, 0, residual)
        res = (CgResult * 1)()
        st = load().hr_cg_solve_force(self.handle, sys, _ptr(b), _ptr(x), ctypes.byref(p), res,
                                      _ptr(Y), coeff, _ptr(F), _stream(stream))
        if check:
            _check(st)
        out = [dict(iters=r.iters, outer_iters=r.outer_iters, true_rel_residual=r.true_rel_residual,
                    status=STATUS.get(r.status, r.status)) for r in res]
        return x, F, Y, out, st

    def cg_solve_multishift(self, sys: int, b, shifts, x=None, nrhs: int = 1, tol: float = 1e-10,
                            max_iter: int = 10000, inner: int = F64, inner_tol: float = 1e-5,
                            stream=None, check: bool = True):
        """x[k] = (A + shifts[k])^-1 b for every shift (hr_cg_solve_multishift).
        x has shape (nshift,) + b.shape; the results are [nshift][nrhs]."""
        shifts = [float(s) for s in shifts]
        ns = len(shifts)
        if x is None:
            x = torch.empty((ns,) + tuple(b.shape), dtype=b.dtype, device=b.device)
        p = CgParams(tol, max_iter, inner, inner_tol, 0, F64)
        res = (CgResult * (ns * nrhs))()
        sh = (ctypes.c_double * ns)(*shifts)
        st = load().hr_cg_solve_multishift(self.handle, sys, _ptr(b), _ptr(x), nrhs, sh, ns,
                                           ctypes.byref(p), res, _stream(stream))
        if check:
            _check(st)
        out = [dict(iters=r.iters, outer_iters=r.outer_iters, true_rel_residual=r.true_rel_residual,
                    status=STATUS.get(r.status, r.status)) for r in res]
        return x, [out[k * nrhs:(k + 1) * nrhs] for k in range(ns)], st

    def force(self, sys: int, X, Y, coeff: float = 1.0, F=None, arith: int = F64, stream=None):
        """F += coeff * the fermion force (hr_dirac_force_prec); arith F64 or
        DF64 (float-float on the handle's DF64 links)."""
        if F is None:
            F = torch.zeros((self.lat.volume, 4, self.lat.N ** 2 - 1), dtype=torch.float64,
                            device=X.device)
        _check(load().hr_dirac_force_prec(self.handle, sys, _ptr(X), _ptr(Y), coeff, _ptr(F), arith,
                                          _stream(stream)))
        return F


def cg_solve_batched(gauges, sys: int, bs, xs, nrhs, tol=1e-10, max_iter=10000, inner=F32,
                     inner_tol=1e-5, residual=F64, stream=None, check=True):
    n = len(gauges)
    P = ctypes.c_void_p
    g_arr = (P * n)(*[g.handle.value for g in gauges])
    b_arr = (P * n)(*[b.data_ptr() for b in bs])
    x_arr = (P * n)(*[x.data_ptr() for x in xs])
    n_arr = (ctypes.c_int * n)(*nrhs)
    p = CgParams(tol, max_iter, inner, inner_tol, 0, residual)
    res = (CgResult * sum(nrhs))()
    st = load().hr_cg_solve_batched(n, g_arr, sys, b_arr, x_arr, n_arr, ctypes.byref(p), res,
                                    _stream(stream))
    if check:
        _check(st)
    return [dict(iters=r.iters, outer_iters=r.outer_iters, true_rel_residual=r.true_rel_residual,
                 status=STATUS.get(r.status, r.status)) for r in res], st
