"""Plain FP64 CPU oracle for the HiRep v2 Wilson-Dirac hot path (arXiv 2503.06721).

TEST INFRASTRUCTURE ONLY.  The arithmetic lives in ``hr_oracle.c`` (plain C,
FP64, one loop per definition of the paper); this module only compiles it and
marshals numpy arrays through ctypes.  Only the test suite, the smoke check and
the benchmark's CPU-baseline leg may import it.  It shares no code with the GPU
library and never imports it.

Layouts (numpy complex128 unless stated):
    gauge links U[V, 4, N, N]           lexicographic site, direction mu, row, col
    represented links UR[V, 4, D, D]    same, in representation R (boundary signs applied)
    spinors psi[V, 4, D]                lexicographic site, spin, colour
    half (parity) fields [V/2, 4, D]    index lex // 2 inside the parity
    force F[V, 4, N*N-1]                float64 Lie-algebra components

Every function below has a "pinned" status recorded in the tests: see
``tests/test_oracle_*.py`` for the closed forms, invariants and brute-force
checks that each one is held against.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "hr_oracle.c"
_HDR = _HERE / "hr_oracle.h"
_LIBDIR = _HERE / "_build"
_LIB = _LIBDIR / "liboracle.so"

FUND, ADJ, SYM, ASYM, ASYM_REAL = 0, 1, 2, 3, 4
REP_NAMES = {"FUND": FUND, "ADJ": ADJ, "SYM": SYM, "ASYM": ASYM, "2AS": ASYM, "ASYM_REAL": ASYM_REAL,
             "2AS_REAL": ASYM_REAL}


def build(force: bool = False) -> Path:
    """Compile hr_oracle.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    _LIBDIR.mkdir(exist_ok=True)
    stamp = max(_SRC.stat().st_mtime, _HDR.stat().st_mtime)
    if force or not _LIB.exists() or _LIB.stat().st_mtime < stamp:
        tmp = _LIBDIR / f"liboracle.{os.getpid()}.so"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
               "-o", str(tmp), str(_SRC), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Lat(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("rep", ctypes.c_int),
                ("dims", ctypes.c_int * 4), ("bc", ctypes.c_int * 4),
                ("m0", ctypes.c_double)]


def lat(N: int, rep, dims, bc=(-1, 1, 1, 1), m0: float = 0.0) -> Lat:
    """Lattice descriptor.  dims = (T, X, Y, Z); bc[mu] = +1 / -1."""
    if isinstance(rep, str):
        rep = REP_NAMES[rep]
    L = Lat()
    L.N, L.rep, L.m0 = int(N), int(rep), float(m0)
    for i in range(4):
        L.dims[i] = int(dims[i])
        L.bc[i] = int(bc[i])
    return L


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(str(build()))
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        LP = ctypes.POINTER(Lat)
        sig = {
            "or_rep_dim": (I, [I, I]),
            "or_gamma": (None, [I, P]),
            "or_generators": (None, [I, P]),
            "or_rep_basis": (I, [I, I, P]),
            "or_represent_link": (I, [I, I, P, P]),
            "or_rep_generators": (None, [I, I, P]),
            "or_represent_field": (None, [LP, P, P]),
            "or_dirac_full": (None, [LP, P, P, P, I]),
            "or_hop_parity": (None, [LP, P, I, P, P, I]),
            "or_dhat": (None, [LP, P, P, P, I]),
            "or_sum_naive": (D, [P, ctypes.c_long]),
            "or_sum_neumaier": (D, [P, ctypes.c_long]),
            "or_sum_neumaier2": (D, [P, ctypes.c_long]),
            "or_sum_double_double": (D, [P, ctypes.c_long]),
            "or_norm2": (D, [P, ctypes.c_long]),
            "or_cg": (I, [LP, P, I, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D)]),
            "or_cg_shifted": (I, [LP, P, I, D, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D)]),
            "or_force": (None, [LP, P, P, P, P]),
            "or_plaquette_action": (D, [LP, P, D]),
            "or_gauge_force": (None, [LP, P, D, P]),
            "or_num_threads": (I, []),
            "or_hop_sites": (None, [LP, P, I, P, P, ctypes.c_long, P, I]),
            "or_hop_local": (None, [LP, P, P, P, P, I]),
            "or_hop_local_rep": (None, [LP, P, P, P, P, I]),
            "or_represent_links": (None, [I, I, ctypes.c_long, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _c(a, dtype=np.complex128):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def rep_dim(N: int, rep) -> int:
    rep = REP_NAMES.get(rep, rep) if isinstance(rep, str) else rep
    return _load().or_rep_dim(N, rep)


def num_threads() -> int:
    return _load().or_num_threads()


def gamma(mu: int) -> np.ndarray:
    g = np.zeros((4, 4), np.complex128)
    _load().or_gamma(mu, _p(g))
    return g


def generators(N: int) -> np.ndarray:
    T = np.zeros((N * N - 1, N, N), np.complex128)
    _load().or_generators(N, _p(T))
    return T


def rep_basis(N: int, rep) -> np.ndarray:
    rep = REP_NAMES.get(rep, rep) if isinstance(rep, str) else rep
    D = rep_dim(N, rep)
    E = np.zeros((max(D, 1), N, N), np.complex128)
    n = _load().or_rep_basis(N, rep, _p(E))
    return E[:n]


def represent_link(N: int, rep, U) -> np.ndarray:
    rep = REP_NAMES.get(rep, rep) if isinstance(rep, str) else rep
    D = rep_dim(N, rep)
    U = _c(U)
    R = np.zeros((D, D), np.complex128)
    _load().or_represent_link(N, rep, _p(U), _p(R))
    return R


def rep_generators(N: int, rep) -> np.ndarray:
    rep = REP_NAMES.get(rep, rep) if isinstance(rep, str) else rep
    D = rep_dim(N, rep)
    TR = np.zeros((N * N - 1, D, D), np.complex128)
    _load().or_rep_generators(N, rep, _p(TR))
    return TR


def volume(L: Lat) -> int:
    return L.dims[0] * L.dims[1] * L.dims[2] * L.dims[3]


def represent_field(L: Lat, UF) -> np.ndarray:
    D = rep_dim(L.N, L.rep)
    UF = _c(UF)
    assert UF.size == volume(L) * 4 * L.N * L.N
    UR = np.zeros((volume(L), 4, D, D), np.complex128)
    _load().or_represent_field(ctypes.byref(L), _p(UF), _p(UR))
    return UR


def dirac_full(L: Lat, UR, psi, dagger: bool = False) -> np.ndarray:
    UR, psi = _c(UR), _c(psi)
    out = np.zeros_like(psi)
    _load().or_dirac_full(ctypes.byref(L), _p(UR), _p(psi), _p(out), int(dagger))
    return out


def hop_parity(L: Lat, UR, out_parity: int, in_half, dagger: bool = False) -> np.ndarray:
    """D_{p,1-p} in_half: the hopping block of D_m from parity 1-p to parity p."""
    UR, in_half = _c(UR), _c(in_half)
    out = np.zeros_like(in_half)
    _load().or_hop_parity(ctypes.byref(L), _p(UR), int(out_parity), _p(in_half), _p(out),
                          int(dagger))
    return out


def dhat(L: Lat, UR, in_e, dagger: bool = False) -> np.ndarray:
    UR, in_e = _c(UR), _c(in_e)
    out = np.zeros_like(in_e)
    _load().or_dhat(ctypes.byref(L), _p(UR), _p(in_e), _p(out), int(dagger))
    return out


def hop_sites(L: Lat, UF, out_parity: int, in_half, sites, dagger: bool = False) -> np.ndarray:
    """(D_{p,1-p} in_half) at the given half-index sites of parity p, links represented
    on the fly from the fundamental field UF."""
    UF, in_half = _c(UF), _c(in_half)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    D = rep_dim(L.N, L.rep)
    out = np.zeros((len(sites), 4, D), np.complex128)
    _load().or_hop_sites(ctypes.byref(L), _p(UF), int(out_parity), _p(in_half), _p(sites),
                         len(sites), _p(out), int(dagger))
    return out


def hop_local(L: Lat, coords, Ulinks, psi, dagger: bool = False, represented: bool = False) -> np.ndarray:
    """Hopping term at output sites from gathered data: coords[n, 4] (t,x,y,z),
    Ulinks[n, 8, N, N] fundamental links U(x,mu) / U(x-mu,mu) (represented =
    True: Ulinks[n, 8, D, D] = R of those links, without boundary signs),
    psi[n, 8, 4, D] neighbour spinors.  Returns [n, 4, D]."""
    coords = np.ascontiguousarray(coords, dtype=np.int32)
    Ulinks, psi = _c(Ulinks), _c(psi)
    D = rep_dim(L.N, L.rep)
    n = coords.shape[0]
    out = np.zeros((n, 4, D), np.complex128)
    f = _load().or_hop_local_rep if represented else _load().or_hop_local
    for k in range(n):
        f(ctypes.byref(L), coords[k].ctypes.data_as(ctypes.c_void_p), _p(Ulinks[k]), _p(psi[k]),
          out[k].ctypes.data_as(ctypes.c_void_p), int(dagger))
    return out


def represent_links(N: int, rep, U) -> np.ndarray:
    """R(U[k]) for a stack of N x N matrices U[..., N, N] (no boundary signs)."""
    rep = REP_NAMES.get(rep, rep) if isinstance(rep, str) else rep
    D = rep_dim(N, rep)
    U = _c(U)
    lead = U.shape[:-2]
    n = int(np.prod(lead)) if lead else 1
    R = np.zeros(lead + (D, D), np.complex128)
    _load().or_represent_links(N, rep, n, _p(U), _p(R))
    return R


def _sum(name, a) -> float:
    a = _c(a, np.float64)
    return getattr(_load(), name)(_p(a), a.size)


def sum_naive(a):
    return _sum("or_sum_naive", a)


def sum_neumaier(a):
    return _sum("or_sum_neumaier", a)


def sum_neumaier2(a):
    return _sum("or_sum_neumaier2", a)


def sum_double_double(a):
    return _sum("or_sum_double_double", a)


def norm2(a) -> float:
    a = _c(a)
    return _load().or_norm2(_p(a), a.size)


def cg(L: Lat, UR, sys: int, b, x0=None, tol: float = 1e-10, max_iter: int = 10000,
       sigma: float = 0.0):
    """CG on (A + sigma) x = b with A = D^dag D (sys 0, full fields) or Dhat^dag Dhat
    (sys 1, even half fields).  Returns (x, converged, iterations, true relative
    residual)."""
    UR, b = _c(UR), _c(b)
    x = np.zeros_like(b) if x0 is None else _c(x0).copy()
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    rc = _load().or_cg_shifted(ctypes.byref(L), _p(UR), int(sys), float(sigma), _p(b), _p(x),
                               float(tol), int(max_iter), ctypes.byref(it), ctypes.byref(rr))
    return x, rc == 0, it.value, rr.value


def cg_multishift(L: Lat, UR, sys: int, b, shifts, tol: float = 1e-10, max_iter: int = 10000):
    """The multi-shift inversion of the RHMC (Sec. 4.3.2) by its definition: one
    shifted CG solve (A + sigma_k) x_k = b per shift.  Returns (x[nshift, ...],
    converged[nshift], iterations[nshift], true relative residuals[nshift])."""
    out = [cg(L, UR, sys, b, tol=tol, max_iter=max_iter, sigma=s) for s in shifts]
    return (np.stack([o[0] for o in out]), [o[1] for o in out], [o[2] for o in out],
            [o[3] for o in out])


def force(L: Lat, UR, X, Y) -> np.ndarray:
    """d/de of S = -2 Re <Y, D_m X> along exp(i e T^a) U_F(x, mu); F[V, 4, N*N-1]."""
    UR, X, Y = _c(UR), _c(X), _c(Y)
    F = np.zeros((volume(L), 4, L.N * L.N - 1), np.float64)
    _load().or_force(ctypes.byref(L), _p(UR), _p(X), _p(Y), _p(F))
    return F


# ---- HMC building blocks (Sec. 2.4, Sec. 2.5, Sec. 4.2) ----

T_FUND = 0.5   # Tr T^a T^b = T_F delta^ab for the fundamental generators


def plaquette_action(L: Lat, UF, beta: float) -> float:
    """S_g = beta sum_{x, mu<nu} (1 - Re tr P_mu_nu(x) / N) (Eq. plaquette)."""
    UF = _c(UF)
    return _load().or_plaquette_action(ctypes.byref(L), _p(UF), float(beta))


def gauge_force(L: Lat, UF, beta: float) -> np.ndarray:
    """d/de S_g along exp(i e T^a) U_mu(x); F[V, 4, N*N-1]."""
    UF = _c(UF)
    F = np.zeros((volume(L), 4, L.N * L.N - 1), np.float64)
    _load().or_gauge_force(ctypes.byref(L), _p(UF), float(beta), _p(F))
    return F


def su_algebra(N: int, pi) -> np.ndarray:
    """sum_a pi^a T^a for pi[..., N*N-1] (Hermitian N x N matrices)."""
    T = generators(N)
    return np.einsum("...a,aij->...ij", np.asarray(pi, np.float64), T)


def link_update(L: Lat, UF, pi, eps: float) -> np.ndarray:
    """U_mu(x) <- exp(i eps pi^a T^a) U_mu(x) (dU/dtau = pi U, Sec. 2.5), the
    exponential of the Hermitian eps pi^a T^a by its eigendecomposition."""
    H = eps * su_algebra(L.N, pi)
    w, Q = np.linalg.eigh(H)
    E = np.einsum("...ij,...j,...kj->...ik", Q, np.exp(1j * w), Q.conj())
    return np.einsum("...ij,...jk->...ik", E, _c(UF))


def kinetic_energy(pi) -> float:
    """H_pi = T_F/2 sum_{x,mu,a} pi^a(x,mu)^2 (Sec. 2.5)."""
    p = np.ascontiguousarray(pi, np.float64).ravel()
    return 0.5 * T_FUND * sum_neumaier(p * p)


def fermion_action_eo(L: Lat, UR, phi_e, tol: float = 1e-14) -> float:
    """S_f = phi^dag (Dhat^dag Dhat)^-1 phi for an even-site pseudofermion
    (two flavours, even/odd preconditioned: det Q^2 = det Dhat^dag Dhat up to a
    constant, Sec. 4.3.3)."""
    x, ok, it, rr = cg(L, UR, 1, phi_e, tol=tol, max_iter=100000)
    if not ok:
        raise RuntimeError("oracle CG did not converge")
    return float(np.real(np.vdot(phi_e.ravel(), x.ravel())))


def fermion_force_eo(L: Lat, UR, phi_e, tol: float = 1e-14) -> np.ndarray:
    """d/de S_f along exp(i e T^a) U_mu(x) for S_f = phi^dag (Dhat^dag Dhat)^-1 phi:
    with x = (Dhat^dag Dhat)^-1 phi and y = Dhat x, dS_f = -2 Re <y, dDhat x>, and
    -2 Re <y, Dhat x> is minus the full-operator form -2 Re <Y', D X'> on
    X' = (x, D_oe x), Y' = (y, (D^dag)_oe y) (the diagonal terms do not depend on U)."""
    x, ok, it, rr = cg(L, UR, 1, phi_e, tol=tol, max_iter=100000)
    if not ok:
        raise RuntimeError("oracle CG did not converge")
    y = dhat(L, UR, x)
    Xp = merge(L, x, hop_parity(L, UR, 1, x))
    Yp = merge(L, y, hop_parity(L, UR, 1, y, dagger=True))
    return -force(L, UR, Xp, Yp)


def hamiltonian(L: Lat, UF, pi, beta: float, phi_e=None, tol: float = 1e-14):
    """(H_pi, S_g, S_f) of Sec. 2.5 (S_f = 0 without a pseudofermion)."""
    Sf = 0.0
    if phi_e is not None:
        Sf = fermion_action_eo(L, represent_field(L, UF), phi_e, tol)
    return kinetic_energy(pi), plaquette_action(L, UF, beta), Sf


# second-order minimum-norm (Omelyan) integrator parameter lambda
OMELYAN_LAMBDA = 0.1931833275037836


def md_trajectory(L: Lat, UF, pi, beta: float, tau: float, nsteps: int, phi_e=None,
                  integrator: str = "omelyan", tol: float = 1e-14):
    """Molecular dynamics (Sec. 2.5, Sec. 4.2): Hamilton's equations dU/dtau = pi U,
    dpi/dtau = F with F^a = -(1/T_F) dS/de^a, integrated over tau in nsteps steps
    by leapfrog (PQP) or the 2nd-order Omelyan scheme (PQPQP,
    P(l h) Q(h/2) P((1-2l) h) Q(h/2) P(l h)).  Returns the new (U, pi)."""
    U = np.array(UF, np.complex128, copy=True)
    p = np.array(pi, np.float64, copy=True)
    h = tau / nsteps

    def P(eps):
        F = gauge_force(L, U, beta)
        if phi_e is not None:
            F = F + fermion_force_eo(L, represent_field(L, U), phi_e, tol)
        p[...] = p - (eps / T_FUND) * F

    def Q(eps):
        U[...] = link_update(L, U, p, eps)

    for _ in range(nsteps):
        if integrator == "leapfrog":
            P(h / 2); Q(h); P(h / 2)
        elif integrator == "omelyan":
            lam = OMELYAN_LAMBDA
            P(lam * h); Q(h / 2); P((1 - 2 * lam) * h); Q(h / 2); P(lam * h)
        else:
            raise ValueError(integrator)
    return U, p


# ---- clover improvement (Sec. 5.1.2, Eqs. clover-term, field-strength-tensor) ----

def _neighbours(L: Lat):
    """nb[s, x, mu] = lex index of x + s mu (s = 0: +mu, s = 1: -mu), periodic."""
    dims = [L.dims[i] for i in range(4)]
    t, x, y, z = np.meshgrid(*[np.arange(d) for d in dims], indexing="ij")
    c = np.stack([t, x, y, z], axis=-1).reshape(-1, 4)
    stride = np.array([dims[1] * dims[2] * dims[3], dims[2] * dims[3], dims[3], 1])
    nb = np.empty((2, len(c), 4), np.int64)
    for mu in range(4):
        for s, d in ((0, 1), (1, -1)):
            e = c.copy()
            e[:, mu] = (e[:, mu] + d) % dims[mu]
            nb[s, :, mu] = e @ stride
    return nb


def sigma(mu: int, nu: int) -> np.ndarray:
    """sigma_mu_nu = (i/2) [gamma_mu, gamma_nu] (Hermitian)."""
    g1, g2 = gamma(mu), gamma(nu)
    return 0.5j * (g1 @ g2 - g2 @ g1)


def clover_leaves(L: Lat, UR) -> np.ndarray:
    """Q[x, mu, nu] = the four plaquettes of the (mu, nu) plane with a corner at
    x (Eq. clover-term), each as the closed loop that starts and ends at x,
    traversed mu before nu; in the representation of UR (whose boundary signs
    cancel around every closed loop)."""
    UR = _c(UR)
    V, D = UR.shape[0], UR.shape[-1]
    nb = _neighbours(L)
    dag = lambda A: np.conj(np.swapaxes(A, -1, -2))
    mm = lambda *Ms: _chain(Ms)
    Q = np.zeros((V, 4, 4, D, D), np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            xp_mu, xp_nu = nb[0, :, mu], nb[0, :, nu]
            xm_mu, xm_nu = nb[1, :, mu], nb[1, :, nu]
            xm_mu_p_nu = nb[0, xm_mu, nu]          # x - mu + nu
            xm_mu_m_nu = nb[1, xm_mu, nu]          # x - mu - nu
            xm_nu_p_mu = nb[0, xm_nu, mu]          # x - nu + mu
            U = lambda x, d: UR[x, d]
            Q[:, mu, nu] = (
                mm(U(np.arange(V), mu), U(xp_mu, nu), dag(U(xp_nu, mu)), dag(U(np.arange(V), nu)))
                + mm(U(np.arange(V), nu), dag(U(xm_mu_p_nu, mu)), dag(U(xm_mu, nu)), U(xm_mu, mu))
                + mm(dag(U(xm_mu, mu)), dag(U(xm_mu_m_nu, nu)), U(xm_mu_m_nu, mu), U(xm_nu, nu))
                + mm(dag(U(xm_nu, nu)), U(xm_nu, mu), U(xm_nu_p_mu, nu), dag(U(np.arange(V), mu))))
    return Q


def _chain(Ms):
    out = Ms[0]
    for M in Ms[1:]:
        out = np.einsum("...ij,...jk->...ik", out, M)
    return out


def field_strength(L: Lat, UR) -> np.ndarray:
    """F_mu_nu(x) = (Q_mu_nu(x) - Q_mu_nu(x)^dag) / 8 (Eq. field-strength-tensor)."""
    Q = clover_leaves(L, UR)
    return (Q - np.conj(np.swapaxes(Q, -1, -2))) / 8.0


def clover_term(L: Lat, UR, csw: float, exponential: bool = False) -> np.ndarray:
    """The site-diagonal block C(x) [V, 4D, 4D] (index spin * D + colour) of
    D_ee + D_oo (Sec. 5.1.2):  (4 + m) + csw (i/4) sum_{mu,nu} sigma_mu_nu F_mu_nu,
    or its exponential form (4 + m) exp(csw / (4 + m) (i/4) sum sigma F)."""
    F = field_strength(L, UR)
    V, D = F.shape[0], F.shape[-1]
    X = np.zeros((V, 4 * D, 4 * D), np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu != nu:
                X += 0.25j * np.einsum("st,xab->xsatb", sigma(mu, nu), F[:, mu, nu]).reshape(V, 4 * D, 4 * D)
    m4 = 4.0 + L.m0
    I = np.eye(4 * D)
    if not exponential:
        return m4 * I + csw * X
    w, Qe = np.linalg.eigh(csw / m4 * X)
    return m4 * np.einsum("xij,xj,xkj->xik", Qe, np.exp(w), Qe.conj())


def _site_mv(C, psi):
    V = C.shape[0]
    return np.einsum("xij,xj->xi", C, psi.reshape(V, -1)).reshape(psi.shape)


def dirac_full_clover(L: Lat, UR, C, psi, dagger: bool = False) -> np.ndarray:
    """D_m with the clover diagonal: C(x) psi(x) + the hopping terms of Eq. D_m^R
    (C is Hermitian, so D^dag keeps C)."""
    psi = _c(psi)
    return dirac_full(L, UR, psi, dagger) - (4.0 + L.m0) * psi + _site_mv(C, psi)


def dhat_clover(L: Lat, UR, C, in_e, dagger: bool = False) -> np.ndarray:
    """Dhat = C_ee - D_eo C_oo^-1 D_oe on even half fields (Sec. 4.3.3 with a
    site-dependent diagonal); Dhat^dag = C_ee - (D^dag)_eo C_oo^-1 (D^dag)_oe."""
    e_sites, o_sites = _parity_sites(L)
    Ce, Co = C[e_sites], C[o_sites]
    t = hop_parity(L, UR, 1, _c(in_e), dagger)
    t = np.linalg.solve(Co, t.reshape(len(o_sites), -1)[..., None])[..., 0].reshape(t.shape)
    return _site_mv(Ce, _c(in_e)) - hop_parity(L, UR, 0, t, dagger)


def _parity_sites(L: Lat):
    """lex indices of the even and the odd sites, in half-index (lex // 2) order."""
    par = parity_of_sites(L)
    lex = np.arange(volume(L))
    return lex[par == 0], lex[par == 1]


def cg_apply(apply_A, b, tol: float = 1e-12, max_iter: int = 10000):
    """Textbook CG on a Hermitian positive definite operator given as a
    function, restarted from the true residual until |b - A x| / |b| <= tol.
    Returns (x, converged, iterations, true relative residual)."""
    b = _c(b)
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    k = 0
    while True:
        r = b - apply_A(x)
        rel = np.linalg.norm(r) / bn
        if rel <= tol or k >= max_iter:
            return x, rel <= tol, k, rel
        p = r.copy()
        rr = np.vdot(r, r).real
        while k < max_iter:
            Ap = apply_A(p)
            alpha = rr / np.vdot(p, Ap).real
            x = x + alpha * p
            r = r - alpha * Ap
            k += 1
            rr_new = np.vdot(r, r).real
            if np.sqrt(rr_new) / bn <= tol:
                break
            p = r + (rr_new / rr) * p
            rr = rr_new


# ---- parity helpers (pure index bookkeeping) ----

def parity_of_sites(L: Lat) -> np.ndarray:
    T, X, Y, Z = (L.dims[i] for i in range(4))
    t, x, y, z = np.meshgrid(np.arange(T), np.arange(X), np.arange(Y), np.arange(Z),
                             indexing="ij")
    return ((t + x + y + z) & 1).reshape(-1)


def split(L: Lat, full):
    """Full lexicographic field -> (even half, odd half), half index lex // 2."""
    par = parity_of_sites(L)
    lex = np.arange(volume(L))
    full = np.asarray(full)
    e = np.zeros((volume(L) // 2,) + full.shape[1:], full.dtype)
    o = np.zeros_like(e)
    e[lex[par == 0] // 2] = full[par == 0]
    o[lex[par == 1] // 2] = full[par == 1]
    return e, o


def merge(L: Lat, even, odd):
    par = parity_of_sites(L)
    lex = np.arange(volume(L))
    even = np.asarray(even)
    full = np.zeros((volume(L),) + even.shape[1:], even.dtype)
    full[par == 0] = even[lex[par == 0] // 2]
    full[par == 1] = np.asarray(odd)[lex[par == 1] // 2]
    return full
