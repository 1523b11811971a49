"""Pins for the oracle's fermion force (Sec. 2.5) and compensated sums
(Sec. 4.1.1).

Force: the analytic Lie derivative is compared with central finite
differences of S_f = phi^dag (D^dag D)^{-1} phi, each S_f evaluated with the
oracle's CG to 1e-14, along random su(N) directions.  Sums: against exact
rational arithmetic (fractions.Fraction)."""
from fractions import Fraction

import numpy as np
import pytest
from scipy.linalg import expm

from tests import _helpers as H


def _action(oracle_mod, L, UF, phi):
    UR = oracle_mod.represent_field(L, UF)
    x, ok, it, res = oracle_mod.cg(L, UR, 0, phi, tol=1e-14, max_iter=20000)
    assert ok
    return float(np.vdot(phi.ravel(), x.ravel()).real), x, UR


@pytest.mark.parametrize("N,rep,dims", [(3, "SYM", (4, 2, 2, 4)), (2, "ADJ", (4, 4, 2, 2)),
                                        (4, "ASYM", (2, 2, 2, 4)), (3, "FUND", (4, 2, 2, 2))])
def test_force_vs_finite_differences(oracle_mod, N, rep, dims):
    V = int(np.prod(dims))
    m0 = 0.1
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), m0)
    D = oracle_mod.rep_dim(N, rep)
    UF = H.links(dims, N, 0.4, seed=51)
    phi = H.spinor(V, D, 53)
    S0, X, UR = _action(oracle_mod, L, UF, phi)
    Y = oracle_mod.dirac_full(L, UR, X)
    F = oracle_mod.force(L, UR, X, Y)
    T = oracle_mod.generators(N)
    eps = 1e-5
    for k in range(2):
        omega = H.hermitian(V * 4, N, seed=60 + k).reshape(V, 4, N, N)
        # components omega^a = 2 Tr(T^a omega)
        wa = 2 * np.einsum("aij,xmji->xma", T, omega).real
        dS = float(np.sum(F * wa))
        Up = np.einsum("xmij,xmjk->xmik", np.stack([expm(1j * eps * o) for o in omega.reshape(-1, N, N)]).reshape(omega.shape), UF)
        Um = np.einsum("xmij,xmjk->xmik", np.stack([expm(-1j * eps * o) for o in omega.reshape(-1, N, N)]).reshape(omega.shape), UF)
        Sp = _action(oracle_mod, L, Up, phi)[0]
        Sm = _action(oracle_mod, L, Um, phi)[0]
        fd = (Sp - Sm) / (2 * eps)
        assert abs(fd - dS) <= 1e-7 * abs(fd), (fd, dS)


def test_force_single_link_component(oracle_mod):
    """One link, one generator: dS/de along exp(i e T^a) U(x,mu) only."""
    N, rep, dims = 3, "SYM", (2, 2, 2, 4)
    V = int(np.prod(dims))
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), 0.2)
    D = oracle_mod.rep_dim(N, rep)
    UF = H.links(dims, N, 0.5, seed=71)
    phi = H.spinor(V, D, 73)
    S0, X, UR = _action(oracle_mod, L, UF, phi)
    F = oracle_mod.force(L, UR, X, oracle_mod.dirac_full(L, UR, X))
    T = oracle_mod.generators(N)
    eps = 1e-5
    for (x, mu, a) in [(0, 0, 0), (5, 3, 7), (31, 0, 4)]:   # (31, 0) crosses t = T-1 -> 0
        Up, Um = UF.copy(), UF.copy()
        Up[x, mu] = expm(1j * eps * T[a]) @ UF[x, mu]
        Um[x, mu] = expm(-1j * eps * T[a]) @ UF[x, mu]
        fd = (_action(oracle_mod, L, Up, phi)[0] - _action(oracle_mod, L, Um, phi)[0]) / (2 * eps)
        assert abs(fd - F[x, mu, a]) <= 1e-7 * max(abs(fd), 1e-3), (x, mu, a, fd, F[x, mu, a])


def _exact(a):
    return sum((Fraction(float(v)) for v in a), Fraction(0))


def test_fast_two_sum_exact(oracle_mod):
    import ctypes
    lib = oracle_mod._load()
    f = lib.or_fast_two_sum
    f.restype = None
    f.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                  ctypes.POINTER(ctypes.c_double)]
    rng = np.random.default_rng(1)
    s, c = ctypes.c_double(), ctypes.c_double()
    for _ in range(200):
        a, b = rng.normal() * 10.0 ** rng.integers(-20, 20), rng.normal() * 10.0 ** rng.integers(-20, 20)
        f(a, b, ctypes.byref(s), ctypes.byref(c))
        assert Fraction(s.value) + Fraction(c.value) == Fraction(a) + Fraction(b)


def test_compensated_sums_adversarial(oracle_mod):
    eps = 2.0 ** -53
    # classic cancellation: naive loses the small terms entirely
    a = np.array([1e16, 1.0, -1e16, 1.0] * 50)
    assert oracle_mod.sum_naive(a) != 100.0
    for f in (oracle_mod.sum_neumaier, oracle_mod.sum_neumaier2, oracle_mod.sum_double_double):
        assert f(a) == 100.0
    rng = np.random.default_rng(7)
    for trial in range(5):
        n = 5000
        big = rng.normal(size=n) * 10.0 ** rng.integers(0, 12, size=n)
        a = np.concatenate([big, -big[::-1] * (1 + 1e-13), rng.normal(size=n)])
        rng.shuffle(a)
        ex = float(_exact(a))
        sabs = float(np.abs(a).sum())
        nv = oracle_mod.sum_naive(a)
        nm = oracle_mod.sum_neumaier(a)
        n2 = oracle_mod.sum_neumaier2(a)
        dd = oracle_mod.sum_double_double(a)
        m = len(a)
        # Neumaier: |err| <= 2 eps |S| + O(n eps^2) sum|a|  (Neumaier 1974)
        assert abs(nm - ex) <= 2 * eps * abs(ex) + 4 * m * eps * eps * sabs
        assert abs(n2 - ex) <= 2 * eps * abs(ex) + 4 * m * eps * eps * sabs
        assert abs(dd - ex) <= 2 * eps * abs(ex) + 4 * m * eps * eps * sabs
        # and they beat the naive sum whenever the naive one is off
        assert abs(nm - ex) <= abs(nv - ex) + eps * abs(ex)


def test_norm_dot(oracle_mod):
    rng = np.random.default_rng(3)
    u = rng.normal(size=64) + 1j * rng.normal(size=64)
    ex = _exact(np.concatenate([u.real * u.real, u.imag * u.imag]))
    assert abs(oracle_mod.norm2(u) - float(ex)) <= 1e-15 * float(ex)
