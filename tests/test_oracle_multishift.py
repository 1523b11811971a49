"""Pins of the oracle's shifted CG, the definition of the multi-shift inversion
that the RHMC needs (Sec. 4.3.2: (Q^2 + beta_k) x_k = phi for every shift
beta_k).  Each check is independent of the oracle's CG: a dense LU solve on a
2^4 lattice, the free-field closed form, and the Neumann series at a large
shift."""
import numpy as np
import pytest

from tests import _helpers as H


def _dense_full(oracle_mod, L, UR, V, D):
    n = V * 4 * D
    M = np.zeros((n, n), np.complex128)
    e = np.zeros(n, np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        M[:, j] = oracle_mod.dirac_full(L, UR, e.reshape(V, 4, D)).ravel()
    return M


def _dense_dhat(oracle_mod, L, UR, V, D):
    nh = V // 2 * 4 * D
    B = np.zeros((nh, nh), np.complex128)
    e = np.zeros(nh, np.complex128)
    for j in range(nh):
        e[:] = 0
        e[j] = 1
        B[:, j] = oracle_mod.dhat(L, UR, e.reshape(V // 2, 4, D)).ravel()
    return B


@pytest.mark.parametrize("N,rep", [(2, "ADJ"), (3, "SYM"), (4, "ASYM")])
def test_shifted_cg_dense_2x2x2x2(oracle_mod, N, rep):
    dims = (2, 2, 2, 2)
    V = 16
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), -0.3)
    D = oracle_mod.rep_dim(N, rep)
    UR = oracle_mod.represent_field(L, H.links(dims, N, 1.0, seed=37))
    M = _dense_full(oracle_mod, L, UR, V, D)
    B = _dense_dhat(oracle_mod, L, UR, V, D)
    b = H.spinor(V, D, 43)
    be = b[: V // 2]
    shifts = [0.0, 1e-3, 0.37, 6.0]
    xs, ok, its, res = oracle_mod.cg_multishift(L, UR, 0, b, shifts, tol=1e-13, max_iter=5000)
    xe, oke, itse, rese = oracle_mod.cg_multishift(L, UR, 1, be, shifts, tol=1e-13, max_iter=5000)
    for k, s in enumerate(shifts):
        assert ok[k] and res[k] <= 1e-13 and oke[k] and rese[k] <= 1e-13
        A = M.conj().T @ M + s * np.eye(M.shape[0])
        ref = np.linalg.solve(A, b.ravel()).reshape(b.shape)
        np.testing.assert_allclose(xs[k], ref, atol=1e-10 * np.abs(ref).max())
        Ah = B.conj().T @ B + s * np.eye(B.shape[0])
        refe = np.linalg.solve(Ah, be.ravel()).reshape(be.shape)
        np.testing.assert_allclose(xe[k], refe, atol=1e-10 * np.abs(refe).max())
    # a larger shift is a better-conditioned system: never more iterations
    assert all(its[k + 1] <= its[k] for k in range(len(shifts) - 1))


@pytest.mark.parametrize("sigma", [0.0, 0.25, 3.0])
def test_shifted_cg_free_field(oracle_mod, sigma):
    """On a plane wave, (D^dag D + sigma) has the eigenvalue
    (m + sum(1 - cos p))^2 + sum sin^2 p + sigma: one CG step is exact."""
    N, rep = 3, "SYM"
    dims = (6, 4, 4, 4)
    m0 = -0.2
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), m0)
    D = oracle_mod.rep_dim(N, rep)
    UR = oracle_mod.represent_field(L, H.unit_links(dims, N))
    x = H.coords(dims)
    p = np.array([np.pi / 6, 2 * np.pi / 4, 2 * np.pi / 4, 0.0])
    chi = np.arange(1, 4 * D + 1).reshape(4, D) * (0.5 - 1j)
    b = np.exp(1j * x @ p)[:, None, None] * chi[None]
    lam = (m0 + np.sum(1 - np.cos(p))) ** 2 + np.sum(np.sin(p) ** 2) + sigma
    xs, ok, it, res = oracle_mod.cg(L, UR, 0, b, tol=1e-12, sigma=sigma)
    assert ok and it == 1
    np.testing.assert_allclose(xs, b / lam, atol=1e-12 * np.abs(b / lam).max())


def test_shifted_cg_neumann_series(oracle_mod):
    """For sigma >> |A|: (A + sigma)^-1 b = b/sigma - A b/sigma^2 + O(|A|^2 |b| / sigma^3)."""
    N, rep = 2, "ADJ"
    dims = (4, 4, 2, 2)
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), -0.1)
    D = oracle_mod.rep_dim(N, rep)
    UR = oracle_mod.represent_field(L, H.links(dims, N, 0.5, seed=53))
    V = int(np.prod(dims))
    be = H.spinor(V // 2, D, 59)
    Ab = oracle_mod.dhat(L, UR, oracle_mod.dhat(L, UR, be), dagger=True)
    # |Dhat| <= (4+m)^2 + 16, so |A| <= ((4+m)^2 + 16)^2
    a_max = ((4 - 0.1) ** 2 + 16) ** 2
    sigma = 1e3 * a_max
    x, ok, it, res = oracle_mod.cg(L, UR, 1, be, tol=1e-14, sigma=sigma)
    assert ok
    approx = be / sigma - Ab / sigma ** 2
    bound = a_max ** 2 * np.linalg.norm(be) / sigma ** 3 * 1.01 / (1 - a_max / sigma)
    assert np.linalg.norm(x - approx) <= bound + 1e-14 * np.linalg.norm(x)
    # the first-order term is resolved: dropping it is far outside the bound
    assert np.linalg.norm(x - be / sigma) > 100 * bound
