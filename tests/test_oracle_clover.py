"""Pins of the oracle's clover term (Sec. 5.1.2, Eqs. clover-term and
field-strength-tensor, plain and exponential): the field strength vanishes
on unit links and is gauge covariant; the clover block is Hermitian and
commutes with gamma5; its spectrum on an abelian constant field is known in
closed form; and on a 2^4 lattice the dense operator with the clover diagonal
keeps gamma5-hermiticity, det D = det C_oo det Dhat (Schur complement), the
even/odd Schur solve equals the LU solve, and CG on Dhat^dag Dhat equals LU."""
import numpy as np
import pytest

from tests import _helpers as H


def test_unit_links_give_mass_term(oracle_mod):
    N, rep, dims = 3, "SYM", (2, 2, 2, 4)
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), -0.2)
    V, D = 32, 6
    UR = oracle_mod.represent_field(L, H.unit_links(dims, N))
    F = oracle_mod.field_strength(L, UR)
    assert np.abs(F).max() < 1e-15
    C = oracle_mod.clover_term(L, UR, 1.7)
    np.testing.assert_allclose(C, np.broadcast_to(3.8 * np.eye(4 * D), C.shape), atol=1e-14)


@pytest.mark.parametrize("N,rep", [(2, "ADJ"), (3, "SYM"), (3, "FUND")])
def test_covariance_hermiticity_chirality(oracle_mod, N, rep):
    dims = (4, 2, 2, 4)
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), -0.1)
    V = int(np.prod(dims))
    D = oracle_mod.rep_dim(N, rep)
    U = H.links(dims, N, 0.8, seed=173)
    g = H.su_n(V, N, 179, eps=1.3)
    c = H.coords(dims)
    stride = np.array([dims[1] * dims[2] * dims[3], dims[2] * dims[3], dims[3], 1])
    Ug = np.empty_like(U)
    for mu in range(4):
        cn = c.copy()
        cn[:, mu] = (cn[:, mu] + 1) % dims[mu]
        Ug[:, mu] = np.einsum("xij,xjk,xlk->xil", g, U[:, mu], g[cn @ stride].conj())
    UR = oracle_mod.represent_field(L, U)
    F = oracle_mod.field_strength(L, UR)
    Fg = oracle_mod.field_strength(L, oracle_mod.represent_field(L, Ug))
    Rg = np.stack([oracle_mod.represent_link(N, rep, g[x]) for x in range(V)])
    np.testing.assert_allclose(Fg, np.einsum("xab,xmnbc,xdc->xmnad", Rg, F, Rg.conj()), atol=1e-13)
    # anti-Hermitian, antisymmetric in (mu, nu)
    np.testing.assert_allclose(F, -np.conj(np.swapaxes(F, -1, -2)), atol=1e-15)
    np.testing.assert_allclose(F, -np.swapaxes(F, 1, 2), atol=1e-15)
    for expo in (False, True):
        C = oracle_mod.clover_term(L, UR, 1.3, exponential=expo)
        np.testing.assert_allclose(C, np.conj(np.swapaxes(C, -1, -2)), atol=1e-13)
        G5 = np.kron(np.diag([1.0, 1, -1, -1]), np.eye(D))
        np.testing.assert_allclose(G5 @ C @ G5, C, atol=1e-13)


@pytest.mark.parametrize("rep", ["FUND", "ADJ", "SYM"])
def test_abelian_constant_field_spectrum(oracle_mod, rep):
    """U_0(x) = diag(e^{i th x1}, e^{-i th x1}), other links 1: every leaf of the
    (0,1) plane is P = diag(e^{-i th}, e^{i th}); with R(P) eigenvalues e^{i phi_k},
    F_01 has eigenvalues i sin phi_k, and the clover block
    (4+m) + c (i/4) 2 sigma_01 F_01 has eigenvalues (4+m) -/+ (c/2) sin phi_k,
    each twice (sigma_01 = +-1); the exponential form (4+m) exp(-/+ c sin phi_k / (2 (4+m)))."""
    N = 2
    dims = (2, 6, 2, 2)
    m0, csw = 0.2, 1.9
    L = oracle_mod.lat(N, rep, dims, (1, 1, 1, 1), m0)
    V = int(np.prod(dims))
    th = 2 * np.pi / dims[1]
    U = np.tile(np.eye(N, dtype=np.complex128), (V, 4, 1, 1))
    x1 = H.coords(dims)[:, 1]
    U[:, 0, 0, 0] = np.exp(1j * th * x1)
    U[:, 0, 1, 1] = np.exp(-1j * th * x1)
    UR = oracle_mod.represent_field(L, U)
    P = np.diag([np.exp(-1j * th), np.exp(1j * th)])
    phi = np.angle(np.linalg.eigvals(oracle_mod.represent_link(N, rep, P)))
    m4 = 4 + m0
    for expo in (False, True):
        C = oracle_mod.clover_term(L, UR, csw, exponential=expo)
        s = np.concatenate([np.sin(phi), -np.sin(phi)] * 2) * csw / 2
        want = np.sort(m4 * np.exp(s / m4) if expo else m4 + s)
        for x in (0, 7, V - 1):
            np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(C[x])), want, atol=1e-13)


def _dense(f, n, shape):
    M = np.zeros((n, n), np.complex128)
    e = np.zeros(n, np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        M[:, j] = f(e.reshape(shape)).ravel()
    return M


@pytest.mark.parametrize("N,rep,expo", [(2, "ADJ", False), (3, "SYM", False), (2, "FUND", True)])
def test_dense_clover_operator_2x2x2x2(oracle_mod, N, rep, expo):
    dims = (2, 2, 2, 2)
    V = 16
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), -0.3)
    D = oracle_mod.rep_dim(N, rep)
    UR = oracle_mod.represent_field(L, H.links(dims, N, 1.0, seed=181))
    C = oracle_mod.clover_term(L, UR, 1.5, exponential=expo)
    n = V * 4 * D
    M = _dense(lambda v: oracle_mod.dirac_full_clover(L, UR, C, v), n, (V, 4, D))
    Md = _dense(lambda v: oracle_mod.dirac_full_clover(L, UR, C, v, dagger=True), n, (V, 4, D))
    np.testing.assert_allclose(Md, M.conj().T, atol=1e-13)
    G5 = np.kron(np.eye(V), np.kron(np.diag([1.0, 1, -1, -1]), np.eye(D)))
    np.testing.assert_allclose(G5 @ M @ G5, Md, atol=1e-13)
    # c_sw = 0 is the plain operator
    C0 = oracle_mod.clover_term(L, UR, 0.0)
    psi = H.spinor(V, D, 191)
    np.testing.assert_allclose(oracle_mod.dirac_full_clover(L, UR, C0, psi), oracle_mod.dirac_full(L, UR, psi),
                               atol=1e-14)
    # parity blocks, Schur complement and determinant identity
    e_s, o_s = oracle_mod._parity_sites(L)
    idx = lambda sites: (sites[:, None] * 4 * D + np.arange(4 * D)[None]).ravel()
    ie, io = idx(e_s), idx(o_s)
    Cee, Ceo, Coe, Coo = M[np.ix_(ie, ie)], M[np.ix_(ie, io)], M[np.ix_(io, ie)], M[np.ix_(io, io)]
    nh = len(ie)
    Bhat = _dense(lambda v: oracle_mod.dhat_clover(L, UR, C, v), nh, (V // 2, 4, D))
    np.testing.assert_allclose(Bhat, Cee - Ceo @ np.linalg.solve(Coo, Coe), atol=1e-12)
    Bhatd = _dense(lambda v: oracle_mod.dhat_clover(L, UR, C, v, dagger=True), nh, (V // 2, 4, D))
    np.testing.assert_allclose(Bhatd, Bhat.conj().T, atol=1e-12)
    s1, l1 = np.linalg.slogdet(M)
    s2, l2 = np.linalg.slogdet(Coo)
    s3, l3 = np.linalg.slogdet(Bhat)
    assert abs(l1 - (l2 + l3)) < 1e-9 and abs(s1 - s2 * s3) < 1e-9
    # Schur solve == LU; CG on Dhat^dag Dhat == LU
    eta = H.spinor(V, D, 193)
    x_lu = np.linalg.solve(M, eta.ravel()).reshape(V, 4, D)
    ee, eo = oracle_mod.split(L, eta)
    t = np.linalg.solve(Coo, eo.ravel()).reshape(eo.shape)
    rhs = ee - oracle_mod.hop_parity(L, UR, 0, t)
    xe = np.linalg.solve(Bhat, rhs.ravel()).reshape(ee.shape)
    xo = np.linalg.solve(Coo, (eo - oracle_mod.hop_parity(L, UR, 1, xe)).ravel()).reshape(eo.shape)
    np.testing.assert_allclose(oracle_mod.merge(L, xe, xo), x_lu, atol=1e-10 * np.abs(x_lu).max())
    A = lambda v: oracle_mod.dhat_clover(L, UR, C, oracle_mod.dhat_clover(L, UR, C, v), dagger=True)
    x_cg, ok, it, rel = oracle_mod.cg_apply(A, ee, tol=1e-13)
    assert ok
    x_ref = np.linalg.solve(Bhat.conj().T @ Bhat, ee.ravel()).reshape(ee.shape)
    np.testing.assert_allclose(x_cg, x_ref, atol=1e-10 * np.abs(x_ref).max())
