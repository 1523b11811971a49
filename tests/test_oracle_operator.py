"""Pins for the oracle's Wilson-Dirac operator (Eq. D_m^R, Sec. 2.3), its
even/odd blocks (Sec. 4.3.3) and its CG (Sec. 4.1.2).

Pins: the free-field momentum-space closed form, gamma5-hermiticity, gauge
covariance, and a brute-force dense matrix on a 2^4 lattice (where x+mu and
x-mu coincide, which exercises the neighbour wrap)."""
import numpy as np
import pytest

from tests import _helpers as H

CASES = [(2, "ADJ"), (3, "SYM"), (3, "ADJ"), (4, "FUND"), (4, "ASYM"), (3, "FUND"), (5, "FUND"), (8, "FUND"),
         (4, "ASYM_REAL"), (4, "ADJ"), (4, "SYM")]


def _gam(oracle_mod):
    return [oracle_mod.gamma(mu) for mu in range(4)]


@pytest.mark.parametrize("N,rep", CASES)
@pytest.mark.parametrize("bc", [(-1, 1, 1, 1), (1, 1, 1, 1), (-1, -1, 1, 1)])
def test_free_field_plane_wave(oracle_mod, N, rep, bc):
    """U = 1, psi(x) = exp(i p.x) chi with p_mu = (2 n_mu + [bc_mu = -1]) pi / L_mu:
    D psi = [m + sum_mu (1 - cos p_mu) + i sum_mu gamma_mu sin p_mu] psi."""
    dims = (4, 6, 2, 4)
    m0 = -0.37
    L = oracle_mod.lat(N, rep, dims, bc, m0)
    D = oracle_mod.rep_dim(N, rep)
    UR = oracle_mod.represent_field(L, H.unit_links(dims, N))
    x = H.coords(dims)
    g = _gam(oracle_mod)
    rng = np.random.default_rng(5)
    for trial in range(3):
        n = rng.integers(0, 7, size=4)
        p = np.array([(2 * n[mu] + (1 if bc[mu] == -1 else 0)) * np.pi / dims[mu]
                      for mu in range(4)])
        chi = rng.normal(size=(4, D)) + 1j * rng.normal(size=(4, D))
        psi = np.exp(1j * x @ p)[:, None, None] * chi[None]
        Dp = (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(
            g[mu] * np.sin(p[mu]) for mu in range(4))
        Ddp = Dp.conj().T
        want = np.exp(1j * x @ p)[:, None, None] * (Dp @ chi)[None]
        wantd = np.exp(1j * x @ p)[:, None, None] * (Ddp @ chi)[None]
        np.testing.assert_allclose(oracle_mod.dirac_full(L, UR, psi), want, atol=1e-13)
        np.testing.assert_allclose(oracle_mod.dirac_full(L, UR, psi, dagger=True), wantd,
                                   atol=1e-13)


@pytest.mark.parametrize("N,rep", CASES)
def test_gamma5_hermiticity_and_dagger(oracle_mod, N, rep):
    dims = (4, 2, 4, 6)
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), -0.21)
    D = oracle_mod.rep_dim(N, rep)
    V = int(np.prod(dims))
    UR = oracle_mod.represent_field(L, H.links(dims, N, 1.0, seed=3))
    phi, psi = H.spinor(V, D, 7, nrhs=2)
    g5 = np.diag([1.0, 1, -1, -1])
    G5 = lambda f: np.einsum("st,xtc->xsc", g5, f)
    dot = lambda a, b: np.vdot(a.ravel(), b.ravel())
    Dphi = oracle_mod.dirac_full(L, UR, phi)
    lhs = dot(phi, G5(oracle_mod.dirac_full(L, UR, G5(psi))))
    assert abs(lhs - dot(Dphi, psi)) < 1e-12 * abs(lhs)
    lhs = dot(phi, oracle_mod.dirac_full(L, UR, psi))
    rhs = dot(oracle_mod.dirac_full(L, UR, phi, dagger=True), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # block form: gamma5 D_eo gamma5 = (D_oe)^dag
    pe, po = oracle_mod.split(L, phi)
    se, so = oracle_mod.split(L, psi)
    a = dot(pe, G5(oracle_mod.hop_parity(L, UR, 0, G5(so))))
    b = dot(oracle_mod.hop_parity(L, UR, 1, pe), so)
    assert abs(a - b) < 1e-12 * abs(a)


@pytest.mark.parametrize("N,rep", CASES)
def test_gauge_covariance(oracle_mod, N, rep):
    """D[U^g] (g_R psi) = g_R D[U] psi, U^g(x,mu) = g(x) U(x,mu) g(x+mu)^dag."""
    import torch
    from paper_2503_06721_gb300 import synth
    dims = (4, 4, 2, 4)
    V = int(np.prod(dims))
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), 0.13)
    D = oracle_mod.rep_dim(N, rep)
    U = H.links(dims, N, 0.8, seed=17)
    g = synth.haar_su_n(V, N, seed=19)
    Ug = synth.gauge_transform_links(torch.as_tensor(U), g, dims).numpy()
    gR = np.stack([oracle_mod.represent_link(N, rep, gx) for gx in g.numpy()])
    psi = H.spinor(V, D, 29)
    gpsi = np.einsum("xab,xsb->xsa", gR, psi)
    lhs = oracle_mod.dirac_full(L, oracle_mod.represent_field(L, Ug), gpsi)
    rhs = np.einsum("xab,xsb->xsa", gR, oracle_mod.dirac_full(L, oracle_mod.represent_field(L, U),
                                                             psi))
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


def _dense(oracle_mod, L, UR, V, D, dagger=False):
    n = V * 4 * D
    M = np.zeros((n, n), np.complex128)
    e = np.zeros(n, np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        M[:, j] = oracle_mod.dirac_full(L, UR, e.reshape(V, 4, D), dagger).ravel()
    return M


@pytest.mark.parametrize("N,rep", [(2, "ADJ"), (3, "SYM"), (3, "ADJ"), (4, "ASYM"), (5, "FUND"), (8, "FUND"),
                                   (4, "ASYM_REAL")])
def test_dense_2x2x2x2(oracle_mod, N, rep):
    dims = (2, 2, 2, 2)
    V = 16
    m0 = -0.3
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), m0)
    D = oracle_mod.rep_dim(N, rep)
    UR = oracle_mod.represent_field(L, H.links(dims, N, 1.0, seed=31))
    M = _dense(oracle_mod, L, UR, V, D)
    Md = _dense(oracle_mod, L, UR, V, D, dagger=True)
    np.testing.assert_allclose(Md, M.conj().T, atol=1e-14)
    G5 = np.kron(np.eye(V), np.kron(np.diag([1.0, 1, -1, -1]), np.eye(D)))
    Q = G5 @ M
    np.testing.assert_allclose(Q, Q.conj().T, atol=1e-14)
    ev = np.linalg.eigvals(M)
    # every eigenvalue has its complex conjugate in the spectrum (det D real)
    dist = np.abs(ev[:, None] - ev.conj()[None, :]).min(axis=1)
    assert dist.max() < 1e-9
    # parity blocks from the dense matrix
    par = oracle_mod.parity_of_sites(L)
    lex = np.arange(V)
    ev_sites, od_sites = lex[par == 0], lex[par == 1]
    idx = lambda sites: (sites[:, None] * 4 * D + np.arange(4 * D)[None]).ravel()
    ie, io = idx(ev_sites), idx(od_sites)
    Dee, Deo = M[np.ix_(ie, ie)], M[np.ix_(ie, io)]
    Doe, Doo = M[np.ix_(io, ie)], M[np.ix_(io, io)]
    m4 = 4 + m0
    np.testing.assert_allclose(Dee, m4 * np.eye(len(ie)), atol=1e-15)
    np.testing.assert_allclose(Doo, m4 * np.eye(len(io)), atol=1e-15)
    # hop blocks: column j of D_eo from or_hop_parity (half index = lex // 2)
    nh = len(io)
    Beo = np.zeros((nh, nh), np.complex128)
    Boe = np.zeros((nh, nh), np.complex128)
    Bhat = np.zeros((nh, nh), np.complex128)
    Bhatd = np.zeros((nh, nh), np.complex128)
    e = np.zeros(nh, np.complex128)
    for j in range(nh):
        e[:] = 0
        e[j] = 1
        f = e.reshape(V // 2, 4, D)
        Beo[:, j] = oracle_mod.hop_parity(L, UR, 0, f).ravel()
        Boe[:, j] = oracle_mod.hop_parity(L, UR, 1, f).ravel()
        Bhat[:, j] = oracle_mod.dhat(L, UR, f).ravel()
        Bhatd[:, j] = oracle_mod.dhat(L, UR, f, dagger=True).ravel()
    # half fields are ordered by lex // 2, which preserves the lex order of each parity
    np.testing.assert_allclose(Beo, Deo, atol=1e-15)
    np.testing.assert_allclose(Boe, Doe, atol=1e-15)
    np.testing.assert_allclose(Bhat, m4 * m4 * np.eye(nh) - Deo @ Doe, atol=1e-13)
    np.testing.assert_allclose(Bhatd, Bhat.conj().T, atol=1e-13)
    # det D = det D_oo det(D_ee - D_eo D_oo^-1 D_oe) = det Dhat  (n_e = n_o)
    s1, l1 = np.linalg.slogdet(M)
    s2, l2 = np.linalg.slogdet(Bhat)
    assert abs(l1 - l2) < 1e-10 and abs(s1 - s2) < 1e-10
    # Schur solve == LU solve
    eta = H.spinor(V, D, 41)
    x_lu = np.linalg.solve(M, eta.ravel()).reshape(V, 4, D)
    ee, eo = oracle_mod.split(L, eta)
    rhs = m4 * ee - oracle_mod.hop_parity(L, UR, 0, eo)
    xe = np.linalg.solve(Bhat, rhs.ravel()).reshape(ee.shape)
    xo = (eo - oracle_mod.hop_parity(L, UR, 1, xe)) / m4
    np.testing.assert_allclose(oracle_mod.merge(L, xe, xo), x_lu, atol=1e-11)
    # CG on D^dag D and on Dhat^dag Dhat == LU
    b = eta
    x_cg, ok, it, res = oracle_mod.cg(L, UR, 0, b, tol=1e-13, max_iter=5000)
    assert ok and res <= 1e-13
    x_ref = np.linalg.solve(M.conj().T @ M, b.ravel()).reshape(b.shape)
    np.testing.assert_allclose(x_cg, x_ref, atol=1e-10 * np.abs(x_ref).max())
    x_cg, ok, it, res = oracle_mod.cg(L, UR, 1, ee, tol=1e-13, max_iter=5000)
    assert ok and res <= 1e-13
    x_ref = np.linalg.solve(Bhat.conj().T @ Bhat, ee.ravel()).reshape(ee.shape)
    np.testing.assert_allclose(x_cg, x_ref, atol=1e-10 * np.abs(x_ref).max())


@pytest.mark.parametrize("N,rep", [(2, "ADJ"), (3, "SYM")])
def test_cg_free_field_exact(oracle_mod, N, rep):
    """D^dag D (p) = (m + sum(1 - cos p))^2 + sum sin^2 p  on plane waves."""
    dims = (6, 4, 4, 4)
    m0 = -0.2
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), m0)
    D = oracle_mod.rep_dim(N, rep)
    UR = oracle_mod.represent_field(L, H.unit_links(dims, N))
    x = H.coords(dims)
    p = np.array([3 * np.pi / 6, 2 * np.pi / 4, 0.0, 2 * 2 * np.pi / 4])
    chi = np.arange(1, 4 * D + 1).reshape(4, D) * (1 + 0.5j)
    b = np.exp(1j * x @ p)[:, None, None] * chi[None]
    lam = (m0 + np.sum(1 - np.cos(p))) ** 2 + np.sum(np.sin(p) ** 2)
    xs, ok, it, res = oracle_mod.cg(L, UR, 0, b, tol=1e-12)
    assert ok
    np.testing.assert_allclose(xs, b / lam, atol=1e-11 * np.abs(b / lam).max())
    # a single plane wave is one eigenvector: CG converges in one iteration
    assert it == 1


def test_antiperiodic_sign_slice(oracle_mod):
    """The -1 sits on the represented links of the slice t = T-1 only (Sec. 5.3.1)."""
    dims = (4, 2, 2, 2)
    L = oracle_mod.lat(3, "ADJ", dims, (-1, 1, 1, 1), 0.0)
    UR = oracle_mod.represent_field(L, H.unit_links(dims, 3))
    t = H.coords(dims)[:, 0]
    for mu in range(4):
        sign = np.where((t == 3) & (mu == 0), -1.0, 1.0)
        np.testing.assert_allclose(UR[:, mu, 0, 0].real, sign)


@pytest.mark.parametrize("N,rep", [(3, "SYM"), (2, "ADJ"), (4, "ASYM")])
@pytest.mark.parametrize("dagger", [False, True])
def test_hop_sites_matches_full(oracle_mod, N, rep, dagger):
    """The sampled-site evaluator reproduces the whole-lattice hopping block."""
    dims = (4, 2, 4, 6)
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, -1), 0.1)
    D = oracle_mod.rep_dim(N, rep)
    V = int(np.prod(dims))
    UF = H.links(dims, N, 0.7, seed=81)
    UR = oracle_mod.represent_field(L, UF)
    psi = H.spinor(V // 2, D, 83)
    for p in (0, 1):
        full = oracle_mod.hop_parity(L, UR, p, psi, dagger)
        sites = np.arange(V // 2)[::3]
        np.testing.assert_allclose(oracle_mod.hop_sites(L, UF, p, psi, sites, dagger), full[sites],
                                   atol=1e-14)


def test_hop_local_matches_full(oracle_mod):
    """The gathered-data single-site evaluator reproduces the hopping block."""
    dims = (4, 2, 4, 6)
    N, rep = 3, "SYM"
    L = oracle_mod.lat(N, rep, dims, (-1, 1, -1, 1), 0.0)
    D = oracle_mod.rep_dim(N, rep)
    V = int(np.prod(dims))
    UF = H.links(dims, N, 0.7, seed=91)
    UR = oracle_mod.represent_field(L, UF)
    psi = H.spinor(V, D, 93)
    full = oracle_mod.dirac_full(L, UR, psi) - (4 + 0.0) * psi
    xs = np.arange(0, V, 5)
    coords = H.coords(dims)[xs]
    Ul = np.zeros((len(xs), 8, N, N), np.complex128)
    ps = np.zeros((len(xs), 8, 4, D), np.complex128)
    for n, x in enumerate(xs):
        for k in range(8):
            mu = k & 3
            nb = oracle_mod_neighbour(dims, x, mu, +1 if k < 4 else -1)
            Ul[n, k] = UF[x if k < 4 else nb, mu]
            ps[n, k] = psi[nb]
    np.testing.assert_allclose(oracle_mod.hop_local(L, coords, Ul, ps), full[xs], atol=1e-14)
    # the represented-link form, given R of the same links, is the same hopping term
    Rl = oracle_mod.represent_links(N, rep, Ul)
    np.testing.assert_allclose(oracle_mod.hop_local(L, coords, Rl, ps, represented=True), full[xs],
                               atol=1e-14)
    np.testing.assert_allclose(oracle_mod.hop_local(L, coords, Rl, ps, dagger=True, represented=True),
                               (oracle_mod.dirac_full(L, UR, psi, True) - 4.0 * psi)[xs], atol=1e-14)


def oracle_mod_neighbour(dims, lex, mu, d):
    c = list(np.unravel_index(lex, dims))
    c[mu] = (c[mu] + d) % dims[mu]
    return int(np.ravel_multi_index(c, dims))


def test_asym_real_operator_and_force_equivalence(oracle_mod):
    """The Wilson-Dirac operator with SU(4) 2AS links in the real basis is the
    2AS operator in rotated colour coordinates: D_real (W^dag psi) =
    W^dag (D_2AS psi), W the fixed basis change; the force, a function of
    basis-independent bilinears, is the same for X, Y and W^dag X, W^dag Y."""
    dims = (4, 2, 2, 4)
    L = oracle_mod.lat(4, "ASYM", dims, (-1, 1, 1, 1), -0.1)
    Lr = oracle_mod.lat(4, "ASYM_REAL", dims, (-1, 1, 1, 1), -0.1)
    W = np.einsum("mij,nij->mn", oracle_mod.rep_basis(4, "ASYM").conj(), oracle_mod.rep_basis(4, "ASYM_REAL"))
    V = int(np.prod(dims))
    UF = H.links(dims, 4, 0.6, seed=301)
    UR = oracle_mod.represent_field(L, UF)
    URr = oracle_mod.represent_field(Lr, UF)
    assert np.abs(URr.imag).max() < 1e-14
    psi = H.spinor(V, 6, 303)
    rot = lambda x: x @ W.conj()   # colour coordinates in the real basis: W^dag x per spin
    for dag in (False, True):
        np.testing.assert_allclose(oracle_mod.dirac_full(Lr, URr, rot(psi), dag),
                                   rot(oracle_mod.dirac_full(L, UR, psi, dag)), atol=1e-13)
    X, Y = H.spinor(V, 6, 305), H.spinor(V, 6, 307)
    np.testing.assert_allclose(oracle_mod.force(Lr, URr, rot(X), rot(Y)), oracle_mod.force(L, UR, X, Y),
                               atol=1e-12)
