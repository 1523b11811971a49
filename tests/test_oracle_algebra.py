"""Pins for the oracle's group-theory layer: gamma matrices (Sec. 2.2),
generators and representations of SU(N) (Sec. 2.3, Table 1).

Every check is against something other than the oracle's own formula: the
printed basis and table (tests/golden/), the Clifford algebra, group
homomorphism and unitarity, characters that are fixed by group theory, and
finite differences of the representation map itself."""
import itertools

import numpy as np
import pytest
from scipy.linalg import expm

from tests import _helpers as H


def test_gamma_matches_printed_basis(oracle_mod):
    e = H.gamma_blocks()
    for mu in range(4):
        g = oracle_mod.gamma(mu)
        np.testing.assert_array_equal(g[:2, :2], 0)
        np.testing.assert_array_equal(g[2:, 2:], 0)
        np.testing.assert_allclose(g[:2, 2:], e[mu], atol=0)
        np.testing.assert_allclose(g[2:, :2], e[mu].conj().T, atol=0)


def test_gamma_clifford_and_gamma5(oracle_mod):
    g = [oracle_mod.gamma(mu) for mu in range(4)]
    one = np.eye(4)
    for mu, nu in itertools.product(range(4), range(4)):
        np.testing.assert_allclose(g[mu] @ g[nu] + g[nu] @ g[mu], 2 * one * (mu == nu),
                                   atol=1e-15)
    for mu in range(4):
        np.testing.assert_allclose(g[mu], g[mu].conj().T, atol=0)
    g5 = oracle_mod.gamma(4)
    np.testing.assert_allclose(g5, g[0] @ g[1] @ g[2] @ g[3], atol=1e-15)
    np.testing.assert_allclose(g5, g5.conj().T, atol=1e-15)
    np.testing.assert_allclose(g5 @ g5, one, atol=1e-15)
    for mu in range(4):
        np.testing.assert_allclose(g5 @ g[mu] + g[mu] @ g5, 0, atol=1e-15)
    # in this chiral basis gamma5 is diagonal
    np.testing.assert_allclose(g5, np.diag([1, 1, -1, -1]), atol=1e-15)


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 8])
def test_generators(oracle_mod, N):
    T = oracle_mod.generators(N)
    assert T.shape == (N * N - 1, N, N)
    for a in range(N * N - 1):
        np.testing.assert_allclose(T[a], T[a].conj().T, atol=0)
        assert abs(np.trace(T[a])) < 1e-15
    G = np.einsum("aij,bji->ab", T, T)
    np.testing.assert_allclose(G, 0.5 * np.eye(N * N - 1), atol=1e-15)
    CF = (N * N - 1) / (2 * N)
    np.testing.assert_allclose(np.einsum("aij,ajk->ik", T, T), CF * np.eye(N), atol=1e-14)
    if N == 2:  # textbook: Pauli matrices / 2
        s = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]),
             np.array([[1, 0], [0, -1]])]
        for a in range(3):
            np.testing.assert_allclose(T[a], s[a] / 2, atol=1e-16)


@pytest.mark.parametrize("row", H.table1(), ids=lambda r: f"{r['rep']}-N{r['N']}")
def test_rep_dims_table1(oracle_mod, row):
    assert oracle_mod.rep_dim(row["N"], row["rep"]) == row["D"]


REPS = [(N, rep) for N in (2, 3, 4) for rep in ("FUND", "ADJ", "SYM", "ASYM")
        if not (N == 2 and rep == "ASYM")] + [(4, "ASYM_REAL")]
# the real basis of the SU(4) 2AS is the same representation (Table 1's 2AS row)
TABLE_REP = {"ASYM_REAL": "ASYM"}


@pytest.mark.parametrize("N,rep", REPS)
def test_represent_homomorphism_unitarity(oracle_mod, N, rep):
    U = H.su_n(6, N, seed=11 + N)
    D = oracle_mod.rep_dim(N, rep)
    for i in range(0, 6, 2):
        RU = oracle_mod.represent_link(N, rep, U[i])
        RV = oracle_mod.represent_link(N, rep, U[i + 1])
        RUV = oracle_mod.represent_link(N, rep, U[i] @ U[i + 1])
        np.testing.assert_allclose(RUV, RU @ RV, atol=1e-13)
        np.testing.assert_allclose(RU @ RU.conj().T, np.eye(D), atol=1e-13)
        RUd = oracle_mod.represent_link(N, rep, U[i].conj().T)
        np.testing.assert_allclose(RUd, RU.conj().T, atol=1e-13)
        if rep in ("ADJ", "ASYM_REAL"):  # real representations (stored real, Sec. 3.1.2)
            assert np.abs(RU.imag).max() < 1e-14
            assert abs(np.linalg.det(RU.real) - 1) < 1e-12
        np.testing.assert_allclose(oracle_mod.represent_link(N, rep, np.eye(N)), np.eye(D),
                                   atol=1e-15)


@pytest.mark.parametrize("N,rep", REPS)
def test_characters(oracle_mod, N, rep):
    """Basis-independent characters fixed by group theory."""
    for U in H.su_n(4, N, seed=23 + N):
        tr = np.trace(U)
        tr2 = np.trace(U @ U)
        chi = np.trace(oracle_mod.represent_link(N, rep, U))
        want = {"FUND": tr, "ADJ": abs(tr) ** 2 - 1, "SYM": (tr * tr + tr2) / 2,
                "ASYM": (tr * tr - tr2) / 2, "ASYM_REAL": (tr * tr - tr2) / 2}[rep]
        assert abs(chi - want) < 1e-13
        if N == 3 and rep == "ASYM":  # 2AS of SU(3) is the anti-fundamental
            assert abs(chi - np.conj(tr)) < 1e-13
        if N == 2 and rep == "SYM":   # SYM of SU(2) is the adjoint (spin 1)
            assert abs(chi - np.trace(oracle_mod.represent_link(2, "ADJ", U))) < 1e-13


@pytest.mark.parametrize("N,rep", REPS)
def test_rep_generators(oracle_mod, N, rep):
    """T_R^a against finite differences of R, trace normalisation T_R and
    Casimir C2(R) of Table 1, and the Lie algebra of the fundamental."""
    T = oracle_mod.generators(N)
    TR = oracle_mod.rep_generators(N, rep)
    D = oracle_mod.rep_dim(N, rep)
    eps = 1e-5
    for a in range(N * N - 1):
        Rp = oracle_mod.represent_link(N, rep, expm(1j * eps * T[a]))
        Rm = oracle_mod.represent_link(N, rep, expm(-1j * eps * T[a]))
        fd = -1j * (Rp - Rm) / (2 * eps)
        np.testing.assert_allclose(TR[a], fd, atol=1e-9)
        np.testing.assert_allclose(TR[a], TR[a].conj().T, atol=1e-14)
    row = [r for r in H.table1() if r["rep"] == TABLE_REP.get(rep, rep) and r["N"] == N][0]
    if rep == "ASYM_REAL":   # generators of a real orthogonal representation: i x real antisymmetric
        assert np.abs(TR.real).max() < 1e-14
        np.testing.assert_allclose(TR.imag, -np.swapaxes(TR.imag, 1, 2), atol=1e-14)
    np.testing.assert_allclose(np.einsum("aij,bji->ab", TR, TR),
                               float(row["T"]) * np.eye(N * N - 1), atol=1e-13)
    np.testing.assert_allclose(np.einsum("aij,ajk->ik", TR, TR), float(row["C2"]) * np.eye(D),
                               atol=1e-13)
    # structure constants of the fundamental carry over: [T_R^a, T_R^b] = i f_abc T_R^c
    f = -2j * np.einsum("aij,bjk,cki->abc", T, T, T) + 2j * np.einsum("bij,ajk,cki->abc", T, T, T)
    lhs = np.einsum("aij,bjk->abik", TR, TR) - np.einsum("bij,ajk->abik", TR, TR)
    rhs = 1j * np.einsum("abc,cik->abik", f, TR)
    np.testing.assert_allclose(lhs, rhs, atol=1e-13)


def test_asym_real_basis_is_equivalent_to_asym(oracle_mod):
    """The real basis of the SU(4) 2AS is the complex basis rotated by one
    fixed unitary W (W_mn = Tr(e_m^dag f_n)): R_real(U) = W^dag R_2AS(U) W for
    every U, and W maps the real basis onto matrices fixed by A -> *conj(A)."""
    E = oracle_mod.rep_basis(4, "ASYM")
    F = oracle_mod.rep_basis(4, "ASYM_REAL")
    assert F.shape == (6, 4, 4)
    np.testing.assert_allclose(np.einsum("nij,mij->nm", F.conj(), F), np.eye(6), atol=1e-15)
    np.testing.assert_allclose(F, -np.swapaxes(F, 1, 2), atol=0)
    eps = np.zeros((4, 4, 4, 4))
    for p in itertools.permutations(range(4)):
        eps[p] = np.linalg.det(np.eye(4)[list(p)])
    for f in F:   # fixed by the antilinear Hodge map
        np.testing.assert_allclose(0.5 * np.einsum("ijkl,kl->ij", eps, f.conj()), f, atol=1e-15)
    W = np.einsum("mij,nij->mn", E.conj(), F)
    np.testing.assert_allclose(W.conj().T @ W, np.eye(6), atol=1e-15)
    for U in H.su_n(5, 4, seed=97):
        np.testing.assert_allclose(oracle_mod.represent_link(4, "ASYM_REAL", U),
                                   W.conj().T @ oracle_mod.represent_link(4, "ASYM", U) @ W, atol=1e-14)


def test_table1_reading_is_consistent():
    """T_R (N^2 - 1) = C2(R) D_R holds for the read column and fails for the
    printed 2AS entry, which is why the (N-2)/2 reading is taken."""
    for r in H.table1():
        assert r["T"] * (r["N"] ** 2 - 1) == r["C2"] * r["D"]
        if r["rep"] == "ASYM":
            assert r["T_printed"] * (r["N"] ** 2 - 1) != r["C2"] * r["D"]


def test_input_generator_philox_known_answers():
    """The seeded generator is Philox4x32-10 (Salmon et al., SC'11): the
    published known-answer vectors of the reference implementation."""
    import torch
    from paper_2503_06721_gb300 import synth
    kat = [((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
           ((0xffffffff,) * 4, (0xffffffff, 0xffffffff), (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
           ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
            (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1))]
    for ctr, key, want in kat:
        got = synth.philox4x32(tuple(torch.tensor([c], dtype=torch.int64) for c in ctr), key)
        assert tuple(int(x) for x in got) == want
