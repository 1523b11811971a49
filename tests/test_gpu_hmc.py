"""GPU parity of the HMC building blocks (Sec. 2.4, Sec. 2.5, Sec. 4.2) with
the oracle: Wilson plaquette action, gauge force, link update, kinetic energy,
and whole molecular-dynamics trajectories (leapfrog and 2nd-order Omelyan,
pure gauge and with an even/odd pseudofermion); then the integrator properties
the paper checks, on the GPU path: the Hamiltonian violation falls as the
step size squared, and a trajectory run back with reversed momenta returns to
its start."""
import numpy as np
import pytest
import torch

from tests import _helpers as H
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

BETA = 2.2


@pytest.fixture(scope="module")
def hr():
    from paper_2503_06721_gb300 import build, hr
    build.build()
    hr.load()
    return hr


def _momenta(V, N, seed):
    return np.random.default_rng(seed).normal(size=(V, 4, N * N - 1)) / np.sqrt(0.5)


def _setup(hr, oracle_mod, N, rep, dims, m0=0.3, eps=0.5, seed=211):
    lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), m0)
    L = oracle_mod.lat(N, rep, dims, (-1, 1, 1, 1), m0)
    U = H.links(dims, N, eps, seed=seed)
    return lat, L, U


@pytest.mark.parametrize("N", [2, 3, 4])
def test_gauge_action_force_update_energy(hr, oracle_mod, N):
    rep = "FUND"
    lat, L, U = _setup(hr, oracle_mod, N, rep, (4, 6, 2, 4), eps=0.8)
    Ud = G.to_gpu(U)
    S = hr.gauge_action(lat, Ud, BETA)
    So = oracle_mod.plaquette_action(L, U, BETA)
    assert abs(S - So) <= 1e-13 * abs(So)
    # force, accumulated with a coefficient onto an existing field
    F0 = np.random.default_rng(5).normal(size=(lat.volume, 4, N * N - 1))
    F = hr.gauge_force(lat, Ud, BETA, coeff=0.7, F=torch.as_tensor(F0).cuda())
    want = F0 + 0.7 * oracle_mod.gauge_force(L, U, BETA)
    np.testing.assert_allclose(F.cpu().numpy(), want, rtol=0, atol=1e-12 * np.abs(want).max())
    # link update, with small and large steps (the large one takes the squaring path)
    pi = _momenta(lat.volume, N, 7)
    for e in (0.05, 3.0):
        Un = hr.link_update(lat, Ud.clone(), torch.as_tensor(pi).cuda(), e)
        want = oracle_mod.link_update(L, U, pi, e)
        np.testing.assert_allclose(Un.cpu().numpy(), want, rtol=0, atol=5e-14)
    # kinetic energy
    Hp = hr.momenta_energy(lat, torch.as_tensor(pi).cuda())
    assert abs(Hp - oracle_mod.kinetic_energy(pi)) <= 1e-13 * Hp


def _hmc_case(hr, oracle_mod, fermions, N=2, rep="FUND", dims=(4, 4, 2, 2), m0=0.3):
    lat, L, U = _setup(hr, oracle_mod, N, rep, dims, m0=m0, eps=0.5, seed=157)
    pi = _momenta(lat.volume, N, 163)
    phi = None
    if fermions:
        eta = H.spinor(lat.volume // 2, lat.D, 167)
        phi = oracle_mod.dhat(L, oracle_mod.represent_field(L, U), eta, dagger=True)
    return lat, L, U, pi, phi


def _gpu_traj(hr, lat, U, pi, phi, tau, nsteps, integrator, tol=1e-13):
    Ud = G.to_gpu(U)
    pd = torch.as_tensor(pi).cuda().clone()
    g = hr.Gauge(lat, Ud, precs=("f64",))
    try:
        st = hr.md_trajectory(g, Ud, pd, G.to_gpu(phi) if phi is not None else None, BETA, tau, nsteps,
                              integrator=integrator, tol=tol)
        Hs = hr.hamiltonian(g, Ud, pd, G.to_gpu(phi) if phi is not None else None, BETA, tol=1e-13)
    finally:
        g.close()
    return Ud.cpu().numpy(), pd.cpu().numpy(), st, Hs


@pytest.mark.parametrize("integrator", [0, 1], ids=["leapfrog", "omelyan"])
@pytest.mark.parametrize("fermions", [False, True], ids=["gauge", "gauge+fermion"])
def test_md_trajectory_matches_oracle(hr, oracle_mod, integrator, fermions):
    lat, L, U, pi, phi = _hmc_case(hr, oracle_mod, fermions)
    tau, nsteps = 0.4, 4
    U1, p1, st, Hs = _gpu_traj(hr, lat, U, pi, phi, tau, nsteps, integrator)
    name = "leapfrog" if integrator == 0 else "omelyan"
    Uo, po = oracle_mod.md_trajectory(L, U, pi, BETA, tau, nsteps, phi, name)
    tolU = 1e-12 if phi is None else 1e-10
    np.testing.assert_allclose(U1, Uo, rtol=0, atol=tolU)
    np.testing.assert_allclose(p1, po, rtol=0, atol=tolU * 10 * np.abs(po).max())
    if fermions:
        assert st["force_evals"] == (nsteps + 1 if integrator == 0 else 2 * nsteps + 1)
        assert st["max_true_rel_residual"] <= 1e-13
    # the Hamiltonian at the end, term by term
    Ho = oracle_mod.hamiltonian(L, Uo, po, BETA, phi)
    for a, b in zip(Hs, Ho):
        assert abs(a - b) <= 1e-9 * max(1.0, abs(b)), (Hs, Ho)


def test_md_energy_violation_and_reversibility(hr, oracle_mod):
    """SU(3) sextet fermions on 8^4: |dH| of an Omelyan trajectory falls by
    ~4 when the step halves (2nd order, Table 2), and the reversed trajectory
    returns to the start."""
    lat, L, U, pi, phi = _hmc_case(hr, oracle_mod, True, N=3, rep="SYM", dims=(8, 8, 8, 8), m0=0.1)
    H0 = sum(oracle_mod.hamiltonian(L, U, pi, BETA, phi))
    dH = []
    for n in (8, 16, 32):
        U1, p1, st, Hs = _gpu_traj(hr, lat, U, pi, phi, 0.5, n, 1)
        dH.append(abs(sum(Hs) - H0))
    r1, r2 = dH[0] / dH[1], dH[1] / dH[2]
    assert 3.0 < r1 < 5.2 and 3.6 < r2 < 4.4, (dH, r1, r2)
    U1, p1, _, _ = _gpu_traj(hr, lat, U, pi, phi, 0.5, 8, 1)
    U2, p2, _, _ = _gpu_traj(hr, lat, U1, -p1, phi, 0.5, 8, 1)
    assert np.abs(U2 - U).max() < 1e-9
    assert np.abs(p2 + pi).max() < 1e-8 * np.abs(pi).max()


def test_hmc_update_matches_oracle(hr, oracle_mod):
    """One HMC update (heat bath phi = Dhat^dag eta, H, trajectory, H,
    Metropolis) against the oracle on the same random draws; a forced
    rejection restores the links and their representation."""
    lat, L, U, pi, _ = _hmc_case(hr, oracle_mod, False)
    eta = H.spinor(lat.volume // 2, lat.D, 307)
    UR = oracle_mod.represent_field(L, U)
    phi = oracle_mod.dhat(L, UR, eta, dagger=True)
    H0 = sum(oracle_mod.hamiltonian(L, U, pi, BETA, phi))
    Uo, po = oracle_mod.md_trajectory(L, U, pi, BETA, 0.4, 4, phi, "omelyan")
    dHo = sum(oracle_mod.hamiltonian(L, Uo, po, BETA, phi)) - H0
    Ud = G.to_gpu(U)
    g = hr.Gauge(lat, Ud, precs=("f64",))
    try:
        r = hr.hmc_trajectory(g, Ud, torch.as_tensor(pi).cuda().clone(), G.to_gpu(eta), BETA, 0.4, 4,
                              u_accept=0.0, tol=1e-13)
        assert r["accepted"] and abs(r["dH"] - dHo) < 1e-8 * max(1.0, abs(dHo)), (r["dH"], dHo)
        np.testing.assert_allclose(Ud.cpu().numpy(), Uo, rtol=0, atol=1e-10)
        # forced rejection: the links and the operator return to the start
        U1 = Ud.clone()
        r = hr.hmc_trajectory(g, Ud, torch.as_tensor(pi).cuda().clone(), G.to_gpu(eta), BETA, 0.4, 4,
                              u_accept=2.0, tol=1e-13)
        assert not r["accepted"]
        assert torch.equal(Ud, U1)
        psi = H.spinor(lat.volume // 2, lat.D, 311)
        y = g.apply(hr.EVEN, hr.F64, G.to_gpu(psi)).cpu().numpy()
        want = oracle_mod.hop_parity(L, oracle_mod.represent_field(L, U1.cpu().numpy()), 0, psi)
        assert G.rel(y, want) <= 1e-13
    finally:
        g.close()
