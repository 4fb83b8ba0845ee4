"""Pins for oracle.exact: ED against dense eigh, closed forms against ED."""
import numpy as np
import pytest

from oracle import exact, mpo


@pytest.mark.parametrize("L,g", [(12, 1.0), (8, 0.5), (6, 1.5)])
def test_ising_free_fermion_matches_ed(L, g):
    H = exact.kron_hamiltonian(L, 2, *exact.ising_terms(L, 1.0, g))
    e_ed = exact.ground_energy(H)
    e_cf = exact.ising_free_fermion_energy(L, 1.0, g)
    assert abs(e_ed - e_cf) < 1e-10 * abs(e_cf)


def test_xx_free_fermion_matches_ed_site_dependent():
    rng = np.random.default_rng(0)
    L = 10
    J = rng.uniform(0.8, 1.2, L - 1)
    h = rng.uniform(-0.5, 0.5, L)
    H = exact.kron_hamiltonian(L, 2, *exact.xxz_terms(L, J, 0.0, h))
    e_ed = exact.ground_energy(H)
    assert abs(e_ed - exact.xx_free_fermion_energy(J, h)) < 1e-10


def test_xx_hellmann_feynman_matches_finite_differences():
    rng = np.random.default_rng(3)
    L = 8
    J = rng.uniform(0.8, 1.2, L - 1)
    h = rng.uniform(-0.5, 0.5, L)
    dJ, dh = exact.xx_free_fermion_gradients(J, h)
    step = 1e-6
    for i in [0, 3, L - 2]:
        Jp, Jm = J.copy(), J.copy()
        Jp[i] += step
        Jm[i] -= step
        fd = (exact.xx_free_fermion_energy(Jp, h) - exact.xx_free_fermion_energy(Jm, h)) / (2 * step)
        assert abs(fd - dJ[i]) < 1e-7
    for i in [0, 4, L - 1]:
        hp, hm = h.copy(), h.copy()
        hp[i] += step
        hm[i] -= step
        fd = (exact.xx_free_fermion_energy(J, hp) - exact.xx_free_fermion_energy(J, hm)) / (2 * step)
        assert abs(fd - dh[i]) < 1e-7


def test_xx_hellmann_feynman_matches_ed_expectations():
    rng = np.random.default_rng(5)
    L = 8
    J = rng.uniform(0.8, 1.2, L - 1)
    h = rng.uniform(-0.5, 0.5, L)
    E, psi = exact.ground_state(exact.kron_hamiltonian(L, 2, *exact.xxz_terms(L, J, 0.0, h)))
    dJ, dh = exact.xx_free_fermion_gradients(J, h)
    one = np.ones(L - 1)
    for i in [1, 5]:
        bond_i = exact.kron_hamiltonian(L, 2, [np.zeros((2, 2))] * L,
                                        exact.xxz_terms(L, one * (np.arange(L - 1) == i), 0.0, 0.0)[1])
        assert abs(psi @ (bond_i @ psi) - dJ[i]) < 1e-9


@pytest.mark.parametrize("L", [6, 8])
def test_aklt_exact_energy(L):
    site, bonds, _ = exact.aklt_terms(L)
    H = exact.kron_hamiltonian(L, 3, site, bonds)
    assert abs(exact.ground_energy(H) - exact.aklt_energy(L)) < 1e-10


def test_eigsh_matches_dense_eigh():
    H = exact.kron_hamiltonian(8, 2, *exact.xxz_terms(8, 1.0, 1.0, 0.0))
    dense = float(np.linalg.eigvalsh(H.toarray())[0])
    import scipy.sparse.linalg as spla
    sparse = float(spla.eigsh(H, k=1, which="SA", tol=1e-14)[0][0])
    assert abs(dense - sparse) < 1e-12


def test_heisenberg_energy_per_site_sanity():
    # open Heisenberg chain: the energy added per site between L=10 and L=12
    # approaches the Bethe-ansatz bulk value 1/4 - ln 2 = -0.4431
    e12 = exact.ground_energy(exact.kron_hamiltonian(12, 2, *exact.xxz_terms(12, 1.0, 1.0, 0.0)))
    e10 = exact.ground_energy(exact.kron_hamiltonian(10, 2, *exact.xxz_terms(10, 1.0, 1.0, 0.0)))
    assert abs((e12 - e10) / 2 - (0.25 - np.log(2.0))) < 5e-3
    # MPO route agrees with the Kronecker route at a smaller size
    W = mpo.xxz_mpo(8, 1.0, 1.0, 0.0)
    assert abs(np.linalg.eigvalsh(mpo.mpo_to_dense(W))[0]
               - exact.ground_energy(exact.kron_hamiltonian(8, 2, *exact.xxz_terms(8)))) < 1e-12


def test_xxz_l20_golden_matches_oracle():
    """tests/golden/xxz_l20_ground_energy.json (the exact chi = 1024 reference
    of the GPU sweeps) is what its script's oracle construction gives."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "xxz_l20_ground_energy.json")
    with open(path) as f:
        stored = json.load(f)["ground_energy"]
    H = exact.kron_hamiltonian(20, 2, *exact.xxz_terms(20, 1.0, 1.0, 0.0))
    assert abs(exact.ground_energy(H) - stored) <= 1e-12 * abs(stored)
