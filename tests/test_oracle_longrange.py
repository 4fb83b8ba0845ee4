"""Pins for the long-range Ising MPO (Eq. LRIsing, couplings as sums of
exponentials): the MPO contracts to the dense pair-sum Hamiltonian; the
library's builder gives the same tensors; a single exponential reproduces a
pure exponential decay; the fit of 1/r^alpha is close on r = 1..L-1."""
import numpy as np

from oracle import exact, mpo
from paper_1703_00387_gb300 import hamiltonians


def test_long_range_mpo_is_pair_sum():
    L, J, g = 6, 0.8, 1.3
    amps, lam = np.array([0.7, -0.2, 0.5]), np.array([0.9, 0.5, 0.3])
    f = lambda r: float(np.sum(amps * lam ** r))
    H = mpo.mpo_to_dense(mpo.long_range_ising_mpo(L, J, g, amps, lam))
    Hd = mpo.long_range_ising_dense(L, J, g, f)
    assert np.abs(H - Hd).max() < 1e-13


def test_library_builder_matches_oracle():
    L = 7
    a, lam, _ = hamiltonians.exponential_fit(lambda r: r ** -1.5, L - 1, 4)
    A = hamiltonians.long_range_ising(L, 1.0, 0.9, a, lam)
    Bo = mpo.long_range_ising_mpo(L, 1.0, 0.9, a, lam)
    for x, y in zip(A, Bo):
        np.testing.assert_allclose(x, y, atol=1e-15)


def test_nearest_neighbour_limit():
    """One exponential with decay -> 0 at fixed amplitude * decay reduces to
    the nearest-neighbour Ising chain (closed form)."""
    L = 8
    lam = 1e-12
    W = mpo.long_range_ising_mpo(L, 1.0, 1.0, [1.0 / lam], [lam])
    e0 = np.linalg.eigvalsh(mpo.mpo_to_dense(W))[0]
    assert abs(e0 - exact.ising_free_fermion_energy(L, 1.0, 1.0)) < 1e-9


def test_power_law_fit_quality():
    a, lam, err = hamiltonians.exponential_fit(lambda r: r ** -1.5, 127, 8)
    assert err < 2e-3
