"""Pins for oracle.variance: the squared shifted MPO equals (H - E)^2 as a
dense matrix, the variance of a random state matches the dense state-vector
formula, and an exact eigenstate has zero variance."""
import numpy as np
import pytest

from oracle import dmrg, exact, mpo, variance
from paper_1703_00387_gb300 import inputs


def test_squared_shifted_mpo_is_dense_square():
    L = 5
    J, h = inputs.random_couplings(L, seed=2)
    W = mpo.xxz_mpo(L, J, 0.8, h)
    H = mpo.mpo_to_dense(W)
    c = 0.37
    Hs = mpo.mpo_to_dense(variance.mpo_square(variance.shifted_mpo(W, c)))
    ref = (H - c * np.eye(len(H))) @ (H - c * np.eye(len(H)))
    assert np.abs(Hs - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("model", ["ising", "xxz"])
def test_variance_matches_dense(model):
    L = 7
    W = mpo.ising_mpo(L, 1.0, 0.7) if model == "ising" else mpo.xxz_mpo(L, 1.0, 1.0, 0.2)
    mps = inputs.random_mps(L, 2, 4, seed=9)
    E, V = variance.mps_variance(W, mps)
    Ed, Vd = variance.dense_variance(W, mps)
    assert abs(E - Ed) < 1e-12 * abs(Ed)
    assert abs(V - Vd) < 1e-11 * Vd
    assert V > 0


def test_eigenstate_has_zero_variance():
    """The exact ground state (full bond dimension, from the oracle DMRG at
    chi = 2^(L/2)) has variance zero to rounding."""
    L = 8
    W = mpo.ising_mpo(L, 1.0, 1.0)
    E, mps, _ = dmrg.dmrg(W, inputs.random_mps(L, 2, 16, seed=0), chi_max=16, n_sweeps=4)
    E2, V = variance.mps_variance(W, mps)
    assert abs(E2 - exact.ising_free_fermion_energy(L, 1.0, 1.0)) < 1e-10
    assert V < 1e-11
