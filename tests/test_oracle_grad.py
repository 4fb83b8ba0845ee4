"""Pins for oracle.grad: finite differences (every quantity is linear in the
varied tensor, so central differences are exact up to rounding) and the
Hellmann-Feynman derivatives of the free-fermion XX chain."""
import numpy as np
import pytest

from oracle import dmrg, exact, grad, mpo
from paper_1703_00387_gb300 import inputs


def test_heff_vjp_matches_finite_differences():
    Lh, W1, W2, Rh, th = inputs.random_heff_operands(5, 2, 3, 4, 3, 4, 2, seed=8)
    gy = np.random.default_rng(9).standard_normal(th.shape)
    f = lambda t, a, b: float(np.vdot(gy, dmrg.heff_apply(Lh, a, b, Rh, t)))
    g_th, g_w1, g_w2 = grad.heff_vjp(Lh, W1, W2, Rh, th, gy)
    rng = np.random.default_rng(1)
    for _ in range(6):
        idx = tuple(rng.integers(0, n) for n in th.shape)
        e = np.zeros_like(th); e[idx] = 1.0
        fd = (f(th + 1e-3 * e, W1, W2) - f(th - 1e-3 * e, W1, W2)) / 2e-3
        assert abs(fd - g_th[idx]) <= 1e-9 * max(1.0, abs(fd))
        idx = tuple(rng.integers(0, n) for n in W1.shape)
        e = np.zeros_like(W1); e[idx] = 1.0
        fd = (f(th, W1 + 1e-3 * e, W2) - f(th, W1 - 1e-3 * e, W2)) / 2e-3
        assert abs(fd - g_w1[idx]) <= 1e-9 * max(1.0, abs(fd))
        idx = tuple(rng.integers(0, n) for n in W2.shape)
        e = np.zeros_like(W2); e[idx] = 1.0
        fd = (f(th, W1, W2 + 1e-3 * e) - f(th, W1, W2 - 1e-3 * e)) / 2e-3
        assert abs(fd - g_w2[idx]) <= 1e-9 * max(1.0, abs(fd))


def test_energy_grad_matches_finite_differences():
    L = 6
    J, h = inputs.random_couplings(L, seed=3)
    W = mpo.xxz_mpo(L, J, 0.9, h)
    mps = inputs.random_mps(L, 2, 4, seed=5)  # not canonical, not normalised
    E, gW = grad.energy_grad_W(W, mps)
    assert abs(E - dmrg.mps_energy(W, mps)) < 1e-12 * abs(E)
    rng = np.random.default_rng(2)
    for _ in range(8):
        k = int(rng.integers(0, L))
        idx = tuple(rng.integers(0, n) for n in W[k].shape)
        Wp = [w.copy() for w in W]; Wm = [w.copy() for w in W]
        Wp[k][idx] += 1e-3; Wm[k][idx] -= 1e-3
        fd = (dmrg.mps_energy(Wp, mps) - dmrg.mps_energy(Wm, mps)) / 2e-3
        assert abs(fd - gW[k][idx]) <= 1e-9


def test_xx_hellmann_feynman_from_energy_grad():
    """At the (exact, chi = 2^(L/2)) ground state of the site-dependent XX
    chain the energy gradient equals the free-fermion Hellmann-Feynman values."""
    L = 10
    J, h = inputs.random_couplings(L, seed=0)
    W = mpo.xxz_mpo(L, J, 0.0, h)
    E, mps, _ = dmrg.dmrg(W, inputs.random_mps(L, 2, 32, seed=1), chi_max=32, n_sweeps=3)
    _, gW = grad.energy_grad_W(W, mps)
    dJ, dh = grad.xxz_coupling_grads(gW, L, J, 0.0, h)
    dJ_ref, dh_ref = exact.xx_free_fermion_gradients(J, h)
    np.testing.assert_allclose(dJ, dJ_ref, atol=1e-8)
    np.testing.assert_allclose(dh, dh_ref, atol=1e-8)
