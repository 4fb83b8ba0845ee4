"""Pins for oracle.u1: the Bose-Hubbard MPO conserves the particle number
(exact diagonalisation: [H, N] = 0, and entry by entry), and the block rules
for theta, L and R are exactly the ones under which H_eff theta stays in the
allowed sector (a wrong sign in any rule leaks weight out of it)."""
import numpy as np
import pytest

from oracle import mpo, u1
from oracle import u1 as ou1
from paper_1703_00387_gb300 import inputs


def test_bose_hubbard_conserves_particle_number():
    L, nmax = 4, 2
    W = mpo.bose_hubbard_mpo(L, 1.0, 4.0, nmax)
    H = mpo.mpo_to_dense(W)
    d = nmax + 1
    n_site = np.arange(d)
    N = np.zeros(d ** L)
    for idx in range(d ** L):
        digits = np.unravel_index(idx, (d,) * L)
        N[idx] = sum(n_site[x] for x in digits)
    comm = H * N[None, :] - N[:, None] * H
    assert np.abs(comm).max() < 1e-12
    q = u1.mpo_channel_charges(W)           # raises if an entry breaks the rule
    assert list(q[2]) == [0, 1, -1, 0]      # done, b^dag applied, b applied, start


def _masked_operands(ql_s, chil, qr_s, chir, d, qwl, qwr, seed):
    ql = u1.index_charges(ql_s, chil)
    qr = u1.index_charges(qr_s, chir)
    rng = np.random.default_rng(seed)
    Lh = rng.standard_normal((len(ql), len(qwl), len(ql))) * u1.env_mask(ql, qwl, ql)
    Rh = rng.standard_normal((len(qr), len(qwr), len(qr))) * u1.env_mask(qr, qwr, qr)
    th = rng.standard_normal((len(ql), d, d, len(qr))) * u1.theta_mask(ql, qr, d, d)
    return ql, qr, Lh, Rh, th


@pytest.mark.parametrize("flip", [None, "L", "R"])
def test_block_rules_keep_heff_in_sector(flip):
    W = mpo.bose_hubbard_mpo(6, 1.0, 4.0, 3)
    W1, W2 = W[2], W[3]
    qw = u1.mpo_channel_charges(W)
    qwl, qwr = qw[2], qw[4]
    ql, qr, Lh, Rh, th = _masked_operands([3, 4, 5, 6], [2, 3, 3, 1], [5, 6, 7, 8, 9],
                                          [1, 2, 3, 2, 1], 4, qwl, qwr, seed=1)
    if flip == "L":   # operands built with the wrong sign of the channel charge
        Lh = np.random.default_rng(2).standard_normal(Lh.shape) * u1.env_mask(ql, -qwl, ql)
    if flip == "R":
        Rh = np.random.default_rng(3).standard_normal(Rh.shape) * u1.env_mask(qr, -qwr, qr)
    from oracle import dmrg
    y = dmrg.heff_apply(Lh, W1, W2, Rh, th)
    leak = np.abs(np.where(u1.theta_mask(ql, qr, 4, 4), 0.0, y)).max()
    if flip is None:
        assert leak < 1e-12 * np.abs(y).max()
    else:
        assert leak > 1e-3 * np.abs(y).max()


def test_sector_profile_recipe():
    q, chi = inputs.u1_sector_profile(31.0, total=512, width=8.0)
    assert sum(chi) == 512 and min(chi) >= 1
    assert list(q) == sorted(q) and len(set(q)) == len(q)
    assert chi[list(q).index(31)] == max(chi)


def test_sector_heff_from_u1_mps_is_symmetric_and_closed():
    """Environments of a random particle-number-conserving MPS give an H_eff
    that maps the sector into itself and is symmetric on it."""
    from oracle import dmrg
    Lc, nmax, N, d = 6, 2, 6, 3
    q = [ou1.index_charges(list(range(max(0, N - (Lc - k) * nmax), min(N, k * nmax) + 1)),
                           [1 if k in (0, Lc) else 2] * (min(N, k * nmax) - max(0, N - (Lc - k) * nmax) + 1))
         for k in range(Lc + 1)]
    A = [inputs.random_dense((len(q[k]), d, len(q[k + 1])), 10 + k) * ou1.mps_mask(q[k], q[k + 1], d)
         for k in range(Lc)]
    W = mpo.bose_hubbard_mpo(Lc, 1.0, 4.0, nmax)
    Le = np.ones((1, 1, 1))
    for k in (0, 1):
        Le = dmrg.env_left(Le, A[k], W[k])
    Re = np.ones((1, 1, 1))
    for k in (5, 4):
        Re = dmrg.env_right(Re, A[k], W[k])
    qw = ou1.mpo_channel_charges(W)
    assert np.abs(np.where(ou1.env_mask(q[2], qw[2], q[2]), 0.0, Le)).max() == 0.0
    assert np.abs(np.where(ou1.env_mask(q[4], qw[4], q[4]), 0.0, Re)).max() == 0.0
    mt = ou1.theta_mask(q[2], q[4], d, d)
    H = ou1.sector_heff_matrix(Le, W[2], W[3], Re, mt)
    assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()
