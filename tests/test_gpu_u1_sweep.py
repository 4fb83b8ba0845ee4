"""Two-site sweeps on a particle-number-conserving MPS (Sec. 3.4 with
symmetries), end to end on the GPU: theta formation, the U(1) Lanczos, the
per-sector split with joint truncation and the block environment updates
through the library's calls. Checked against exact diagonalisation of the
oracle's MPO restricted to the fixed-N sector, and the final state against
the oracle's float64 contractions of its dense site tensors (canonical form,
particle number, energy)."""
import numpy as np
import pytest

from oracle import dmrg as od
from oracle import mpo as ompo
from paper_1703_00387_gb300 import binding as B
from paper_1703_00387_gb300 import hamiltonians
from paper_1703_00387_gb300 import u1sweep as us

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import os
    if not os.path.exists(B.LIB_PATH):
        from paper_1703_00387_gb300 import build
        build.build()
    c = B.Context(0)
    yield c
    c.close()


def _sector_ground_energy(W_oracle, L, d, N):
    H = ompo.mpo_to_dense(W_oracle)
    digits = np.array(np.unravel_index(np.arange(d ** L), (d,) * L)).sum(axis=0)
    idx = np.nonzero(digits == N)[0]
    return float(np.linalg.eigvalsh(H[np.ix_(idx, idx)])[0])


def _check_state(mps, W_oracle, N, res):
    dense = mps.dense()
    for k in range(1, mps.L):
        assert od.right_isometry_defect(dense[k]) < 1e-10
    psi = od.mps_to_vector(dense)
    d, L = mps.d, mps.L
    digits = np.array(np.unravel_index(np.arange(d ** L), (d,) * L)).sum(axis=0)
    assert np.abs(psi[digits != N]).max() == 0.0
    e_oracle = od.mps_energy(W_oracle, dense)
    assert abs(res["energy"] - e_oracle) <= 1e-10 * max(1.0, abs(e_oracle))


@pytest.mark.parametrize("prec,tol", [("tf32x3", 1e-9), ("bf16x3", 1e-7)])
def test_bose_hubbard_sweep_reaches_sector_ground_state(ctx, prec, tol):
    L, nmax, N = 6, 2, 6
    W = hamiltonians.bose_hubbard(L, 1.0, 4.0, nmax)
    Wo = ompo.bose_hubbard_mpo(L, 1.0, 4.0, nmax)
    ex = us.DeviceExecutor(ctx)
    mps = us.random_u1_mps(ex, L, nmax + 1, N, chi=8, seed=11)
    res = us.u1_sweep(mps, W, n_sweeps=3, chi_max=64, eps_local=0.0, precision=prec,
                      lanczos_tol=1e-11, lanczos_max_iter=100)
    e0 = _sector_ground_energy(Wo, L, nmax + 1, N)
    assert abs(res["energy"] - e0) <= tol * abs(e0), (res["energy"], e0)
    assert res["max_discarded"] <= 1e-12
    _check_state(mps, Wo, N, res)


def test_xxz_half_filling_sweep(ctx):
    L, N = 10, 5
    W = hamiltonians.xxz(L, 1.0, 1.0, 0.0)
    Wo = ompo.xxz_mpo(L, 1.0, 1.0, 0.0)
    ex = us.DeviceExecutor(ctx)
    mps = us.random_u1_mps(ex, L, 2, N, chi=4, seed=3)
    res = us.u1_sweep(mps, W, n_sweeps=3, chi_max=64, eps_local=0.0, precision="tf32x3",
                      lanczos_tol=1e-11)
    e0 = _sector_ground_energy(Wo, L, 2, N)
    assert abs(res["energy"] - e0) <= 1e-9 * abs(e0), (res["energy"], e0)
    _check_state(mps, Wo, N, res)


def test_truncated_sweep_keeps_chi_max_and_bounds_the_energy(ctx):
    L, nmax, N = 8, 2, 8
    W = hamiltonians.bose_hubbard(L, 1.0, 4.0, nmax)
    Wo = ompo.bose_hubbard_mpo(L, 1.0, 4.0, nmax)
    ex = us.DeviceExecutor(ctx)
    mps = us.random_u1_mps(ex, L, nmax + 1, N, chi=8, seed=5)
    chi = 12
    res = us.u1_sweep(mps, W, n_sweeps=3, chi_max=chi, eps_local=0.0, precision="tf32x3",
                      lanczos_tol=1e-10)
    assert max(b.dim for b in mps.bonds) <= chi
    e0 = _sector_ground_energy(Wo, L, nmax + 1, N)
    # variational: above the sector's ground energy, and close to it at chi = 12
    assert res["energy"] >= e0 - 1e-10
    assert res["energy"] - e0 <= 1e-3 * abs(e0)
    assert res["max_discarded"] > 0.0
    _check_state(mps, Wo, N, res)
