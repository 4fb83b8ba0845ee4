"""Pins for oracle.dmrg: brute-force effective Hamiltonians, textbook Lanczos,
truncation identities of Sec. 2 / the overlap appendix, and full two-site
sweeps against exact diagonalisation and closed forms."""
import numpy as np
import pytest

from oracle import dmrg, exact, mpo
from paper_1703_00387_gb300 import inputs


def _mixed_canonical(mps, k):
    """Left-canonical sites < k, right-canonical sites > k+1 (via the oracle's
    RQ sweep followed by left QR shifts)."""
    m = dmrg.right_canonicalize(mps)
    for j in range(k):
        chl, d, chr_ = m[j].shape
        Q, Rm = np.linalg.qr(m[j].reshape(chl * d, chr_))
        m[j] = Q.reshape(chl, d, Q.shape[1])
        m[j + 1] = np.tensordot(Rm, m[j + 1], axes=([1], [0]))
    return m


def _projector(mps, k):
    """P maps theta (a s1 s2 c) to the full d^L vector: psi = P theta."""
    left = np.ones((1, 1))
    for A in mps[:k]:
        left = np.tensordot(left, A, axes=([left.ndim - 1], [0]))
    left = left.reshape(-1, mps[k].shape[0])           # (d^k, a)
    right = np.ones((1, 1))
    for A in reversed(mps[k + 2:]):
        right = np.tensordot(A, right, axes=([2], [0]))
        right = right.reshape(A.shape[0], -1)
    d1, d2 = mps[k].shape[1], mps[k + 1].shape[1]
    P = np.einsum("xa,st,uv,cy->xsuyatvc", left, np.eye(d1), np.eye(d2), right)
    n_full = left.shape[0] * d1 * d2 * right.shape[1]
    return P.reshape(n_full, -1)


@pytest.mark.parametrize("model,k", [("ising", 2), ("xxz", 0), ("xxz", 4), ("aklt", 1)])
def test_heff_equals_projected_hamiltonian(model, k):
    if model == "ising":
        L, d, W = 7, 2, mpo.ising_mpo(7, 1.0, 0.9)
    elif model == "xxz":
        J, h = inputs.random_couplings(6, seed=2)
        L, d, W = 6, 2, mpo.xxz_mpo(6, J, 0.8, h)
    else:
        L, d, W = 5, 3, mpo.aklt_mpo(5)
    mps = _mixed_canonical(inputs.random_mps(L, d, 6, seed=1), k)
    for j in range(k):
        assert dmrg.left_isometry_defect(mps[j]) < 1e-13
    for j in range(k + 2, L):
        assert dmrg.right_isometry_defect(mps[j]) < 1e-13
    Lenv = np.ones((1, 1, 1))
    for j in range(k):
        Lenv = dmrg.env_left(Lenv, mps[j], W[j])
    Renv = np.ones((1, 1, 1))
    for j in range(L - 1, k + 1, -1):
        Renv = dmrg.env_right(Renv, mps[j], W[j])
    Hfull = mpo.mpo_to_dense(W)
    P = _projector(mps, k)
    Heff_bf = P.T @ Hfull @ P
    Heff = dmrg.heff_dense(Lenv, W[k], W[k + 1], Renv)
    np.testing.assert_allclose(Heff, Heff_bf, atol=1e-12)
    np.testing.assert_allclose(Heff, Heff.T, atol=1e-12)
    theta = np.tensordot(mps[k], mps[k + 1], axes=([2], [0]))
    y = dmrg.heff_apply(Lenv, W[k], W[k + 1], Renv, theta)
    np.testing.assert_allclose(y.ravel(), Heff_bf @ theta.ravel(), atol=1e-12)
    # <theta|H_eff|theta> = <psi|H|psi> in mixed-canonical form
    psi = dmrg.mps_to_vector(mps)
    assert abs(theta.ravel() @ y.ravel() - psi @ Hfull @ psi) < 1e-12
    assert abs(dmrg.mpo_expectation(W, mps) - psi @ Hfull @ psi) < 1e-12


def test_heff_symmetry_random_vectors():
    W = mpo.xxz_mpo(8, 1.0, 1.0, 0.0)
    mps = dmrg.right_canonicalize(inputs.random_mps(8, 2, 8, seed=4))
    Renv = dmrg.build_right_envs(W, mps)
    rng = np.random.default_rng(9)
    x = rng.standard_normal(mps[0].shape[:2] + mps[1].shape[1:])
    yv = rng.standard_normal(x.shape)
    Lenv = np.ones((1, 1, 1))
    hx = dmrg.heff_apply(Lenv, W[0], W[1], Renv[2], x)
    hy = dmrg.heff_apply(Lenv, W[0], W[1], Renv[2], yv)
    a, b = float(np.vdot(yv, hx)), float(np.vdot(hy, x))
    assert abs(a - b) <= 1e-13 * max(abs(a), 1.0)


def test_lanczos_random_symmetric_matrix():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((500, 500))
    A = (A + A.T) / 2
    e, x, iters, resid = dmrg.lanczos_ground(lambda v: A @ v, rng.standard_normal(500),
                                             max_iter=500, tol=1e-12)
    assert abs(e - np.linalg.eigvalsh(A)[0]) < 1e-12 * abs(e)
    assert np.linalg.norm(A @ x - e * x) < 1e-10
    assert abs(np.linalg.norm(x) - 1.0) < 1e-14


def test_lanczos_small_space_exhausted():
    A = np.diag([3.0, -1.0, 2.0])
    e, x, iters, _ = dmrg.lanczos_ground(lambda v: A @ v, np.ones(3), max_iter=100, tol=1e-14)
    assert abs(e + 1.0) < 1e-14 and iters <= 3


@pytest.mark.parametrize("chi", [1, 3, 8, 16])
def test_truncation_overlap_identity(chi):
    # overlap <psi'|psi> = sqrt(sum_{i<=chi} lambda_i^2) (Eq. overlap) and
    # 1 - <psi'|psi> <= discarded weight (Eq. elocal)
    L, k = 10, 4
    mps = _mixed_canonical(inputs.random_mps(L, 2, 32, seed=7), k)
    psi = dmrg.mps_to_vector(mps)
    theta = np.tensordot(mps[k], mps[k + 1], axes=([2], [0]))
    for split in (dmrg.split_svd, dmrg.split_eig):
        Ak, Ak1, info = split(theta, chi, 0.0, move_right=True)
        trunc = list(mps)
        trunc[k], trunc[k + 1] = Ak, Ak1
        psi_t = dmrg.mps_to_vector(trunc)
        assert abs(np.linalg.norm(psi_t) - 1.0) < 1e-13
        overlap = psi_t @ psi
        kept = np.sum(info["lam2"][:info["keep"]])
        assert abs(overlap - np.sqrt(kept)) < 1e-12
        assert 1.0 - overlap <= info["discarded"] + 1e-14
        assert dmrg.left_isometry_defect(Ak) < 1e-12


def test_split_eig_matches_svd_spectrum_and_product():
    rng = np.random.default_rng(1)
    theta = rng.standard_normal((6, 2, 2, 5))
    theta /= np.linalg.norm(theta)
    for move_right in (True, False):
        a1, b1, i1 = dmrg.split_svd(theta, 100, 0.0, move_right)
        a2, b2, i2 = dmrg.split_eig(theta, 100, 0.0, move_right)
        n = len(i1["lam2"])
        big = i1["lam2"] > 1e-12
        np.testing.assert_allclose(i2["lam2"][:n][big], i1["lam2"][big], rtol=1e-12)
        assert np.all(np.abs(i2["lam2"][n:]) < 1e-14)  # Gram of the larger side: rank-deficient tail
        t1 = np.tensordot(a1, b1, axes=([2], [0]))
        t2 = np.tensordot(a2, b2, axes=([2], [0]))
        np.testing.assert_allclose(t1, theta, atol=1e-13)
        np.testing.assert_allclose(t2, theta, atol=1e-13)
        if move_right:
            assert dmrg.left_isometry_defect(a2) < 1e-13
        else:
            assert dmrg.right_isometry_defect(b2) < 1e-13


def test_truncation_rank_rule():
    lam2 = np.array([0.5, 0.3, 0.15, 0.04, 0.009, 0.001])
    assert dmrg.truncation_rank(lam2, 100, 0.0) == 6
    assert dmrg.truncation_rank(lam2, 100, 0.0011) == 5    # tail from index 5 is 0.001
    assert dmrg.truncation_rank(lam2, 100, 0.0101) == 4
    assert dmrg.truncation_rank(lam2, 3, 0.0) == 3
    assert dmrg.truncation_rank(lam2, 100, 1.0) == 1


def test_ghz_entropy_ln2():
    # near g -> 0 the Ising ground state approaches the GHZ state, with
    # centre-bond entropy ln 2 (Sec. 2)
    # (centre-bond entropy ln 2, Sec. 2). The two lowest states are split by
    # ~g^L, so the even-parity sector is selected by lifting the odd one.
    L = 8
    import scipy.sparse as sps
    H = exact.kron_hamiltonian(L, 2, *exact.ising_terms(L, 1.0, 1e-4))
    P = sps.csr_matrix(np.array([[1.0]]))
    for _ in range(L):
        P = sps.kron(P, sps.csr_matrix(np.array([[0.0, 1.0], [1.0, 0.0]])), format="csr")
    E, psi = exact.ground_state(H + 5.0 * (sps.identity(2 ** L) - P))
    M = psi.reshape(2 ** (L // 2), 2 ** (L // 2))
    theta = M.reshape(2 ** (L // 2 - 1), 2, 2, 2 ** (L // 2 - 1))
    _, _, info = dmrg.split_svd(theta, 100, 0.0)
    assert abs(info["entropy"] - np.log(2.0)) < 1e-6


def test_right_canonicalize_preserves_state():
    mps = inputs.random_mps(7, 2, 8, seed=3)
    v0 = dmrg.mps_to_vector(mps)
    rc = dmrg.right_canonicalize(mps)
    v1 = dmrg.mps_to_vector(rc)
    np.testing.assert_allclose(v1, v0 / np.linalg.norm(v0), atol=1e-13)
    for A in rc[1:]:
        assert dmrg.right_isometry_defect(A) < 1e-13


def test_dmrg_ising_chain_l12_chi32():
    # TFI, J=1, g=1, L=12, chi_max=32, 4 sweeps, Lanczos tol 1e-12, seed 0
    W = mpo.ising_mpo(12, 1.0, 1.0)
    E, mps, hist = dmrg.dmrg(W, inputs.random_mps(12, 2, 32, seed=0), chi_max=32, n_sweeps=4,
                             lanczos_tol=1e-12, lanczos_max_iter=100)
    e_cf = exact.ising_free_fermion_energy(12, 1.0, 1.0)
    assert E >= e_cf - 1e-12                      # variational bound
    assert abs(E - e_cf) < 1e-9 * abs(e_cf)
    assert abs(dmrg.mps_norm2(mps) - 1.0) < 1e-13
    assert abs(hist[-1]["energy"] - E) < 1e-10
    for A in mps[1:]:
        assert dmrg.right_isometry_defect(A) < 1e-12
    # energies do not rise across sweeps beyond the truncation error
    per_sweep = [hist[i * 22 + 21]["energy"] for i in range(4)]
    assert all(b <= a + 1e-10 for a, b in zip(per_sweep, per_sweep[1:]))


def test_dmrg_aklt_exact():
    L = 8
    E, mps, _ = dmrg.dmrg(mpo.aklt_mpo(L), inputs.random_mps(L, 3, 4, seed=0), chi_max=8,
                          n_sweeps=3)
    assert abs(E - exact.aklt_energy(L)) < 1e-10


def test_dmrg_xx_site_dependent_exact():
    L = 10
    J, h = inputs.random_couplings(L, seed=0)
    E, _, _ = dmrg.dmrg(mpo.xxz_mpo(L, J, 0.0, h), inputs.random_mps(L, 2, 32, seed=1),
                        chi_max=32, n_sweeps=3, split="eig")
    assert abs(E - exact.xx_free_fermion_energy(J, h)) < 1e-10


def test_dmrg_bose_hubbard_small():
    L, nmax = 5, 3
    E, _, _ = dmrg.dmrg(mpo.bose_hubbard_mpo(L, 1.0, 4.0, nmax),
                        inputs.random_mps(L, nmax + 1, 32, seed=2), chi_max=32, n_sweeps=3)
    e_ed = exact.ground_energy(exact.kron_hamiltonian(L, nmax + 1,
                                                      *exact.bose_hubbard_terms(L, 1.0, 4.0, nmax)))
    assert abs(E - e_ed) < 1e-10


def test_right_canonicalize_long_random_chain_stays_finite():
    # a random L=128 chain has norm ~ (d chi^2)^(L/2): the shifts must rescale
    mps = dmrg.right_canonicalize(inputs.random_mps(128, 2, 32, seed=0))
    assert all(np.isfinite(A).all() for A in mps)
    assert abs(dmrg.mps_norm2(mps) - 1.0) < 1e-12
    assert max(dmrg.right_isometry_defect(A) for A in mps[1:]) < 1e-12
