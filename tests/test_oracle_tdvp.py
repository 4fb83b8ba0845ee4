"""Pins of the TDVP oracle (oracle.tdvp) against exact dense evolution, the
matrix exponential and brute-force contractions: every check compares the
oracle with something computed another way."""
import numpy as np
import pytest
import scipy.linalg

from oracle import dmrg as od
from oracle import mpo
from oracle import tdvp as T


def _random_hermitian(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return 0.5 * (A + A.conj().T)


def _random_complex_mps(L, d, chi, seed):
    rng = np.random.default_rng(seed)
    dims = [min(d ** k, d ** (L - k), chi) for k in range(L + 1)]
    return [rng.standard_normal((dims[k], d, dims[k + 1]))
            + 1j * rng.standard_normal((dims[k], d, dims[k + 1])) for k in range(L)]


@pytest.mark.parametrize("n,tau", [(120, 0.3), (120, -0.7), (60, 2.0)])
def test_krylov_expm_matches_matrix_exponential(n, tau):
    H = _random_hermitian(n, seed=n)
    v = np.random.default_rng(5).standard_normal(n) + 1j * np.random.default_rng(6).standard_normal(n)
    x, m, err = T.krylov_expm(lambda y: H @ y, v, tau, max_iter=n, tol=1e-13)
    ref = scipy.linalg.expm(-1j * tau * H) @ v
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(v)
    assert m < n  # stopped on the error estimate, not on the dimension
    # unitary: the norm is kept
    assert abs(np.linalg.norm(x) - np.linalg.norm(v)) <= 1e-12 * np.linalg.norm(v)


def test_krylov_expm_exhausted_space_is_exact():
    # v0 in a 3-dimensional invariant subspace: exact after 3 vectors
    H = np.diag([1.0, -2.0, 0.5, 3.0, 7.0]).astype(np.complex128)
    v = np.array([1.0, 1j, 2.0, 0.0, 0.0])
    x, m, err = T.krylov_expm(lambda y: H @ y, v, 1.3, max_iter=5, tol=0.0)
    assert m == 3 and err == 0.0
    assert np.allclose(x, np.exp(-1.3j * np.diag(H)) * v, atol=1e-14, rtol=0)


def test_krylov_expm_stops_at_cap():
    H = _random_hermitian(80, seed=3)
    v = np.ones(80, dtype=np.complex128)
    _, m, err = T.krylov_expm(lambda y: H @ y, v, 5.0, max_iter=4, tol=1e-15)
    assert m == 4 and err > 0.0


def test_complex_expectation_matches_dense():
    # <psi|H|psi> through the complex environments against the dense vector:
    # a conjugate on the wrong tensor changes the value for a complex state
    L = 5
    W = mpo.xxz_mpo(L, 1.0, 0.7, 0.3)
    mps = _random_complex_mps(L, 2, 4, seed=2)
    psi = T.mps_to_vector_c(mps)
    H = mpo.mpo_to_dense(W)
    e, nrm = T.mps_expectation_c(W, mps)
    assert abs(nrm - np.vdot(psi, psi).real) <= 1e-12 * nrm
    assert abs(e - np.vdot(psi, H @ psi)) <= 1e-12 * abs(e)


def test_heff_forms_match_projected_hamiltonian():
    # <theta|H_eff theta> = <psi|H|psi> in mixed canonical form, for the
    # two-site and the one-site effective Hamiltonians, and H_eff is Hermitian
    L = 6
    W = mpo.ising_mpo(L, 1.0, 1.3)
    mps = T.right_canonicalize_c(_random_complex_mps(L, 2, 8, seed=4))
    Renv = T.build_right_envs_c(W, mps)
    Lenv = [np.ones((1, 1, 1), dtype=np.complex128)]
    for k in range(2):  # move the centre to site 2 by QR
        chl, d, chr_ = mps[k].shape
        Q, Rm = np.linalg.qr(mps[k].reshape(chl * d, chr_))
        mps[k] = Q.reshape(chl, d, Q.shape[1])
        mps[k + 1] = np.tensordot(Rm, mps[k + 1], axes=([1], [0]))
        Lenv.append(T.env_left_c(Lenv[k], mps[k], W[k]))
    H = mpo.mpo_to_dense(W)
    psi = T.mps_to_vector_c(mps)
    e_ref = np.vdot(psi, H @ psi).real
    th = np.tensordot(mps[2], mps[3], axes=([2], [0]))
    y = T.heff2_apply(Lenv[2], W[2], W[3], Renv[4], th)
    assert abs(np.vdot(th, y) - e_ref) <= 1e-12 * abs(e_ref)
    c = mps[2]
    y1 = T.heff1_apply(Lenv[2], W[2], Renv[3], c)
    assert abs(np.vdot(c, y1) - e_ref) <= 1e-12 * abs(e_ref)
    rng = np.random.default_rng(9)
    a = rng.standard_normal(th.shape) + 1j * rng.standard_normal(th.shape)
    b = rng.standard_normal(th.shape) + 1j * rng.standard_normal(th.shape)
    lhs = np.vdot(a, T.heff2_apply(Lenv[2], W[2], W[3], Renv[4], b))
    rhs = np.vdot(T.heff2_apply(Lenv[2], W[2], W[3], Renv[4], a), b)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("model", ["xxz", "ising"])
def test_tdvp_at_full_bond_dimension_is_exact_evolution(model):
    # With no truncation the projector-splitting integrator reproduces the
    # exact evolution exp(-i H t) psi0 (up to the Krylov tolerance)
    L = 6
    W = mpo.xxz_mpo(L, 1.0, 0.5, 0.2) if model == "xxz" else mpo.ising_mpo(L, 1.0, 1.2)
    H = mpo.mpo_to_dense(W)
    mps0 = _random_complex_mps(L, 2, 64, seed=1)
    psi0 = T.mps_to_vector_c(T.right_canonicalize_c(mps0))
    dt, n = 0.1, 4
    mps, hist = T.tdvp2_evolve(W, mps0, dt, n, chi_max=64)
    ref = scipy.linalg.expm(-1j * H * dt * n) @ psi0
    assert np.linalg.norm(T.mps_to_vector_c(mps) - ref) <= 1e-10
    e0 = np.vdot(psi0, H @ psi0).real
    for _, e, nrm in hist:  # energy and norm conserved
        assert abs(e - e0) <= 1e-11 * max(1.0, abs(e0))
        assert abs(nrm - 1.0) <= 1e-12


def test_tdvp_ground_state_only_gains_a_phase():
    # a DMRG ground state (truncated, chi = 16 at L = 10) is stationary:
    # psi(t) = exp(-i E0 t) psi0 up to the truncation
    L = 10
    W = mpo.ising_mpo(L, 1.0, 1.0)
    rng = np.random.default_rng(0)
    dims = od.initial_bond_dims(L, 2, 16)
    start = [rng.standard_normal((dims[k], 2, dims[k + 1])) for k in range(L)]
    E0, gs, _ = od.dmrg(W, start, chi_max=16, n_sweeps=4)
    psi0 = T.mps_to_vector_c(T.right_canonicalize_c(gs))
    dt, n = 0.05, 4
    mps, _ = T.tdvp2_evolve(W, gs, dt, n, chi_max=16, eps_local=1e-14)
    psi = T.mps_to_vector_c(mps)
    ov = np.vdot(psi0, psi)
    assert abs(abs(ov) - 1.0) <= 1e-8
    assert abs(np.angle(ov * np.exp(1j * E0 * dt * n))) <= 1e-8


def test_tdvp_truncated_converges_with_bond_dimension():
    # a Neel-state quench of the XXZ chain at L = 8, the product state held
    # at the full bond dimensions (zero padding, made orthonormal by the
    # canonicalisation): the error against exact evolution falls as chi_max
    # grows and vanishes at the full dimension 16
    L = 8
    W = mpo.xxz_mpo(L, 1.0, 1.0, 0.0)
    H = mpo.mpo_to_dense(W)
    dims = [min(2 ** k, 2 ** (L - k)) for k in range(L + 1)]
    neel = [np.zeros((dims[k], 2, dims[k + 1])) for k in range(L)]
    for k in range(L):
        neel[k][0, k % 2, 0] = 1.0
    psi0 = T.mps_to_vector_c(neel)
    t_end, dt = 0.6, 0.05
    ref = scipy.linalg.expm(-1j * H * t_end) @ psi0
    errs = []
    for chi in (2, 4, 16):
        mps, _ = T.tdvp2_evolve(W, neel, dt, int(round(t_end / dt)), chi_max=chi)
        errs.append(np.linalg.norm(T.mps_to_vector_c(mps) - ref))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] <= 1e-10


@pytest.mark.parametrize("mistake", ["backward_sign", "no_backward", "full_dt", "no_conj"])
def test_exactness_pin_catches_planted_mistakes(monkeypatch, mistake):
    # each plausible slip in the step, planted in the oracle, breaks the
    # full-bond-dimension exactness pin by far more than its 1e-10 bar
    L = 6
    W = mpo.xxz_mpo(L, 1.0, 0.5, 0.2)
    H = mpo.mpo_to_dense(W)
    mps0 = _random_complex_mps(L, 2, 64, seed=1)
    psi0 = T.mps_to_vector_c(T.right_canonicalize_c(mps0))
    real_expm = T.krylov_expm
    if mistake == "backward_sign":
        monkeypatch.setattr(T, "krylov_expm", lambda mv, v, tau, *a: real_expm(mv, v, abs(tau), *a))
    elif mistake == "no_backward":
        monkeypatch.setattr(T, "krylov_expm",
                            lambda mv, v, tau, *a: (v, 1, 0.0) if tau < 0 else real_expm(mv, v, tau, *a))
    elif mistake == "full_dt":
        monkeypatch.setattr(T, "krylov_expm",
                            lambda mv, v, tau, *a: real_expm(mv, v, 2 * tau if tau > 0 else tau, *a))
    else:
        def env_left_noconj(Lenv, A, Wk):
            X = np.tensordot(Lenv, A, axes=([2], [0]))
            Y = np.tensordot(X, Wk, axes=([1, 2], [0, 2]))
            return np.ascontiguousarray(np.tensordot(A, Y, axes=([0, 1], [0, 2])).transpose(0, 2, 1))
        monkeypatch.setattr(T, "env_left_c", env_left_noconj)
    mps, _ = T.tdvp2_evolve(W, mps0, 0.1, 4, chi_max=64)
    ref = scipy.linalg.expm(-1j * H * 0.4) @ psi0
    assert np.linalg.norm(T.mps_to_vector_c(mps) - ref) > 1e-4


@pytest.mark.parametrize("move_right", [True, False])
def test_complex_split_is_the_best_rank_k_approximation(move_right):
    # Eckart-Young: the truncated split reproduces theta up to exactly the
    # discarded singular values; the isometric factor is orthonormal and the
    # other one carries the renormalised Schmidt values
    rng = np.random.default_rng(7)
    chl, d1, d2, chr_ = 5, 2, 3, 4
    theta = rng.standard_normal((chl, d1, d2, chr_)) + 1j * rng.standard_normal((chl, d1, d2, chr_))
    M = theta.reshape(chl * d1, d2 * chr_)
    S = np.linalg.svd(M, compute_uv=False)
    k = 4
    A1, A2, info = T.split_svd_c(theta, k, 0.0, move_right=move_right)
    assert info["keep"] == k
    kept = np.sqrt(np.sum(S[:k] ** 2))
    approx = np.tensordot(A1, A2, axes=([2], [0])).reshape(M.shape) * kept
    assert abs(np.linalg.norm(M - approx) ** 2 - np.sum(S[k:] ** 2)) <= 1e-12 * np.sum(S ** 2)
    assert abs(info["discarded"] - np.sum(S[k:] ** 2) / np.sum(S ** 2)) <= 1e-14
    if move_right:
        U = A1.reshape(chl * d1, k)
        assert np.abs(U.conj().T @ U - np.eye(k)).max() <= 1e-13
        sv = np.linalg.svd(A2.reshape(k, d2 * chr_), compute_uv=False)
    else:
        V = A2.reshape(k, d2 * chr_)
        assert np.abs(V @ V.conj().T - np.eye(k)).max() <= 1e-13
        sv = np.linalg.svd(A1.reshape(chl * d1, k), compute_uv=False)
    assert np.allclose(sv, S[:k] / kept, rtol=1e-12, atol=0)
