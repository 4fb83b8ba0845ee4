"""GPU Krylov propagator exp(-i tau H_eff) theta (the local step of the
two-site TDVP) against the complex128 oracle, element by element."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mpo
from oracle import tdvp as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1703_00387_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(0)
    yield c
    c.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _operator(L, k, chi, seed, model="xxz"):
    """Complex environments around the pair (k, k+1) of a random complex MPS
    (left part left-canonical, right part right-canonical), the MPO tensors
    and the centre theta."""
    W = mpo.xxz_mpo(L, 1.0, 0.8, 0.3) if model == "xxz" else mpo.ising_mpo(L, 1.0, 1.1)
    rng = np.random.default_rng(seed)
    dims = [min(2 ** j, 2 ** (L - j), chi) for j in range(L + 1)]
    mps = [rng.standard_normal((dims[j], 2, dims[j + 1]))
           + 1j * rng.standard_normal((dims[j], 2, dims[j + 1])) for j in range(L)]
    mps = T.right_canonicalize_c(mps)
    Renv = T.build_right_envs_c(W, mps)
    Lenv = np.ones((1, 1, 1), dtype=np.complex128)
    for j in range(k):
        chl, d, chr_ = mps[j].shape
        Q, Rm = np.linalg.qr(mps[j].reshape(chl * d, chr_))
        mps[j] = Q.reshape(chl, d, Q.shape[1])
        mps[j + 1] = np.tensordot(Rm, mps[j + 1], axes=([1], [0]))
        Lenv = T.env_left_c(Lenv, mps[j], W[j])
    theta = np.tensordot(mps[k], mps[k + 1], axes=([2], [0]))
    return Lenv, W[k], W[k + 1], Renv[k + 2], theta


# (L, k, chi, seed): theta 1x2x2x2, 16x2x2x16 and 24x2x2x24 (ragged tiles)
CASES = [(3, 0, 8, 1), (10, 4, 24, 2), (12, 5, 24, 3)]


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-11), ("fp64emu", 1e-11), ("bf16x3", 3e-5)])
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("tau", [0.05, -0.2])
def test_heff_expm_matches_oracle(B, ctx, prec, bar, case, tau):
    Lh, W1, W2, Rh, theta = _operator(*case)
    mv = lambda x: T.heff2_apply(Lh, W1, W2, Rh, x)
    ref, m_ref, _ = T.krylov_expm(mv, theta, tau, max_iter=40, tol=1e-12)
    th = dev(theta)
    m, err, ok = B.osmps_heff_expm(ctx, dev(Lh), dev(W1), dev(W2), dev(Rh), th, tau,
                                   max_iter=40, tol=1e-12, precision=prec)
    got = th.cpu().numpy()
    assert ok
    assert np.linalg.norm(got - ref) <= bar * np.linalg.norm(ref)
    assert np.max(np.abs(got - ref)) <= bar * np.max(np.abs(ref)) * 4
    if prec != "bf16x3":
        assert abs(m - m_ref) <= 1
    # unitary: the norm is kept
    assert abs(np.linalg.norm(got) - np.linalg.norm(theta)) <= max(bar, 1e-12) * np.linalg.norm(theta)


def test_heff_expm_equals_matrix_exponential(B, ctx):
    # the dense matrix exponential of the explicit H_eff, not the oracle's Krylov loop
    Lh, W1, W2, Rh, theta = _operator(10, 4, 24, 7)
    n = theta.size
    H = np.einsum("xwa,wtsv,vuqz,yzc->xtuyasqc", Lh, W1, W2, Rh).reshape(n, n)
    assert np.abs(H - H.conj().T).max() <= 1e-12 * np.abs(H).max()
    tau = 0.1
    ref = (__import__("scipy.linalg").linalg.expm(-1j * tau * H) @ theta.reshape(-1)).reshape(theta.shape)
    th = dev(theta)
    m, err, ok = B.osmps_heff_expm(ctx, dev(Lh), dev(W1), dev(W2), dev(Rh), th, tau,
                                   max_iter=60, tol=1e-13, precision="fp64")
    assert ok and err <= 1e-13
    assert np.linalg.norm(th.cpu().numpy() - ref) <= 1e-11 * np.linalg.norm(ref)


def test_heff_expm_exhausted_space_is_exact(B, ctx):
    # n_c = 8 at the left end of an L = 3 chain: the Krylov space runs out
    Lh, W1, W2, Rh, theta = _operator(3, 0, 8, 4)
    n = theta.size
    H = np.einsum("xwa,wtsv,vuqz,yzc->xtuyasqc", Lh, W1, W2, Rh).reshape(n, n)
    import scipy.linalg
    ref = (scipy.linalg.expm(-0.7j * H) @ theta.reshape(-1)).reshape(theta.shape)
    th = dev(theta)
    m, err, ok = B.osmps_heff_expm(ctx, dev(Lh), dev(W1), dev(W2), dev(Rh), th, 0.7,
                                   max_iter=40, tol=0.0, precision="fp64")
    assert ok and m <= n and err <= 1e-13
    assert np.linalg.norm(th.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-11), ("bf16x3", 3e-5)])
def test_one_site_backward_step_matches_oracle(B, ctx, prec, bar):
    # the one-site H_eff as d2 = 1 with an identity second MPO tensor,
    # evolved backwards as in the TDVP sweep
    Lh, W1, _, _, _ = _operator(10, 4, 24, 5)
    Rh2 = _operator(10, 3, 24, 5)[3]  # R environment of sites 5..9 of the same state
    rng = np.random.default_rng(11)
    chl, chr_ = Lh.shape[0], Rh2.shape[0]
    wr = W1.shape[3]
    assert Rh2.shape[1] == wr
    C = rng.standard_normal((chl, 2, chr_)) + 1j * rng.standard_normal((chl, 2, chr_))
    mv = lambda x: T.heff1_apply(Lh, W1, Rh2, x)
    ref, _, _ = T.krylov_expm(mv, C, -0.05, max_iter=40, tol=1e-12)
    Wid = np.zeros((wr, 1, 1, wr))
    for w in range(wr):
        Wid[w, 0, 0, w] = 1.0
    th = dev(C.reshape(chl, 2, 1, chr_))
    m, err, ok = B.osmps_heff_expm(ctx, dev(Lh), dev(W1), dev(Wid), dev(Rh2), th, -0.05,
                                   max_iter=40, tol=1e-12, precision=prec)
    assert ok
    got = th.cpu().numpy().reshape(C.shape)
    assert np.linalg.norm(got - ref) <= bar * np.linalg.norm(ref)


def test_heff_expm_cap_and_validation(B, ctx):
    Lh, W1, W2, Rh, theta = _operator(10, 4, 24, 2)
    ops = [dev(x) for x in (Lh, W1, W2, Rh)]
    th = dev(theta)
    m, err, ok = B.osmps_heff_expm(ctx, *ops, th, 3.0, max_iter=3, tol=1e-14, precision="fp64")
    assert not ok and m == 3 and err > 1e-14
    # the capped result is still the 3-vector Krylov approximation of the oracle
    mv = lambda x: T.heff2_apply(Lh, W1, W2, Rh, x)
    ref, m_ref, _ = T.krylov_expm(mv, theta, 3.0, max_iter=3, tol=1e-14)
    assert m_ref == 3
    assert np.linalg.norm(th.cpu().numpy() - ref) <= 1e-11 * np.linalg.norm(ref)
    for kw in (dict(max_iter=0), dict(max_iter=129)):
        with pytest.raises(B.OsmpsError):
            B.osmps_heff_expm(ctx, *ops, dev(theta), 0.1, precision="fp64", **kw)
    with pytest.raises(B.OsmpsError):
        B.osmps_heff_expm(ctx, *ops, dev(theta), float("nan"), precision="fp64")
    with pytest.raises(B.OsmpsError):
        B.osmps_heff_expm(ctx, *ops, dev(np.zeros_like(theta)), 0.1, precision="fp64")


# ---------------------------------------------------------------------------
# Complex split and the whole TDVP evolution
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("move_right", [1, 0])
@pytest.mark.parametrize("chi_max", [5, 64])
def test_split_complex_matches_oracle(B, ctx, prec, move_right, chi_max):
    # precision only selects the float64 GEMM (DMMA or emulated): both exact
    rng = np.random.default_rng(21 + move_right)
    chl, d1, d2, chr_ = 6, 2, 2, 7
    theta = rng.standard_normal((chl, d1, d2, chr_)) + 1j * rng.standard_normal((chl, d1, d2, chr_))
    m, n = chl * d1, d2 * chr_
    kmax = min(chi_max, m, n)
    A1 = torch.zeros(m * kmax, dtype=torch.complex128, device="cuda")
    A2 = torch.zeros(kmax * n, dtype=torch.complex128, device="cuda")
    keep, disc, ent, lam2 = B.osmps_split_complex(ctx, dev(theta), A1, A2, move_right, chi_max,
                                                  0.0, precision=prec)
    a1, a2, info = T.split_svd_c(theta, chi_max, 0.0, move_right=bool(move_right))
    assert keep == info["keep"]
    # only the largest min(chi_max, rank) values are computed
    big = info["lam2"][:keep] > 1e-6
    assert np.allclose(lam2[:keep][big], info["lam2"][:keep][big], rtol=1e-11, atol=0)
    assert abs(disc - info["discarded"]) <= 1e-12
    assert abs(ent - info["entropy"]) <= 1e-11
    g1 = A1.cpu().numpy()[: m * keep].reshape(chl, d1, keep)
    g2 = A2.cpu().numpy()[: keep * n].reshape(keep, d2, chr_)
    # the product is gauge free (the kept singular vectors carry phases)
    rec = np.tensordot(g1, g2, axes=([2], [0]))
    ref = np.tensordot(a1, a2, axes=([2], [0]))
    assert np.linalg.norm(rec - ref) <= 1e-11 * np.linalg.norm(ref)
    if move_right:
        M = g1.reshape(m, keep)
        assert np.abs(M.conj().T @ M - np.eye(keep)).max() <= 1e-12
    else:
        M = g2.reshape(keep, n)
        assert np.abs(M @ M.conj().T - np.eye(keep)).max() <= 1e-12


def _rc_state(L, chi, seed):
    return T.right_canonicalize_c(_random_complex_mps_(L, chi, seed))


def _random_complex_mps_(L, chi, seed):
    rng = np.random.default_rng(seed)
    dims = [min(2 ** j, 2 ** (L - j), chi) for j in range(L + 1)]
    return [rng.standard_normal((dims[j], 2, dims[j + 1]))
            + 1j * rng.standard_normal((dims[j], 2, dims[j + 1])) for j in range(L)]


@pytest.mark.parametrize("model", ["xxz", "ising"])
def test_tdvp_full_bond_dimension_is_exact_evolution(B, ctx, model):
    import scipy.linalg
    L = 6
    W = mpo.xxz_mpo(L, 1.0, 0.5, 0.2) if model == "xxz" else mpo.ising_mpo(L, 1.0, 1.2)
    H = mpo.mpo_to_dense(W)
    mps0 = _rc_state(L, 64, 1)
    psi0 = T.mps_to_vector_c(mps0)
    dt, n = 0.1, 4
    h = B.MPO(ctx, W)
    out, energy, norm, stats = B.osmps_tdvp_evolve(ctx, h, mps0, dt, n, chi_max=64,
                                                   krylov_tol=1e-13, precision="fp64")
    ref = scipy.linalg.expm(-1j * H * dt * n) @ psi0
    assert np.linalg.norm(T.mps_to_vector_c(out) - ref) <= 1e-9
    e0 = np.vdot(psi0, H @ psi0).real
    assert np.all(np.abs(energy - e0) <= 1e-10 * max(1.0, abs(e0)))
    assert np.all(np.abs(norm - 1.0) <= 1e-12)
    assert stats["nonconverged"] == 0 and stats["krylov_calls"] == n * (2 * (L - 1) + 2 * (L - 2))


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-9), ("fp64emu", 1e-9), ("bf16x3", 1e-4)])
def test_tdvp_truncated_matches_oracle(B, ctx, prec, bar):
    # L = 10 XXZ with a field (no Schmidt multiplets at the cut), complex random
    # start with bond dimension 2, chi_max = 6: both sides truncate the same way
    L = 10
    W = mpo.xxz_mpo(L, 1.0, 0.7, 0.35)
    mps0 = _rc_state(L, 2, 5)
    dt, n, chi = 0.05, 6, 6
    ref_mps, ref_hist = T.tdvp2_evolve(W, mps0, dt, n, chi_max=chi, krylov_tol=1e-13)
    h = B.MPO(ctx, W)
    out, energy, norm, stats = B.osmps_tdvp_evolve(ctx, h, mps0, dt, n, chi_max=chi,
                                                   krylov_tol=1e-13, precision=prec)
    assert [A.shape for A in out] == [A.shape for A in ref_mps]
    psi, ref = T.mps_to_vector_c(out), T.mps_to_vector_c(ref_mps)
    assert np.linalg.norm(psi - ref) <= bar
    assert np.allclose(energy, [e for _, e, _ in ref_hist], rtol=0, atol=bar * 10)
    assert stats["max_chi"] == chi


def test_tdvp_ground_state_gains_only_a_phase(B, ctx):
    # a GPU DMRG ground state evolved on the GPU: psi(t) = exp(-i E0 t) psi0
    L = 10
    W = mpo.ising_mpo(L, 1.0, 1.0)
    rng = np.random.default_rng(0)
    from oracle import dmrg as od
    dims = od.initial_bond_dims(L, 2, 16)
    start = [rng.standard_normal((dims[k], 2, dims[k + 1])) for k in range(L)]
    E0, gs, _ = od.dmrg(W, start, chi_max=16, n_sweeps=4)
    gs_c = T.right_canonicalize_c(gs)
    psi0 = T.mps_to_vector_c(gs_c)
    dt, n = 0.05, 4
    h = B.MPO(ctx, W)
    out, energy, norm, _ = B.osmps_tdvp_evolve(ctx, h, gs_c, dt, n, chi_max=16, eps_local=1e-14,
                                               krylov_tol=1e-13, precision="fp64")
    ov = np.vdot(psi0, T.mps_to_vector_c(out))
    assert abs(abs(ov) - 1.0) <= 1e-8
    assert abs(np.angle(ov * np.exp(1j * E0 * dt * n))) <= 1e-8
    assert np.all(np.abs(energy - E0) <= 1e-9 * abs(E0))


# ---------------------------------------------------------------------------
# Edge cases of the evolution
# ---------------------------------------------------------------------------


def _random_rc(L, d, chi, seed):
    rng = np.random.default_rng(seed)
    dims = [min(d ** j, d ** (L - j), chi) for j in range(L + 1)]
    return T.right_canonicalize_c([rng.standard_normal((dims[j], d, dims[j + 1]))
                                   + 1j * rng.standard_normal((dims[j], d, dims[j + 1]))
                                   for j in range(L)])


@pytest.mark.parametrize("L,model", [(2, "xxz"), (4, "aklt")])
def test_tdvp_short_chains_and_spin_one_are_exact(B, ctx, L, model):
    # L = 2: one pair, no one-site steps; spin-1 AKLT (d = 3, w = 14) at L = 4
    import scipy.linalg
    W = mpo.xxz_mpo(L, 1.0, 0.6, 0.4) if model == "xxz" else mpo.aklt_mpo(L)
    d = W[0].shape[1]
    H = mpo.mpo_to_dense(W)
    mps0 = _random_rc(L, d, 64, seed=8)
    psi0 = T.mps_to_vector_c(mps0)
    dt, n = 0.07, 3
    out, energy, norm, stats = B.osmps_tdvp_evolve(ctx, B.MPO(ctx, W), mps0, dt, n, chi_max=64,
                                                   krylov_tol=1e-13, precision="fp64")
    ref = scipy.linalg.expm(-1j * H * dt * n) @ psi0
    assert np.linalg.norm(T.mps_to_vector_c(out) - ref) <= 1e-9
    assert stats["krylov_calls"] == n * (2 * (L - 1) + 2 * max(L - 2, 0))


def test_tdvp_product_manifold_chi1_matches_oracle(B, ctx):
    # chi_max = 1: both sides keep the leading Schmidt vector at every split
    L = 6
    W = mpo.xxz_mpo(L, 1.0, 0.5, 0.8)
    rng = np.random.default_rng(4)
    mps0 = T.right_canonicalize_c([rng.standard_normal((1, 2, 1)) + 1j * rng.standard_normal((1, 2, 1))
                                   for _ in range(L)])
    ref_mps, _ = T.tdvp2_evolve(W, mps0, 0.05, 3, chi_max=1, krylov_tol=1e-13)
    out, _, norm, stats = B.osmps_tdvp_evolve(ctx, B.MPO(ctx, W), mps0, 0.05, 3, chi_max=1,
                                              krylov_tol=1e-13, precision="fp64")
    assert stats["max_chi"] == 1
    assert np.linalg.norm(T.mps_to_vector_c(out) - T.mps_to_vector_c(ref_mps)) <= 1e-9
    assert np.all(np.abs(norm - 1.0) <= 1e-12)


def test_tdvp_krylov_cap_matches_oracle(B, ctx):
    # a cap of 3 Krylov vectors stops most propagators early; the capped
    # approximation is still the same on both sides
    L = 8
    W = mpo.ising_mpo(L, 1.0, 1.3)
    mps0 = _random_rc(L, 2, 8, seed=12)
    ref_mps, _ = T.tdvp2_evolve(W, mps0, 0.2, 2, chi_max=8, krylov_tol=1e-14, krylov_max_iter=3)
    out, _, _, stats = B.osmps_tdvp_evolve(ctx, B.MPO(ctx, W), mps0, 0.2, 2, chi_max=8,
                                           krylov_tol=1e-14, krylov_max_iter=3, precision="fp64")
    assert stats["nonconverged"] > 0 and stats["max_krylov"] == 3
    assert np.linalg.norm(T.mps_to_vector_c(out) - T.mps_to_vector_c(ref_mps)) <= 1e-9


def test_tdvp_zero_steps_and_validation(B, ctx):
    L = 5
    W = mpo.ising_mpo(L, 1.0, 1.0)
    h = B.MPO(ctx, W)
    mps0 = _random_rc(L, 2, 4, seed=2)
    scaled = [A.copy() for A in mps0]
    scaled[0] = 3.0 * scaled[0]  # the centre is normalised on entry
    out, e, nrm, stats = B.osmps_tdvp_evolve(ctx, h, scaled, 0.1, 0, chi_max=4, precision="fp64")
    assert len(e) == 0 and stats["krylov_calls"] == 0
    assert np.linalg.norm(T.mps_to_vector_c(out) - T.mps_to_vector_c(mps0)) <= 1e-13
    with pytest.raises(B.OsmpsError):  # a bond above chi_max
        B.osmps_tdvp_evolve(ctx, h, mps0, 0.1, 1, chi_max=2, precision="fp64")
    with pytest.raises(B.OsmpsError):
        B.osmps_tdvp_evolve(ctx, h, mps0, float("nan"), 1, chi_max=4, precision="fp64")
    with pytest.raises(B.OsmpsError):
        B.osmps_tdvp_evolve(ctx, h, mps0, 0.1, 1, chi_max=4, krylov_max_iter=200, precision="fp64")
