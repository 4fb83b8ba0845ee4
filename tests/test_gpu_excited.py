"""Excited states (eMPS, Eq. emps_lagrange): the projected Lanczos against the
lowest eigenvalue of the explicit H_eff restricted to the complement of the
projector rows, and whole excited-state sweeps against exact
diagonalisation (first and second excited energies, orthogonality)."""
import numpy as np
import pytest

from oracle import dmrg as od
from oracle import mpo as ompo
from paper_1703_00387_gb300 import binding as B
from paper_1703_00387_gb300 import hamiltonians, inputs

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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _operator(L, k, chi, seed):
    W = hamiltonians.xxz(L, 1.0, 1.0, 0.0)
    mps = od.right_canonicalize(inputs.random_mps(L, 2, chi, seed=seed))
    Renv = od.build_right_envs(W, mps)
    Lenv = np.ones((1, 1, 1))
    for j in range(k):
        chl, d, chr_ = mps[j].shape
        Q, Rm = np.linalg.qr(mps[j].reshape(chl * d, chr_))
        mps[j] = Q.reshape(chl, d, Q.shape[1])
        mps[j + 1] = np.tensordot(Rm, mps[j + 1], axes=([1], [0]))
        Lenv = od.env_left(Lenv, mps[j], W[j])
    theta = np.tensordot(mps[k], mps[k + 1], axes=([2], [0]))
    return Lenv, W[k], W[k + 1], Renv[k + 2], theta


@pytest.mark.parametrize("k", [0, 1, 3])
def test_projected_lanczos_matches_restricted_eigenvalue(ctx, k):
    Lh, W1, W2, Rh, th = _operator(10, 4, 8, seed=5)
    n = th.size
    H = np.zeros((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        H[:, c] = od.heff_apply(Lh, W1, W2, Rh, e.reshape(th.shape)).ravel()
    P = np.random.default_rng(7).standard_normal((k, n))
    if k:
        Q, _ = np.linalg.qr(P.T)
        C = np.linalg.svd(np.eye(n) - Q @ Q.T)[0][:, : n - k]  # basis of the complement
    else:
        C = np.eye(n)
    ref = np.linalg.eigvalsh(C.T @ H @ C)[0]
    t = dev(th.copy())
    e, it, res, conv = B.osmps_lanczos_ground_projected(ctx, dev(Lh), dev(W1), dev(W2), dev(Rh), t,
                                                        dev(P) if k else None, max_iter=200,
                                                        tol=1e-11, precision="fp64")
    assert conv and abs(e - ref) <= 1e-10 * abs(ref)
    v = t.cpu().numpy().ravel()
    if k:
        assert np.abs(P @ v).max() <= 1e-10 * np.abs(P).max() * np.sqrt(n)


def test_overlap_environment_gives_overlap(ctx):
    """The left overlap environment over all sites is <psi|phi> (dense check)."""
    L = 6
    a = inputs.random_mps(L, 2, 4, seed=1)
    b = inputs.random_mps(L, 2, 3, seed=2)
    o = dev(np.ones((1, 1)))
    for k in range(L):
        nxt = torch.empty((a[k].shape[2], b[k].shape[2]), dtype=torch.float64, device="cuda:0")
        B.osmps_overlap_env_update(ctx, 0, o, dev(a[k]), dev(b[k]), nxt)
        o = nxt
    def dense(m):
        v = m[0]
        for t in m[1:]:
            v = np.tensordot(v, t, axes=([v.ndim - 1], [0]))
        return v.ravel()
    ref = float(dense(a) @ dense(b))
    assert abs(float(o.cpu().numpy()[0, 0]) - ref) <= 1e-12 * max(1.0, abs(ref))
    o = dev(np.ones((1, 1)))
    for k in range(L - 1, -1, -1):
        nxt = torch.empty((a[k].shape[0], b[k].shape[0]), dtype=torch.float64, device="cuda:0")
        B.osmps_overlap_env_update(ctx, 1, o, dev(a[k]), dev(b[k]), nxt)
        o = nxt
    assert abs(float(o.cpu().numpy()[0, 0]) - ref) <= 1e-12 * max(1.0, abs(ref))


def test_excited_states_match_exact_diagonalisation(ctx):
    """TFI L=8, g=1.5 (gapped, non-degenerate low levels), exact bond
    dimension 16: ground state by the sweeps, then the first and second
    excited states by eMPS, each orthogonal to the ones below."""
    from paper_1703_00387_gb300.excited import excited_state
    L, g = 8, 1.5
    W = hamiltonians.ising(L, 1.0, g)
    ev = np.linalg.eigvalsh(ompo.mpo_to_dense(ompo.ising_mpo(L, 1.0, g)))
    mps = B.MPS(ctx, inputs.random_mps(L, 2, 16, seed=0), chi_cap=16)
    mpo = B.MPO(ctx, W)
    st = B.osmps_sweep(ctx, mps, mpo, B.sweep_params(16, 4, "fp64", lanczos_tol=1e-13), record_steps=False)
    assert abs(st["energy"] - ev[0]) <= 1e-10 * abs(ev[0])
    ground = mps.tensors()
    mps.close()
    mpo.close()
    r1 = excited_state(ctx, W, [ground], inputs.random_mps(L, 2, 16, seed=1), 16, n_sweeps=6,
                       lanczos_tol=1e-13)
    assert abs(r1["energy"] - ev[1]) <= 1e-9 * abs(ev[1])
    assert abs(r1["overlaps"][0]) <= 1e-9
    r2 = excited_state(ctx, W, [ground, r1["tensors"]], inputs.random_mps(L, 2, 16, seed=2), 16,
                       n_sweeps=6, lanczos_tol=1e-13)
    assert abs(r2["energy"] - ev[2]) <= 1e-9 * abs(ev[2])
    assert max(abs(x) for x in r2["overlaps"]) <= 1e-9
