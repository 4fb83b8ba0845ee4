"""Plain complex128 two-site time-dependent variational principle (Sec. 5.4);
the local propagators are the Krylov approximation of Sec. 5.2 (Eq. propSE,
Eq. krylov:approx), applied to the centre tensor only, as the appendix on the
details of the Krylov method shows is exact in canonical form.

TEST INFRASTRUCTURE, like the rest of ``oracle``: only tests, ``smoke()`` and
the bench's CPU legs use it; it shares no code with the GPU library.

The paper names the method (the two-site TDVP of Haegeman et al., which lets
the bond dimension grow and propagates with the many-body operator projected
onto a local subspace) without printing its steps. This module takes the
standard symmetric second-order two-site scheme of that reference, in the
conventions of ``oracle.dmrg``:

* one time step dt = a left-to-right half sweep with dt/2 and a right-to-left
  half sweep with dt/2;
* left to right, at the pair (k, k+1): theta = A_k A_{k+1}, evolve
  theta <- exp(-i H_eff dt/2) theta, split theta = U S V^dagger (truncated as
  in the ground-state search), A_k = U, grow the left environment; unless
  k+1 is the last site, evolve the centre C = S V^dagger backwards,
  C <- exp(+i H1_eff dt/2) C, with the one-site effective Hamiltonian of
  site k+1; A_{k+1} = C;
* right to left mirrored: A_{k+1} = V^dagger, grow the right environment,
  C = U S evolved backwards at site k unless k = 0.

Complex tensors keep the index conventions of ``oracle.dmrg``. The bra of an
environment is the complex conjugate of the site tensor:
L2[b2,w2,b] = sum conj(A[a2,t,b2]) L[a2,w,a] W[w,t,s,w2] A[a,s,b].
"""
import numpy as np
import scipy.linalg

from .dmrg import bond_entropy, truncation_rank

# ----------------------------------------------------------------------------
# Complex environments and effective Hamiltonians
# ----------------------------------------------------------------------------


def env_left_c(Lenv, A, W):
    """L2[b2,w2,b] = sum conj(A[a2,t,b2]) L[a2,w,a] W[w,t,s,w2] A[a,s,b]."""
    X = np.tensordot(Lenv, A, axes=([2], [0]))              # [a2, w, s, b]
    Y = np.tensordot(X, W, axes=([1, 2], [0, 2]))           # [a2, b, t, w2]
    Ln = np.tensordot(np.conj(A), Y, axes=([0, 1], [0, 2]))  # [b2, b, w2]
    return np.ascontiguousarray(Ln.transpose(0, 2, 1))


def env_right_c(Renv, A, W):
    """R2[a2,w,a] = sum conj(A[a2,t,b2]) W[w,t,s,w2] R[b2,w2,b] A[a,s,b]."""
    X = np.tensordot(A, Renv, axes=([2], [2]))              # [a, s, b2, w2]
    Y = np.tensordot(X, W, axes=([1, 3], [2, 3]))           # [a, b2, w, t]
    Rn = np.tensordot(np.conj(A), Y, axes=([1, 2], [3, 1]))  # [a2, a, w]
    return np.ascontiguousarray(Rn.transpose(0, 2, 1))


def heff2_apply(Lenv, W1, W2, Renv, theta):
    """Two-site H_eff.theta, the same contraction as the ground-state search:
    y[a2,t1,t2,c2] = sum L[a2,w,a] W1[w,t1,s1,w1] W2[w1,t2,s2,w2] R[c2,w2,c] theta[a,s1,s2,c]."""
    T1 = np.tensordot(Lenv, theta, axes=([2], [0]))       # [a2, w, s1, s2, c]
    T2 = np.tensordot(T1, W1, axes=([1, 2], [0, 2]))      # [a2, s2, c, t1, w1]
    T3 = np.tensordot(T2, W2, axes=([4, 1], [0, 2]))      # [a2, c, t1, t2, w2]
    return np.tensordot(T3, Renv, axes=([4, 1], [1, 2]))  # [a2, t1, t2, c2]


def heff1_apply(Lenv, W, Renv, x):
    """One-site H_eff.x: y[a2,t,c2] = sum L[a2,w,a] W[w,t,s,w2] R[c2,w2,c] x[a,s,c]."""
    T1 = np.tensordot(Lenv, x, axes=([2], [0]))          # [a2, w, s, c]
    T2 = np.tensordot(T1, W, axes=([1, 2], [0, 2]))      # [a2, c, t, w2]
    return np.tensordot(T2, Renv, axes=([3, 1], [1, 2]))  # [a2, t, c2]


# ----------------------------------------------------------------------------
# Krylov propagator (Eq. krylov:approx)
# ----------------------------------------------------------------------------


def _expm_tridiag_e1(alpha, beta, tau):
    """exp(-i tau T) e_1 for the real symmetric tridiagonal T (diagonal alpha,
    off-diagonal beta), through its eigendecomposition T = S diag(l) S^T."""
    if len(alpha) == 1:
        return np.array([np.exp(-1j * tau * alpha[0])])
    lam, S = scipy.linalg.eigh_tridiagonal(alpha, beta)
    return S @ (np.exp(-1j * tau * lam) * S[0, :])


def krylov_expm(matvec, v0, tau, max_iter=40, tol=1e-12):
    """exp(-i tau H) v0 for a Hermitian operator H given by matvec (Eq. propSE,
    Eq. krylov:approx).

    The Krylov basis V = [v_1, v_2, ...] starts from v_1 = v0/||v0|| and is
    built by the Lanczos recurrence with full reorthogonalisation (two
    classical Gram-Schmidt passes, complex inner products), so V^dagger H V is
    the real tridiagonal T. With m vectors the result is
    ||v0|| V exp(-i tau T_m) e_1. The basis stops growing when the weight that
    would leave the space, beta_m |[exp(-i tau T_m) e_1]_m|, is <= tol, when
    the Krylov space is exhausted (beta_m = 0 up to rounding: the result is
    then exact), or at max_iter vectors.

    Returns (vector, number of basis vectors, last error estimate).
    """
    shape = v0.shape
    nrm = np.linalg.norm(v0)
    V = [np.asarray(v0, dtype=np.complex128).reshape(-1) / nrm]
    alpha, beta = [], []
    n = V[0].size
    for j in range(min(max_iter, n)):
        w = matvec(V[j].reshape(shape)).reshape(-1).astype(np.complex128)
        alpha.append(float(np.real(np.vdot(V[j], w))))
        B = np.array(V)
        for _ in range(2):
            w = w - B.T @ (np.conj(B) @ w)
        b = float(np.linalg.norm(w))
        u = _expm_tridiag_e1(np.array(alpha), np.array(beta), tau)
        err = b * abs(u[-1])
        scale = max(abs(a) for a in alpha) + (max(beta) if beta else 0.0)
        exhausted = b <= 1e-14 * max(scale, 1e-300)
        if exhausted or err <= tol or j + 1 == min(max_iter, n):
            x = np.array(V).T @ u
            return (nrm * x).reshape(shape), j + 1, (0.0 if exhausted else err)
        beta.append(b)
        V.append(w / b)
    raise AssertionError("unreachable")


# ----------------------------------------------------------------------------
# Split with truncation (the SVD form of Sec. 2, complex)
# ----------------------------------------------------------------------------


def split_svd_c(theta, chi_max, eps_local, move_right=True):
    """theta[a,s1,s2,c] = U S V^dagger over (a s1) x (s2 c), truncated by the
    ground-state search's rule (``truncation_rank``) and the kept Schmidt
    values renormalised. move_right: returns (U, S V^dagger, info);
    otherwise (U S, V^dagger, info)."""
    chl, d1, d2, chr_ = theta.shape
    M = theta.reshape(chl * d1, d2 * chr_)
    U, S, Vh = scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesdd")
    lam2 = S ** 2 / np.sum(S ** 2)
    keep = truncation_rank(lam2, chi_max, eps_local)
    lamk = S[:keep] / np.sqrt(np.sum(S[:keep] ** 2))
    if move_right:
        Ak = U[:, :keep].reshape(chl, d1, keep)
        C = (lamk[:, None] * Vh[:keep]).reshape(keep, d2, chr_)
    else:
        C = (U[:, :keep] * lamk[None, :]).reshape(chl, d1, keep)
        Ak = Vh[:keep].reshape(keep, d2, chr_)
    info = dict(lam2=lam2, keep=keep, discarded=float(np.sum(lam2[keep:])),
                entropy=bond_entropy(lam2[:keep] / np.sum(lam2[:keep])))
    return (Ak, C, info) if move_right else (C, Ak, info)


# ----------------------------------------------------------------------------
# Complex states
# ----------------------------------------------------------------------------


def right_canonicalize_c(mps):
    """Complex form of ``oracle.dmrg.right_canonicalize``: RQ decompositions
    from the right (M = R Q with Q's rows orthonormal, from the QR of
    M^dagger), every site k >= 1 right-canonical
    (sum_{s,b} A[a,s,b] conj(A[a2,s,b]) = delta), the state normalised."""
    mps = [np.array(A, dtype=np.complex128, copy=True) for A in mps]
    for k in range(len(mps) - 1, 0, -1):
        chl, d, chr_ = mps[k].shape
        M = mps[k].reshape(chl, d * chr_)
        Q, Rm = np.linalg.qr(M.conj().T)  # M = Rm^dagger Q^dagger
        m = Q.shape[1]
        mps[k] = Q.conj().T.reshape(m, d, chr_)
        mps[k - 1] = np.tensordot(mps[k - 1], Rm.conj().T, axes=([2], [0]))
        mps[k - 1] = mps[k - 1] / np.linalg.norm(mps[k - 1])
    mps[0] = mps[0] / np.linalg.norm(mps[0])
    return mps


def mps_to_vector_c(mps):
    """The d^L state vector of a complex MPS, site 1 most significant."""
    v = mps[0]
    for A in mps[1:]:
        v = np.tensordot(v, A, axes=([v.ndim - 1], [0]))
    return v.reshape(-1)


def mps_expectation_c(W, mps):
    """(<psi|H|psi>, <psi|psi>) by contracting the MPO sandwich from the left;
    <psi|H|psi> is real for a Hermitian MPO (its imaginary part is returned
    too, as a check)."""
    env = np.ones((1, 1, 1), dtype=np.complex128)
    nrm = np.ones((1, 1), dtype=np.complex128)
    for A, Wk in zip(mps, W):
        env = env_left_c(env, A, Wk)
        nrm = np.tensordot(np.tensordot(nrm, A, axes=([1], [0])), np.conj(A), axes=([0, 1], [0, 1]))
        nrm = nrm.T
    return complex(env[0, 0, 0]), float(np.real(nrm[0, 0]))


def build_right_envs_c(W, mps):
    """R environments of a right-canonical complex MPS: Renv[k] covers sites k..L-1."""
    L = len(mps)
    Renv = [None] * (L + 1)
    Renv[L] = np.ones((1, 1, 1), dtype=np.complex128)
    for k in range(L - 1, 0, -1):
        Renv[k] = env_right_c(Renv[k + 1], mps[k], W[k])
    return Renv


# ----------------------------------------------------------------------------
# Two-site TDVP time step
# ----------------------------------------------------------------------------


def tdvp2_step(W, mps, Lenv, Renv, dt, chi_max, eps_local=0.0, krylov_tol=1e-12,
               krylov_max_iter=40):
    """One second-order two-site TDVP step of length dt (see the module
    docstring). On entry the orthogonality centre is site 0, every other site
    right-canonical, Renv[k] built for k >= 2 and Lenv[0] the boundary; on
    exit the same holds for the evolved state. mps, Lenv, Renv are modified in
    place. Returns a list of per-pair stats."""
    L = len(mps)
    half = 0.5 * dt
    stats = []
    # left to right
    for k in range(0, L - 1):
        theta = np.tensordot(mps[k], mps[k + 1], axes=([2], [0]))
        mv = lambda x, k=k: heff2_apply(Lenv[k], W[k], W[k + 1], Renv[k + 2], x)
        theta, m2, e2 = krylov_expm(mv, theta, half, krylov_max_iter, krylov_tol)
        Ak, C, info = split_svd_c(theta, chi_max, eps_local, move_right=True)
        mps[k] = Ak
        Lenv[k + 1] = env_left_c(Lenv[k], Ak, W[k])
        m1 = 0
        if k + 1 < L - 1:
            mv1 = lambda x, k=k: heff1_apply(Lenv[k + 1], W[k + 1], Renv[k + 2], x)
            C, m1, _ = krylov_expm(mv1, C, -half, krylov_max_iter, krylov_tol)
        mps[k + 1] = C
        stats.append(dict(k=k, dir="R", krylov2=m2, krylov1=m1, err2=e2, keep=info["keep"],
                          discarded=info["discarded"]))
    # right to left
    for k in range(L - 2, -1, -1):
        theta = np.tensordot(mps[k], mps[k + 1], axes=([2], [0]))
        mv = lambda x, k=k: heff2_apply(Lenv[k], W[k], W[k + 1], Renv[k + 2], x)
        theta, m2, e2 = krylov_expm(mv, theta, half, krylov_max_iter, krylov_tol)
        C, Bk1, info = split_svd_c(theta, chi_max, eps_local, move_right=False)
        mps[k + 1] = Bk1
        Renv[k + 1] = env_right_c(Renv[k + 2], Bk1, W[k + 1])
        m1 = 0
        if k > 0:
            mv1 = lambda x, k=k: heff1_apply(Lenv[k], W[k], Renv[k + 1], x)
            C, m1, _ = krylov_expm(mv1, C, -half, krylov_max_iter, krylov_tol)
        mps[k] = C
        stats.append(dict(k=k, dir="L", krylov2=m2, krylov1=m1, err2=e2, keep=info["keep"],
                          discarded=info["discarded"]))
    return stats


def tdvp2_evolve(W, mps0, dt, n_steps, chi_max, eps_local=0.0, krylov_tol=1e-12,
                 krylov_max_iter=40):
    """n_steps TDVP steps of length dt from mps0 (right-canonicalised first).
    Returns (mps, list of (time, <H>, <psi|psi>) after each step)."""
    L = len(W)
    mps = right_canonicalize_c(mps0)
    Renv = build_right_envs_c(W, mps)
    Lenv = [None] * (L + 1)
    Lenv[0] = np.ones((1, 1, 1), dtype=np.complex128)
    history = []
    for n in range(n_steps):
        tdvp2_step(W, mps, Lenv, Renv, dt, chi_max, eps_local, krylov_tol, krylov_max_iter)
        e, nrm = mps_expectation_c(W, mps)
        history.append(((n + 1) * dt, e.real / nrm, nrm))
    return mps, history
