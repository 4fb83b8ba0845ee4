"""Plain FP64 two-site variational ground-state search (Sec. 3.4 of the paper).

Tensor conventions (shared with the GPU library only as a documented
interface, never as code):

* MPS site tensor ``A[a, s, b]`` (left bond, physical, right bond), Eq. mps.
* MPO site tensor ``W[w, t, s, w2]`` (see ``oracle.mpo``).
* Environments ``L[a2, w, a]`` and ``R[b2, w, b]``: first index bra
  (conjugated MPS), middle index MPO bond, last index ket. The boundary
  environments are ``ones((1, 1, 1))``.
* Two-site tensor ``theta[a, s1, s2, c]``.

All arithmetic is float64, with ``numpy.tensordot`` as the contraction step.
"""
import numpy as np
import scipy.linalg

# ----------------------------------------------------------------------------
# Canonical forms (Eq. oc) and shifting of the orthogonality centre by QR/RQ
# ----------------------------------------------------------------------------


def right_canonicalize(mps):
    """Move the orthogonality centre to site 0 by RQ decompositions from the
    right (the 'shifting' operation of Sec. 2) and normalise the state.

    Every site k >= 1 becomes right-canonical: sum_{s,b} A[a,s,b] A[a2,s,b] =
    delta(a, a2). Returns a new list; bond dimensions may shrink to the rank.
    The state is only defined up to a scalar, so the site receiving R is
    rescaled to unit norm at each shift; otherwise the norm of a long random
    chain (about sqrt(d chi^2) per site) overflows float64.
    """
    mps = [np.array(A, dtype=np.float64, copy=True) for A in mps]
    for k in range(len(mps) - 1, 0, -1):
        chl, d, chr_ = mps[k].shape
        M = mps[k].reshape(chl, d * chr_)
        Q, Rm = np.linalg.qr(M.T)  # M = Rm^T Q^T, rows of Q^T orthonormal
        m = Q.shape[1]
        mps[k] = Q.T.reshape(m, d, chr_)
        mps[k - 1] = np.tensordot(mps[k - 1], Rm.T, axes=([2], [0]))
        mps[k - 1] = mps[k - 1] / np.linalg.norm(mps[k - 1])
    mps[0] = mps[0] / np.linalg.norm(mps[0])
    return mps


def left_isometry_defect(A):
    """max |sum_{a,s} A[a,s,b] A[a,s,b2] - delta| (left-canonical condition, Eq. oc)."""
    chl, d, chr_ = A.shape
    M = A.reshape(chl * d, chr_)
    return float(np.max(np.abs(M.T @ M - np.eye(chr_))))


def right_isometry_defect(A):
    """max |sum_{s,b} A[a,s,b] A[a2,s,b] - delta| (right-canonical condition, Eq. oc)."""
    chl, d, chr_ = A.shape
    M = A.reshape(chl, d * chr_)
    return float(np.max(np.abs(M @ M.T - np.eye(chl))))


# ----------------------------------------------------------------------------
# Environments (the fixed sites contracted into L and R, Sec. 3.4)
# ----------------------------------------------------------------------------


def env_left(Lenv, A, W):
    """Grow the left environment by one site:
    L2[b2, w2, b] = sum A[a2,t,b2] L[a2,w,a] W[w,t,s,w2] A[a,s,b]."""
    X = np.tensordot(Lenv, A, axes=([2], [0]))        # [a2, w, s, b]
    Y = np.tensordot(X, W, axes=([1, 2], [0, 2]))     # [a2, b, t, w2]
    Ln = np.tensordot(A, Y, axes=([0, 1], [0, 2]))    # [b2, b, w2]
    return np.ascontiguousarray(Ln.transpose(0, 2, 1))


def env_right(Renv, A, W):
    """Grow the right environment by one site:
    R2[a2, w, a] = sum A[a2,t,b2] W[w,t,s,w2] R[b2,w2,b] A[a,s,b]."""
    X = np.tensordot(A, Renv, axes=([2], [2]))        # [a, s, b2, w2]
    Y = np.tensordot(X, W, axes=([1, 3], [2, 3]))     # [a, b2, w, t]
    Rn = np.tensordot(A, Y, axes=([1, 2], [3, 1]))    # [a2, a, w]
    return np.ascontiguousarray(Rn.transpose(0, 2, 1))


# ----------------------------------------------------------------------------
# Effective Hamiltonian (Fig. LanczosMPS): contract L, M^[k], M^[k+1], R with
# theta step by step instead of forming the chi^2 d^2 square matrix.
# ----------------------------------------------------------------------------


def heff_apply(Lenv, W1, W2, Renv, theta):
    """y[a2,t1,t2,c2] = sum L[a2,w,a] W1[w,t1,s1,w1] W2[w1,t2,s2,w2] R[c2,w2,c] theta[a,s1,s2,c]."""
    T1 = np.tensordot(Lenv, theta, axes=([2], [0]))       # [a2, w, s1, s2, c]
    T2 = np.tensordot(T1, W1, axes=([1, 2], [0, 2]))      # [a2, s2, c, t1, w1]
    T3 = np.tensordot(T2, W2, axes=([4, 1], [0, 2]))      # [a2, c, t1, t2, w2]
    y = np.tensordot(T3, Renv, axes=([4, 1], [1, 2]))     # [a2, t1, t2, c2]
    return y


def heff_dense(Lenv, W1, W2, Renv):
    """The effective Hamiltonian as an explicit (chi_l d1 d2 chi_r)^2 matrix,
    for small test cases only: H[(a2 t1 t2 c2), (a s1 s2 c)]."""
    H = np.einsum("xwa,wtsv,vuqz,yzc->xtuyasqc", Lenv, W1, W2, Renv)
    n = Lenv.shape[0] * W1.shape[1] * W2.shape[1] * Renv.shape[0]
    return H.reshape(n, n)


# ----------------------------------------------------------------------------
# Lanczos (Sec. 3.4: lowest eigenpair of H_eff from matrix-vector products)
# ----------------------------------------------------------------------------


def lanczos_ground(matvec, v0, max_iter=100, tol=1e-12):
    """Lowest eigenpair of a symmetric operator by Lanczos with full
    reorthogonalisation (two classical Gram-Schmidt passes per step).

    Stops when the residual estimate beta_j |s_j| of the lowest Ritz pair is
    <= tol, when max_iter Krylov vectors have been used, or when the Krylov
    space is exhausted. Returns (energy, normalised Ritz vector, iterations,
    residual estimate).
    """
    shape = v0.shape
    n = v0.size
    V = [np.ravel(v0) / np.linalg.norm(v0)]
    alpha, beta = [], []
    e, s, resid = None, None, None
    for j in range(max_iter):
        w = np.ravel(matvec(V[j].reshape(shape)))
        a = float(V[j] @ w)
        alpha.append(a)
        w = w - a * V[j]
        if j > 0:
            w = w - beta[-1] * V[j - 1]
        Vm = np.array(V)
        for _ in range(2):
            w = w - Vm.T @ (Vm @ w)
        b = float(np.linalg.norm(w))
        if j == 0:
            e, s = alpha[0], np.array([1.0])
        else:
            ev, es = scipy.linalg.eigh_tridiagonal(
                np.array(alpha), np.array(beta), select="i", select_range=(0, 0))
            e, s = float(ev[0]), es[:, 0]
        resid = b * abs(s[-1])
        if resid <= tol or j + 1 == max_iter or j + 1 == n or b == 0.0:
            break
        beta.append(b)
        V.append(w / b)
    x = np.array(V[: len(s)]).T @ s
    x = x / np.linalg.norm(x)
    return e, x.reshape(shape), len(alpha), resid


# ----------------------------------------------------------------------------
# Splitting and truncation (Sec. 2: SVD / eigendecomposition, Eq. elocal)
# ----------------------------------------------------------------------------


def truncation_rank(lam2, chi_max, eps_local):
    """Number of Schmidt values to keep.

    lam2: squared Schmidt values in descending order, normalised to sum 1.
    Keeps n = min(chi_max, smallest n >= 1 whose discarded weight
    sum_{i >= n} lam2_i is <= eps_local): the local tolerance decides unless
    the maximal bond dimension is reached first (Sec. 3.4).
    """
    lam2 = np.clip(np.asarray(lam2, dtype=np.float64), 0.0, None)
    tail = np.concatenate([np.cumsum(lam2[::-1])[::-1], [0.0]])  # tail[n] = sum_{i>=n}
    n = 1
    while n < len(lam2) and tail[n] > eps_local:
        n += 1
    return int(min(chi_max, n))


def split_svd(theta, chi_max, eps_local, move_right=True):
    """Split theta[a,s1,s2,c] by an SVD of the (a s1) x (s2 c) matrix (Sec. 2).

    move_right=True (left-to-right sweep): A_k = U (left-canonical),
    A_{k+1} = lambda' V (orthogonality centre moves to k+1).
    move_right=False: A_{k+1} = V (right-canonical), A_k = U lambda'.
    lambda' are the kept Schmidt values renormalised (appendix on the overlap).
    Returns (A_k, A_{k+1}, info) with info = dict(lam2 (all, normalised),
    keep, discarded, entropy).
    """
    chl, d1, d2, chr_ = theta.shape
    M = theta.reshape(chl * d1, d2 * chr_)
    U, S, Vt = scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesdd")
    lam2 = S ** 2 / np.sum(S ** 2)
    keep = truncation_rank(lam2, chi_max, eps_local)
    lamk = S[:keep] / np.sqrt(np.sum(S[:keep] ** 2))
    if move_right:
        Ak = U[:, :keep].reshape(chl, d1, keep)
        Ak1 = (lamk[:, None] * Vt[:keep]).reshape(keep, d2, chr_)
    else:
        Ak1 = Vt[:keep].reshape(keep, d2, chr_)
        Ak = (U[:, :keep] * lamk[None, :]).reshape(chl, d1, keep)
    info = dict(lam2=lam2, keep=keep, discarded=float(np.sum(lam2[keep:])),
                entropy=bond_entropy(lam2[:keep] / np.sum(lam2[:keep])))
    return Ak, Ak1, info


def split_eig(theta, chi_max, eps_local, move_right=True):
    """Split theta by the eigendecomposition route of Eq. AAD_ULLUD.

    move_right=True: G = M M^T = U lambda^2 U^T; A_k = U (kept columns,
    descending lambda); A_{k+1} = U^T M (= lambda V, Eq. ThetaAL), renormalised.
    move_right=False: G = M^T M = V lambda^2 V^T; A_{k+1} = V^T; A_k = M V.
    """
    chl, d1, d2, chr_ = theta.shape
    M = theta.reshape(chl * d1, d2 * chr_)
    G = M @ M.T if move_right else M.T @ M
    ev, Q = np.linalg.eigh(G)
    order = np.argsort(ev)[::-1]
    ev, Q = ev[order], Q[:, order]
    ev = np.clip(ev, 0.0, None)
    lam2 = ev / np.sum(ev)
    keep = truncation_rank(lam2, chi_max, eps_local)
    Qk = Q[:, :keep]
    if move_right:
        Ak = Qk.reshape(chl, d1, keep)
        B = Qk.T @ M
        Ak1 = (B / np.linalg.norm(B)).reshape(keep, d2, chr_)
    else:
        Ak1 = Qk.T.reshape(keep, d2, chr_)
        B = M @ Qk
        Ak = (B / np.linalg.norm(B)).reshape(chl, d1, keep)
    info = dict(lam2=lam2, keep=keep, discarded=float(np.sum(lam2[keep:])),
                entropy=bond_entropy(lam2[:keep] / np.sum(lam2[:keep])))
    return Ak, Ak1, info


def bond_entropy(lam2):
    """Von Neumann bond entropy S = -sum lambda^2 log lambda^2 (Sec. 2)."""
    p = np.asarray(lam2, dtype=np.float64)
    p = p[p > 0.0]
    return float(-np.sum(p * np.log(p)))


# ----------------------------------------------------------------------------
# Whole-state quantities
# ----------------------------------------------------------------------------


def mps_to_vector(mps):
    """Contract an MPS (Eq. mps) to its d^L state vector, site 1 most significant."""
    v = mps[0]
    for A in mps[1:]:
        v = np.tensordot(v, A, axes=([v.ndim - 1], [0]))
    return v.reshape(-1)


def mpo_expectation(W, mps):
    """<psi|H|psi> by contracting the full MPO sandwich from the left."""
    env = np.ones((1, 1, 1))
    for A, Wk in zip(mps, W):
        env = env_left(env, A, Wk)
    return float(env[0, 0, 0])


def mps_norm2(mps):
    env = np.ones((1, 1))
    for A in mps:
        env = np.tensordot(np.tensordot(env, A, axes=([1], [0])), A, axes=([0, 1], [0, 1]))
    return float(env[0, 0])


def mps_energy(W, mps):
    """E = <psi|H|psi> / <psi|psi> in FP64."""
    return mpo_expectation(W, mps) / mps_norm2(mps)


def initial_bond_dims(L, d, chi_init):
    """chi_k = min(d^k, d^(L-k), chi_init) for the L+1 bonds (chi_0 = chi_L = 1)."""
    return [int(min(d ** k, d ** (L - k), chi_init)) for k in range(L + 1)]


# ----------------------------------------------------------------------------
# Two-site sweeps (Sec. 3.4)
# ----------------------------------------------------------------------------


def build_right_envs(W, mps):
    """R environments for a right-canonical MPS: Renv[k] covers sites k..L-1."""
    L = len(mps)
    Renv = [None] * (L + 1)
    Renv[L] = np.ones((1, 1, 1))
    for k in range(L - 1, 0, -1):
        Renv[k] = env_right(Renv[k + 1], mps[k], W[k])
    return Renv


def two_site_step(W, mps, Lenv, Renv, k, move_right, chi_max, eps_local,
                  lanczos_tol, lanczos_max_iter, split="svd"):
    """One optimisation of the pair (k, k+1): form theta, Lanczos on H_eff,
    split with truncation, update the environment on the side the centre
    leaves. Modifies mps/Lenv/Renv in place; returns a stats dict."""
    theta = np.tensordot(mps[k], mps[k + 1], axes=([2], [0]))
    mv = lambda x: heff_apply(Lenv[k], W[k], W[k + 1], Renv[k + 2], x)
    E, theta, iters, resid = lanczos_ground(mv, theta, lanczos_max_iter, lanczos_tol)
    splitter = split_svd if split == "svd" else split_eig
    Ak, Ak1, info = splitter(theta, chi_max, eps_local, move_right)
    mps[k], mps[k + 1] = Ak, Ak1
    if move_right:
        Lenv[k + 1] = env_left(Lenv[k], Ak, W[k])
    else:
        Renv[k + 1] = env_right(Renv[k + 2], Ak1, W[k + 1])
    return dict(k=k, energy=E, iters=iters, resid=resid, keep=info["keep"],
                discarded=info["discarded"], entropy=info["entropy"])


def dmrg(W, mps0, chi_max, n_sweeps, eps_local=None, lanczos_tol=1e-12,
         lanczos_max_iter=100, split="svd"):
    """Two-site variational ground-state search.

    One sweep optimises the pairs (0,1)...(L-2,L-1) left to right, then
    (L-2,L-1)...(0,1) right to left, so every pair is optimised twice
    (2(L-1) steps). The initial MPS is right-canonicalised first. eps_local
    defaults to 1e-12 / (4 L), the paper's default with a variance target of
    1e-12. Returns (final FP64 MPO energy, mps, list of per-step stats).
    """
    L = len(W)
    if eps_local is None:
        eps_local = 1e-12 / (4 * L)
    mps = right_canonicalize(mps0)
    Renv = build_right_envs(W, mps)
    Lenv = [None] * (L + 1)
    Lenv[0] = np.ones((1, 1, 1))
    history = []
    for _ in range(n_sweeps):
        for k in range(0, L - 1):
            history.append(two_site_step(W, mps, Lenv, Renv, k, True, chi_max, eps_local,
                                         lanczos_tol, lanczos_max_iter, split))
        for k in range(L - 2, -1, -1):
            history.append(two_site_step(W, mps, Lenv, Renv, k, False, chi_max, eps_local,
                                         lanczos_tol, lanczos_max_iter, split))
    return mps_energy(W, mps), mps, history
