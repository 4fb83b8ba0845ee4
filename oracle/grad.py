"""Plain FP64 gradients for the differentiation workload (oracle side).

* ``heff_vjp``: for y = H_eff(L, W1, W2, R) theta (Fig. LanczosMPS) and an
  output cotangent gy, the cotangents of theta, W1 and W2. H_eff is linear
  in each of them, so each cotangent is the full contraction of gy with
  every other factor (written out step by step).
* ``energy_grad_W``: E = <psi|H|psi> / <psi|psi> for a fixed MPS, and the
  derivative of E with respect to every MPO site tensor W_k (Eq. mpo). H is
  linear in each W_k, so dE/dW_k[w,t,s,w2] = G_k / <psi|psi> with
  G_k = sum L_k[a2,w,a] A_k[a2,t,b2] A_k[a,s,b] R_{k+1}[b2,w2,b], the left
  and right environments built from the tensors as they are (no canonical
  form assumed).
* ``xxz_coupling_grads``: the chain rule from dE/dW_k to the site-dependent
  couplings J_i and fields h_i of the XXZ MPO built by ``oracle.mpo``; at a
  ground state these are the Hellmann-Feynman derivatives of the energy.
"""
import numpy as np

from . import dmrg, mpo


def heff_vjp(Lenv, W1, W2, Renv, theta, gy):
    """Returns (g_theta, g_W1, g_W2) of f = <gy, H_eff theta>."""
    # g_theta[a,s1,s2,c] = sum gy[a2,t1,t2,c2] L[a2,w,a] W1[w,t1,s1,w1] W2[w1,t2,s2,w2] R[c2,w2,c]
    X = np.tensordot(gy, Lenv, axes=([0], [0]))               # [t1, t2, c2, w, a]
    X = np.tensordot(X, W1, axes=([0, 3], [1, 0]))            # [t2, c2, a, s1, w1]
    X = np.tensordot(X, W2, axes=([0, 4], [1, 0]))            # [c2, a, s1, s2, w2]
    g_theta = np.tensordot(X, Renv, axes=([0, 4], [0, 1]))    # [a, s1, s2, c]
    # shared pieces
    T1 = np.tensordot(Lenv, theta, axes=([2], [0]))           # [a2, w, s1, s2, c]
    Q = np.tensordot(gy, Renv, axes=([3], [0]))               # [a2, t1, t2, w2, c]
    # g_W1[w,t1,s1,w1] = sum T1[a2,w,s1,s2,c] W2[w1,t2,s2,w2] Q[a2,t1,t2,w2,c]
    P = np.tensordot(Q, W2, axes=([2, 3], [1, 3]))            # [a2, t1, c, w1, s2]
    g_W1 = np.tensordot(T1, P, axes=([0, 3, 4], [0, 4, 2]))   # [w, s1, t1, w1]
    g_W1 = np.ascontiguousarray(g_W1.transpose(0, 2, 1, 3))
    # g_W2[w1,t2,s2,w2] = sum T2[a2,t1,w1,s2,c] Q[a2,t1,t2,w2,c]
    T2 = np.tensordot(T1, W1, axes=([1, 2], [0, 2]))          # [a2, s2, c, t1, w1]
    g_W2 = np.tensordot(T2, Q, axes=([0, 3, 2], [0, 1, 4]))   # [s2, w1, t2, w2]
    g_W2 = np.ascontiguousarray(g_W2.transpose(1, 2, 0, 3))
    return g_theta, g_W1, g_W2


def _left_envs(W, mps):
    envs = [np.ones((1, 1, 1))]
    for A, Wk in zip(mps, W):
        envs.append(dmrg.env_left(envs[-1], A, Wk))
    return envs


def _right_envs(W, mps):
    L = len(mps)
    envs = [None] * (L + 1)
    envs[L] = np.ones((1, 1, 1))
    for k in range(L - 1, -1, -1):
        envs[k] = dmrg.env_right(envs[k + 1], mps[k], W[k])
    return envs


def energy_grad_W(W, mps):
    """Returns (E, [dE/dW_k]) for the fixed MPS."""
    norm = dmrg.mps_norm2(mps)
    Ls = _left_envs(W, mps)
    Rs = _right_envs(W, mps)
    E = float(Ls[-1][0, 0, 0]) / norm
    grads = []
    for k, A in enumerate(mps):
        X = np.tensordot(Ls[k], A, axes=([2], [0]))            # [a2, w, s, b]
        Y = np.tensordot(A, Rs[k + 1], axes=([2], [0]))        # [a2, t, w2, b]
        G = np.tensordot(X, Y, axes=([0, 3], [0, 3]))          # [w, s, t, w2]
        grads.append(np.ascontiguousarray(G.transpose(0, 2, 1, 3)) / norm)
    return E, grads


def xxz_coupling_grads(grads_W, L, J, delta, h):
    """dE/dJ_i (L-1 values) and dE/dh_i (L values) from dE/dW_k, using that the
    XXZ MPO of ``oracle.mpo.xxz_mpo`` is affine in each coupling."""
    J = np.broadcast_to(np.asarray(J, dtype=np.float64), (L - 1,)).copy()
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (L,)).copy()
    base = mpo.xxz_mpo(L, J, delta, h)
    dJ = np.zeros(L - 1)
    dh = np.zeros(L)
    for i in range(L - 1):
        Jp = J.copy()
        Jp[i] += 1.0
        Wp = mpo.xxz_mpo(L, Jp, delta, h)
        dJ[i] = sum(float(np.sum(g * (a - b))) for g, a, b in zip(grads_W, Wp, base))
    for i in range(L):
        hp = h.copy()
        hp[i] += 1.0
        Wp = mpo.xxz_mpo(L, J, delta, hp)
        dh[i] = sum(float(np.sum(g * (a - b))) for g, a, b in zip(grads_W, Wp, base))
    return dJ, dh
