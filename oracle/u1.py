"""U(1) block structure, oracle side (test infrastructure only).

With a conserved particle number every bond index carries a charge (the
number of particles to the left of the bond) and a local state s carries
charge s. An MPO channel carries the charge its operators have added so far.
The tensors of the effective Hamiltonian (Sec. 3.4) are then block sparse:

  theta[a,s1,s2,c] may be nonzero only if q(a) + s1 + s2 = q(c),
  L[a2,w,a]        only if q(a2) = q(a) + q_w,
  R[c2,w,c]        only if q(c2) = q(c) + q_w,
  W[w,t,s,w2]      only if q_w2 = q_w + t - s.

The block-sparse product is by definition the dense product of the masked
tensors, restricted to the allowed entries of the result; that is what this
module computes, with the dense contraction of ``oracle.dmrg``.
"""
import numpy as np

from . import dmrg


def index_charges(charges, sizes):
    """Charge of every index of a bond given as sectors (charge, size) in order."""
    return np.repeat(np.asarray(charges, dtype=np.int64), np.asarray(sizes, dtype=np.int64))


def theta_mask(q_left, q_right, d1, d2):
    """Allowed entries of theta[a, s1, s2, c] (per-index charge arrays)."""
    s1 = np.arange(d1)[None, :, None, None]
    s2 = np.arange(d2)[None, None, :, None]
    return q_left[:, None, None, None] + s1 + s2 == q_right[None, None, None, :]


def env_mask(q_bra, q_w, q_ket):
    """Allowed entries of an environment E[x, w, y] with q(x) = q(y) + q_w."""
    q_w = np.asarray(q_w, dtype=np.int64)
    return q_bra[:, None, None] == q_ket[None, None, :] + q_w[None, :, None]


def channel_charges(W, q_first=0):
    """Charges of the right channels of site tensor W[w, t, s, w2] given the
    charges of its left channels (q_first: scalar or array), read off the
    nonzero entries (q_w2 = q_w + t - s). Raises if W does not conserve
    the charge or a right channel is never reached."""
    wl, d, _, wr = W.shape
    ql = np.broadcast_to(np.asarray(q_first, dtype=np.int64), (wl,))
    qr = [None] * wr
    for w, t, s, w2 in zip(*np.nonzero(W)):
        q = int(ql[w] + t - s)
        if qr[w2] is None:
            qr[w2] = q
        elif qr[w2] != q:
            raise ValueError(f"channel {w2} reached with charges {qr[w2]} and {q}")
    if any(q is None for q in qr):
        raise ValueError("a right channel carries no operator")
    return np.array(qr, dtype=np.int64)


def mpo_channel_charges(W_list):
    """Charges of all MPO bonds of a chain (the left boundary channel has 0)."""
    q = [np.zeros(W_list[0].shape[0], dtype=np.int64)]
    for W in W_list:
        q.append(channel_charges(W, q[-1]))
    return q


def heff_apply_u1(Lenv, W1, W2, Renv, theta, q_left, q_right, q_wl, q_wr):
    """Dense H_eff theta of the masked operands, masked to the allowed
    entries of the result (dense arrays in, dense array out)."""
    d1, d2 = W1.shape[1], W2.shape[1]
    mt = theta_mask(q_left, q_right, d1, d2)
    ml = env_mask(q_left, q_wl, q_left)
    mr = env_mask(q_right, q_wr, q_right)
    y = dmrg.heff_apply(np.where(ml, Lenv, 0.0), W1, W2, np.where(mr, Renv, 0.0),
                        np.where(mt, theta, 0.0))
    return np.where(mt, y, 0.0)


def mps_mask(q_left, q_right, d):
    """Allowed entries of an MPS tensor A[a, s, b]: q(a) + s = q(b)."""
    return q_left[:, None, None] + np.arange(d)[None, :, None] == q_right[None, None, :]


def sector_heff_matrix(Lenv, W1, W2, Renv, mask):
    """H_eff as an explicit matrix on the allowed entries of theta (column i =
    H_eff applied to the i-th allowed unit vector), for small sectors."""
    idx = np.flatnonzero(mask)
    H = np.zeros((idx.size, idx.size))
    for col, i in enumerate(idx):
        e = np.zeros(mask.shape)
        e.flat[i] = 1.0
        H[:, col] = dmrg.heff_apply(Lenv, W1, W2, Renv, e).flat[idx]
    return H
