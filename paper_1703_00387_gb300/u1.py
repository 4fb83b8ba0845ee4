"""Host-side helpers for the U(1)-symmetric H_eff (block-sparse tensors).

Packed format (the library's): the entries allowed by the charge rules, in C
order of the dense tensor. A bond is a list of sectors (charge, size) in index
order; a local state s carries charge s; an MPO channel carries the charge its
operators have added. Rules: theta[a,s1,s2,c]: q(a)+s1+s2 = q(c);
L[a2,w,a]: q(a2) = q(a)+q_w; R[c2,w,c]: q(c2) = q(c)+q_w.
"""
import numpy as np

from . import binding


def bond_charges(sectors_q, sectors_chi):
    """Per-index charges of a bond."""
    return np.concatenate([np.full(int(c), int(q), dtype=np.int64)
                           for q, c in zip(sectors_q, sectors_chi)])


def channel_charges(W_sites):
    """Charges of every MPO bond (list of arrays, L+1 of them), from the
    nonzero pattern of the site tensors W[w,t,s,w2] (q_w2 - q_w = t - s),
    starting from charge 0 on the left boundary channel. A channel that no
    operator reaches from the left (a zero coupling, e.g. a field h = 0 on
    the first site) takes its charge from the operators it feeds on the
    right; one connected to nothing at all gets charge 0 (its environment
    blocks are zero whatever the charge)."""
    unset = np.iinfo(np.int64).min
    out = [np.zeros(W_sites[0].shape[0], dtype=np.int64)]
    out += [np.full(W.shape[3], unset, dtype=np.int64) for W in W_sites]
    nz = [np.nonzero(W) for W in W_sites]
    changed = True
    while changed:  # propagate along nonzeros in both directions
        changed = False
        for k in range(len(W_sites)):
            for a, b, c, e in zip(*nz[k]):
                if out[k][a] != unset and out[k + 1][e] == unset:
                    out[k + 1][e] = out[k][a] + b - c
                    changed = True
                elif out[k][a] == unset and out[k + 1][e] != unset:
                    out[k][a] = out[k + 1][e] - b + c
                    changed = True
    for q in out:
        q[q == unset] = 0
    for k in range(len(W_sites)):
        for a, b, c, e in zip(*nz[k]):
            if out[k + 1][e] != out[k][a] + b - c:
                raise ValueError("the MPO does not conserve the charge")
    return out


def theta_allowed(qa, qc, d1, d2):
    s12 = np.arange(d1)[:, None] + np.arange(d2)[None, :]
    return (qa[:, None, None, None] + s12[None, :, :, None]) == qc[None, None, None, :]


def env_allowed(q_bra, q_w, q_ket):
    return q_bra[:, None, None] == (q_ket[None, None, :] + np.asarray(q_w)[None, :, None])


def pack(dense, mask):
    return np.ascontiguousarray(dense[mask])


def unpack(packed, mask):
    out = np.zeros(mask.shape)
    out[mask] = packed
    return out


class U1Operator:
    """One U(1) two-site operator structure: the library plan plus the masks
    used to pack and unpack dense arrays."""

    def __init__(self, ctx, left, right, d1, d2, W1, W2, q_wl, q_wr):
        (ql_s, chil), (qr_s, chir) = left, right
        self.qa = bond_charges(ql_s, chil)
        self.qc = bond_charges(qr_s, chir)
        self.m_theta = theta_allowed(self.qa, self.qc, d1, d2)
        self.m_L = env_allowed(self.qa, q_wl, self.qa)
        self.m_R = env_allowed(self.qc, q_wr, self.qc)
        self.plan = binding.U1Heff(ctx, ql_s, chil, qr_s, chir, d1, d2, W1.shape[0], W1.shape[3],
                                   W2.shape[3], q_wl, q_wr)
        assert self.plan.n_theta == int(self.m_theta.sum())
        assert self.plan.n_L == int(self.m_L.sum()) and self.plan.n_R == int(self.m_R.sum())

    def close(self):
        self.plan.close()
