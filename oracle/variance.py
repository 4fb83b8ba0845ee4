"""Energy variance of an MPS (oracle side, test infrastructure only).

The paper's convergence criterion (Sec. 3.4, convergence parameters) is the
variance V = <H^2> - <H>^2 of the normalised state, with the outer sweeps
lowering the local tolerance as eps' = eps eps_V / V (Eq. linearExtrap).

Near an eigenstate V is tiny next to E^2, so V is formed as <(H - E)^2>:
the MPO of H - E (each site's local term shifted by -E/L) is squared site by
site and contracted with the state. ``dense_variance`` is the same quantity
from the full state vector, for small chains.
"""
import numpy as np

from . import dmrg, mpo


def shifted_mpo(W, shift):
    """MPO of H - shift * 1 for the nearest-neighbour form of ``oracle.mpo``
    (channel 0 'done', the last channel 'start'; site k's local term sits at
    [start, :, :, done]): shift / L is subtracted from every local term."""
    L = len(W)
    out = [w.copy() for w in W]
    for k, w in enumerate(out):
        d = w.shape[1]
        out[k][w.shape[0] - 1, :, :, 0] -= (shift / L) * np.eye(d)
    return out


def mpo_square(W):
    """Site tensors of the product MPO H H: (W W)[(a,b), t, s, (a2,b2)] =
    sum_u W[a, t, u, a2] W[b, u, s, b2]."""
    out = []
    for w in W:
        wl, d, _, wr = w.shape
        sq = np.einsum("atux,busy->abtsxy", w, w)
        out.append(sq.reshape(wl * wl, d, d, wr * wr))
    return out


def mps_variance(W, mps):
    """(E, V) with V = <psi|(H - E)^2|psi> / <psi|psi>."""
    E = dmrg.mps_energy(W, mps)
    Wsq = mpo_square(shifted_mpo(W, E))
    return E, dmrg.mpo_expectation(Wsq, mps) / dmrg.mps_norm2(mps)


def dense_variance(W, mps):
    """(E, V) from the dense Hamiltonian and state vector (small L)."""
    H = mpo.mpo_to_dense(W)
    psi = mps[0]
    for A in mps[1:]:
        psi = np.tensordot(psi, A, axes=([psi.ndim - 1], [0]))
    psi = psi.reshape(-1)
    nrm = psi @ psi
    E = psi @ H @ psi / nrm
    r = H @ psi - E * psi
    return float(E), float(r @ r / nrm)
