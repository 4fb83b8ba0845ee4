"""Matrix product operators for the oracle (Sec. 3.2, Eq. mpo and Eq. MPOdef).

Convention (fixed for the whole project): a site tensor is ``W[w, t, s, w2]``
with ``w``/``w2`` the left/right auxiliary (MPO bond) indices, ``t`` the
outgoing physical index (the paper's i') and ``s`` the incoming one (i), so
``W[w, :, :, w2]`` is the operator in row ``w`` and column ``w2`` of the
paper's operator-valued matrix M^{[k]}.

The paper's nearest-neighbour structure (Eq. MPOdef and the Ising example
right after it): M^{[k]} is lower triangular; the top-left entry is the
identity that has not yet met any term, the bottom-right entry is the
identity after all terms; the local term sits in the bottom-left corner; a
bond term O_k (x) P_{k+1} puts O_k (with its coupling) in the last row of
site k and P_{k+1} in the first column of site k+1. The first site keeps only
the last row (a row vector), the last site only the first column.
"""
import numpy as np

from . import ops


def nearest_neighbour_mpo(site_terms, bond_terms):
    """Build W tensors from local terms and bond terms.

    site_terms: list of L (d x d) matrices h_k (may be zero matrices).
    bond_terms: list of L-1 lists; bond_terms[k] = [(O, P), ...] meaning the
        term O acting on site k times P acting on site k+1 (the coupling is
        already folded into O). Every bond must list the same number n_b of
        pairs (pad with zero matrices) so the MPO bond dimension is n_b + 2.
    Returns a list of L arrays W[k] of shape (w_left, d, d, w_right).
    """
    L = len(site_terms)
    d = site_terms[0].shape[0]
    nb = len(bond_terms[0]) if L > 1 else 0
    w = nb + 2
    eye = np.eye(d)
    bulk = []
    for k in range(L):
        M = np.zeros((w, d, d, w))
        M[0, :, :, 0] = eye
        M[w - 1, :, :, w - 1] = eye
        M[w - 1, :, :, 0] = site_terms[k]
        if k > 0:  # right partner of the bond (k-1, k): first column
            for j, (_, P) in enumerate(bond_terms[k - 1]):
                M[1 + j, :, :, 0] = P
        if k < L - 1:  # left operator of the bond (k, k+1): last row
            for j, (O, _) in enumerate(bond_terms[k]):
                M[w - 1, :, :, 1 + j] = O
        bulk.append(M)
    if L == 1:
        return [bulk[0][w - 1:w, :, :, 0:1].copy()]
    W = [bulk[0][w - 1:w].copy()]  # first site: last row
    W += [bulk[k] for k in range(1, L - 1)]
    W.append(bulk[L - 1][:, :, :, 0:1].copy())  # last site: first column
    return W


def ising_mpo(L, J=1.0, g=1.0):
    """Transverse-field Ising H = -J sum sz sz - J g sum sx (Eq. Ising), w = 3."""
    o = ops.spin_half()
    site = [-J * g * o["sigma_x"] for _ in range(L)]
    bonds = [[(-J * o["sigma_z"], o["sigma_z"])] for _ in range(L - 1)]
    return nearest_neighbour_mpo(site, bonds)


def xxz_mpo(L, J=1.0, delta=1.0, h=0.0):
    """Spin-1/2 XXZ chain with S = sigma/2 (the paper never defines XXZ; this
    is the reading used throughout the project):

        H = sum_i J_i (Sx Sx + Sy Sy + delta Sz Sz)_{i,i+1} + sum_i h_i Sz_i,

    written with real operators as J_i [ (S+ S- + S- S+)/2 + delta Sz Sz ].
    J may be a scalar or an array of L-1 bond couplings, h a scalar or an
    array of L fields. w = 5.
    """
    o = ops.spin_half()
    Jb = np.broadcast_to(np.asarray(J, dtype=np.float64), (max(L - 1, 0),))
    hs = np.broadcast_to(np.asarray(h, dtype=np.float64), (L,))
    site = [hs[k] * o["Sz"] for k in range(L)]
    bonds = []
    for k in range(L - 1):
        bonds.append([
            (0.5 * Jb[k] * o["Sp"], o["Sm"]),
            (0.5 * Jb[k] * o["Sm"], o["Sp"]),
            (delta * Jb[k] * o["Sz"], o["Sz"]),
        ])
    return nearest_neighbour_mpo(site, bonds)


def bose_hubbard_mpo(L, J=1.0, U=4.0, nmax=4):
    """Bose-Hubbard H = -J sum (b^dag_i b_{i+1} + h.c.) + U/2 sum n (n - 1)
    (Eq. bosehubbard with the hopping read with its dagger; the chemical
    potential is a constant at fixed particle number and is dropped). w = 4.
    """
    o = ops.boson(nmax)
    n = o["n"]
    site = [0.5 * U * n @ (n - o["id"]) for _ in range(L)]
    bonds = [[(-J * o["bd"], o["b"]), (-J * o["b"], o["bd"])] for _ in range(L - 1)]
    return nearest_neighbour_mpo(site, bonds)


def aklt_mpo(L):
    """Spin-1 AKLT chain H = sum [S.S + (S.S)^2 / 3] (not in the paper; used as a
    pin because its open-chain ground energy is exactly -2/3 (L-1)). w = 14.

    With T^x = Sx, T^y = i Sy, T^z = Sz (all real), S^a S^b (x) S^a S^b equals
    (-1)^{n_y} T^a T^b (x) T^a T^b where n_y counts the y's among (a, b).
    """
    o = ops.spin_one()
    T = {"x": o["Sx"], "y": o["iSy"], "z": o["Sz"]}
    pairs = []
    for a in "xyz":
        sign = -1.0 if a == "y" else 1.0
        pairs.append((sign * T[a], T[a]))
    for a in "xyz":
        for b in "xyz":
            ny = (a == "y") + (b == "y")
            sign = (-1.0) ** ny / 3.0
            pairs.append((sign * T[a] @ T[b], T[a] @ T[b]))
    site = [np.zeros((3, 3)) for _ in range(L)]
    return nearest_neighbour_mpo(site, [list(pairs) for _ in range(L - 1)])


def mpo_to_dense(W):
    """Contract an MPO into the full d^L x d^L matrix (Eq. mpo), for small L.

    Row index = outgoing configuration (t_1 ... t_L), column = incoming, both
    with site 1 as the most significant digit.
    """
    acc = W[0][0]  # (d, d, w): operator-valued row vector, left bond is 1
    for Wk in W[1:]:
        # acc[o, i, w] * Wk[w, t, s, w2] -> new[(o, t), (i, s), w2]
        new = np.einsum("oiw,wtsv->otisv", acc, Wk)
        D_o, d_t, D_i, d_s, w2 = new.shape
        acc = new.reshape(D_o * d_t, D_i * d_s, w2)
    assert acc.shape[2] == 1
    return acc[:, :, 0]


def long_range_ising_mpo(L, J, g, amps, decays):
    """Eq. LRIsing with the distance dependence f(r) = sum_k amps_k decays_k^r
    (the paper's exponential rule: a channel per exponential whose diagonal
    entry is the decay times the identity). Channel layout as in
    nearest_neighbour_mpo: 0 'done', 1..K the open exponential terms, K+1
    'start'."""
    o = ops.spin_half()
    K = len(amps)
    w = K + 2
    bulk = np.zeros((w, 2, 2, w))
    bulk[0, :, :, 0] = o["id"]
    bulk[w - 1, :, :, w - 1] = o["id"]
    bulk[w - 1, :, :, 0] = -J * g * o["sigma_x"]
    for c, (a, lam) in enumerate(zip(amps, decays)):
        bulk[w - 1, :, :, 1 + c] = -J * a * lam * o["sigma_z"]   # open: amplitude and first decay
        bulk[1 + c, :, :, 1 + c] = lam * o["id"]             # pass one more site
        bulk[1 + c, :, :, 0] = o["sigma_z"]                       # close
    W = [bulk.copy() for _ in range(L)]
    W[0] = W[0][w - 1:w].copy()
    W[-1] = W[-1][..., 0:1].copy()
    return W


def long_range_ising_dense(L, J, g, coupling):
    """Dense Eq. LRIsing from its pair sum, coupling(r) for r = j - i."""
    o = ops.spin_half()
    dim = 2 ** L

    def site_op(op, i):
        out = np.array([[1.0]])
        for k in range(L):
            out = np.kron(out, op if k == i else o["id"])
        return out

    H = np.zeros((dim, dim))
    for i in range(L):
        H -= J * g * site_op(o["sigma_x"], i)
        for j in range(i + 1, L):
            H -= J * coupling(j - i) * site_op(o["sigma_z"], i) @ site_op(o["sigma_z"], j)
    return H
