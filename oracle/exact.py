"""Exact diagonalisation and closed forms that pin the oracle.

Hamiltonians here are assembled by brute force from Kronecker products of
local operators, with no MPO involved, so they check ``oracle.mpo``
independently. Ground energies come from textbook routines
(``numpy.linalg.eigh``, ``scipy.sparse.linalg.eigsh``) or from closed forms.
"""
import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import ops


def _embed(op_list, L, d):
    """Kronecker product of a list of (site, operator) placements, identity elsewhere."""
    placed = dict(op_list)
    out = sp.identity(1, format="csr", dtype=np.float64)
    for k in range(L):
        m = placed.get(k)
        m = sp.identity(d, format="csr", dtype=np.float64) if m is None else sp.csr_matrix(m)
        out = sp.kron(out, m, format="csr")
    return out


def kron_hamiltonian(L, d, site_terms, bond_terms):
    """H = sum_k h_k + sum_k sum_j O_kj (x) P_{k+1,j}, as a sparse CSR matrix.

    Same input format as ``oracle.mpo.nearest_neighbour_mpo`` but assembled
    directly from Kronecker products.
    """
    D = d ** L
    H = sp.csr_matrix((D, D), dtype=np.float64)
    for k in range(L):
        if np.any(site_terms[k]):
            H = H + _embed([(k, site_terms[k])], L, d)
    for k in range(L - 1):
        for O, P in bond_terms[k]:
            if np.any(O) and np.any(P):
                H = H + _embed([(k, O), (k + 1, P)], L, d)
    return H


def ising_terms(L, J=1.0, g=1.0):
    o = ops.spin_half()
    site = [-J * g * o["sigma_x"]] * L
    bonds = [[(-J * o["sigma_z"], o["sigma_z"])] for _ in range(L - 1)]
    return site, bonds


def xxz_terms(L, J=1.0, delta=1.0, h=0.0):
    """XXZ with S = sigma/2, written with Sx and i*Sy: Sy(x)Sy = -(iSy)(x)(iSy)."""
    o = ops.spin_half()
    Jb = np.broadcast_to(np.asarray(J, dtype=np.float64), (max(L - 1, 0),))
    hs = np.broadcast_to(np.asarray(h, dtype=np.float64), (L,))
    site = [hs[k] * o["Sz"] for k in range(L)]
    bonds = []
    for k in range(L - 1):
        bonds.append([
            (Jb[k] * o["Sx"], o["Sx"]),
            (-Jb[k] * o["iSy"], o["iSy"]),
            (delta * Jb[k] * o["Sz"], o["Sz"]),
        ])
    return site, bonds


def bose_hubbard_terms(L, J=1.0, U=4.0, nmax=4):
    o = ops.boson(nmax)
    n = o["n"]
    site = [0.5 * U * (n @ n - n)] * L
    bonds = [[(-J * o["bd"], o["b"]), (-J * o["b"], o["bd"])] for _ in range(L - 1)]
    return site, bonds


def aklt_terms(L):
    """h_bond = S.S + (S.S)^2/3 assembled as a dense 9x9 matrix and split by an
    operator SVD into O (x) P pairs, so it does not share the channel layout of
    ``oracle.mpo.aklt_mpo``."""
    o = ops.spin_one()
    Sx, Sz, iSy = o["Sx"], o["Sz"], o["iSy"]
    SS = np.kron(Sx, Sx) - np.kron(iSy, iSy) + np.kron(Sz, Sz)
    hb = SS + SS @ SS / 3.0
    # operator Schmidt decomposition: hb[(t1 t2),(s1 s2)] -> [(t1 s1),(t2 s2)]
    R = hb.reshape(3, 3, 3, 3).transpose(0, 2, 1, 3).reshape(9, 9)
    U, S, Vt = np.linalg.svd(R)
    pairs = [(S[i] * U[:, i].reshape(3, 3), Vt[i].reshape(3, 3)) for i in range(9) if S[i] > 1e-12]
    site = [np.zeros((3, 3))] * L
    return site, [list(pairs) for _ in range(L - 1)], hb


def ground_energy(H, dense_limit=600):
    """Lowest eigenvalue: dense eigh for small matrices, eigsh otherwise."""
    if H.shape[0] <= dense_limit:
        return float(np.linalg.eigvalsh(H.toarray() if sp.issparse(H) else H)[0])
    vals = spla.eigsh(H, k=1, which="SA", tol=1e-14, maxiter=100000)[0]
    return float(vals[0])


def ground_state(H):
    """(E0, psi0) via eigsh (sparse) or eigh (dense)."""
    if H.shape[0] <= 600:
        Hd = H.toarray() if sp.issparse(H) else H
        w, v = np.linalg.eigh(Hd)
        return float(w[0]), v[:, 0]
    w, v = spla.eigsh(H, k=1, which="SA", tol=1e-14, maxiter=100000)
    return float(w[0]), v[:, 0]


def ising_free_fermion_energy(L, J=1.0, g=1.0):
    """Closed-form ground energy of the open transverse-field Ising chain.

    After a Jordan-Wigner transformation the chain is quadratic; its
    single-particle energies are 2x the singular values of the L x L
    upper-bidiagonal matrix with J g on the diagonal and J on the
    superdiagonal, and E0 = -sum of them. Written with the factor 2 folded in:
    B has 2 J g on the diagonal, 2 J on the superdiagonal, E0 = -1/2 sum sigma(B).
    """
    B = np.diag(np.full(L, 2.0 * J * g)) + np.diag(np.full(L - 1, 2.0 * J), 1)
    return -0.5 * float(np.sum(np.linalg.svd(B, compute_uv=False)))


def xx_free_fermion_energy(J, h):
    """Closed-form ground energy of the open XX chain (XXZ at delta = 0),
    H = sum J_i (Sx Sx + Sy Sy) + sum h_i Sz, site-dependent couplings.

    Jordan-Wigner with Sz = n - 1/2 gives free fermions with hopping J_i/2 and
    on-site energy h_i: E0 = sum of the negative eigenvalues of the tridiagonal
    single-particle matrix minus 1/2 sum h_i.
    """
    J = np.asarray(J, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    eps = scipy.linalg.eigh_tridiagonal(h, J / 2.0, eigvals_only=True)
    return float(np.sum(eps[eps < 0.0]) - 0.5 * np.sum(h))


def xx_free_fermion_gradients(J, h):
    """Hellmann-Feynman derivatives of the XX ground energy from the Slater
    determinant: dE/dh_i = <Sz_i> = <n_i> - 1/2, dE/dJ_i = <Sx Sx + Sy Sy>_i
    = Re <c_i^dag c_{i+1}>, with the correlation matrix C = sum over occupied
    modes of phi phi^T.
    """
    J = np.asarray(J, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    eps, phi = scipy.linalg.eigh_tridiagonal(h, J / 2.0)
    occ = phi[:, eps < 0.0]
    C = occ @ occ.T
    dh = np.diag(C) - 0.5
    dJ = np.array([C[i, i + 1] for i in range(len(J))])
    return dJ, dh


def aklt_energy(L):
    """Exact open-chain AKLT ground energy -2/3 (L - 1) (every bond projector
    term S.S + (S.S)^2/3 has minimum -2/3 and the valence-bond state reaches it
    on all bonds at once)."""
    return -2.0 / 3.0 * (L - 1)
