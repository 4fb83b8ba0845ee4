"""Host-side MPO construction for the library (Sec. 3.2, Eq. MPOdef).

A nearest-neighbour Hamiltonian is described as a small automaton on the
MPO bond: channel 0 = "every term is complete", channel w-1 = "no term
started yet", channels 1..n_b = "the left half of bond term j was applied".
Each site tensor W[w, t, s, w2] is the operator that moves channel w (left
bond) to channel w2 (right bond):
    done -> done : identity          start -> start : identity
    start -> done: local term h_k    start -> j     : left factor of bond term j
    j -> done    : right factor of bond term j
The first site keeps only the "start" row, the last site only the "done"
column, so the product of all site matrices is the 1 x 1 Hamiltonian.
Real operators only: S^y S^y terms are written with S^+ S^- + S^- S^+.
"""
import numpy as np


def _spin_half():
    sp = np.array([[0.0, 1.0], [0.0, 0.0]])
    return {"sx": np.array([[0.0, 1.0], [1.0, 0.0]]), "sz": np.diag([1.0, -1.0]),
            "Sz": np.diag([0.5, -0.5]), "Sp": sp, "Sm": sp.T.copy(), "1": np.eye(2)}


def _spin_one():
    r = np.sqrt(2.0)
    sp = np.array([[0.0, r, 0.0], [0.0, 0.0, r], [0.0, 0.0, 0.0]])
    return {"Sz": np.diag([1.0, 0.0, -1.0]), "Sp": sp, "Sm": sp.T.copy(), "1": np.eye(3)}


def _boson(nmax):
    b = np.diag(np.sqrt(np.arange(1, nmax + 1, dtype=np.float64)), 1)
    return {"b": b, "bd": b.T.copy(), "n": np.diag(np.arange(nmax + 1, dtype=np.float64)),
            "1": np.eye(nmax + 1)}


class NearestNeighbourAutomaton:
    """Collects local terms and bond terms, then emits the MPO site tensors."""

    def __init__(self, L, d):
        self.L, self.d = L, d
        self.local = [np.zeros((d, d)) for _ in range(L)]
        self.bond = [[] for _ in range(L - 1)]  # bond[k] = list of (left op, right op)

    def add_local(self, k, op):
        self.local[k] = self.local[k] + op

    def add_bond(self, k, left, right):
        self.bond[k].append((left, right))

    def tensors(self):
        nb = max((len(b) for b in self.bond), default=0)
        w = nb + 2
        d, L = self.d, self.L
        done, start = 0, w - 1
        out = []
        for k in range(L):
            W = np.zeros((w, d, d, w))
            W[done, :, :, done] = np.eye(d)
            W[start, :, :, start] = np.eye(d)
            W[start, :, :, done] = self.local[k]
            if k + 1 < L:
                for j, (left, _) in enumerate(self.bond[k]):
                    W[start, :, :, 1 + j] = left
            if k >= 1:
                for j, (_, right) in enumerate(self.bond[k - 1]):
                    W[1 + j, :, :, done] = right
            if k == 0:
                W = W[start:start + 1]
            if k == L - 1:
                W = W[..., done:done + 1]
            out.append(np.ascontiguousarray(W))
        return out


def ising(L, J=1.0, g=1.0):
    """H = -J sum sz_i sz_{i+1} - J g sum sx_i (Eq. Ising)."""
    o = _spin_half()
    a = NearestNeighbourAutomaton(L, 2)
    for k in range(L):
        a.add_local(k, -J * g * o["sx"])
    for k in range(L - 1):
        a.add_bond(k, -J * o["sz"], o["sz"])
    return a.tensors()


def xxz(L, J=1.0, delta=1.0, h=0.0):
    """H = sum_i J_i (Sx Sx + Sy Sy + delta Sz Sz) + sum_i h_i Sz_i, S = sigma/2.
    J: scalar or L-1 couplings; h: scalar or L fields."""
    o = _spin_half()
    Jv = np.broadcast_to(np.asarray(J, dtype=np.float64), (L - 1,))
    hv = np.broadcast_to(np.asarray(h, dtype=np.float64), (L,))
    a = NearestNeighbourAutomaton(L, 2)
    for k in range(L):
        a.add_local(k, hv[k] * o["Sz"])
    for k in range(L - 1):
        a.add_bond(k, 0.5 * Jv[k] * o["Sp"], o["Sm"])
        a.add_bond(k, 0.5 * Jv[k] * o["Sm"], o["Sp"])
        a.add_bond(k, delta * Jv[k] * o["Sz"], o["Sz"])
    return a.tensors()


def bose_hubbard(L, J=1.0, U=4.0, nmax=4):
    """H = -J sum (b^dag_i b_{i+1} + b^dag_{i+1} b_i) + U/2 sum n_i (n_i - 1)."""
    o = _boson(nmax)
    a = NearestNeighbourAutomaton(L, nmax + 1)
    onsite = 0.5 * U * (o["n"] @ o["n"] - o["n"])
    for k in range(L):
        a.add_local(k, onsite)
    for k in range(L - 1):
        a.add_bond(k, -J * o["bd"], o["b"])
        a.add_bond(k, -J * o["b"], o["bd"])
    return a.tensors()


def aklt(L):
    """Spin-1 H = sum S.S + (S.S)^2 / 3, with S.S = Sz Sz + (S+ S- + S- S+)/2 and
    (S.S)^2 expanded over the nine products of {Sz, S+/sqrt2, S-/sqrt2}."""
    o = _spin_one()
    r = 1.0 / np.sqrt(2.0)
    # S.S = sum_a X_a (x) Y_a with X = (Sz, S+/r2, S-/r2), Y = (Sz, S-/r2, S+/r2)
    X = [o["Sz"], r * o["Sp"], r * o["Sm"]]
    Y = [o["Sz"], r * o["Sm"], r * o["Sp"]]
    a = NearestNeighbourAutomaton(L, 3)
    for k in range(L - 1):
        for i in range(3):
            a.add_bond(k, X[i], Y[i])
        for i in range(3):
            for j in range(3):
                a.add_bond(k, (X[i] @ X[j]) / 3.0, Y[i] @ Y[j])
    return a.tensors()


def xxz_coupling_basis(L, delta=1.0):
    """The XXZ MPO of ``xxz`` as an affine function of its couplings
    p = (J_0 .. J_{L-2}, h_0 .. h_{L-1}):  W(p) = W_0 + sum_j p_j B_j.

    Returns (W_0, row_ptr, col, val): W_0 the site tensors at p = 0 and the
    B_j in compressed sparse rows over the concatenated site tensors (row j
    lists the flat indices and values of the nonzero entries of B_j)."""
    n_par = 2 * L - 1
    W0 = xxz(L, np.zeros(L - 1), delta, np.zeros(L))
    flat0 = np.concatenate([w.ravel() for w in W0])
    row_ptr = [0]
    cols, vals = [], []
    for j in range(n_par):
        p = np.zeros(n_par)
        p[j] = 1.0
        flat = np.concatenate([w.ravel() for w in xxz(L, p[:L - 1], delta, p[L - 1:])]) - flat0
        nz = np.flatnonzero(flat)
        cols.append(nz)
        vals.append(flat[nz])
        row_ptr.append(row_ptr[-1] + nz.size)
    return (W0, np.asarray(row_ptr, dtype=np.int64), np.concatenate(cols).astype(np.int64),
            np.concatenate(vals))


def exponential_fit(f, rmax, n_exp):
    """Amplitudes a_k and decays l_k with sum_k a_k l_k^r ~ f(r) for r = 1..rmax
    (the paper expresses every infinite-range coupling as a sum of
    exponentials): decays on a geometric grid of length scales from 1/2 to
    rmax, amplitudes by linear least squares. Returns (a, l, max |error|)."""
    r = np.arange(1, rmax + 1, dtype=np.float64)
    scales = np.geomspace(0.5, max(float(rmax), 1.0), n_exp)
    lam = np.exp(-1.0 / scales)
    V = lam[None, :] ** r[:, None]
    a, *_ = np.linalg.lstsq(V, f(r), rcond=None)
    return a, lam, float(np.abs(V @ a - f(r)).max())


def long_range_ising(L, J=1.0, g=1.0, amps=(), decays=()):
    """Long-range transverse-field Ising chain (Eq. LRIsing) with the coupling
    as a sum of exponentials, f(r) = sum_k amps_k decays_k^r:
        H = -J sum_{i<j} f(j - i) sz_i sz_j - J g sum_i sx_i.
    Channel 1 + k carries the term started by amps_k decays_k sz on the left
    and multiplies by decays_k on every site it passes (the decay factor on
    the MPO diagonal); sz closes it into 'done'. w = len(amps) + 2."""
    o = _spin_half()
    K = len(amps)
    w = K + 2
    done, start = 0, w - 1
    out = []
    for k in range(L):
        W = np.zeros((w, 2, 2, w))
        W[done, :, :, done] = o["1"]
        W[start, :, :, start] = o["1"]
        W[start, :, :, done] = -J * g * o["sx"]
        for c in range(K):
            W[start, :, :, 1 + c] = -J * amps[c] * decays[c] * o["sz"]
            W[1 + c, :, :, 1 + c] = decays[c] * o["1"]
            W[1 + c, :, :, done] = o["sz"]
        if k == 0:
            W = W[start:start + 1]
        if k == L - 1:
            W = W[..., done:done + 1]
        out.append(np.ascontiguousarray(W))
    return out
