"""Pins for oracle.mpo: the paper's worked three-site Ising product (Sec. 3.2)
and brute-force Kronecker-sum Hamiltonians."""
import os

import numpy as np
import pytest

from oracle import exact, mpo, ops

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ising_3site_mpo.txt")
PAULI = {"X": np.array([[0.0, 1.0], [1.0, 0.0]]), "Z": np.diag([1.0, -1.0]), "I": np.eye(2)}


def _coef(sym, J, g):
    val = 1.0
    sym = sym.strip()
    if sym.startswith("-"):
        val, sym = -1.0, sym[1:]
    for f in sym.split("*"):
        val *= {"J": J, "g": g, "1": 1.0}[f]
    return val


def _term_sum(expr, J, g):
    out = 0.0
    for term in expr.split(" + "):
        c, word = term.strip().split()
        m = np.array([[1.0]])
        for ch in word:
            m = np.kron(m, PAULI[ch])
        out = out + _coef(c, J, g) * m
    return out


def _load_golden():
    rows, H = {}, None
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        key, expr = line.split(":", 1)
        if key.startswith("row"):
            rows[int(key.split()[1])] = expr
        else:
            H = expr
    return rows, H


@pytest.mark.parametrize("J,g", [(1.0, 1.0), (0.7, 1.3), (-1.1, 0.4)])
def test_three_site_ising_matches_paper(J, g):
    rows, Hexpr = _load_golden()
    W = mpo.ising_mpo(3, J, g)
    # intermediate product M[1] x M[2]: acc[(t1 t2),(s1 s2), channel]
    acc = np.einsum("tsw,wuvx->tusvx", W[0][0], W[1]).reshape(4, 4, -1)
    for ch, expr in rows.items():
        np.testing.assert_allclose(acc[:, :, ch], _term_sum(expr, J, g), atol=1e-15)
    np.testing.assert_allclose(mpo.mpo_to_dense(W), _term_sum(Hexpr, J, g), atol=1e-14)


def test_mpo_shapes_and_boundaries():
    for W, w in [(mpo.ising_mpo(5), 3), (mpo.xxz_mpo(5), 5), (mpo.bose_hubbard_mpo(5), 4),
                 (mpo.aklt_mpo(5), 14)]:
        assert W[0].shape[0] == 1 and W[-1].shape[3] == 1
        for k in range(1, 4):
            assert W[k].shape[0] == w and W[k].shape[3] == w
        # lower triangular in the auxiliary indices (Eq. MPOdef)
        Wb = W[2]
        for a in range(w):
            for b in range(a + 1, w):
                assert not np.any(Wb[a, :, :, b])


def _cases():
    rng = np.random.default_rng(11)
    J = rng.uniform(0.8, 1.2, 5)
    h = rng.uniform(-0.5, 0.5, 6)
    return [
        ("ising", mpo.ising_mpo(6, 1.0, 0.8), exact.ising_terms(6, 1.0, 0.8), 2),
        ("xxz", mpo.xxz_mpo(6, J, 0.7, h), exact.xxz_terms(6, J, 0.7, h), 2),
        ("bh", mpo.bose_hubbard_mpo(4, 1.0, 4.0, 3), exact.bose_hubbard_terms(4, 1.0, 4.0, 3), 4),
        ("aklt", mpo.aklt_mpo(4), exact.aklt_terms(4)[:2], 3),
    ]


@pytest.mark.parametrize("name,W,terms,d", _cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_mpo_equals_kronecker_hamiltonian(name, W, terms, d):
    site, bonds = terms
    L = len(W)
    Hk = exact.kron_hamiltonian(L, d, site, bonds).toarray()
    Hm = mpo.mpo_to_dense(W)
    np.testing.assert_allclose(Hm, Hk, atol=1e-13)
    np.testing.assert_allclose(Hm, Hm.T, atol=1e-13)


def test_aklt_bond_is_projector_form():
    # S.S + (S.S)^2/3 = 2 P_2 - 2/3 on two spin-1 sites: eigenvalues -2/3 (x4) and 4/3 (x5)
    hb = exact.aklt_terms(2)[2]
    ev = np.sort(np.linalg.eigvalsh(hb))
    np.testing.assert_allclose(ev[:4], -2 / 3, atol=1e-13)
    np.testing.assert_allclose(ev[4:], 4 / 3, atol=1e-13)


def test_operator_algebra():
    o = ops.spin_half()
    np.testing.assert_allclose(o["Sp"] @ o["Sm"] - o["Sm"] @ o["Sp"], 2 * o["Sz"], atol=1e-15)
    s1 = ops.spin_one()
    # S^2 = s(s+1) = 2 with Sy Sy = -(iSy)(iSy)
    S2 = s1["Sx"] @ s1["Sx"] - s1["iSy"] @ s1["iSy"] + s1["Sz"] @ s1["Sz"]
    np.testing.assert_allclose(S2, 2 * np.eye(3), atol=1e-14)
    b = ops.boson(4)
    np.testing.assert_allclose(b["bd"] @ b["b"], b["n"], atol=1e-14)
