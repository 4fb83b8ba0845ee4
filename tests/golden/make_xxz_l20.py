"""Writes xxz_l20_ground_energy.json: the exact ground energy of the open
spin-1/2 XXZ chain (J = 1, Delta = 1, h = 0; S = sigma/2) at L = 20, by
sparse exact diagonalisation of the Kronecker-product Hamiltonian
(oracle.exact.kron_hamiltonian with oracle.exact.xxz_terms, eigsh). The same
construction is pinned against dense diagonalisation and closed forms at
L <= 12 by tests/test_oracle_exact.py.

At L = 20 the largest Schmidt rank of any state is 2^10 = 1024 (the middle
bond), so two-site DMRG at chi_max = 1024 represents the ground state
without truncation and must reach this energy: the float64 reference for
the chi = 1024 split-precision sweeps (the model of Sec. 3.4's variational
search at full bond dimension). Calls only oracle/; run from the repository
root: python tests/golden/make_xxz_l20.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact  # noqa: E402


def main():
    L = 20
    t0 = time.time()
    H = exact.kron_hamiltonian(L, 2, *exact.xxz_terms(L, 1.0, 1.0, 0.0))
    e0 = float(exact.ground_energy(H))
    out = {"model": "open XXZ chain, S = sigma/2", "L": L, "J": 1.0, "Delta": 1.0, "h": 0.0,
           "ground_energy": e0, "method": "sparse exact diagonalisation (scipy eigsh) of the "
           "Kronecker-product Hamiltonian from oracle.exact", "seconds": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, "xxz_l20_ground_energy.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
