"""FP64 CPU oracle for the two-site variational ground-state search.

This package is TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The product (``paper_1703_00387_gb300``) never imports it, and it never
imports the product: the two share no code. Inputs (random MPS tensors,
couplings) are drawn by the caller and passed in as arrays.

Everything here is plain NumPy/SciPy in float64, written for readability,
following the paper's steps in order:

* ``ops``    -- local operators (spin-1/2, spin-1, bosons with a cutoff).
* ``mpo``    -- matrix product operators built as in Sec. 3.2 (Eq. MPOdef and
                the Ising example that follows it), plus dense contraction of
                an MPO for small L.
* ``exact``  -- exact diagonalisation and closed-form ground energies used to
                pin the rest (free fermions, AKLT).
* ``dmrg``   -- the two-site variational search of Sec. 3.4: effective
                Hamiltonian application, environment updates, Lanczos,
                eigendecomposition/SVD split with truncation (Sec. 2,
                Eq. AAD_ULLUD, Eq. elocal), sweeps and the MPO energy.
* ``grad``   -- gradients for the differentiation workload: the vector-Jacobian
                product of H_eff.theta and dE/dW_k of the MPO energy at a
                fixed state, with the chain rule to XXZ couplings.
* ``tdvp``   -- real-time evolution (Sec. 5.4, two-site TDVP) in complex128:
                complex environments, one- and two-site H_eff, the Krylov
                propagator of Eq. krylov:approx, the complex SVD split and the
                symmetric second-order time step.

Parity status: every function is pinned by a test in ``tests/test_oracle_*.py``
against exact diagonalisation, a closed form, the paper's worked example, or a
brute-force construction. No function is "parity unpinned".
"""
