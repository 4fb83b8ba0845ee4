"""GPU two-site sweeps against the FP64 oracle, exact diagonalisation and
closed forms. Energies are gauge invariant, so they are what is compared;
ground energies must agree to 1e-10 relative (float64 path and the
split-precision path after its float64 refinement sweep)."""
import numpy as np
import pytest

from oracle import dmrg as od
from oracle import exact, mpo as ompo
from paper_1703_00387_gb300 import binding as B
from paper_1703_00387_gb300 import hamiltonians, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import os
    if not os.path.exists(B.LIB_PATH):
        from paper_1703_00387_gb300 import build
        build.build()
    c = B.Context(0)
    yield c
    c.close()


def run_gpu(ctx, W, mps0, chi_max, n_sweeps, precision="fp64", refine=0, tol=1e-12, eps=-1.0):
    mpo = B.MPO(ctx, W)
    mps = B.MPS(ctx, mps0, chi_cap=chi_max)
    p = B.sweep_params(chi_max, n_sweeps, precision, eps_local=eps, lanczos_tol=tol,
                       lanczos_max_iter=100, refine_sweeps=refine)
    stats = B.osmps_sweep(ctx, mps, mpo, p)
    out = dict(stats=stats, tensors=mps.tensors(), chi=mps.bond_dims())
    mps.close()
    mpo.close()
    return out


def test_ising_l12_chi32_matches_oracle_and_closed_form(ctx):
    """TFI J=1 g=1, L=12, chi_max=32, 4 sweeps, Lanczos tol 1e-12, seed 0."""
    mps0 = inputs.random_mps(12, 2, 32, seed=0)
    r = run_gpu(ctx, hamiltonians.ising(12, 1.0, 1.0), mps0, 32, 4)
    E_ref, mps_ref, hist = od.dmrg(ompo.ising_mpo(12, 1.0, 1.0), mps0, 32, 4)
    e_cf = exact.ising_free_fermion_energy(12, 1.0, 1.0)
    E = r["stats"]["energy"]
    assert abs(E - E_ref) <= 1e-10 * abs(E_ref)
    assert abs(E - e_cf) <= 1e-9 * abs(e_cf)
    assert E >= e_cf - 1e-11
    # per-step Lanczos energies follow the oracle's to 1e-9 (same schedule, same truncation)
    ref_steps = np.array([h["energy"] for h in hist])
    np.testing.assert_allclose(r["stats"]["step_energies"][-22:], ref_steps[-22:], rtol=1e-9)
    # final state: normalised, right-canonical except the centre (site 0)
    t = r["tensors"]
    assert abs(od.mps_norm2(t) - 1.0) < 1e-12
    for A in t[1:]:
        assert od.right_isometry_defect(A) < 1e-11
    assert abs(od.mps_energy(ompo.ising_mpo(12, 1.0, 1.0), t) - E) < 1e-11


def test_aklt_exact_energy(ctx):
    L = 10
    r = run_gpu(ctx, hamiltonians.aklt(L), inputs.random_mps(L, 3, 4, seed=0), 8, 3)
    assert abs(r["stats"]["energy"] - exact.aklt_energy(L)) <= 1e-10 * abs(exact.aklt_energy(L))


def test_xx_site_dependent_closed_form(ctx):
    L = 12
    J, h = inputs.random_couplings(L, seed=0)
    r = run_gpu(ctx, hamiltonians.xxz(L, J, 0.0, h), inputs.random_mps(L, 2, 64, seed=1), 64, 3)
    e_cf = exact.xx_free_fermion_energy(J, h)
    assert abs(r["stats"]["energy"] - e_cf) <= 1e-10 * abs(e_cf)


def test_bose_hubbard_small_matches_ed(ctx):
    L, nmax = 5, 3
    r = run_gpu(ctx, hamiltonians.bose_hubbard(L, 1.0, 4.0, nmax),
                inputs.random_mps(L, nmax + 1, 32, seed=2), 32, 3)
    e_ed = exact.ground_energy(exact.kron_hamiltonian(L, nmax + 1,
                                                      *exact.bose_hubbard_terms(L, 1.0, 4.0, nmax)))
    assert abs(r["stats"]["energy"] - e_ed) <= 1e-10 * abs(e_ed)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_mixed_precision_with_refinement_matches_oracle(ctx, prec):
    """XXZ (Heisenberg) L=16, chi=64: split-precision sweeps, then one float64
    refinement sweep; the float64 energy matches the oracle to 1e-10."""
    L, chi = 16, 64
    mps0 = inputs.random_mps(L, 2, 16, seed=0)
    W = hamiltonians.xxz(L, 1.0, 1.0, 0.0)
    r = run_gpu(ctx, W, mps0, chi, 3, precision=prec, refine=1, tol=1e-9)
    E_ref, _, _ = od.dmrg(ompo.xxz_mpo(L, 1.0, 1.0, 0.0), mps0, chi, 4)
    assert abs(r["stats"]["energy"] - E_ref) <= 1e-10 * abs(E_ref)
    e_ed = exact.ground_energy(exact.kron_hamiltonian(L, 2, *exact.xxz_terms(L, 1.0, 1.0, 0.0)))
    assert r["stats"]["energy"] >= e_ed - 1e-10


def test_sweep_step_api_walks_the_centre(ctx):
    L = 10
    W = hamiltonians.xxz(L, 1.0, 1.0, 0.0)
    mps0 = inputs.random_mps(L, 2, 16, seed=5)
    mpo = B.MPO(ctx, W)
    mps = B.MPS(ctx, mps0, chi_cap=32)  # 2^5 = 32: exact, nothing is truncated
    B.osmps_mps_canonicalize(ctx, mps, mpo, 3, "fp64")
    p = B.sweep_params(32, 1, "fp64")
    E_prev = None
    for k in range(3, 7):
        out = B.osmps_sweep_step(ctx, mps, mpo, k, 1, p)
        assert out["chi_new"] <= 32
        if E_prev is not None:
            assert out["energy"] <= E_prev + 1e-10  # variational: each step cannot raise E
        E_prev = out["energy"]
    t = mps.tensors()
    for A in t[:7]:
        assert od.left_isometry_defect(A) < 1e-11
    assert abs(B.osmps_energy(ctx, mps, mpo) - E_prev) < 1e-9
    mps.close()
    mpo.close()


def test_fp64_emulated_sweep_matches_oracle(ctx):
    """Sweeps whose contractions and split are float64-accurate on the tensor
    cores (emulated float64) reach the oracle's energy to 1e-10."""
    L, chi = 14, 48
    mps0 = inputs.random_mps(L, 2, 16, seed=4)
    r = run_gpu(ctx, hamiltonians.xxz(L, 1.0, 1.0, 0.0), mps0, chi, 3, precision="fp64emu")
    E_ref, _, _ = od.dmrg(ompo.xxz_mpo(L, 1.0, 1.0, 0.0), mps0, chi, 3)
    assert abs(r["stats"]["energy"] - E_ref) <= 1e-10 * abs(E_ref)


@pytest.mark.parametrize("precision,refine", [("fp64", 0), ("bf16x3", 1)])
def test_long_range_ising_matches_exact(ctx, precision, refine):
    """Eq. LRIsing, alpha = 1.5 fitted by 4 exponentials (MPO w = 6), L = 10 at
    the exact bond dimension 32: the GPU ground energy equals exact
    diagonalisation of the same MPO Hamiltonian to 1e-10."""
    L = 10
    a, lam, _ = hamiltonians.exponential_fit(lambda r: r ** -1.5, L - 1, 4)
    E0 = np.linalg.eigvalsh(ompo.mpo_to_dense(ompo.long_range_ising_mpo(L, 1.0, 0.7, a, lam)))[0]
    r = run_gpu(ctx, hamiltonians.long_range_ising(L, 1.0, 0.7, a, lam),
                inputs.random_mps(L, 2, 32, seed=3), 32, 4, precision=precision, refine=refine)
    assert abs(r["stats"]["energy"] - E0) <= 1e-10 * abs(E0)
