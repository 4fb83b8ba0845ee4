"""GPU energy variance against the oracle (squared shifted MPO and the dense
state vector), and the paper's convergence loop (variance check, Eq.
linearExtrap) reaching an exact ground state."""
import numpy as np
import pytest

from oracle import exact, mpo as ompo, variance as ovar
from paper_1703_00387_gb300 import binding as B
from paper_1703_00387_gb300 import convergence, hamiltonians, inputs

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


@pytest.mark.parametrize("model", ["ising", "xxz"])
def test_variance_random_state(ctx, model):
    L = 9
    if model == "ising":
        Wp, Wo = hamiltonians.ising(L, 1.0, 0.8), ompo.ising_mpo(L, 1.0, 0.8)
    else:
        J, h = inputs.random_couplings(L, seed=4)
        Wp, Wo = hamiltonians.xxz(L, J, 0.9, h), ompo.xxz_mpo(L, J, 0.9, h)
    tensors = inputs.random_mps(L, 2, 8, seed=6)
    mps = B.MPS(ctx, tensors, chi_cap=8)
    mpo = B.MPO(ctx, Wp)
    E, V = B.osmps_variance(ctx, mps, mpo)
    Eo, Vo = ovar.mps_variance(Wo, tensors)
    Ed, Vd = ovar.dense_variance(Wo, tensors)
    assert abs(E - Eo) <= 1e-12 * abs(Eo)
    assert abs(V - Vo) <= 1e-11 * Vo and abs(V - Vd) <= 1e-11 * Vd
    mps.close()
    mpo.close()


def test_variance_of_converged_state_matches_oracle(ctx):
    L = 12
    mps = B.MPS(ctx, inputs.random_mps(L, 2, 64, seed=0), chi_cap=64)
    mpo = B.MPO(ctx, hamiltonians.ising(L, 1.0, 1.0))
    B.osmps_sweep(ctx, mps, mpo, B.sweep_params(64, 3, "fp64", lanczos_tol=1e-13), record_steps=False)
    E, V = B.osmps_variance(ctx, mps, mpo)
    Eo, Vo = ovar.mps_variance(ompo.ising_mpo(L, 1.0, 1.0), mps.tensors())
    assert abs(E - Eo) <= 1e-12 * abs(Eo)
    assert abs(V - Vo) <= 1e-12 and V < 1e-10
    mps.close()
    mpo.close()


def test_convergence_loop_reaches_exact_ground_state(ctx):
    """TFI L=12, g=1, chi_max=64 (exact): the loop stops once V <= L eps_V."""
    L = 12
    mps = B.MPS(ctx, inputs.random_mps(L, 2, 32, seed=0), chi_cap=64)
    mpo = B.MPO(ctx, hamiltonians.ising(L, 1.0, 1.0))
    out = convergence.ground_state(ctx, mps, mpo, 64, eps_var=1e-12, n_inner=2, n_outer=4,
                                   lanczos_tol=1e-13)
    assert out["converged"]
    assert out["variance"] <= L * 1e-12
    e_cf = exact.ising_free_fermion_energy(L, 1.0, 1.0)
    assert abs(out["energy"] - e_cf) <= 1e-10 * abs(e_cf)
    mps.close()
    mpo.close()


def test_variance_unsupported_block(ctx):
    mps = B.MPS(ctx, inputs.random_mps(6, 5, 4, seed=1), chi_cap=4)
    mpo = B.MPO(ctx, hamiltonians.bose_hubbard(6, 1.0, 4.0, 4))  # w^2 d = 80
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_variance(ctx, mps, mpo)
    assert e.value.status == B.EUNSUPPORTED
    mps.close()
    mpo.close()
