"""Split precision at chi = 1024 against an exact float64 reference.

The open XXZ chain at L = 20 needs bond dimension 2^10 = 1024 at its middle
bond and no more, so two-site sweeps with chi_max = 1024 carry no
truncation beyond eps_local and must reach the exact ground energy. That
energy comes from sparse exact diagonalisation by the oracle
(tests/golden/make_xxz_l20.py). The bf16x3 sweeps plus one float64-accurate
refinement sweep must reach it to 1e-10 relative (the bar for ground
energies after refinement), exactly like the plain float64 path; the
largest split here is a 1024 x 1024 Gram matrix of a 512 x 2 x 2 x 512
two-site tensor."""
import json
import os

import numpy as np
import pytest

from paper_1703_00387_gb300 import binding as B
from paper_1703_00387_gb300 import hamiltonians, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "xxz_l20_ground_energy.json")


@pytest.fixture(scope="module")
def ctx():
    if not os.path.exists(B.LIB_PATH):
        from paper_1703_00387_gb300 import build
        build.build()
    c = B.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("prec,sweeps,refine", [("bf16x3", 3, 1), ("fp64", 3, 0)])
def test_xxz_l20_chi1024_reaches_exact_energy(ctx, prec, sweeps, refine):
    with open(GOLDEN) as f:
        e0 = json.load(f)["ground_energy"]
    L, chi = 20, 1024
    mpo = B.MPO(ctx, hamiltonians.xxz(L, 1.0, 1.0, 0.0))
    mps = B.MPS(ctx, inputs.random_mps(L, 2, chi, seed=0), chi_cap=chi)
    assert max(mps.bond_dims()) == chi
    p = B.sweep_params(chi, sweeps, prec, lanczos_tol=1e-12, lanczos_max_iter=100,
                       refine_sweeps=refine)
    st = B.osmps_sweep(ctx, mps, mpo, p, record_steps=False)
    mps.close()
    mpo.close()
    assert abs(st["energy"] - e0) <= 1e-10 * abs(e0), (st["energy"], e0)
