"""Host-side checks that need no GPU: the library builds and exports every
symbol declared in include/osmps.h, the binding covers them, and the
library's MPO builder agrees with the oracle's."""
import os
import re

import numpy as np
import pytest

from oracle import mpo as ompo
from paper_1703_00387_gb300 import binding, hamiltonians, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "osmps.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(osmps_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def built_lib():
    if not os.path.exists(binding.LIB_PATH):
        from paper_1703_00387_gb300 import build
        build.build()
    return binding.lib()


def test_library_exports_every_declared_symbol(built_lib):
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(built_lib, name), f"{name} declared in osmps.h but not exported"


def test_binding_covers_header():
    assert sorted(binding.exported_symbols()) == _declared()


def test_status_strings(built_lib):
    for code, name in binding.STATUS.items():
        assert built_lib.osmps_status_string(code).decode() == name


def test_ctx_create_without_gpu_reports_error(built_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes
    p = ctypes.c_void_p()
    st = built_lib.osmps_ctx_create(0, 0, ctypes.byref(p))
    assert st != 0
    assert b"device" in built_lib.osmps_last_error().lower() or st == 4


@pytest.mark.parametrize("name", ["ising", "xxz", "bh"])
def test_mpo_builders_agree_with_oracle(name):
    if name == "ising":
        a, b = hamiltonians.ising(7, 0.9, 1.3), ompo.ising_mpo(7, 0.9, 1.3)
    elif name == "xxz":
        J, h = inputs.random_couplings(7, seed=4)
        a, b = hamiltonians.xxz(7, J, 0.6, h), ompo.xxz_mpo(7, J, 0.6, h)
    else:
        a, b = hamiltonians.bose_hubbard(5, 1.0, 4.0, 4), ompo.bose_hubbard_mpo(5, 1.0, 4.0, 4)
    assert len(a) == len(b)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x.shape, y.shape)
        np.testing.assert_allclose(x, y, atol=1e-15)


def test_aklt_builder_same_operator():
    np.testing.assert_allclose(ompo.mpo_to_dense(hamiltonians.aklt(4)),
                               ompo.mpo_to_dense(ompo.aklt_mpo(4)), atol=1e-13)


def test_seeded_inputs_are_deterministic():
    a = inputs.random_mps(10, 2, 16, seed=0)
    b = inputs.random_mps(10, 2, 16, seed=0)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    assert [t.shape[0] for t in a] == inputs.bond_dims(10, 2, 16)[:10]
    batch = inputs.chain_batch(64, seed=0)
    assert len(batch) == 64 and all(16 <= c["L"] <= 128 for c in batch)


def test_xxz_coupling_basis_rebuilds_oracle_mpo():
    """W_0 + sum_j p_j B_j equals the oracle's XXZ MPO at random couplings,
    and every basis row touches only its own site (J_i: site i, h_i: site i)."""
    L = 9
    W0, row_ptr, col, val = hamiltonians.xxz_coupling_basis(L, 0.7)
    rng = np.random.default_rng(3)
    p = rng.standard_normal(2 * L - 1)
    flat = np.concatenate([w.ravel() for w in W0])
    for j in range(2 * L - 1):
        sl = slice(row_ptr[j], row_ptr[j + 1])
        np.add.at(flat, col[sl], p[j] * val[sl])
    ref = np.concatenate([w.ravel() for w in ompo.xxz_mpo(L, p[:L - 1], 0.7, p[L - 1:])])
    np.testing.assert_array_equal(flat, ref)
    ends = np.cumsum([w.size for w in W0])
    site_of = np.searchsorted(ends, col, side="right")
    for j in range(2 * L - 1):
        k = j if j < L - 1 else j - (L - 1)
        assert set(site_of[row_ptr[j]:row_ptr[j + 1]]) == {k}


def test_tdvp_binding_rejects_mismatched_states_on_the_host():
    # shape checks run before any device work: a wrong site count would make
    # the library read past the bond-dimension array
    import numpy as np
    from paper_1703_00387_gb300 import binding as B

    class FakeMPO:
        L = 3
        shapes = [(1, 2, 2, 5), (5, 2, 2, 5), (5, 2, 2, 1)]
        ptr = None

    good = [np.zeros((1, 2, 2)), np.zeros((2, 2, 2)), np.zeros((2, 2, 1))]
    with pytest.raises(ValueError):
        B.osmps_tdvp_evolve(None, FakeMPO(), good[:2], 0.1, 1, chi_max=4)
    with pytest.raises(ValueError):
        B.osmps_tdvp_evolve(None, FakeMPO(), [good[0], np.zeros((2, 3, 2)), good[2]], 0.1, 1, chi_max=4)
    with pytest.raises(ValueError):
        B.osmps_tdvp_evolve(None, FakeMPO(), [good[0], np.zeros((2, 2, 3)), good[2]], 0.1, 1, chi_max=4)
