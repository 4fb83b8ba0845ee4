"""Many chains at once (osmps_sweep_batch): every chain's result equals the
same chain swept alone, small chains reach their exact ground energies, and
failures are reported per chain."""
import numpy as np
import pytest

from oracle import exact
from paper_1703_00387_gb300 import binding as B
from paper_1703_00387_gb300 import hamiltonians, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctxs():
    import os
    if not os.path.exists(B.LIB_PATH):
        from paper_1703_00387_gb300 import build
        build.build()
    cs = [B.Context(0) for _ in range(3)]
    yield cs
    for c in cs:
        c.close()


CHAINS = [("tfi", 10, 32, 1.0), ("xxz", 12, 16, 1.0), ("tfi", 8, 16, 0.5), ("xxz", 9, 8, 0.7),
          ("tfi", 12, 24, 1.5), ("xxz", 10, 32, 1.3), ("tfi", 6, 8, 1.2)]


def _xxz_ground_energy(L, delta):
    from scipy.sparse.linalg import eigsh
    from oracle import mpo as ompo
    H = ompo.mpo_to_dense(ompo.xxz_mpo(L, 1.0, delta, 0.0))
    return float(eigsh(H, k=1, which="SA", tol=1e-13)[0][0])


def _mpo_W(model, L, p):
    return hamiltonians.ising(L, 1.0, p) if model == "tfi" else hamiltonians.xxz(L, 1.0, p, 0.0)


def _make(ctx, seed):
    mps, mpo, par = [], [], []
    for i, (model, L, chi, p) in enumerate(CHAINS):
        mpo.append(B.MPO(ctx, _mpo_W(model, L, p)))
        mps.append(B.MPS(ctx, inputs.random_mps(L, 2, chi, seed=seed + i), chi_cap=chi))
        par.append(B.sweep_params(chi, 3, "fp64", lanczos_tol=1e-12))
    return mps, mpo, par


def test_batch_equals_sequential_and_exact(ctxs):
    mps, mpo, par = _make(ctxs[0], 100)
    stats, st = B.osmps_sweep_batch(ctxs, mps, mpo, par)
    assert st == [0] * len(CHAINS)
    mps2, mpo2, par2 = _make(ctxs[0], 100)
    for i, (model, L, chi, p) in enumerate(CHAINS):
        ref = B.osmps_sweep(ctxs[0], mps2[i], mpo2[i], par2[i], record_steps=False)
        assert abs(stats[i]["energy"] - ref["energy"]) <= 1e-12 * abs(ref["energy"])
        assert stats[i]["steps"] == ref["steps"] == 2 * (L - 1) * 3
        if model == "tfi" and chi >= 2 ** (L // 2):  # exact bond dimension
            e = exact.ising_free_fermion_energy(L, 1.0, p)
            assert abs(stats[i]["energy"] - e) <= 1e-9 * abs(e)
        if model == "xxz":  # exact diagonalisation of the oracle's own MPO
            e = _xxz_ground_energy(L, p)
            if chi >= 2 ** (L // 2):
                assert abs(stats[i]["energy"] - e) <= 1e-9 * abs(e)
            else:  # truncated: variational, and close
                assert e - 1e-10 <= stats[i]["energy"] <= e + 1e-3 * abs(e)
    for x in mps + mpo + mps2 + mpo2:
        x.close()


def test_batch_reports_failing_chain(ctxs):
    mps, mpo, par = _make(ctxs[0], 200)
    bad = B.MPO(ctxs[0], hamiltonians.ising(CHAINS[2][1] + 1, 1.0, 1.0))  # one site too many
    mpo_list = list(mpo)
    mpo_list[2] = bad
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_sweep_batch(ctxs, mps, mpo_list, par)
    assert e.value.status == B.ESHAPE
    assert e.value.chain_status[2] == B.ESHAPE
    assert all(s in (0, -1) for i, s in enumerate(e.value.chain_status) if i != 2)
    for x in mps + mpo + [bad]:
        x.close()


def test_batch_rejects_shared_mps_and_shared_context(ctxs):
    mps, mpo, par = _make(ctxs[0], 300)
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_sweep_batch(ctxs, [mps[0], mps[0]], mpo[:2], par[:2])
    assert e.value.status == B.EINVAL
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_sweep_batch([ctxs[0], ctxs[0]], mps[:2], mpo[:2], par[:2])
    assert e.value.status == B.EINVAL
    for x in mps + mpo:
        x.close()
