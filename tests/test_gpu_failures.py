"""Device-side failure paths, exercised without faulting or hanging the GPU.

* Bounded waits: every wait in the library's kernels gives up after a time
  limit. osmps_selftest_wait_timeout makes one run out on purpose (an
  mbarrier that no thread arrives at, in a kernel holding tensor memory; a
  grid barrier one block never reaches) with a 2 ms limit: the call returns
  OSMPS_ETIMEOUT within a second or so, and the context, its tensor memory
  and its kernels stay usable (a tcgen05 product then still matches the
  oracle).
* Non-finite data: a NaN in the Lanczos start vector, an infinity in an
  environment, and a NaN in an MPO tensor under osmps_sweep_step all return
  OSMPS_ENAN, and the context works afterwards."""
import os
import time

import numpy as np
import pytest

from oracle import dmrg as od
from paper_1703_00387_gb300 import binding as B
from paper_1703_00387_gb300 import hamiltonians, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not os.path.exists(B.LIB_PATH):
        from paper_1703_00387_gb300 import build
        build.build()
    c = B.Context(0)
    yield c
    c.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _tcgen05_product_ok(ctx):
    Lh, W1, W2, Rh, th = inputs.random_heff_operands(96, 2, 2, 80, 5, 5, 5, seed=7)
    ref = od.heff_apply(Lh, W1, W2, Rh, th)
    t = [dev(x) for x in (Lh, W1, W2, Rh, th)]
    y = torch.empty_like(t[4])
    B.osmps_heff_apply(ctx, *t, y, precision="bf16x3")
    torch.cuda.synchronize()
    return np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-5


@pytest.mark.parametrize("which", [0, 1], ids=["mbarrier_holding_tmem", "grid_barrier"])
def test_bounded_wait_gives_up_with_etimeout(ctx, which):
    t0 = time.perf_counter()
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_selftest_wait_timeout(ctx, which, limit_us=2000.0)
    assert e.value.status == B.ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert _tcgen05_product_ok(ctx)  # tensor memory freed, context usable
    with pytest.raises(B.OsmpsError) as e:  # and the failure repeats the same way
        B.osmps_selftest_wait_timeout(ctx, which, limit_us=500.0)
    assert e.value.status == B.ETIMEOUT


def test_selftest_rejects_bad_arguments(ctx):
    for which, limit in ((2, 100.0), (0, 0.0), (1, 2e6)):
        with pytest.raises(B.OsmpsError) as e:
            B.osmps_selftest_wait_timeout(ctx, which, limit_us=limit)
        assert e.value.status == B.EINVAL


def _xxz_operator(L, k, chi, seed):
    W = hamiltonians.xxz(L, 1.0, 1.0, 0.0)
    mps = od.right_canonicalize(inputs.random_mps(L, 2, chi, seed=seed))
    Renv = od.build_right_envs(W, mps)
    theta = np.tensordot(mps[0], mps[1], axes=([2], [0]))
    return np.ones((1, 1, 1)), W[0], W[1], Renv[2], theta


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_nonfinite_start_vector_gives_enan(ctx, prec):
    Lenv, W1, W2, Renv, theta = _xxz_operator(10, 0, 16, seed=4)
    theta = theta.copy()
    theta.flat[3] = np.nan
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_lanczos_ground(ctx, dev(Lenv), dev(W1), dev(W2), dev(Renv), dev(theta),
                               max_iter=20, tol=1e-10, precision=prec)
    assert e.value.status == B.ENAN
    assert _tcgen05_product_ok(ctx)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_nonfinite_environment_gives_enan(ctx, prec):
    Lenv, W1, W2, Renv, theta = _xxz_operator(10, 0, 16, seed=5)
    Renv = Renv.copy()
    Renv.flat[Renv.size // 2] = np.inf
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_lanczos_ground(ctx, dev(Lenv), dev(W1), dev(W2), dev(Renv), dev(theta),
                               max_iter=20, tol=1e-10, precision=prec)
    assert e.value.status == B.ENAN


def test_sweep_step_with_nonfinite_mpo_gives_enan_and_recovers(ctx):
    L, chi = 10, 16
    W = hamiltonians.xxz(L, 1.0, 1.0, 0.0)
    mpo = B.MPO(ctx, W)
    mps = B.MPS(ctx, inputs.random_mps(L, 2, chi, seed=6), chi_cap=chi)
    p = B.sweep_params(chi, 1, "bf16x3", lanczos_tol=1e-10, lanczos_max_iter=20)
    B.osmps_mps_canonicalize(ctx, mps, mpo, 4, "bf16x3")
    bad = [w.copy() for w in W]
    bad[5][1, 0, 0, 1] = np.nan
    mpo.set(bad)
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_sweep_step(ctx, mps, mpo, 4, 1, p)
    assert e.value.status == B.ENAN
    # restore the operator and the state: the same step then succeeds
    mpo.set(W)
    mps.close()
    mps = B.MPS(ctx, inputs.random_mps(L, 2, chi, seed=6), chi_cap=chi)
    B.osmps_mps_canonicalize(ctx, mps, mpo, 4, "bf16x3")
    out = B.osmps_sweep_step(ctx, mps, mpo, 4, 1, p)
    assert np.isfinite(out["energy"]) and out["chi_new"] >= 1
    mps.close()
    mpo.close()
