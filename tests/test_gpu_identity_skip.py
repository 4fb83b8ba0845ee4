"""Identity environment channels (Sec. 3.2: the MPO's identity corners make
one channel of a left-canonical L and of a right-canonical R the unit
matrix). The split-precision H_eff.theta leaves such a channel out of both
GEMMs; the product must still match the oracle's full contraction at the
reduced-precision bar, and the GEMMs must do only the work of the other
channels (tensor-core FLOPs read back from the library's kernel timing)."""
import numpy as np
import pytest

from oracle import dmrg as od
from paper_1703_00387_gb300 import binding as B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import os
    if not os.path.exists(B.LIB_PATH):
        from paper_1703_00387_gb300 import build
        build.build()
    c = B.Context(0)
    c.set_identity_skip("always")  # single products look for identity channels too
    yield c
    c.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _operands(chi_l, chi_r, w, l_id, r_id, seed):
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((chi_l, w, chi_l))
    R = rng.standard_normal((chi_r, w, chi_r))
    if l_id is not None:
        L[:, l_id, :] = np.eye(chi_l)
    if r_id is not None:
        R[:, r_id, :] = np.eye(chi_r)
    W1 = rng.standard_normal((w, 2, 2, w))
    W2 = rng.standard_normal((w, 2, 2, w))
    W1[np.abs(W1) < 0.8] = 0.0  # sparse, like an MPO
    W2[np.abs(W2) < 0.8] = 0.0
    theta = rng.standard_normal((chi_l, 2, 2, chi_r))
    return L, W1, W2, R, theta


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("l_id,r_id", [(4, 0), (0, 4), (4, None), (None, 0), (None, None)])
@pytest.mark.parametrize("chi_l,chi_r", [(96, 130), (257, 64)])
def test_identity_channels_skipped_and_exact(ctx, prec, l_id, r_id, chi_l, chi_r):
    w = 5
    L, W1, W2, R, theta = _operands(chi_l, chi_r, w, l_id, r_id, seed=chi_l + 7 * chi_r)
    ref = od.heff_apply(L, W1, W2, R, theta)
    t = [dev(x) for x in (L, W1, W2, R, theta)]
    y = torch.empty_like(t[4])
    B.osmps_profile_enable(ctx, True)
    B.osmps_heff_apply(ctx, *t, y, precision=prec)
    torch.cuda.synchronize()
    p = B.osmps_profile_read(ctx, "gemm_tc")
    B.osmps_profile_enable(ctx, False)
    err = np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err
    wl_g = w - (l_id is not None)
    wr_g = w - (r_id is not None)
    n1 = 4 * chi_r
    expect = 2.0 * chi_l * wl_g * n1 * chi_l + 2.0 * (chi_l * 4) * chi_r * (wr_g * chi_r)
    assert p["flops"] == pytest.approx(expect, rel=1e-12)


def test_near_identity_channel_is_not_skipped(ctx):
    """A channel off the unit matrix by more than the tolerance (1e-3) runs
    through the GEMM as usual."""
    w, chi = 5, 80
    L, W1, W2, R, theta = _operands(chi, chi, w, 4, 0, seed=3)
    L[3, 4, 5] = 2e-3
    ref = od.heff_apply(L, W1, W2, R, theta)
    t = [dev(x) for x in (L, W1, W2, R, theta)]
    y = torch.empty_like(t[4])
    B.osmps_profile_enable(ctx, True)
    B.osmps_heff_apply(ctx, *t, y, precision="bf16x3")
    torch.cuda.synchronize()
    p = B.osmps_profile_read(ctx, "gemm_tc")
    B.osmps_profile_enable(ctx, False)
    assert np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-5
    expect = 2.0 * chi * w * 4 * chi * chi + 2.0 * (chi * 4) * chi * ((w - 1) * chi)
    assert p["flops"] == pytest.approx(expect, rel=1e-12)


def test_identity_skip_modes(ctx):
    """'off' runs every channel; 'solver' skips in solvers, not in single
    products; a bad mode is refused."""
    w, chi = 5, 64
    L, W1, W2, R, theta = _operands(chi, chi, w, 4, 0, seed=9)
    t = [dev(x) for x in (L, W1, W2, R, theta)]
    y = torch.empty_like(t[4])
    full = 2.0 * chi * w * 4 * chi * chi + 2.0 * (chi * 4) * chi * (w * chi)
    try:
        for mode in ("off", "solver"):
            ctx.set_identity_skip(mode)
            B.osmps_profile_enable(ctx, True)
            B.osmps_heff_apply(ctx, *t, y, precision="bf16x3")
            torch.cuda.synchronize()
            p = B.osmps_profile_read(ctx, "gemm_tc")
            B.osmps_profile_enable(ctx, False)
            assert p["flops"] == pytest.approx(full, rel=1e-12)
        with pytest.raises(B.OsmpsError) as e:
            ctx.set_identity_skip(3)
        assert e.value.status == B.EINVAL
    finally:
        ctx.set_identity_skip("always")


def test_split_precision_environment_identity_is_skipped(ctx):
    """An environment updated in bf16x3 from a left-canonical tensor keeps its
    identity channel only to a few 1e-6: still skipped, and the product is
    within the bar of the product with the exact identity channel."""
    from paper_1703_00387_gb300 import hamiltonians, inputs
    chi, w = 192, 5
    W = hamiltonians.xxz(8, 1.0, 1.0, 0.0)[3]
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((2 * chi, chi)))
    A = Q.reshape(chi, 2, chi)
    L0 = inputs.random_symmetric_env(chi, w, seed=2)
    L0[:, w - 1, :] = np.eye(chi)
    Lg = torch.empty((chi, w, chi), dtype=torch.float64, device="cuda")
    B.osmps_env_update(ctx, 0, dev(L0), dev(A), dev(W), Lg, precision="bf16x3")
    Lh = Lg.cpu().numpy()
    dev_id = np.abs(Lh[:, w - 1, :] - np.eye(chi)).max()
    assert 0.0 < dev_id <= 1e-4
    R = inputs.random_symmetric_env(chi, w, seed=3)
    R[:, 0, :] = np.eye(chi)
    theta = rng.standard_normal((chi, 2, 2, chi))
    Lexact = Lh.copy()
    Lexact[:, w - 1, :] = np.eye(chi)
    ref = od.heff_apply(Lexact, W, W, R, theta)
    y = torch.empty((chi, 2, 2, chi), dtype=torch.float64, device="cuda")
    B.osmps_profile_enable(ctx, True)
    B.osmps_heff_apply(ctx, Lg, dev(W), dev(W), dev(R), dev(theta), y, precision="bf16x3")
    torch.cuda.synchronize()
    p = B.osmps_profile_read(ctx, "gemm_tc")
    B.osmps_profile_enable(ctx, False)
    assert np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-5
    expect = 2.0 * chi * (w - 1) * 4 * chi * chi + 2.0 * (chi * 4) * chi * ((w - 1) * chi)
    assert p["flops"] == pytest.approx(expect, rel=1e-12)
