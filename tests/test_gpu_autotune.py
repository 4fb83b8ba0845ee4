"""Tile-width autotuning of the tcgen05 GEMMs: the first product of a size
class is timed at widths 256, 128 and 64 and the fastest kept; every width
gives the same bits (the per-element arithmetic does not depend on it), on
ragged shapes of the dense H_eff.theta and of the U(1) grouped product."""
import numpy as np
import pytest

from oracle import dmrg as od
from paper_1703_00387_gb300 import binding as B
from paper_1703_00387_gb300 import hamiltonians, inputs
from paper_1703_00387_gb300 import u1 as pu1

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx():
    import os
    if not os.path.exists(B.LIB_PATH):
        from paper_1703_00387_gb300 import build
        build.build()
    c = B.Context(0)
    yield c
    c.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("chi_l,chi_r", [(200, 130), (77, 300)])
def test_widths_give_identical_products(ctx, prec, chi_l, chi_r):
    Lh, W1, W2, Rh, th = inputs.random_heff_operands(chi_l, 2, 2, chi_r, 5, 5, 5, seed=chi_l)
    ref = od.heff_apply(Lh, W1, W2, Rh, th)
    t = [dev(x) for x in (Lh, W1, W2, Rh, th)]
    y = torch.empty_like(t[4])
    B.osmps_heff_apply(ctx, *t, y, precision=prec)  # tunes both stages' classes
    table = ctx.tuning()
    assert len(table) >= 2
    for e in table:
        assert e["width"] in (64, 128, 256)
        assert all(v > 0.0 for v in e["us"].values())
        assert e["width"] == int(min(e["us"], key=lambda k: e["us"][k]))
    outs = []
    for width in (256, 128, 64):
        for e in table:
            ctx.set_tuning(e["key"], width)
        B.osmps_heff_apply(ctx, *t, y, precision=prec)
        outs.append(y.cpu().numpy().copy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    assert np.linalg.norm(outs[0] - ref) / np.linalg.norm(ref) <= 1e-5


def test_autotune_off_uses_full_width(ctx):
    ctx.set_autotune(False)
    Lh, W1, W2, Rh, th = inputs.random_heff_operands(64, 2, 2, 64, 5, 5, 5, seed=1)
    t = [dev(x) for x in (Lh, W1, W2, Rh, th)]
    y = torch.empty_like(t[4])
    B.osmps_heff_apply(ctx, *t, y, precision="bf16x3")
    assert ctx.tuning() == []
    with pytest.raises(B.OsmpsError) as e:
        ctx.set_tuning([0, 0, 0, 1, 1, 1], 96)
    assert e.value.status == B.EINVAL


def test_u1_grouped_widths_identical(ctx):
    L_chain, nmax = 8, 2
    W = hamiltonians.bose_hubbard(L_chain, 1.0, 4.0, nmax)
    q = pu1.channel_charges(W)
    left = inputs.u1_sector_profile(3.0, total=90, width=3.0)
    right = inputs.u1_sector_profile(5.0, total=110, width=3.0)
    outs = []
    for width in (None, 256, 128, 64):
        op = pu1.U1Operator(ctx, left, right, nmax + 1, nmax + 1, W[3], W[4], q[3], q[5])
        pl = op.plan
        Lp = dev(inputs.random_dense((pl.n_L,), 1))
        Rp = dev(inputs.random_dense((pl.n_R,), 2))
        th = dev(inputs.random_dense((pl.n_theta,), 3))
        if width is not None:
            for e in ctx.tuning():
                if e["key"][0] == 1:
                    ctx.set_tuning(e["key"], width)
        B.osmps_u1_heff_prepare(ctx, pl, Lp, dev(W[3]), dev(W[4]), Rp, precision="bf16x3")
        y = torch.empty_like(th)
        B.osmps_u1_heff_apply(ctx, pl, th, y)
        outs.append(y.cpu().numpy().copy())
        op.close()
    assert any(e["key"][0] == 1 for e in ctx.tuning())
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)
