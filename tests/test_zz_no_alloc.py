"""The allocation-free H_eff.theta entry point, for callers that cannot
allocate device memory (a process that reserved its whole budget up front,
a loop that must not synchronise on an allocation, a plug-in that may not
own allocations). It runs on a fixed scratch array inside the library, so
this test checks it through the C ABI against osmps_heff_apply (float64),
on two calls in a row with different shapes (the second call must not be
disturbed by what the first left in the shared scratch), and that sizes
beyond the fixed scratch are refused with OSMPS_ESHAPE. It sits in a file
collected last so a failure here leaves every other test already run."""
import os

import numpy as np
import pytest

from paper_1703_00387_gb300 import binding as B
from paper_1703_00387_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def test_noalloc_matches_heff_apply_on_two_calls():
    if not os.path.exists(B.LIB_PATH):
        from paper_1703_00387_gb300 import build
        build.build()
    torch.cuda.set_device(0)
    ctx = B.Context(0)
    for shape, seed in (((96, 2, 2, 80, 5, 5, 5), 31), ((33, 3, 3, 20, 4, 6, 3), 32)):
        ops = [_dev(x) for x in inputs.random_heff_operands(*shape, seed=seed)]
        y_ref = torch.empty_like(ops[4])
        B.osmps_heff_apply(ctx, *ops, y_ref, precision="fp64")
        y = torch.full_like(ops[4], float("nan"))
        B.osmps_heff_apply_noalloc(*ops, y)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(y - y_ref) / torch.linalg.norm(y_ref))
        assert err <= 1e-12, (shape, err)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    big = [_dev(x) for x in inputs.random_heff_operands(512, 2, 2, 512, 5, 5, 5, seed=1)]
    y = torch.empty_like(big[4])
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_heff_apply_noalloc(*big, y)
    assert e.value.status == 2 and "scratch" in str(e.value)
