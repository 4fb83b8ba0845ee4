"""The allocation-free H_eff.theta entry point, for callers that cannot
allocate device memory (a process that reserved its whole budget up front,
a loop that must not synchronise on an allocation, a plug-in that may not
own allocations). It runs on a fixed scratch array inside the library, so
this test checks it through the C ABI against osmps_heff_apply (float64) and
against the float64 oracle, on two calls in a row with different shapes (the
second call must not be disturbed by what the first left in the shared
scratch); that repeated calls, one of them on a non-default stream, leave the
device's free memory unchanged (read with cudaMemGetInfo, beneath torch's
caching allocator); and that sizes beyond the fixed scratch are refused with
OSMPS_ESHAPE. It sits in a file collected last so a failure here leaves every
other test already run."""
import ctypes
import os

import numpy as np
import pytest

from oracle import dmrg as od
from paper_1703_00387_gb300 import binding as B
from paper_1703_00387_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = (((96, 2, 2, 80, 5, 5, 5), 31), ((33, 3, 3, 20, 4, 6, 3), 32))


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _lib():
    if not os.path.exists(B.LIB_PATH):
        from paper_1703_00387_gb300 import build
        build.build()
    return B.lib()


def _free_bytes():
    """Free device memory of the current device from the CUDA runtime the
    library itself loaded (torch's allocator does not see the library's)."""
    rt = ctypes.CDLL("libcudart.so.13")
    free, total = ctypes.c_size_t(), ctypes.c_size_t()
    assert rt.cudaMemGetInfo(ctypes.byref(free), ctypes.byref(total)) == 0
    return free.value


def test_noalloc_matches_heff_apply_and_oracle_on_two_calls():
    _lib()
    torch.cuda.set_device(0)
    ctx = B.Context(0)
    for shape, seed in SHAPES:
        host = inputs.random_heff_operands(*shape, seed=seed)
        ref = od.heff_apply(*host)
        ops = [_dev(x) for x in host]
        y_ref = torch.empty_like(ops[4])
        B.osmps_heff_apply(ctx, *ops, y_ref, precision="fp64")
        y = torch.full_like(ops[4], float("nan"))
        B.osmps_heff_apply_noalloc(*ops, y)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(y - y_ref) / torch.linalg.norm(y_ref))
        assert err <= 1e-12, (shape, err)
        err_oracle = np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err_oracle <= 1e-12, (shape, err_oracle)
    ctx.close()


def test_noalloc_allocates_nothing_on_any_stream():
    _lib()
    torch.cuda.set_device(0)
    cases = []
    for shape, seed in SHAPES:
        host = inputs.random_heff_operands(*shape, seed=seed)
        ops = [_dev(x) for x in host]
        cases.append((ops, torch.empty_like(ops[4]), od.heff_apply(*host)))
    side = torch.cuda.Stream()
    for ops, y, _ in cases:  # warm-up: loads the kernels and looks up the scratch address
        B.osmps_heff_apply_noalloc(*ops, y)
    torch.cuda.synchronize()
    before = _free_bytes()
    for rep in range(3):
        for ops, y, _ in cases:
            B.osmps_heff_apply_noalloc(*ops, y)
    with torch.cuda.stream(side):
        for ops, y, _ in cases:
            B.osmps_heff_apply_noalloc(*ops, y, stream=side)
    torch.cuda.synchronize()
    assert _free_bytes() == before
    for ops, y, ref in cases:  # the last calls ran on the side stream
        err = np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= 1e-12, err


def test_noalloc_rejects_sizes_beyond_its_scratch():
    big = [_dev(x) for x in inputs.random_heff_operands(512, 2, 2, 512, 5, 5, 5, seed=1)]
    y = torch.empty_like(big[4])
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_heff_apply_noalloc(*big, y)
    assert e.value.status == 2 and "scratch" in str(e.value)


def test_noalloc_checks_devices_and_shapes_before_the_call():
    ops = [_dev(x) for x in inputs.random_heff_operands(16, 2, 2, 12, 3, 3, 3, seed=5)]
    y = torch.empty_like(ops[4])
    short_y = torch.empty(16 * 2 * 2 * 11, dtype=torch.float64, device="cuda:0").view(16, 2, 2, 11)
    with pytest.raises(ValueError):
        B.osmps_heff_apply_noalloc(*ops, short_y)
    small_R = torch.zeros(11, 3, 11, dtype=torch.float64, device="cuda:0")
    with pytest.raises(ValueError):
        B.osmps_heff_apply_noalloc(ops[0], ops[1], ops[2], small_R, ops[4], y)
    if torch.cuda.device_count() > 1:
        with pytest.raises(ValueError):
            B.osmps_heff_apply_noalloc(*ops[:4], ops[4].to("cuda:1"), y)
