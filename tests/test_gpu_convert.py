"""The integer-field float conversions used by the kernels (narrowing with
round to nearest, ties to even; exact widening) equal the IEEE-754
conversions bit for bit, on random values over the whole range and on the
edge cases: exact ties at both parities, carries into the exponent, the
largest finite floats and overflow, the subnormal boundary, zeros of both
signs, infinities and NaN."""
import numpy as np
import pytest

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
    yield c
    c.close()


def _edge_doubles():
    f32max = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    xs = [0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, f32max, -f32max, tiny, -tiny, tiny / 2, tiny * 0.75,
          1e-300, 1e300, 3.5e38, np.nextafter(f32max, np.inf)]
    # ties: 1 + (2k+1) 2^-24 lies halfway between two floats (both parities)
    for k in range(8):
        xs += [1.0 + (2 * k + 1) * 2.0 ** -24, -(1.0 + (2 * k + 1) * 2.0 ** -24),
               2.0 ** 60 * (1.0 + (2 * k + 1) * 2.0 ** -24)]
    # just around ties, and a carry into the exponent (all-ones fraction rounds up)
    xs += [1.0 + 2.0 ** -24 + 2.0 ** -52, 1.0 + 2.0 ** -24 - 2.0 ** -53, 2.0 - 2.0 ** -25, 2.0 - 2.0 ** -24,
           4.0 - 2.0 ** -23 - 2.0 ** -30]
    return np.array(xs, dtype=np.float64)


def test_conversions_match_ieee(ctx):
    rng = np.random.default_rng(0)
    n = 1 << 20
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-160, 140, n)
    x64 = np.ldexp(mant, expo) * rng.choice([-1.0, 1.0], n)
    x64 = np.concatenate([x64, _edge_doubles(), [np.nan]])
    x32 = (rng.standard_normal(x64.size) * np.exp(rng.uniform(-80, 80, x64.size))).astype(np.float32)
    x32[:6] = np.array([0.0, -0.0, np.inf, -np.inf, np.finfo(np.float32).tiny / 4, np.nan], np.float32)
    y32, y64 = B.osmps_selftest_convert(ctx, torch.from_numpy(x64).cuda(), torch.from_numpy(x32).cuda())
    with np.errstate(over="ignore"):  # values past the float32 range become infinities
        r32 = x64.astype(np.float32)
    g32 = y32.cpu().numpy()
    nan = np.isnan(r32)
    assert np.isnan(g32[nan]).all()
    np.testing.assert_array_equal(g32[~nan].view(np.uint32), r32[~nan].view(np.uint32))
    r64 = x32.astype(np.float64)
    g64 = y64.cpu().numpy()
    nan = np.isnan(r64)
    assert np.isnan(g64[nan]).all()
    np.testing.assert_array_equal(g64[~nan].view(np.uint64), r64[~nan].view(np.uint64))


def test_bf16_rounding_matches_cuda(ctx):
    """The U(1) operand split rounds float64 to bf16 through float32 rounded
    to odd (integer fields): bit for bit CUDA's __double2bfloat16 on random
    values over the float range and beyond, on values exactly halfway
    between two bf16 numbers (both parities, which a plain double rounding
    through float would get wrong when float rounds onto the halfway point),
    carries into the exponent, zeros, infinities, subnormals and NaN."""
    rng = np.random.default_rng(1)
    n = 1 << 20
    x = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-140, 135, n)) * rng.choice([-1.0, 1.0], n)
    edge = [0.0, -0.0, np.inf, -np.inf, np.nan, 1e-300, -1e-300, 1e300, 3.4e38, -3.4e38,
            float(np.finfo(np.float32).tiny), float(np.finfo(np.float32).tiny) / 3]
    for k in range(8):
        m = 1.0 + (2 * k + 1) * 2.0 ** -8  # halfway between bf16 neighbours
        edge += [m, -m, m + 2.0 ** -40, m - 2.0 ** -40, m + 2.0 ** -52, m * 2.0 ** 100]
    edge += [2.0 - 2.0 ** -9, 2.0 - 2.0 ** -30, 1.0 + 2.0 ** -8 + 2.0 ** -33]
    x = np.concatenate([x, np.array(edge)])
    yi, yh = B.osmps_selftest_bf16(ctx, torch.from_numpy(x).cuda())
    np.testing.assert_array_equal(yi.cpu().numpy(), yh.cpu().numpy())
