"""Worst case for the exact partial sums of the emulated float64 GEMM: a TMEM
partial sum adds up to 1024 products of the top slices (16 K blocks of 64,
each product at most 2^14, top digits |d_0| <= 128) or 2048 products on any
other diagonal (each at most 128 * 64 = 2^13), so it stays within 2^24,
where float32 still holds every integer. Constant matrices with entries
1 - 2^-10 make every top digit 128 (diagonal 0 reaches exactly 2^24 per
partial sum); entries 1 - 2^-8 make the top digit 128 and the next -64
(diagonal 1 reaches 2^24); with one sign or alternating signs the product
must be exact (it is representable). Random matrices at long K check the
ordinary case against NumPy."""
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


@pytest.mark.parametrize("x", [1.0 - 2.0 ** -10, 1.0 - 2.0 ** -8])
@pytest.mark.parametrize("K", [1024, 4096, 5120])
@pytest.mark.parametrize("signs", ["same", "opposite", "alternating"])
def test_full_top_digits_are_exact(ctx, x, K, signs):
    M = N = 160
    A = np.full((M, K), x)
    Bm = np.full((K, N), x)
    if signs == "opposite":
        Bm = -Bm
    elif signs == "alternating":
        A[:, 1::2] = -x
    C = torch.empty((M, N), dtype=torch.float64, device="cuda")
    B.osmps_dgemm_emu(ctx, torch.from_numpy(A).cuda(), torch.from_numpy(Bm).cuda(), C)
    ref = A @ Bm  # exact here: every term is x^2, sums of powers-of-two multiples
    np.testing.assert_array_equal(C.cpu().numpy(), ref)


@pytest.mark.parametrize("M,N,K", [(300, 200, 8192), (128, 640, 2048)])
def test_long_k_random(ctx, M, N, K):
    rng = np.random.default_rng(K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-5, 5, (M, 1)))
    Bm = rng.standard_normal((K, N))
    C = torch.empty((M, N), dtype=torch.float64, device="cuda")
    B.osmps_dgemm_emu(ctx, torch.from_numpy(A).cuda(), torch.from_numpy(Bm).cuda(), C)
    ref = A @ Bm
    scale = np.abs(A) @ np.abs(Bm)
    assert np.max(np.abs(C.cpu().numpy() - ref) / scale) <= 4e-16
