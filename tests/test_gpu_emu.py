"""Float64-accurate GEMM emulated on the bf16 tensor cores (error-free slices):
parity with NumPy float64 products at 1e-14 norm-wise relative error (float64
rounding of the reference itself is ~1e-16), over ragged shapes, long K and
rows whose magnitudes differ by many orders (each row has its own scale)."""
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


def _run(ctx, A, Bm):
    a = torch.from_numpy(A).cuda()
    b = torch.from_numpy(Bm).cuda()
    c = torch.empty((A.shape[0], Bm.shape[1]), dtype=torch.float64, device="cuda")
    B.osmps_dgemm_emu(ctx, a, b, c)
    torch.cuda.synchronize()
    return c.cpu().numpy()


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (129, 257, 65), (300, 150, 200), (256, 384, 2048),
                                   (2048, 2048, 2048)])
def test_emulated_gemm_matches_float64(ctx, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K))
    Bm = rng.standard_normal((K, N))
    C = _run(ctx, A, Bm)
    ref = A @ Bm
    assert np.linalg.norm(C - ref) <= 1e-14 * np.linalg.norm(ref)


def test_emulated_gemm_row_scales_and_zeros(ctx):
    rng = np.random.default_rng(7)
    A = rng.standard_normal((200, 300)) * 10.0 ** rng.uniform(-8, 8, size=(200, 1))
    Bm = rng.standard_normal((300, 100)) * 10.0 ** rng.uniform(-8, 8, size=(1, 100))
    A[5] = 0.0
    Bm[:, 7] = 0.0
    C = _run(ctx, A, Bm)
    ref = A @ Bm
    # each entry is accurate relative to its own row and column scale
    scale = np.abs(A).max(axis=1, keepdims=True) * np.abs(Bm).max(axis=0, keepdims=True) * 300
    assert np.all(np.abs(C - ref) <= 1e-15 * scale + 1e-300)
    assert np.all(C[5] == 0.0) and np.all(C[:, 7] == 0.0)


def test_emulated_gemm_gram_matrix(ctx):
    """The split's Gram matrix at the chi = 1024 workload shape."""
    rng = np.random.default_rng(3)
    M = rng.standard_normal((2048, 2048)) * np.exp(-0.004 * np.arange(2048))
    M /= np.linalg.norm(M)
    G = _run(ctx, M, np.ascontiguousarray(M.T))
    ref = M @ M.T
    assert np.linalg.norm(G - ref) <= 1e-14 * np.linalg.norm(ref)
