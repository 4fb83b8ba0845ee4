"""GPU parity of the single operations against the FP64 oracle.

Bars (norm-wise relative error of the output): 1e-12 for OSMPS_PREC_FP64
and the emulated float64 mode, 1e-5 for both reduced-precision modes
(bf16x3, tf32x3) at every shape. A bf16 hi+lo pair carries 16 significant
bits (|x - hi - lo| <= 2^-16 |x|); over the four split factors of H_eff.theta
the norm-wise error measures about 6e-6 on every shape here. Environment
updates of under 2^20 multiply-adds run in float64 in every precision (too
few terms meet there for the split errors to average). Shapes cover a single
tile, several tiles with ragged tails in M, N and K, and the full chi = 1024
shape the benchmark times."""
import numpy as np
import pytest

from oracle import dmrg as od
from paper_1703_00387_gb300 import binding as B
from paper_1703_00387_gb300 import hamiltonians, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "bf16x3": 1e-5, "tf32x3": 1e-5, "fp64emu": 1e-12}
TOL_FULL = TOL


@pytest.fixture(scope="module")
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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


HEFF_SHAPES = [
    (5, 2, 2, 7, 3, 3, 3),        # single tile, tiny
    (130, 2, 2, 70, 5, 5, 5),     # ragged M (650 rows), N (280), K (130 -> 192)
    (64, 2, 2, 64, 1, 5, 5),      # left boundary (wl = 1)
    (40, 3, 3, 33, 14, 14, 14),   # AKLT-sized MPO (w = 14, d = 3)
    (48, 5, 5, 40, 4, 4, 4),      # Bose-Hubbard local dimension d = 5
    (200, 2, 2, 256, 5, 5, 1),    # right boundary (wr = 1), exact N tile
]


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32x3", "fp64emu"])
@pytest.mark.parametrize("shape", HEFF_SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_heff_apply_parity(ctx, prec, shape):
    Lh, W1, W2, Rh, th = inputs.random_heff_operands(*shape, seed=sum(shape))
    ref = od.heff_apply(Lh, W1, W2, Rh, th)
    t = [dev(x) for x in (Lh, W1, W2, Rh, th)]
    y = torch.empty_like(t[4])
    B.osmps_heff_apply(ctx, *t, y, precision=prec)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "fp64", "fp64emu"])
def test_heff_apply_full_size_chi1024(ctx, prec):
    """The benchmark's shape: chi_l = chi_r = 1024, d = 2, w = 5 (XXZ)."""
    Lh, W1, W2, Rh, th = inputs.random_heff_operands(1024, 2, 2, 1024, 5, 5, 5, seed=1024)
    ref = od.heff_apply(Lh, W1, W2, Rh, th)
    t = [dev(x) for x in (Lh, W1, W2, Rh, th)]
    y = torch.empty_like(t[4])
    B.osmps_heff_apply(ctx, *t, y, precision=prec)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), ref) <= TOL_FULL[prec]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_heff_apply_many_ragged_tiles(ctx, prec):
    """GEMMs of more tiles than the GPU has SMs but not a whole number of
    waves (stage 1: 51 x 5 = 255 tiles, stage 4: 41 x 2 = 82, on 152 SMs),
    with ragged M and N edges and K padded to the slice size. Parity with the
    oracle at the full-size bar, and bit-identical repeats."""
    Lh, W1, W2, Rh, th = inputs.random_heff_operands(1300, 2, 2, 300, 5, 5, 5, seed=1300)
    ref = od.heff_apply(Lh, W1, W2, Rh, th)
    t = [dev(x) for x in (Lh, W1, W2, Rh, th)]
    ys = []
    for _ in range(2):
        y = torch.empty_like(t[4])
        B.osmps_heff_apply(ctx, *t, y, precision=prec)
        torch.cuda.synchronize()
        ys.append(y.cpu().numpy())
    assert rel(ys[0], ref) <= TOL_FULL[prec]
    np.testing.assert_array_equal(ys[0], ys[1])


def test_heff_apply_repeat_is_deterministic(ctx):
    Lh, W1, W2, Rh, th = inputs.random_heff_operands(96, 2, 2, 96, 5, 5, 5, seed=3)
    t = [dev(x) for x in (Lh, W1, W2, Rh, th)]
    ys = []
    for _ in range(2):
        y = torch.empty_like(t[4])
        B.osmps_heff_apply(ctx, *t, y, precision="bf16x3")
        ys.append(y.cpu().numpy())
    np.testing.assert_array_equal(ys[0], ys[1])


ENV_SHAPES = [(6, 2, 9, 3, 3), (130, 2, 100, 5, 5), (64, 3, 50, 14, 14), (1, 2, 2, 1, 5), (33, 5, 40, 4, 4),
              (600, 2, 500, 5, 5)]  # the last: 96-tile GEMMs


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32x3", "fp64emu"])
@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("shape", ENV_SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_env_update_parity(ctx, prec, side, shape):
    chi_l, d, chi_r, w_in, w_out = shape
    env, A, W = inputs.random_env_operands(chi_l, d, chi_r, w_in, w_out, side, seed=sum(shape) + side)
    if side == 0:
        ref = od.env_left(env, A, W)
        out = torch.empty((chi_r, w_out, chi_r), dtype=torch.float64, device="cuda:0")
    else:
        ref = od.env_right(env, A, W)
        out = torch.empty((chi_l, w_out, chi_l), dtype=torch.float64, device="cuda:0")
    B.osmps_env_update(ctx, side, dev(env), dev(A), dev(W), out, precision=prec)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), ref) <= TOL[prec]


@pytest.mark.parametrize("shape", [(3, 2, 5, 2, 4), (100, 2, 70, 3, 90), (1024, 2, 1024, 2, 1024)])
def test_theta_form_parity(ctx, shape):
    chi_l, d1, chi_m, d2, chi_r = shape
    rng = np.random.default_rng(5)
    A1 = rng.standard_normal((chi_l, d1, chi_m))
    A2 = rng.standard_normal((chi_m, d2, chi_r))
    ref = np.tensordot(A1, A2, axes=([2], [0]))
    th = torch.empty(ref.shape, dtype=torch.float64, device="cuda:0")
    B.osmps_theta_form(ctx, dev(A1), dev(A2), th)
    torch.cuda.synchronize()
    assert rel(th.cpu().numpy(), ref) <= 1e-13


def _split_case(seed, shape, decay):
    """theta with a prescribed, decaying Schmidt spectrum (random orthogonal factors)."""
    chi_l, d1, d2, chi_r = shape
    rng = np.random.default_rng(seed)
    m, n = chi_l * d1, d2 * chi_r
    r = min(m, n)
    U, _ = np.linalg.qr(rng.standard_normal((m, r)))
    V, _ = np.linalg.qr(rng.standard_normal((n, r)))
    s = np.exp(-decay * np.arange(r))
    M = (U * s) @ V.T
    return (M / np.linalg.norm(M)).reshape(shape)


# The Gram route resolves the discarded weight 1 - (kept sum)/||theta||^2 to a
# few eps ||theta||^2: a cut whose oracle tail lies that close to eps_local can
# fall on either side of it.
DISC_RES = 8 * 2.2e-16


def _oracle_split_at(theta, chi_max, eps, move_right, chn):
    """The oracle's SVD split for the GPU's kept count chn: its own truncation,
    or, where chn is one off it and the oracle's discarded weight at chn lies
    within DISC_RES of eps (||theta|| = 1), its split truncated at chn."""
    a_ref, b_ref, info = od.split_svd(theta, chi_max, eps, bool(move_right))
    if chn != info["keep"]:
        tail = float(np.sum(info["lam2"][chn:]))
        assert abs(chn - info["keep"]) == 1 and abs(tail - eps) <= DISC_RES, \
            (chn, info["keep"], tail, eps)
        a_ref, b_ref, info = od.split_svd(theta, chn, 0.0, bool(move_right))
    return a_ref, b_ref, info


@pytest.mark.parametrize("split_prec", ["fp64", "fp64emu", "bf16x3"])
@pytest.mark.parametrize("move_right", [1, 0])
@pytest.mark.parametrize("shape,chi_max,eps", [((8, 2, 2, 8), 100, 0.0), ((40, 2, 2, 30), 20, 0.0),
                                               ((64, 2, 2, 64), 1000, 1e-10), ((20, 5, 5, 16), 50, 1e-12),
                                               ((512, 2, 2, 512), 512, 1e-14)])
def test_split_parity(ctx, move_right, shape, chi_max, eps, split_prec):
    """fp64: Gram and projection on the float64 DMMA GEMM; other precisions:
    on the float64-accurate emulated GEMM; eigenpairs from float64 cuSOLVER
    in both. All must give the float64 answer."""
    theta = _split_case(11, shape, 0.35)
    chi_l, d1, d2, chi_r = shape
    cap = min(chi_l * d1, d2 * chi_r)
    A1 = torch.empty(chi_l * d1 * cap, dtype=torch.float64, device="cuda:0")
    A2 = torch.empty(cap * d2 * chi_r, dtype=torch.float64, device="cuda:0")
    chn, disc, ent, lam2 = B.osmps_split(ctx, dev(theta), A1, A2, move_right, chi_max, eps,
                                         precision=split_prec)
    a_ref, b_ref, info = _oracle_split_at(theta, chi_max, eps, move_right, chn)
    assert chn == info["keep"]
    # only the largest min(chi_max, rank) values are computed; the Gram route
    # squares the singular values, so lambda^2 carries an absolute error of a
    # few eps * ||theta||^2 (||theta|| = 1)
    k = min(chi_max, len(info["lam2"]))
    np.testing.assert_allclose(lam2[:k], info["lam2"][:k], rtol=1e-12, atol=1e-14)
    assert abs(disc - info["discarded"]) <= 1e-13
    assert abs(ent - info["entropy"]) <= 1e-12
    a = A1[: chi_l * d1 * chn].cpu().numpy().reshape(chi_l, d1, chn)
    b = A2[: chn * d2 * chi_r].cpu().numpy().reshape(chn, d2, chi_r)
    # gauge-invariant comparison: the truncated, renormalised two-site tensor.
    # From the Gram matrix an eigenvector with eigenvalue gap g is resolved to
    # ~eps / g, so the smallest kept singular value s_min contributes an error
    # ~eps / s_min to the product (the SVD oracle has no such loss).
    s_min = np.sqrt(info["lam2"][chn - 1])
    np.testing.assert_allclose(np.tensordot(a, b, axes=([2], [0])),
                               np.tensordot(a_ref, b_ref, axes=([2], [0])),
                               atol=1e-11 + 10 * 2.2e-16 / s_min)
    if move_right:
        assert od.left_isometry_defect(a) < 1e-12
    else:
        assert od.right_isometry_defect(b) < 1e-12


def _xxz_operator(L, k, chi, seed):
    W = hamiltonians.xxz(L, 1.0, 1.0, 0.0)
    mps = od.right_canonicalize(inputs.random_mps(L, 2, chi, seed=seed))
    Renv = od.build_right_envs(W, mps)
    Lenv = np.ones((1, 1, 1))
    for j in range(k):  # shift centre to k with QR so that L is built on isometries
        chl, d, chr_ = mps[j].shape
        Q, Rm = np.linalg.qr(mps[j].reshape(chl * d, chr_))
        mps[j] = Q.reshape(chl, d, Q.shape[1])
        mps[j + 1] = np.tensordot(Rm, mps[j + 1], axes=([1], [0]))
        Lenv = od.env_left(Lenv, mps[j], W[j])
    theta = np.tensordot(mps[k], mps[k + 1], axes=([2], [0]))
    return Lenv, W[k], W[k + 1], Renv[k + 2], theta


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x3"])
def test_lanczos_parity(ctx, prec):
    Lenv, W1, W2, Renv, theta = _xxz_operator(12, 5, 32, seed=2)
    mv = lambda x: od.heff_apply(Lenv, W1, W2, Renv, x)
    e_ref, x_ref, it_ref, _ = od.lanczos_ground(mv, theta, 100, 1e-12)
    th = dev(theta)
    tol = 1e-12 if prec == "fp64" else 1e-5
    e, it, res, ok = B.osmps_lanczos_ground(ctx, dev(Lenv), dev(W1), dev(W2), dev(Renv), th,
                                            max_iter=100, tol=tol, precision=prec)
    x = th.cpu().numpy()
    assert abs(np.linalg.norm(x) - 1.0) < 1e-12
    if prec == "fp64":
        assert ok
        assert abs(e - e_ref) <= 1e-10 * abs(e_ref)
        assert abs(abs(np.vdot(x, x_ref)) - 1.0) < 1e-9
    else:
        # a perturbed operator: the Ritz value carries the matvec error linearly,
        # the Rayleigh quotient with the exact operator is accurate to second order
        assert abs(e - e_ref) <= 1e-5 * abs(e_ref)
        rq = float(np.vdot(x, mv(x)))
        assert abs(rq - e_ref) <= 1e-8 * abs(e_ref)


def test_lanczos_max_iter_reports_noconv(ctx):
    Lenv, W1, W2, Renv, theta = _xxz_operator(10, 4, 16, seed=3)
    th = dev(theta)
    e, it, res, ok = B.osmps_lanczos_ground(ctx, dev(Lenv), dev(W1), dev(W2), dev(Renv), th,
                                            max_iter=2, tol=1e-14, precision="fp64")
    assert not ok and it == 2
    assert abs(torch.linalg.norm(th).item() - 1.0) < 1e-12  # best pair still written


def test_invalid_arguments_are_reported(ctx):
    Lh, W1, W2, Rh, th = (dev(x) for x in inputs.random_heff_operands(4, 2, 2, 4, 3, 3, 3))
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_heff_apply(ctx, Lh, W1, W2, Rh, th, th, precision="fp64")
    assert e.value.status == 1  # y aliases theta
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_heff_apply(ctx, Lh, W1, W2, Rh, th, torch.empty_like(th), precision=7)
    assert e.value.status == 1
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_lanczos_ground(ctx, Lh, W1, W2, Rh, th, max_iter=0)
    assert e.value.status == 1
    z = torch.zeros_like(th)
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_lanczos_ground(ctx, Lh, W1, W2, Rh, z, max_iter=5)
    assert e.value.status == 1  # zero start vector


def _split_case_spectrum(seed, shape, s):
    chi_l, d1, d2, chi_r = shape
    rng = np.random.default_rng(seed)
    m, n = chi_l * d1, d2 * chi_r
    r = len(s)
    U, _ = np.linalg.qr(rng.standard_normal((m, r)))
    V, _ = np.linalg.qr(rng.standard_normal((n, r)))
    M = (U * s) @ V.T
    return (M / np.linalg.norm(M)).reshape(shape)


SPECTRA = {  # (fast decay to the noise floor is covered by test_split_parity)
    "slow_decay": lambda r: np.exp(-0.01 * np.arange(r)),
    "multiplets": lambda r: np.repeat(np.exp(-0.05 * np.arange((r + 2) // 3)), 3)[:r],
    "rank_deficient": lambda r: np.r_[np.exp(-0.02 * np.arange(r // 3)), np.zeros(r - r // 3)],
}


@pytest.mark.parametrize("solver", ["tridiag", "cusolver"])
@pytest.mark.parametrize("move_right", [1, 0])
@pytest.mark.parametrize("spectrum", list(SPECTRA))
@pytest.mark.parametrize("shape,chi_max", [((100, 2, 2, 90), 60), ((300, 2, 2, 256), 255),
                                           ((24, 5, 5, 30), 81)])
def test_split_eigensolvers(ctx, solver, move_right, spectrum, shape, chi_max):
    """Both float64 eigensolvers of the split (cuSOLVER dsyevdx and the
    tridiagonal route: bisection, inverse iteration, Cholesky QR, blocked
    back-transformation) against the oracle's SVD truncation, on spectra
    with slow decay, exact multiplets and exact zeros."""
    chi_l, d1, d2, chi_r = shape
    r = min(chi_l * d1, d2 * chi_r)
    theta = _split_case_spectrum(7, shape, SPECTRA[spectrum](r))
    # exact zeros: a tolerance stops both sides at the rank (cuts are multiples of 3 so
    # that no exact multiplet is split)
    eps = 1e-14 if spectrum == "rank_deficient" else 0.0
    cap = r
    A1 = torch.empty(chi_l * d1 * cap, dtype=torch.float64, device="cuda:0")
    A2 = torch.empty(cap * d2 * chi_r, dtype=torch.float64, device="cuda:0")
    ctx.set_eig_solver(solver)
    try:
        chn, disc, ent, lam2 = B.osmps_split(ctx, dev(theta), A1, A2, move_right, chi_max, eps,
                                             precision="fp64emu")
    finally:
        ctx.set_eig_solver("auto")
    a_ref, b_ref, info = _oracle_split_at(theta, chi_max, eps, move_right, chn)
    assert chn == info["keep"]
    k = min(chi_max, len(info["lam2"]))
    np.testing.assert_allclose(lam2[:k], info["lam2"][:k], rtol=1e-12, atol=1e-14)
    assert abs(disc - info["discarded"]) <= 1e-13
    a = A1[: chi_l * d1 * chn].cpu().numpy().reshape(chi_l, d1, chn)
    b = A2[: chn * d2 * chi_r].cpu().numpy().reshape(chn, d2, chi_r)
    s_min = np.sqrt(info["lam2"][chn - 1])
    tol = 1e-11 + 10 * 2.2e-16 / s_min
    np.testing.assert_allclose(np.tensordot(a, b, axes=([2], [0])),
                               np.tensordot(a_ref, b_ref, axes=([2], [0])), atol=tol)
    if move_right:
        assert od.left_isometry_defect(a) < 1e-12
    else:
        assert od.right_isometry_defect(b) < 1e-12


@pytest.mark.parametrize("n,offset", [(2, 0), (37, 0), (300, 0), (301, 1), (1000, 0)])
def test_sytrd_matches_lapack(ctx, n, offset):
    """osmps_sytrd (cooperative panels + emulated-GEMM trailing updates)
    against LAPACK dsytrd: Q^T G Q = T with Q rebuilt from the stored
    reflectors, the spectrum of T, and d, e, tau (same reflector convention).
    offset 1: the matrix starts 8 bytes past a 16-byte boundary, so every row
    of an odd n begins on the other parity for the panel's paired loads."""
    from scipy.linalg import lapack
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    G = M @ M.T
    A = torch.empty(n * n + offset, dtype=torch.float64, device="cuda:0")[offset:].view(n, n)
    A.copy_(dev(G.copy()))
    assert (A.data_ptr() % 16 == 8) == bool(offset)
    d = torch.empty(n, dtype=torch.float64, device="cuda:0")
    e = torch.empty(max(n - 1, 1), dtype=torch.float64, device="cuda:0")
    tau = torch.empty(max(n - 1, 1), dtype=torch.float64, device="cuda:0")
    B.osmps_sytrd(ctx, A, d, e, tau)
    torch.cuda.synchronize()
    Ah, dh, eh, th = A.cpu().numpy(), d.cpu().numpy(), e.cpu().numpy()[: n - 1], tau.cpu().numpy()[: n - 1]
    T = np.diag(dh) + np.diag(eh, 1) + np.diag(eh, -1)
    Q = np.eye(n)
    for j in range(n - 1):  # Q = H(0) ... H(n-2); the reflector of column j is row j of Ah
        v = np.zeros(n)
        v[j + 1] = 1.0
        v[j + 2:] = Ah[j, j + 2:]
        Q = Q @ (np.eye(n) - th[j] * np.outer(v, v))
    scale = np.abs(G).max()
    assert np.abs(Q.T @ G @ Q - T).max() <= 1e-12 * scale
    np.testing.assert_allclose(np.linalg.eigvalsh(T), np.linalg.eigvalsh(G), rtol=0, atol=1e-13 * scale)
    _, dl, el, taul, _ = lapack.dsytrd(G.copy(order="F"), lower=1)
    np.testing.assert_allclose(dh, dl, rtol=0, atol=1e-10 * scale)
    np.testing.assert_allclose(np.abs(eh), np.abs(el), rtol=0, atol=1e-10 * scale)
