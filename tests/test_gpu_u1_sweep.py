"""Two-site sweeps on a particle-number-conserving MPS (Sec. 3.4 with
symmetries), end to end on the GPU: theta formation, the U(1) Lanczos, the
per-sector split with joint truncation and the block environment updates
through the library's calls. Checked against exact diagonalisation of the
oracle's MPO restricted to the fixed-N sector, and the final state against
the oracle's float64 contractions of its dense site tensors (canonical form,
particle number, energy)."""
import numpy as np
import pytest

from oracle import dmrg as od
from oracle import mpo as ompo
from paper_1703_00387_gb300 import binding as B
from paper_1703_00387_gb300 import hamiltonians
from paper_1703_00387_gb300 import u1sweep as us

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


def _sector_ground_energy(W_oracle, L, d, N):
    H = ompo.mpo_to_dense(W_oracle)
    digits = np.array(np.unravel_index(np.arange(d ** L), (d,) * L)).sum(axis=0)
    idx = np.nonzero(digits == N)[0]
    return float(np.linalg.eigvalsh(H[np.ix_(idx, idx)])[0])


def _check_state(mps, W_oracle, N, res):
    dense = mps.dense()
    for k in range(1, mps.L):
        assert od.right_isometry_defect(dense[k]) < 1e-10
    psi = od.mps_to_vector(dense)
    d, L = mps.d, mps.L
    digits = np.array(np.unravel_index(np.arange(d ** L), (d,) * L)).sum(axis=0)
    assert np.abs(psi[digits != N]).max() == 0.0
    e_oracle = od.mps_energy(W_oracle, dense)
    assert abs(res["energy"] - e_oracle) <= 1e-10 * max(1.0, abs(e_oracle))


@pytest.mark.parametrize("prec,tol", [("tf32x3", 1e-9), ("bf16x3", 1e-7)])
def test_bose_hubbard_sweep_reaches_sector_ground_state(ctx, prec, tol):
    L, nmax, N = 6, 2, 6
    W = hamiltonians.bose_hubbard(L, 1.0, 4.0, nmax)
    Wo = ompo.bose_hubbard_mpo(L, 1.0, 4.0, nmax)
    ex = us.DeviceExecutor(ctx)
    mps = us.random_u1_mps(ex, L, nmax + 1, N, chi=8, seed=11)
    res = us.u1_sweep(mps, W, n_sweeps=3, chi_max=64, eps_local=0.0, precision=prec,
                      lanczos_tol=1e-11, lanczos_max_iter=100)
    e0 = _sector_ground_energy(Wo, L, nmax + 1, N)
    assert abs(res["energy"] - e0) <= tol * abs(e0), (res["energy"], e0)
    assert res["max_discarded"] <= 1e-12
    _check_state(mps, Wo, N, res)


def test_xxz_half_filling_sweep(ctx):
    L, N = 10, 5
    W = hamiltonians.xxz(L, 1.0, 1.0, 0.0)
    Wo = ompo.xxz_mpo(L, 1.0, 1.0, 0.0)
    ex = us.DeviceExecutor(ctx)
    mps = us.random_u1_mps(ex, L, 2, N, chi=4, seed=3)
    res = us.u1_sweep(mps, W, n_sweeps=3, chi_max=64, eps_local=0.0, precision="tf32x3",
                      lanczos_tol=1e-11)
    e0 = _sector_ground_energy(Wo, L, 2, N)
    assert abs(res["energy"] - e0) <= 1e-9 * abs(e0), (res["energy"], e0)
    _check_state(mps, Wo, N, res)


def test_truncated_sweep_keeps_chi_max_and_bounds_the_energy(ctx):
    L, nmax, N = 8, 2, 8
    W = hamiltonians.bose_hubbard(L, 1.0, 4.0, nmax)
    Wo = ompo.bose_hubbard_mpo(L, 1.0, 4.0, nmax)
    ex = us.DeviceExecutor(ctx)
    mps = us.random_u1_mps(ex, L, nmax + 1, N, chi=8, seed=5)
    chi = 12
    res = us.u1_sweep(mps, W, n_sweeps=3, chi_max=chi, eps_local=0.0, precision="tf32x3",
                      lanczos_tol=1e-10)
    assert max(b.dim for b in mps.bonds) <= chi
    e0 = _sector_ground_energy(Wo, L, nmax + 1, N)
    # variational: above the sector's ground energy, and close to it at chi = 12
    assert res["energy"] >= e0 - 1e-10
    assert res["energy"] - e0 <= 1e-3 * abs(e0)
    assert res["max_discarded"] > 0.0
    _check_state(mps, Wo, N, res)


def test_concurrent_sector_eigensolves_match_sequential(ctx):
    """The split's sector eigensolves on four worker contexts at once (the
    Householder panels of the larger sectors as concurrent cooperative
    launches) give the same sweep as one after another on one context."""
    L, nmax, N = 16, 3, 16
    W = hamiltonians.bose_hubbard(L, 1.0, 4.0, nmax)
    runs = []
    for workers in (1, 4):
        ex = us.DeviceExecutor(ctx, eig_workers=workers)
        sizes = []
        many = ex.eig_top_many
        ex.eig_top_many = lambda jobs, many=many, sizes=sizes: (sizes.extend(j[1] for j in jobs),
                                                                many(jobs))[1]
        mps = us.random_u1_mps(ex, L, nmax + 1, N, chi=32, seed=7)
        res = us.u1_sweep(mps, W, n_sweeps=2, chi_max=96, eps_local=0.0, precision="tf32x3",
                          lanczos_tol=1e-10, lanczos_max_iter=60)
        assert max(sizes) >= 64  # some sectors take the cooperative route
        runs.append((res["energy"], res["max_discarded"], [b.dim for b in mps.bonds],
                     [b.m.tolist() for b in mps.bonds]))
        ex.close()
    (e1, d1, dims1, m1), (e4, d4, dims4, m4) = runs
    assert dims1 == dims4 and m1 == m4
    assert abs(e1 - e4) <= 1e-12 * abs(e1) and abs(d1 - d4) <= 1e-12 + 1e-9 * d1


def test_gemm_grouped_matches_numpy(ctx):
    """Grouped products on strided views: several terms per output (K
    ragged across 16-wide steps), transposed and reversed (negative-stride)
    operands, an output with no terms (zeroed), beta accumulation, and
    outputs spanning several 64 x 64 tiles."""
    rng = np.random.default_rng(0)
    buf = rng.standard_normal(200_000)
    out = np.full(60_000, np.nan)
    out[40_000:] = rng.standard_normal(20_000)
    dbuf, dout = torch.from_numpy(buf).cuda(), torch.from_numpy(out.copy()).cuda()
    pb, po = dbuf.data_ptr(), dout.data_ptr()

    def view(a, off, rows, cols, rs, cs):  # element (r, c) at off + r rs + c cs, any sign
        return a[off + rs * np.arange(rows)[:, None] + cs * np.arange(cols)[None, :]]

    outs, terms, expect = [], [], []
    # out 0: 130 x 70 at 0, row stride 70; 3 terms K = 17, 1, 40
    specs = [
        (0, 70, 1, 130, 70, 0.0, [(100, 17, 1, 5000, 70, 1, 17, 1.5),
                                  (9000, 1, 130, 20000, 1, 1, 1, -2.0),     # A transposed
                                  (30000, 40, 1, 60000, 1, 40, 40, 0.25)]),  # B transposed
        (20000, 9, 1, 9, 9, 0.0, []),                                         # no terms: zero
        (20100, 1, 33, 33, 20, 0.0, [(120000, 50, 1, 140000, 20, 1, 50, 1.0)]),  # C transposed
        (40000, 100, 1, 64, 100, 0.5, [(150000 + 63 * 77, -77, 1, 170000, 100, 1, 77, 1.0)]),  # A rows reversed, beta
    ]
    for (co, scm, scn, M, N, beta, tl) in specs:
        outs.append((po + 8 * co, scm, scn, M, N, beta, len(terms), len(tl)))
        ref = np.zeros((M, N))
        for (ao, sam, sak, bo, sbk, sbn, K, alpha) in tl:
            terms.append((pb + 8 * ao, sam, sak, pb + 8 * bo, sbk, sbn, K, alpha))
            ref += alpha * view(buf, ao, M, K, sam, sak) @ view(buf, bo, K, N, sbk, sbn)
        C0 = view(out, co, M, N, scm, scn)
        expect.append((co, M, N, scm, scn, ref + (beta * C0 if beta != 0.0 else 0.0)))
    B.osmps_gemm_grouped(ctx, np.array(outs, dtype=B.GEMM_OUT_DTYPE), np.array(terms, dtype=B.GEMM_TERM_DTYPE))
    got = dout.cpu().numpy()
    for (co, M, N, scm, scn, ref) in expect:
        np.testing.assert_allclose(view(got, co, M, N, scm, scn), ref, rtol=1e-13, atol=1e-12)
    # untouched entries stay untouched
    assert np.isnan(got[130 * 70: 20000]).all()


def test_gemm_grouped_rejects_bad_ranges(ctx):
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    terms = np.array([(p, 8, 1, p, 8, 1, 8, 1.0)], dtype=B.GEMM_TERM_DTYPE)
    for bad in ((p, 8, 1, 8, 8, 0.0, 0, 2), (p, 8, 1, 8, 8, 0.0, -1, 1)):
        with pytest.raises(B.OsmpsError) as e:
            B.osmps_gemm_grouped(ctx, np.array([bad], dtype=B.GEMM_OUT_DTYPE), terms)
        assert e.value.status == B.EINVAL
    zero_k = np.array([(p, 8, 1, p, 8, 1, 0, 1.0)], dtype=B.GEMM_TERM_DTYPE)
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_gemm_grouped(ctx, np.array([(p, 8, 1, 8, 8, 0.0, 0, 1)], dtype=B.GEMM_OUT_DTYPE), zero_k)
    assert e.value.status == B.ESHAPE
