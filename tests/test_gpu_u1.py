"""U(1)-symmetric H_eff.theta on the GPU (grouped sector-block launches)
against the oracle's dense product of the masked tensors. Bars as for the
dense split-precision path: 1e-5 norm-wise for bf16x3 and tf32x3, at every
shape."""
import numpy as np
import pytest

from oracle import mpo as ompo
from oracle import u1 as ou1
from paper_1703_00387_gb300 import binding as B
from paper_1703_00387_gb300 import hamiltonians, inputs
from paper_1703_00387_gb300 import u1 as pu1

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"bf16x3": 1e-5, "tf32x3": 1e-5}


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


def _run(ctx, left, right, nmax, sites, prec, seed, L_chain=8):
    """sites: which two sites of a Bose-Hubbard chain give W1, W2."""
    d = nmax + 1
    Wp = hamiltonians.bose_hubbard(L_chain, 1.0, 4.0, nmax)
    Wo = ompo.bose_hubbard_mpo(L_chain, 1.0, 4.0, nmax)
    k1, k2 = sites
    qp = pu1.channel_charges(Wp)
    qo = ou1.mpo_channel_charges(Wo)
    op = pu1.U1Operator(ctx, left, right, d, d, Wp[k1], Wp[k2], qp[k1], qp[k2 + 1])
    ql = ou1.index_charges(*left)
    qr = ou1.index_charges(*right)
    wl, wr = Wo[k1].shape[0], Wo[k2].shape[3]
    Lh = inputs.random_dense((len(ql), wl, len(ql)), seed)
    Rh = inputs.random_dense((len(qr), wr, len(qr)), seed + 1)
    th = inputs.random_dense((len(ql), d, d, len(qr)), seed + 2)
    ref = ou1.heff_apply_u1(Lh, Wo[k1], Wo[k2], Rh, th, ql, qr, qo[k1], qo[k2 + 1])
    ref_packed = ref[ou1.theta_mask(ql, qr, d, d)]
    t = [dev(pu1.pack(Lh, op.m_L)), dev(Wp[k1]), dev(Wp[k2]), dev(pu1.pack(Rh, op.m_R)),
         dev(pu1.pack(th, op.m_theta))]
    y = torch.empty_like(t[4])
    B.osmps_heff_apply_u1(ctx, op.plan, *t, y, precision=prec)
    torch.cuda.synchronize()
    out = y.cpu().numpy()
    flops = op.plan.flops
    op.close()
    return out, ref_packed, flops


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = {
    "small": (([3, 4, 5, 6], [2, 3, 3, 1]), ([5, 6, 7, 8, 9], [1, 2, 3, 2, 1]), 3, (2, 3)),
    "multi_tile": (([10, 11, 12], [70, 130, 90]), ([12, 13, 14, 15], [100, 150, 60, 40]), 4, (3, 4)),
    "gaps": (([0, 2, 3], [5, 7, 1]), ([1, 4, 9], [6, 3, 2]), 2, (1, 2)),
    "left_boundary": (([0], [1]), ([0, 1, 2, 3, 4], [1, 1, 1, 1, 1]), 2, (0, 1)),
    "right_boundary": (([4, 5, 6], [3, 2, 1]), ([6], [1]), 2, (6, 7)),
}


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("case", list(CASES))
def test_u1_heff_parity(ctx, case, prec):
    left, right, nmax, sites = CASES[case]
    y, ref, _ = _run(ctx, left, right, nmax, sites, prec, seed=len(case))
    assert y.shape == ref.shape
    assert rel(y, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_u1_heff_bose_hubbard_workload(ctx, prec):
    """L = 64, N = 64, n <= 4 (d = 5), chi = 512 per bond, sector sizes from
    the Gaussian profile around N k / L at bonds 31 and 33 (sites 31, 32)."""
    left = inputs.u1_sector_profile(31.0, total=512, width=8.0)
    right = inputs.u1_sector_profile(33.0, total=512, width=8.0)
    y, ref, flops = _run(ctx, left, right, 4, (31, 32), prec, seed=64, L_chain=64)
    assert rel(y, ref) <= 1e-5
    assert flops > 0


def test_u1_errors(ctx):
    with pytest.raises(B.OsmpsError) as e:
        B.U1Heff(ctx, [1, 1], [2, 2], [1], [1], 2, 2, 4, 4, 4, [0, 1, -1, 0], [0, 1, -1, 0])
    assert e.value.status == B.EINVAL
    with pytest.raises(B.OsmpsError) as e:
        B.U1Heff(ctx, [1], [0], [1], [1], 2, 2, 4, 4, 4, [0, 1, -1, 0], [0, 1, -1, 0])
    assert e.value.status == B.ESHAPE
    plan = B.U1Heff(ctx, [0, 1], [2, 2], [1, 2], [2, 2], 2, 2, 4, 4, 4, [0, 1, -1, 0], [0, 1, -1, 0])
    z = lambda n: torch.zeros(n, dtype=torch.float64, device="cuda:0")
    W = dev(np.zeros((4, 2, 2, 4)))
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_heff_apply_u1(ctx, plan, z(plan.n_L), W, W, z(plan.n_R), z(plan.n_theta),
                              z(plan.n_theta), precision="fp64")
    assert e.value.status == B.EUNSUPPORTED
    with pytest.raises(ValueError):
        B.osmps_heff_apply_u1(ctx, plan, z(plan.n_L + 1), W, W, z(plan.n_R), z(plan.n_theta),
                              z(plan.n_theta))
    plan.close()


def _u1_chain_operator(Lc=6, nmax=2, N=6, chi_sec=2, seed=10):
    """Environments of a random particle-number-conserving Bose-Hubbard MPS
    (oracle contractions) around sites 2, 3, with the sector structure."""
    from oracle import dmrg
    d = nmax + 1
    sectors = []
    for k in range(Lc + 1):
        qs = list(range(max(0, N - (Lc - k) * nmax), min(N, k * nmax) + 1))
        sectors.append((qs, [1 if k in (0, Lc) else chi_sec] * len(qs)))
    q = [ou1.index_charges(*s) for s in sectors]
    A = [inputs.random_dense((len(q[k]), d, len(q[k + 1])), seed + k) * ou1.mps_mask(q[k], q[k + 1], d)
         for k in range(Lc)]
    Wo = ompo.bose_hubbard_mpo(Lc, 1.0, 4.0, nmax)
    Le = np.ones((1, 1, 1))
    for k in range(2):
        Le = dmrg.env_left(Le, A[k], Wo[k])
    Re = np.ones((1, 1, 1))
    for k in range(Lc - 1, 3, -1):
        Re = dmrg.env_right(Re, A[k], Wo[k])
    return sectors, q, Wo, Le, Re, d


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_u1_lanczos_ground_matches_sector_eigenvalue(ctx, prec):
    sectors, q, Wo, Le, Re, d = _u1_chain_operator()
    mt = ou1.theta_mask(q[2], q[4], d, d)
    E0 = np.linalg.eigvalsh(ou1.sector_heff_matrix(Le, Wo[2], Wo[3], Re, mt))[0]
    Wp = hamiltonians.bose_hubbard(6, 1.0, 4.0, 2)
    qp = pu1.channel_charges(Wp)
    op = pu1.U1Operator(ctx, sectors[2], sectors[4], d, d, Wp[2], Wp[3], qp[2], qp[4])
    th = dev(pu1.pack(inputs.random_dense(mt.shape, 5), op.m_theta))
    e, it, res, conv = B.osmps_lanczos_ground_u1(ctx, op.plan, dev(pu1.pack(Le, op.m_L)), dev(Wp[2]),
                                                 dev(Wp[3]), dev(pu1.pack(Re, op.m_R)), th,
                                                 max_iter=200, tol=1e-9, precision=prec)
    assert conv
    assert abs(e - E0) <= 1e-5 * abs(E0)
    # the Ritz vector is normalised and is an eigenvector of the oracle matrix
    v = th.cpu().numpy()
    assert abs(np.linalg.norm(v) - 1.0) < 1e-12
    H = ou1.sector_heff_matrix(Le, Wo[2], Wo[3], Re, mt)
    assert np.linalg.norm(H @ v - E0 * v) <= 1e-4 * abs(E0)
    op.close()


def test_u1_prepare_apply_matches_combined(ctx):
    left, right, nmax, sites = CASES["multi_tile"]
    Wp = hamiltonians.bose_hubbard(8, 1.0, 4.0, nmax)
    qp = pu1.channel_charges(Wp)
    k1, k2 = sites
    op = pu1.U1Operator(ctx, left, right, nmax + 1, nmax + 1, Wp[k1], Wp[k2], qp[k1], qp[k2 + 1])
    pl = op.plan
    L = dev(inputs.random_dense((pl.n_L,), 1))
    R = dev(inputs.random_dense((pl.n_R,), 2))
    th = dev(inputs.random_dense((pl.n_theta,), 3))
    W1, W2 = dev(Wp[k1]), dev(Wp[k2])
    y1 = torch.empty_like(th)
    y2 = torch.empty_like(th)
    B.osmps_heff_apply_u1(ctx, pl, L, W1, W2, R, th, y1, precision="tf32x3")
    B.osmps_u1_heff_prepare(ctx, pl, L, W1, W2, R, precision="tf32x3")
    B.osmps_u1_heff_apply(ctx, pl, th, y2)
    B.osmps_u1_heff_apply(ctx, pl, th, y2)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    op.close()


@pytest.mark.parametrize("prec,piece_bytes", [("bf16x3", 2), ("tf32x3", 4)])
def test_u1_wstep_profile_counts_its_bytes(ctx, prec, piece_bytes):
    """The fused W-step's profile record: one launch per product, credited
    with 4 n_T1 + 2 piece_bytes n_A4 bytes, where n_A4 (the stage-4 A entries)
    is counted here from its definition: for every right sector j of c2 and
    every left sector reached by q(c2) - t1 - t2, chi_left rows of K_j = sum
    over the right channels w2 of the size of the sector q(c2) - q_w2."""
    left, right, nmax, sites = CASES["multi_tile"]
    d = nmax + 1
    Wp = hamiltonians.bose_hubbard(8, 1.0, 4.0, nmax)
    qp = pu1.channel_charges(Wp)
    k1, k2 = sites
    q_wr = qp[k2 + 1]
    op = pu1.U1Operator(ctx, left, right, d, d, Wp[k1], Wp[k2], qp[k1], q_wr)
    (ql, chil), (qr, chir) = left, right
    n_a4 = 0
    for j, qj in enumerate(qr):
        K = sum(chir[qr.index(qj - q)] for q in q_wr if (qj - q) in qr)
        rows = sum(chil[ql.index(qj - t1 - t2)] for t1 in range(d) for t2 in range(d)
                   if (qj - t1 - t2) in ql)
        n_a4 += rows * K
    assert op.plan.n_A4 == n_a4 > 0 and op.plan.n_T1 > 0
    t = [dev(np.zeros(op.plan.n_L)), dev(Wp[k1]), dev(Wp[k2]), dev(np.zeros(op.plan.n_R)),
         dev(np.ones(op.plan.n_theta))]
    y = torch.empty_like(t[4])
    B.osmps_heff_apply_u1(ctx, op.plan, *t, y, precision=prec)  # warm-up (tile tuning)
    B.osmps_profile_enable(ctx, True)
    try:
        for _ in range(3):
            B.osmps_heff_apply_u1(ctx, op.plan, *t, y, precision=prec)
        p = B.osmps_profile_read(ctx, "u1_wstep")
    finally:
        B.osmps_profile_enable(ctx, False)
        op.close()
    assert p["launches"] == 3 and p["ms"] > 0.0
    assert p["flops"] == 3 * (4 * op.plan.n_T1 + 2 * piece_bytes * n_a4)
