"""Host logic of the U(1) sweep, without a GPU: the sector layouts agree with
the oracle's masks (the packed format is the allowed entries in C order of
the dense tensor), and the block operation lists that theta formation, the
split and the environment updates hand to the library compute the dense
definitions when run by a plain NumPy executor (strided views of flat
arrays). The dense references here are the textbook contractions."""
import numpy as np
import pytest

from oracle import dmrg as od
from oracle import u1 as ou1
from paper_1703_00387_gb300 import hamiltonians
from paper_1703_00387_gb300 import u1sweep as us
from paper_1703_00387_gb300.u1 import channel_charges


class NumpyExecutor:
    """Runs the operation records on flat NumPy arrays (test only)."""

    def empty(self, n):
        return np.full(max(int(n), 1), np.nan)

    @staticmethod
    def view(ref, rows, cols, rs, cs):
        buf, off = ref
        return np.lib.stride_tricks.as_strided(buf[int(off):], (rows, cols),
                                               (rs * 8, cs * 8), writeable=True)

    def products(self, ops):
        for o in ops:
            acc = np.zeros((o.M, o.N))
            for t in o.terms:
                acc += t.alpha * (self.view(t.A, o.M, t.K, t.sam, t.sak) @ self.view(t.B, t.K, o.N, t.sbk, t.sbn))
            C = self.view(o.C, o.M, o.N, o.scm, o.scn)
            C[...] = acc + (o.beta * C if o.beta != 0.0 else 0.0)

    def copies(self, ops):
        vals = []
        for c in ops:
            vals.append(0.0 if c.src is None else c.alpha * self.view(c.src, c.rows, c.cols, c.srs, c.scs).copy())
        for c, v in zip(ops, vals):
            self.view(c.dst, c.rows, c.cols, c.drs, 1)[...] = v

    def norm2(self, buf, n):
        return float(np.dot(buf[:n], buf[:n]))

    def eig_top(self, G, n, nev):
        w, v = np.linalg.eigh(G[: n * n].reshape(n, n))
        return w[n - nev:], np.ascontiguousarray(v[:, n - nev:].T).ravel()

    def eig_top_many(self, jobs):
        return [self.eig_top(*j) for j in jobs]

    def upload(self, a):
        return np.array(a, dtype=np.float64).ravel()

    def download(self, buf, n):
        return buf[:n].copy()

    def sync(self):
        pass

    def ground(self, Lk, W1, W2, Rk, theta, left, right, d, q_wl, q_wr, wm, precision, tol, max_iter):
        """The oracle's sector H_eff as an explicit matrix, lowest eigenpair."""
        wl, wr = len(q_wl), len(q_wr)
        W1 = W1.reshape(wl, d, d, wm)
        W2 = W2.reshape(wm, d, d, wr)
        ql, qr = left.charges(), right.charges()
        ml, mr = ou1.env_mask(ql, q_wl, ql), ou1.env_mask(qr, q_wr, qr)
        Ld, Rd = np.zeros(ml.shape), np.zeros(mr.shape)
        Ld[ml] = Lk[: int(ml.sum())]
        Rd[mr] = Rk[: int(mr.sum())]
        mt = ou1.theta_mask(ql, qr, d, d)
        H = ou1.sector_heff_matrix(Ld, W1, W2, Rd, mt)
        w, v = np.linalg.eigh(0.5 * (H + H.T))
        theta[: int(mt.sum())] = v[:, 0]
        return float(w[0]), 1


def _bond(rng, charges):
    return us.Bond(charges, rng.integers(1, 4, size=len(charges)))


def test_layouts_match_oracle_masks():
    rng = np.random.default_rng(0)
    left, right = _bond(rng, [0, 1, 2, 4]), _bond(rng, [1, 2, 3, 5, 6])
    d = 3
    lay = us.MpsLayout(left, right, d)
    mask = ou1.mps_mask(left.charges(), right.charges(), d)
    assert lay.size == int(mask.sum())
    dense = np.where(mask, rng.standard_normal(mask.shape), 0.0)
    packed = dense[mask]
    ro = np.concatenate([[0], np.cumsum(left.m)])
    co = np.concatenate([[0], np.cumsum(right.m)])
    for i in range(len(left.q)):
        for s in range(d):
            j = lay.right_sector[i, s]
            if j < 0:
                continue
            blk = packed[lay.row_off[i]:lay.row_off[i] + left.m[i] * lay.row_len[i]].reshape(
                left.m[i], lay.row_len[i])[:, lay.col_off[i, s]:lay.col_off[i, s] + right.m[j]]
            np.testing.assert_array_equal(blk, dense[ro[i]:ro[i + 1], s, co[j]:co[j + 1]])
    layt = us.ThetaLayout(left, right, d, d)
    tm = ou1.theta_mask(left.charges(), right.charges(), d, d)
    assert layt.size == int(tm.sum())
    for q_w in ([0, 1, -1, 0], [0, 2]):
        el = us.EnvLayout(left, np.array(q_w))
        assert el.size == int(ou1.env_mask(left.charges(), np.array(q_w), left.charges()).sum())


def _random_u1_dense(rng, left, right, d):
    m = ou1.mps_mask(left.charges(), right.charges(), d)
    return np.where(m, rng.standard_normal(m.shape), 0.0), m


def test_theta_formation_ops():
    rng = np.random.default_rng(1)
    d = 3
    left, mid, right = _bond(rng, [0, 1, 2]), _bond(rng, [1, 2, 3, 4]), _bond(rng, [2, 3, 4, 5, 6])
    A1, m1 = _random_u1_dense(rng, left, mid, d)
    A2, m2 = _random_u1_dense(rng, mid, right, d)
    ex = NumpyExecutor()
    layt = us.ThetaLayout(left, right, d, d)
    th = ex.empty(layt.size)
    ex.products(us.theta_ops(A1[m1].copy(), us.MpsLayout(left, mid, d), A2[m2].copy(),
                          us.MpsLayout(mid, right, d), mid, left, th, layt))
    ref = np.tensordot(A1, A2, axes=([2], [0]))
    tm = ou1.theta_mask(left.charges(), right.charges(), d, d)
    np.testing.assert_allclose(th[: layt.size], ref[tm], rtol=1e-13, atol=1e-13)
    assert np.abs(ref[~tm]).max() == 0.0


@pytest.mark.parametrize("move_right", [True, False])
def test_split_ops_match_svd_truncation(move_right):
    rng = np.random.default_rng(2)
    d = 3
    left, right = _bond(rng, [0, 1, 2, 3]), _bond(rng, [2, 3, 4, 5, 6])
    tm = ou1.theta_mask(left.charges(), right.charges(), d, d)
    theta = np.where(tm, rng.standard_normal(tm.shape), 0.0)
    theta /= np.linalg.norm(theta)
    ex = NumpyExecutor()
    layt = us.ThetaLayout(left, right, d, d)
    th = theta[tm].copy()
    chi_max = 7
    mid, A1, A2, disc, ent = us.split(ex, th, layt, left, right, d, d, move_right, chi_max, 0.0)
    a1 = np.zeros(ou1.mps_mask(left.charges(), mid.charges(), d).shape)
    a1[ou1.mps_mask(left.charges(), mid.charges(), d)] = A1[: us.MpsLayout(left, mid, d).size]
    a2 = np.zeros(ou1.mps_mask(mid.charges(), right.charges(), d).shape)
    a2[ou1.mps_mask(mid.charges(), right.charges(), d)] = A2[: us.MpsLayout(mid, right, d).size]
    # the dense SVD truncation: the symmetric theta's singular vectors carry one charge each,
    # and the kept space is the top chi_max (no ties here)
    _, _, info = od.split_svd(theta, chi_max, 0.0, move_right)
    assert mid.dim == info["keep"]
    assert abs(disc - info["discarded"]) <= 1e-12
    prod = np.tensordot(a1, a2, axes=([2], [0]))
    a_ref, b_ref, _ = od.split_svd(theta, chi_max, 0.0, move_right)
    np.testing.assert_allclose(prod, np.tensordot(a_ref, b_ref, axes=([2], [0])), atol=1e-11)
    if move_right:
        assert od.left_isometry_defect(a1) < 1e-12
    else:
        assert od.right_isometry_defect(a2) < 1e-12


def test_environment_update_ops():
    L, d = 6, 3
    W = hamiltonians.bose_hubbard(L, 1.0, 4.0, d - 1)
    qw = channel_charges(W)
    rng = np.random.default_rng(3)
    k = 2
    left, mid, right = _bond(rng, [0, 1, 2, 3]), _bond(rng, [1, 2, 3, 4]), _bond(rng, [2, 3, 4, 5])
    A, mA = _random_u1_dense(rng, left, mid, d)
    ex = NumpyExecutor()
    # left update: L_new over mid from L_old over left
    ml = ou1.env_mask(left.charges(), qw[k], left.charges())
    Lold = np.where(ml, rng.standard_normal(ml.shape), 0.0)
    elo, eln = us.EnvLayout(left, qw[k]), us.EnvLayout(mid, qw[k + 1])
    Ln = ex.empty(eln.size)
    _, _, nx = us.env_left_ops(None, elo, None, us.MpsLayout(left, mid, d), None, eln, W[k], left, mid, None)
    X = ex.empty(nx)
    s1, s2, _ = us.env_left_ops(Lold[ml].copy(), elo, A[mA].copy(), us.MpsLayout(left, mid, d), Ln, eln,
                                W[k], left, mid, X)
    ex.products(s1)
    ex.products(s2)
    ref = od.env_left(Lold, A, W[k])
    mln = ou1.env_mask(mid.charges(), qw[k + 1], mid.charges())
    np.testing.assert_allclose(Ln[: eln.size], ref[mln], rtol=1e-12, atol=1e-12)
    assert np.abs(ref[~mln]).max() < 1e-12
    # right update: R_new over left from R_old over mid (site tensor A: left -> mid)
    mr = ou1.env_mask(mid.charges(), qw[k + 1], mid.charges())
    Rold = np.where(mr, rng.standard_normal(mr.shape), 0.0)
    ero, ern = us.EnvLayout(mid, qw[k + 1]), us.EnvLayout(left, qw[k])
    Rn = ex.empty(ern.size)
    _, _, nz = us.env_right_ops(None, ero, None, us.MpsLayout(left, mid, d), None, ern, W[k], left, mid, None)
    Z = ex.empty(nz)
    s1, s2, _ = us.env_right_ops(Rold[mr].copy(), ero, A[mA].copy(), us.MpsLayout(left, mid, d), Rn, ern,
                                 W[k], left, mid, Z)
    ex.products(s1)
    ex.products(s2)
    ref = od.env_right(Rold, A, W[k])
    mrn = ou1.env_mask(left.charges(), qw[k], left.charges())
    np.testing.assert_allclose(Rn[: ern.size], ref[mrn], rtol=1e-12, atol=1e-12)
    assert np.abs(ref[~mrn]).max() < 1e-12


def test_sweep_orchestration_reaches_sector_ground_state():
    """The whole U(1) sweep (right-canonical start, theta, split with joint
    truncation, environment updates, final energy) with exact sector
    eigenpairs in place of Lanczos: Bose-Hubbard L = 5, n_max = 2, N = 5,
    against exact diagonalisation of the oracle's MPO in the N sector."""
    from oracle import mpo as ompo
    L, nmax, N = 5, 2, 5
    d = nmax + 1
    W = hamiltonians.bose_hubbard(L, 1.0, 4.0, nmax)
    ex = NumpyExecutor()
    mps = us.random_u1_mps(ex, L, d, N, chi=4, seed=1)
    res = us.u1_sweep(mps, W, n_sweeps=2, chi_max=64, eps_local=0.0)
    H = ompo.mpo_to_dense(ompo.bose_hubbard_mpo(L, 1.0, 4.0, nmax))
    n_of = np.array(np.unravel_index(np.arange(d ** L), (d,) * L)).sum(axis=0)
    idx = np.nonzero(n_of == N)[0]
    e0 = np.linalg.eigvalsh(H[np.ix_(idx, idx)])[0]
    assert abs(res["energy"] - e0) <= 1e-10 * abs(e0)
    dense = mps.dense()
    for k in range(1, L):
        assert od.right_isometry_defect(dense[k]) < 1e-12
    psi = od.mps_to_vector(dense)
    assert np.abs(psi[n_of != N]).max() == 0.0
    assert abs(od.mps_energy(ompo.bose_hubbard_mpo(L, 1.0, 4.0, nmax), dense) - res["energy"]) < 1e-11


def test_truncated_sweep_orchestration():
    """chi_max below the exact bond dimension: every bond at most chi_max,
    energy variational and near the sector's ground energy."""
    from oracle import mpo as ompo
    L, nmax, N = 6, 2, 6
    d = nmax + 1
    W = hamiltonians.bose_hubbard(L, 1.0, 4.0, nmax)
    ex = NumpyExecutor()
    mps = us.random_u1_mps(ex, L, d, N, chi=6, seed=2)
    res = us.u1_sweep(mps, W, n_sweeps=3, chi_max=9, eps_local=0.0)
    assert max(b.dim for b in mps.bonds) <= 9
    H = ompo.mpo_to_dense(ompo.bose_hubbard_mpo(L, 1.0, 4.0, nmax))
    n_of = np.array(np.unravel_index(np.arange(d ** L), (d,) * L)).sum(axis=0)
    idx = np.nonzero(n_of == N)[0]
    e0 = np.linalg.eigvalsh(H[np.ix_(idx, idx)])[0]
    assert e0 - 1e-10 <= res["energy"] <= e0 + 1e-2 * abs(e0)
    assert res["max_discarded"] > 0.0


def test_xxz_sweep_orchestration_with_empty_field_channel():
    """XXZ at h = 0 (a channel with no operator on the first site, channels
    of charge -1, 0, +1): L = 8 at half filling against exact
    diagonalisation in the N = 4 sector."""
    from oracle import mpo as ompo
    L, N = 8, 4
    W = hamiltonians.xxz(L, 1.0, 0.7, 0.0)
    ex = NumpyExecutor()
    mps = us.random_u1_mps(ex, L, 2, N, chi=4, seed=3)
    res = us.u1_sweep(mps, W, n_sweeps=2, chi_max=64, eps_local=0.0)
    H = ompo.mpo_to_dense(ompo.xxz_mpo(L, 1.0, 0.7, 0.0))
    n_of = np.array(np.unravel_index(np.arange(2 ** L), (2,) * L)).sum(axis=0)
    idx = np.nonzero(n_of == N)[0]
    e0 = np.linalg.eigvalsh(H[np.ix_(idx, idx)])[0]
    assert abs(res["energy"] - e0) <= 1e-10 * abs(e0)


class _Buf:
    """A device buffer stand-in that only knows its length."""

    def __init__(self, n):
        self.n = max(int(n), 1)


class BoundsExecutor:
    """Checks every operation a sweep hands to the library, without running
    it: each strided view (output, A and B operands of every term, copy
    source and destination, the Gram matrix of every eigensolve) lies inside
    its buffer, a grouped stage writes no buffer it reads, and the outputs of
    one stage never overlap (the grouped GEMM runs them concurrently)."""

    def __init__(self):
        self.rng = np.random.default_rng(0)
        self.views = 0

    @staticmethod
    def _span(off, rows, cols, rs, cs):
        assert rows >= 1 and cols >= 1
        lo = off + min(0, (rows - 1) * rs) + min(0, (cols - 1) * cs)
        hi = off + max(0, (rows - 1) * rs) + max(0, (cols - 1) * cs)
        return lo, hi

    def _check(self, ref, rows, cols, rs, cs):
        buf, off = ref
        lo, hi = self._span(int(off), rows, cols, rs, cs)
        assert 0 <= lo and hi < buf.n, (lo, hi, buf.n)
        self.views += 1

    def empty(self, n):
        return _Buf(n)

    def upload(self, a):
        return _Buf(np.size(a))

    def download(self, buf, n):
        assert n <= buf.n
        return np.ones(n)

    def sync(self):
        pass

    def norm2(self, buf, n):
        assert n <= buf.n
        return 1.0

    def ground(self, Lk, W1, W2, Rk, theta, left, right, d, q_wl, q_wr, wm, precision, tol, max_iter):
        assert int(ou1.theta_mask(left.charges(), right.charges(), d, d).sum()) <= theta.n
        return -1.0, 1

    def products(self, ops):
        written, read = set(), set()
        rows = []
        for o in ops:
            self._check(o.C, o.M, o.N, o.scm, o.scn)
            written.add(id(o.C[0]))
            if o.scn == 1:
                off = int(o.C[1])
                rows += [(id(o.C[0]), off + r * o.scm, off + r * o.scm + o.N) for r in range(o.M)]
            for t in o.terms:
                assert t.K >= 1
                self._check(t.A, o.M, t.K, t.sam, t.sak)
                self._check(t.B, t.K, o.N, t.sbk, t.sbn)
                read.update((id(t.A[0]), id(t.B[0])))
        assert not (written & read)
        rows.sort()
        for (b0, _, e0), (b1, s1, _) in zip(rows, rows[1:]):
            assert b0 != b1 or e0 <= s1  # output rows of one stage are disjoint

    def copies(self, ops):
        for c in ops:
            if c.src is not None:
                self._check(c.src, c.rows, c.cols, c.srs, c.scs)
            self._check(c.dst, c.rows, c.cols, c.drs, 1)

    def eig_top_many(self, jobs):
        out = []
        for G, n, nev in jobs:
            assert 1 <= nev <= n and n * n <= G.n
            out.append((np.sort(np.exp(-0.05 * np.arange(nev)) * self.rng.uniform(0.5, 1.0)), _Buf(nev * n)))
        tot = sum(e.sum() for e, _ in out)
        return [(e / tot, y) for e, y in out]


@pytest.mark.parametrize("model", ["bose_hubbard", "xxz"])
def test_sweep_block_lists_stay_inside_their_buffers(model):
    """A whole sweep's block operations (canonicalisation, theta, split with
    truncation at chi_max, both environment updates, the final energy) at
    bond dimensions where the sectors span many blocks, checked for bounds
    and overlaps before they could ever reach a GPU."""
    if model == "bose_hubbard":
        L, d, N = 12, 4, 12
        W = hamiltonians.bose_hubbard(L, 1.0, 4.0, d - 1)
    else:
        L, d, N = 16, 2, 8
        W = hamiltonians.xxz(L, 1.0, 0.7, 0.0)
    ex = BoundsExecutor()
    mps = us.random_u1_mps(ex, L, d, N, chi=32, seed=4)
    res = us.u1_sweep(mps, W, n_sweeps=1, chi_max=48, eps_local=0.0)
    assert res["max_chi"] <= 48 and res["max_chi"] > 16
    assert ex.views > 10000


def test_coop_blocks_follow_the_panel_grid():
    """The budget counts the panel grid the library launches: ceil(n / 8)
    blocks, at most one per SM and at most 160, only where its own route
    solves (auto: n >= 64; tridiag: n >= 2; cuSOLVER: never)."""
    assert us.coop_blocks(63, 152) == 0 and us.coop_blocks(64, 152) == 8
    assert us.coop_blocks(195, 152) == 25 and us.coop_blocks(2048, 152) == 152
    assert us.coop_blocks(4096, 200) == 160
    assert us.coop_blocks(10, 152, "tridiag") == 2 and us.coop_blocks(1000, 152, "cusolver") == 0


def test_block_budget_never_oversubscribes():
    """Threads acquiring random block counts (up to the whole budget) hold
    at most the budget between them at any time, and all of them finish."""
    import threading
    budget = us.BlockBudget(152)
    state = {"held": 0, "peak": 0}
    lock = threading.Lock()

    def worker(seed):
        rng = np.random.default_rng(seed)
        for _ in range(300):
            need = int(rng.choice([0, 8, 25, 64, 152]))
            budget.acquire(need)
            with lock:
                state["held"] += need
                state["peak"] = max(state["peak"], state["held"])
                assert state["held"] <= 152
            with lock:
                state["held"] -= need
            budget.release(need)

    threads = [threading.Thread(target=worker, args=(s,)) for s in range(8)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=60)
    assert not any(t.is_alive() for t in threads)
    assert budget.busy == 0 and 0 < state["peak"] <= 152
    with pytest.raises(ValueError):
        budget.acquire(153)
