"""Two-site DMRG sweeps on a particle-number-conserving (U(1)) MPS.

With a conserved particle number (Sec. 3.4 with symmetries) every bond index
carries a charge, the number of particles to its left, and every tensor of
the sweep is block sparse: A[a, s, b] is nonzero only where q(a) + s = q(b),
theta[a, s1, s2, c] only where q(a) + s1 + s2 = q(c), and the environments
only where q(bra) = q(ket) + q_w. One step of the sweep keeps that structure:

  1. theta = A_k A_{k+1}: one float64 product per (left sector, s1);
  2. the lowest eigenpair of the U(1) block of H_eff by Lanczos, the block
     products in one grouped tcgen05 launch per GEMM stage (osmps_u1_*);
  3. the split (Eq. AAD_ULLUD) per middle charge q: theta restricted to the
     rows (a, s1) with q(a) + s1 = q is one dense block M_q, so the Gram
     matrix is block diagonal; the float64 eigenpairs of each block's Gram
     matrix, then the truncation rule (Eq. elocal) applied to the spectra of
     all blocks jointly, which decides how many states each sector keeps;
  4. the environment update, as float64 products of blocks.

Storage: a tensor is the list of its allowed entries in C order of the dense
tensor (the library's packed format). A bond is a list of sectors (charge,
size) in ascending charge. This module is host orchestration: it builds the
lists of block products and copies from the sector bookkeeping and hands them
to the library (osmps_gemm_grouped: one launch per stage of products,
osmps_copy_list, osmps_sym_eig_top, osmps_lanczos_ground_u1); all
arithmetic runs in the library's kernels.
"""
import time

import numpy as np

from . import binding as B
from .u1 import channel_charges


class Bond:
    """Sectors (charge, size) of one bond, charges ascending."""

    def __init__(self, q, m):
        q = np.asarray(q, dtype=np.int64)
        m = np.asarray(m, dtype=np.int64)
        order = np.argsort(q, kind="stable")
        self.q, self.m = q[order], m[order]
        if (self.m < 1).any() or len(set(self.q.tolist())) != len(self.q):
            raise ValueError("a bond needs distinct charges and sizes >= 1")
        self._idx = {int(c): i for i, c in enumerate(self.q)}
        self.dim = int(self.m.sum())

    def find(self, charge):
        return self._idx.get(int(charge), -1)

    def charges(self):
        """Charge of every index of the bond."""
        return np.repeat(self.q, self.m)


class MpsLayout:
    """A[a, s, b] (q(a) + s = q(b)): the rows of left sector i form one dense
    block of row_len[i] columns, in which (s, b) for local state s occupy the
    columns col_off[i, s] .. + m[right_sector[i, s]]."""

    def __init__(self, left, right, d):
        nl = len(left.q)
        self.right_sector = np.full((nl, d), -1, dtype=np.int64)
        self.col_off = np.full((nl, d), -1, dtype=np.int64)
        self.row_len = np.zeros(nl, dtype=np.int64)
        for i, qi in enumerate(left.q):
            c = 0
            for s in range(d):
                j = right.find(qi + s)
                if j >= 0:
                    self.right_sector[i, s], self.col_off[i, s] = j, c
                    c += int(right.m[j])
            self.row_len[i] = c
        sizes = left.m * self.row_len
        self.row_off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        self.size = int(sizes.sum())


class ThetaLayout:
    """theta[a, s1, s2, c] (q(a) + s1 + s2 = q(c)): rows of left sector i form
    one dense block; for each s1, the columns (s2, c) start at col_off[i, s1]
    and number width(q(a) + s1) = sum over s2 of the size of right sector
    q(a) + s1 + s2 (the row length of the middle sector's A_{k+1} block)."""

    def __init__(self, left, right, d1, d2):
        nl = len(left.q)
        self.col_off = np.full((nl, d1), -1, dtype=np.int64)
        self.width = np.zeros((nl, d1), dtype=np.int64)
        self.row_len = np.zeros(nl, dtype=np.int64)
        for i, qi in enumerate(left.q):
            c = 0
            for s1 in range(d1):
                w = sum(int(right.m[right.find(qi + s1 + s2)]) for s2 in range(d2)
                        if right.find(qi + s1 + s2) >= 0)
                if w > 0:
                    self.col_off[i, s1], self.width[i, s1] = c, w
                    c += w
            self.row_len[i] = c
        sizes = left.m * self.row_len
        self.row_off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        self.size = int(sizes.sum())


class EnvLayout:
    """E[x, w, y] with q(x) = q(y) + q_w[w] over one bond: the rows of bra
    sector i form one dense block; channel w occupies the columns col_off[i,
    w] .. + m[ket[i, w]]."""

    def __init__(self, bond, q_w):
        nb, nw = len(bond.q), len(q_w)
        self.ket = np.full((nb, nw), -1, dtype=np.int64)
        self.col_off = np.full((nb, nw), -1, dtype=np.int64)
        self.row_len = np.zeros(nb, dtype=np.int64)
        for i, qi in enumerate(bond.q):
            c = 0
            for w in range(nw):
                j = bond.find(qi - q_w[w])
                if j >= 0:
                    self.ket[i, w], self.col_off[i, w] = j, c
                    c += int(bond.m[j])
            self.row_len[i] = c
        sizes = bond.m * self.row_len
        self.row_off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        self.size = int(sizes.sum())


# ---------------------------------------------------------------------------
# Operation records: (buffer, element offset) pairs, resolved by an executor
# ---------------------------------------------------------------------------
class Term:
    """alpha A B for one output: A (M x K) at (buffer, offset) with element
    strides (sam, sak), B (K x N) likewise."""
    __slots__ = ("A", "sam", "sak", "B", "sbk", "sbn", "K", "alpha")

    def __init__(self, A, sam, sak, B, sbk, sbn, K, alpha=1.0):
        self.A, self.sam, self.sak = A, int(sam), int(sak)
        self.B, self.sbk, self.sbn = B, int(sbk), int(sbn)
        self.K, self.alpha = int(K), float(alpha)


class Product:
    """C = sum over terms of alpha A B + beta C, C (M x N) at (buffer,
    offset) with element strides (scm, scn); no terms: C = beta C."""
    __slots__ = ("C", "scm", "scn", "M", "N", "beta", "terms")

    def __init__(self, C, scm, scn, M, N, terms=(), beta=0.0):
        self.C, self.scm, self.scn = C, int(scm), int(scn)
        self.M, self.N, self.beta = int(M), int(N), float(beta)
        self.terms = list(terms)


class Copy:
    """dst[r drs + c] = alpha src[r srs + c scs] (src None: zero), rows x cols."""
    __slots__ = ("src", "dst", "rows", "cols", "srs", "scs", "drs", "alpha")

    def __init__(self, src, dst, rows, cols, srs, scs, drs, alpha=1.0):
        self.src, self.dst = src, dst
        self.rows, self.cols = int(rows), int(cols)
        self.srs, self.scs, self.drs = int(srs), int(scs), int(drs)
        self.alpha = float(alpha)


class BlockBudget:
    """At most `total` blocks of cooperative launches in flight at once, held
    by threads that acquire a number of blocks before their solve and
    release it after. A cooperative grid's blocks must all be resident: with
    one block per SM counted, grids running together never wait on each
    other for room, only on kernels that end on their own."""

    def __init__(self, total):
        import threading
        self.total, self.busy = int(total), 0
        self._cond = threading.Condition()

    def acquire(self, need):
        if need > self.total:
            raise ValueError(f"{need} blocks requested of a budget of {self.total}")
        with self._cond:
            self._cond.wait_for(lambda: self.busy + need <= self.total)
            self.busy += need

    def release(self, need):
        with self._cond:
            self.busy -= need
            self._cond.notify_all()


def coop_blocks(n, sms, solver=None):
    """Blocks of the Householder panel's cooperative launch for an n x n
    eigenproblem: min(SMs, 160, ceil(n / 8)) on the library's own route
    (from n = 64 under 'auto', from n = 2 under 'tridiag'), 0 where cuSOLVER
    solves it (no cooperative launch)."""
    own_from = {None: 64, "auto": 64, "tridiag": 2}.get(solver)
    if own_from is None or n < own_from:
        return 0
    return max(1, min(sms, 160, (n + 7) // 8))


class DeviceExecutor:
    """Runs operation records on the GPU through the library (buffers are
    float64 CUDA tensors). eig_workers: how many sector eigensolves of a
    split may run at once (1: one after another on ctx); eig_solver: the
    eigensolver route of the worker contexts ('auto' when None)."""

    def __init__(self, ctx, eig_workers=8, eig_solver=None):
        import torch
        self.ctx, self.torch = ctx, torch
        self.eig_workers, self.eig_solver = int(eig_workers), eig_solver
        self._pool = None
        self._sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count

    def empty(self, n):
        return self.torch.empty(max(int(n), 1), dtype=self.torch.float64, device="cuda")

    @staticmethod
    def _p(ref):
        buf, off = ref
        return buf.data_ptr() + 8 * int(off)

    def products(self, ops):
        """All products of one stage in one grouped launch (outputs disjoint)."""
        if not ops:
            return
        p = self._p
        outs, terms = [], []
        for o in ops:
            outs.append((p(o.C), o.scm, o.scn, o.M, o.N, o.beta, len(terms), len(o.terms)))
            terms.extend((p(t.A), t.sam, t.sak, p(t.B), t.sbk, t.sbn, t.K, t.alpha) for t in o.terms)
        B.osmps_gemm_grouped(self.ctx, np.array(outs, dtype=B.GEMM_OUT_DTYPE),
                             np.array(terms, dtype=B.GEMM_TERM_DTYPE))

    def copies(self, ops):
        if ops:
            B.osmps_copy_list(self.ctx, [(self._p(c.src) if c.src is not None else 0,
                                          self._p(c.dst), c.rows, c.cols, c.srs, c.scs, c.drs,
                                          c.alpha) for c in ops])

    def norm2(self, buf, n):
        return B.osmps_vec_norm2(self.ctx, buf[:n]) if n > 0 else 0.0

    def eig_top(self, G, n, nev):
        """Largest nev eigenpairs of the n x n matrix at G (overwritten):
        (eigenvalues ascending, device array of the eigenvectors as rows)."""
        Y = self.empty(nev * n)
        ev = B.osmps_sym_eig_top(self.ctx, G[: n * n].view(n, n), nev, Y[: nev * n].view(nev, n))
        return ev, Y

    def eig_top_many(self, jobs):
        """eig_top for every (G, n, nev) of jobs: the sectors of one split are
        independent, so up to eig_workers of them run at once, each on a
        worker thread with its own context and stream. The Householder panels
        of this library's eigensolver are cooperative launches of
        min(SMs, n / 8) blocks from n = 64 on, which must all be resident: the
        solves running together are kept within one block per SM. Largest
        first, as the sectors' costs differ the most."""
        if self.eig_workers <= 1 or len(jobs) <= 1:
            return [self.eig_top(*j) for j in jobs]
        import threading
        from concurrent.futures import ThreadPoolExecutor
        if self._pool is None:
            self._tls = threading.local()
            self._lock = threading.Lock()
            self._budget = BlockBudget(self._sms)
            self._workers = []  # (context, stream) of every worker thread
            self._pool = ThreadPoolExecutor(max_workers=self.eig_workers)
        torch = self.torch
        ready = torch.cuda.Event()
        ready.record()  # the Gram matrices, written on this thread's stream

        def run(job):
            G, n, nev = job
            tl = self._tls
            if not hasattr(tl, "ctx"):
                tl.ctx = B.Context(self.ctx.device)
                if self.eig_solver is not None:
                    tl.ctx.set_eig_solver(self.eig_solver)
                tl.stream = torch.cuda.Stream()
                with self._lock:
                    self._workers.append((tl.ctx, tl.stream))
            need = coop_blocks(n, self._sms, self.eig_solver)
            self._budget.acquire(need)
            try:
                tl.stream.wait_event(ready)
                Y = torch.empty(max(nev * n, 1), dtype=torch.float64, device="cuda")
                ev = B.osmps_sym_eig_top(tl.ctx, G[: n * n].view(n, n), nev, Y[: nev * n].view(nev, n),
                                         stream=tl.stream)  # synchronises tl.stream
                return ev, Y
            finally:
                self._budget.release(need)

        order = sorted(range(len(jobs)), key=lambda i: -jobs[i][1])
        futures = {i: self._pool.submit(run, jobs[i]) for i in order}
        return [futures[i].result() for i in range(len(jobs))]

    def close(self):
        """Stop the eigensolve workers and release their contexts."""
        if self._pool is not None:
            self._pool.shutdown(wait=True)
            for c, st in self._workers:
                st.synchronize()
                c.close()
            self._pool, self._workers = None, []

    def upload(self, a):
        return self.torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).to("cuda")

    def download(self, buf, n):
        return buf[:n].cpu().numpy()

    def ground(self, Lk, W1, W2, Rk, theta, left, right, d, q_wl, q_wr, wm, precision, tol, max_iter):
        """Lowest eigenpair of the U(1) block of H_eff (theta: start vector in,
        Ritz vector out). Returns (energy, Lanczos iterations)."""
        plan = B.U1Heff(self.ctx, left.q, left.m, right.q, right.m, d, d, len(q_wl), wm, len(q_wr),
                        q_wl, q_wr)
        try:
            e, it, _, _ = B.osmps_lanczos_ground_u1(self.ctx, plan, Lk, W1, W2, Rk, theta[: plan.n_theta],
                                                    max_iter=max_iter, tol=tol, precision=precision)
        finally:
            plan.close()
        return e, it

    def sync(self):
        self.torch.cuda.synchronize()


# ---------------------------------------------------------------------------
# Block operations of one step
# ---------------------------------------------------------------------------
def theta_ops(A1, lay1, A2, lay2, mid, left, theta, layt):
    """theta = A_k A_{k+1}: one product per block (left sector i, s1) of
    theta, a single term A_k(i, s1) A_{k+1}(middle sector q(i) + s1); blocks
    whose middle charge the bond does not carry are zeroed."""
    ops = []
    for i in range(len(left.q)):
        for s1 in range(layt.col_off.shape[1]):
            if layt.col_off[i, s1] < 0:
                continue
            out = ((theta, layt.row_off[i] + layt.col_off[i, s1]), layt.row_len[i], 1,
                   left.m[i], layt.width[i, s1])
            jm = lay1.right_sector[i, s1]
            if jm < 0:
                ops.append(Product(*out))
                continue
            assert lay2.row_len[jm] == layt.width[i, s1]
            ops.append(Product(*out, terms=[Term((A1, lay1.row_off[i] + lay1.col_off[i, s1]),
                                                 lay1.row_len[i], 1, (A2, lay2.row_off[jm]),
                                                 lay2.row_len[jm], 1, mid.m[jm])]))
    return ops


def middle_groups(left, layt, d1):
    """Middle charge q -> [(left sector i, s1, row offset in M_q)], width W_q
    and row count n_q of M_q (theta restricted to q(a) + s1 = q)."""
    groups = {}
    for i, qi in enumerate(left.q):
        for s1 in range(d1):
            if layt.col_off[i, s1] < 0:
                continue
            q = int(qi + s1)
            g = groups.setdefault(q, {"rows": [], "n": 0, "W": int(layt.width[i, s1])})
            g["rows"].append((i, s1, g["n"]))
            g["n"] += int(left.m[i])
    return groups


def truncation(values, tr, chi_max, eps_local, rank):
    """The local truncation rule (Eq. elocal, Sec. 3.4) on a joint spectrum:
    values (lambda^2, any order) and tr = ||theta||^2; keep the largest,
    chi' = min(chi_max, rank, smallest n with discarded weight <= eps_local),
    at least one. Returns (indices kept, discarded weight, entropy)."""
    order = np.argsort(-np.asarray(values), kind="stable")
    lam2 = np.maximum(np.asarray(values)[order], 0.0) / tr
    cap = max(1, min(int(chi_max), int(rank), len(lam2)))
    kept, comp, keep = 0.0, 0.0, 0
    while keep < len(lam2):
        y = lam2[keep] - comp
        u = kept + y
        comp = (u - kept) - y
        kept = u
        keep += 1
        if 1.0 - kept <= eps_local or keep >= cap:
            break
    p = lam2[:keep] / kept
    p = p[p > 0]
    return order[:keep], max(1.0 - kept, 0.0), float(-(p * np.log(p)).sum())


def _nonzero_w(W, group):
    """Nonzero entries of W[w, t, s, w2] as lists of (key..., value) grouped
    by the axes in `group`, each list in C order of the remaining axes."""
    out = {}
    for idx in zip(*np.nonzero(W)):
        idx = tuple(int(x) for x in idx)
        key = tuple(idx[a] for a in group)
        rest = tuple(idx[a] for a in range(4) if a not in group)
        out.setdefault(key, []).append(rest + (float(W[idx]),))
    return out


def _scratch(X, n):
    """X itself, or X(n) when X is an allocator."""
    return X(n) if callable(X) else X


def env_left_ops(Lold, elo, A, lay, Lnew, eln, W, left, mid, X):
    """L_new[b', w', b] = sum A[a', t, b'] L_old[a', w, a] W[w, t, s, w'] A[a, s, b]
    in two grouped stages: X(i2, w) = L_old(i2, w) A(i), all s at once (one
    product per bra sector i2 and channel w), then one product per block
    (j2, w') of L_new whose terms are W[w, t, s, w'] A(i2, t)^T X(i2, w)[s]
    over every nonzero W entry and sector pair that reaches it (blocks with
    no term are zeroed). X: scratch buffer, or a function that allocates one
    of the size it is given. Returns (stage-1 products, stage-2 products, X
    elements needed)."""
    xoff, off = [], 0
    for i2 in range(len(left.q)):
        for w in range(elo.ket.shape[1]):
            i = int(elo.ket[i2, w])
            if i < 0 or lay.row_len[i] == 0:
                continue
            xoff.append((i2, w, i, off))
            off += int(left.m[i2] * lay.row_len[i])
    X = _scratch(X, off)
    s1_ops = [Product((X, xo), lay.row_len[i], 1, left.m[i2], lay.row_len[i],
                      terms=[Term((Lold, elo.row_off[i2] + elo.col_off[i2, w]), elo.row_len[i2], 1,
                                  (A, lay.row_off[i]), lay.row_len[i], 1, left.m[i])])
              for (i2, w, i, xo) in xoff]
    nzw = _nonzero_w(W, (0,))  # per w: (t, s, w2, value); ordered by s below
    by_w = {w: sorted(v, key=lambda e: (e[1], e[0], e[2])) for (w,), v in nzw.items()}
    rs, co, rl, ro = lay.right_sector, lay.col_off, lay.row_len, lay.row_off
    blocks = {}
    for (i2, w, i, xo) in xoff:
        m2 = left.m[i2]
        for (t, s_, w2, val) in by_w.get(w, ()):
            j, j2 = rs[i, s_], rs[i2, t]
            if j < 0 or j2 < 0:
                continue
            assert eln.ket[j2, w2] == j
            blocks.setdefault((int(j2), w2), []).append(
                Term((A, ro[i2] + co[i2, t]), 1, rl[i2], (X, xo + co[i, s_]), rl[i], 1, m2, alpha=val))
    s2_ops = []
    for j2 in range(len(mid.q)):
        for w2 in range(eln.ket.shape[1]):
            j = eln.ket[j2, w2]
            if j < 0:
                continue
            s2_ops.append(Product((Lnew, eln.row_off[j2] + eln.col_off[j2, w2]), eln.row_len[j2], 1,
                                  mid.m[j2], mid.m[j], terms=blocks.get((j2, w2), ())))
    return s1_ops, s2_ops, off


def env_right_ops(Rold, ero, A, lay, Rnew, ern, W, mid, right, Z):
    """R_new[a2, w, a] = sum A[a2, t, c2] W[w, t, s, w2] R_old[c2, w2, c] A[a, s, c]
    in two grouped stages: Z(j, s, jc2, w2) = A(j, s) R_old(jc2, w2)^T, then
    one product per block (j2, w) of R_new whose terms are
    W[w, t, s, w2] A(j2, t) Z(j, s, jc2, w2)^T (blocks with no term are
    zeroed). Z: scratch buffer, or a function that allocates one of the size
    it is given."""
    # the (jc2, w2) pairs of R_old whose ket sector is jc, in C order
    by_ket = {}
    for jc2 in range(len(right.q)):
        for w2 in range(ero.ket.shape[1]):
            if ero.ket[jc2, w2] >= 0:
                by_ket.setdefault(int(ero.ket[jc2, w2]), []).append((jc2, w2))
    zoff, off = [], 0
    d = lay.col_off.shape[1]
    for j in range(len(mid.q)):
        for s_ in range(d):
            jc = int(lay.right_sector[j, s_])
            if jc < 0:
                continue
            for (jc2, w2) in by_ket.get(jc, ()):
                zoff.append((j, s_, jc, jc2, w2, off))
                off += int(mid.m[j] * right.m[jc2])
    Z = _scratch(Z, off)
    s1_ops = [Product((Z, zo), right.m[jc2], 1, mid.m[j], right.m[jc2],
                      terms=[Term((A, lay.row_off[j] + lay.col_off[j, s_]), lay.row_len[j], 1,
                                  (Rold, ero.row_off[jc2] + ero.col_off[jc2, w2]), 1,
                                  ero.row_len[jc2], right.m[jc])])
              for (j, s_, jc, jc2, w2, zo) in zoff]
    nzw = _nonzero_w(W, (2, 3))  # per (s, w2): (w, t, value); ordered by t below
    by_sw = {k: sorted(v, key=lambda e: (e[1], e[0])) for k, v in nzw.items()}
    rs, co, rl, ro = lay.right_sector, lay.col_off, lay.row_len, lay.row_off
    blocks = {}
    for (j, s_, jc, jc2, w2, zo) in zoff:
        terms = by_sw.get((s_, w2))
        if not terms:
            continue
        qc2, mc2 = right.q[jc2], right.m[jc2]
        for (w, t, val) in terms:
            j2 = mid.find(qc2 - t)
            if j2 < 0 or rs[j2, t] != jc2:
                continue
            assert ern.ket[j2, w] == j
            blocks.setdefault((j2, w), []).append(
                Term((A, ro[j2] + co[j2, t]), rl[j2], 1, (Z, zo), 1, mc2, mc2, alpha=val))
    s2_ops = []
    for j2 in range(len(mid.q)):
        for w in range(ern.ket.shape[1]):
            j = ern.ket[j2, w]
            if j < 0:
                continue
            s2_ops.append(Product((Rnew, ern.row_off[j2] + ern.col_off[j2, w]), ern.row_len[j2], 1,
                                  mid.m[j2], mid.m[j], terms=blocks.get((j2, w), ())))
    return s1_ops, s2_ops, off


def split(ex, theta, layt, left, right, d1, d2, move_right, chi_max, eps_local):
    """Split theta (packed over left, right bonds) by the eigendecomposition
    route per middle charge with joint truncation. Returns the new middle
    bond, A1 (left -> mid) and A2 (mid -> right) packed, the discarded weight
    and the entropy. move_right: A1 left-canonical, A2 renormalised; else A2
    right-canonical, A1 renormalised."""
    groups = middle_groups(left, layt, d1)
    tr = ex.norm2(theta, layt.size)
    if not (tr > 0.0) or not np.isfinite(tr):
        raise B.OsmpsError(B.ENAN, "u1 split: theta has zero or non-finite norm")
    vecs, jobs, ops = {}, [], []
    for q, g in sorted(groups.items()):
        n, Wq = g["n"], g["W"]
        gdim = n if move_right else Wq          # Gram of the rows (L->R) or columns (R->L)
        nev = min(n, Wq, int(chi_max))
        if nev < 1:
            continue
        G = ex.empty(gdim * gdim)
        if move_right:   # G[g, g'] = theta_g theta_g'^T
            for (i, s1, r0) in g["rows"]:
                for (i2, s2, r2) in g["rows"]:
                    ops.append(Product((G, r0 * gdim + r2), gdim, 1, left.m[i], left.m[i2], terms=[
                        Term((theta, layt.row_off[i] + layt.col_off[i, s1]), layt.row_len[i], 1,
                             (theta, layt.row_off[i2] + layt.col_off[i2, s2]), 1, layt.row_len[i2], Wq)]))
        else:            # G = sum_g theta_g^T theta_g
            ops.append(Product((G, 0), gdim, 1, Wq, Wq, terms=[
                Term((theta, layt.row_off[i] + layt.col_off[i, s1]), 1, layt.row_len[i],
                     (theta, layt.row_off[i] + layt.col_off[i, s1]), layt.row_len[i], 1, left.m[i])
                for (i, s1, r0) in g["rows"]]))
        jobs.append((q, G, gdim, nev))
    if not jobs:
        raise B.OsmpsError(B.ESHAPE, "u1 split: no middle sector carries a state")
    ex.products(ops)  # every sector's Gram matrix in one grouped launch
    results = ex.eig_top_many([(G, gdim, nev) for (_, G, gdim, nev) in jobs])
    # the joint spectrum: sector by sector (ascending charge), largest first
    # within a sector (the c-th largest is row nev - 1 - c of Y)
    vals, qs = [], []
    for (q, _, gdim, nev), (ev, Y) in zip(jobs, results):
        vecs[q] = (Y, gdim, nev)
        vals.append(np.asarray(ev[:nev], dtype=np.float64)[::-1])
        qs.append(np.full(nev, q, dtype=np.int64))
    vals, qs = np.concatenate(vals), np.concatenate(qs)
    rank = len(vals)
    keep_idx, discarded, entropy = truncation(vals, tr, chi_max, eps_local, rank)
    kept_q, kept_n = np.unique(qs[keep_idx], return_counts=True)
    kq = {int(q): int(c) for q, c in zip(kept_q, kept_n)}
    mid = Bond(sorted(kq), [kq[q] for q in sorted(kq)])
    lay1, lay2 = MpsLayout(left, mid, d1), MpsLayout(mid, right, d2)
    A1, A2 = ex.empty(lay1.size), ex.empty(lay2.size)
    prods, copies = [], []
    for jm, q in enumerate(mid.q):
        q = int(q)
        k = kq[q]
        g = groups[q]
        Y, gdim, nev = vecs[q]
        top = (nev - 1) * gdim  # row of the largest eigenvector; next ones at -gdim
        if move_right:
            terms = []
            for (i, s1, r0) in g["rows"]:
                # A1 block (i, s1) = U_q[rows of the group, :k]
                copies.append(Copy((Y, top + r0), (A1, lay1.row_off[i] + lay1.col_off[i, s1]),
                                   left.m[i], k, 1, -gdim, lay1.row_len[i]))
                terms.append(Term((Y, top + r0), -gdim, 1,
                                  (theta, layt.row_off[i] + layt.col_off[i, s1]), layt.row_len[i], 1,
                                  left.m[i]))
            # A2 rows of sector q = U_q[:, :k]^T M_q (a sum over the groups' rows)
            prods.append(Product((A2, lay2.row_off[jm]), lay2.row_len[jm], 1, k, g["W"], terms=terms))
        else:
            # A2 rows of sector q = V_q[:, :k]^T
            copies.append(Copy((Y, top), (A2, lay2.row_off[jm]), k, g["W"], -gdim, 1,
                               lay2.row_len[jm]))
            for (i, s1, r0) in g["rows"]:
                # A1 block (i, s1) = theta_g V_q[:, :k]
                prods.append(Product((A1, lay1.row_off[i] + lay1.col_off[i, s1]), lay1.row_len[i], 1,
                                     left.m[i], k, terms=[
                                         Term((theta, layt.row_off[i] + layt.col_off[i, s1]), layt.row_len[i], 1,
                                              (Y, top), 1, -gdim, g["W"])]))
    ex.copies(copies)
    ex.products(prods)
    # renormalise the non-isometric factor (the kept Schmidt values sum to 1)
    other, size = (A2, lay2.size) if move_right else (A1, lay1.size)
    nrm2 = ex.norm2(other, size)
    ex.copies([Copy((other, 0), (other, 0), 1, size, 0, 1, size, 1.0 / np.sqrt(nrm2))])
    return mid, A1, A2, discarded, entropy


class U1MPS:
    """A particle-number-conserving MPS on the device: bonds (L+1 Bond) and
    packed site tensors (CUDA float64 tensors)."""

    def __init__(self, ex, bonds, tensors, d):
        self.ex, self.bonds, self.d = ex, list(bonds), int(d)
        self.L = len(self.bonds) - 1
        self.A = []
        for k in range(self.L):
            lay = MpsLayout(self.bonds[k], self.bonds[k + 1], self.d)
            t = np.ascontiguousarray(tensors[k], dtype=np.float64).ravel()
            if t.size != lay.size:
                raise ValueError(f"site {k}: {t.size} entries, the sectors allow {lay.size}")
            self.A.append(ex.upload(t))

    def layout(self, k):
        return MpsLayout(self.bonds[k], self.bonds[k + 1], self.d)

    def tensors(self):
        """Host copies of the packed site tensors."""
        return [self.ex.download(a, self.layout(k).size) for k, a in enumerate(self.A)]

    def dense(self):
        """Dense site tensors (host) for checks."""
        out = []
        for k, a in enumerate(self.tensors()):
            ql, qr = self.bonds[k].charges(), self.bonds[k + 1].charges()
            mask = ql[:, None, None] + np.arange(self.d)[None, :, None] == qr[None, None, :]
            t = np.zeros(mask.shape)
            t[mask] = a
            out.append(t)
        return out


def random_u1_mps(ex, L, d, N, chi, seed=0):
    """Seeded random particle-number-conserving MPS with N particles on L
    sites (local states 0 .. d-1): bond k carries the charges reachable from
    both ends, each sector min(states on the left, states on the right,
    chi / (number of charges)) deep (at least 1); entries N(0,1) from
    default_rng(seed), site by site in packed order."""
    def counts(n_sites):
        c = np.zeros(n_sites * (d - 1) + 1)
        c[0] = 1.0
        for _ in range(n_sites):
            nxt = np.zeros_like(c)
            for s in range(d):
                nxt[s:] += c[: len(c) - s]
            c = nxt
        return c
    bonds = []
    for k in range(L + 1):
        lo, hi = max(0, N - (L - k) * (d - 1)), min(N, k * (d - 1))
        qs = np.arange(lo, hi + 1)
        cl, cr = counts(k), counts(L - k)
        per = max(1, chi // max(1, len(qs)))
        ms = [int(min(cl[q], cr[N - q], per)) for q in qs]
        bonds.append(Bond(qs, ms))
    rng = np.random.default_rng(seed)
    tensors = [rng.standard_normal(MpsLayout(bonds[k], bonds[k + 1], d).size) for k in range(L)]
    return U1MPS(ex, bonds, tensors, d)


def u1_sweep(mps, W, n_sweeps=1, chi_max=64, eps_local=0.0, precision="tf32x3",
             lanczos_tol=1e-10, lanczos_max_iter=100, phase_timing=False):
    """Two-site sweeps on a U(1) MPS for the MPO W (list of dense site tensors
    W[w, t, s, w2] that conserve the particle number). The state is first
    brought to right-canonical form by right-to-left splits without
    truncation; then each sweep optimises the pairs (0,1) ... (L-2,L-1) and
    back. Returns a dict with the float64 energy <psi|H|psi> / <psi|psi> of
    the final state (block environments contracted through the chain), the
    largest discarded weight, Lanczos iterations and timings (phase_timing:
    also seconds per phase of the steps, synchronising after each phase)."""
    ex = mps.ex
    L, d = mps.L, mps.d
    qw = channel_charges(W)
    Wd = [ex.upload(w) for w in W]
    t0 = time.perf_counter()

    def form_theta(k):
        left, mid, right = mps.bonds[k], mps.bonds[k + 1], mps.bonds[k + 2]
        layt = ThetaLayout(left, right, d, d)
        th = ex.empty(layt.size)
        ex.products(theta_ops(mps.A[k], mps.layout(k), mps.A[k + 1], mps.layout(k + 1), mid, left,
                           th, layt))
        return th, layt

    def do_split(k, th, layt, move_right, chi, eps):
        mid, A1, A2, disc, ent = split(ex, th, layt, mps.bonds[k], mps.bonds[k + 2], d, d,
                                       move_right, chi, eps)
        mps.bonds[k + 1] = mid
        mps.A[k], mps.A[k + 1] = A1, A2
        return disc

    # right-canonical start: right-to-left splits, no truncation beyond rank
    for k in range(L - 2, -1, -1):
        th, layt = form_theta(k)
        do_split(k, th, layt, False, 1 << 30, 1e-15)
    nrm2 = ex.norm2(mps.A[0], mps.layout(0).size)
    ex.copies([Copy((mps.A[0], 0), (mps.A[0], 0), 1, mps.layout(0).size, 0, 1,
                    mps.layout(0).size, 1.0 / np.sqrt(nrm2))])

    def env_left(k, Lk):
        left, mid = mps.bonds[k], mps.bonds[k + 1]
        elo, eln = EnvLayout(left, qw[k]), EnvLayout(mid, qw[k + 1])
        Ln = ex.empty(eln.size)
        s1, s2, _ = env_left_ops(Lk, elo, mps.A[k], mps.layout(k), Ln, eln, W[k], left, mid, ex.empty)
        ex.products(s1)
        ex.products(s2)
        return Ln

    def env_right(k, Rk1):
        mid, right = mps.bonds[k], mps.bonds[k + 1]
        ero, ern = EnvLayout(right, qw[k + 1]), EnvLayout(mid, qw[k])
        Rn = ex.empty(ern.size)
        s1, s2, _ = env_right_ops(Rk1, ero, mps.A[k], mps.layout(k), Rn, ern, W[k], mid, right, ex.empty)
        ex.products(s1)
        ex.products(s2)
        return Rn

    one = lambda: ex.upload(np.ones(1))
    Lenv = [None] * (L + 1)
    Renv = [None] * (L + 1)
    Lenv[0], Renv[L] = one(), one()
    for k in range(L - 1, 1, -1):
        Renv[k] = env_right(k, Renv[k + 1])
    t_setup = time.perf_counter() - t0

    iters, max_disc, energy_step, steps = 0, 0.0, None, 0
    phase = {"theta": 0.0, "lanczos": 0.0, "split": 0.0, "env": 0.0}

    def mark(name, t):
        # phase seconds (synchronising after each phase) when asked for
        if not phase_timing:
            return t
        ex.sync()
        now = time.perf_counter()
        phase[name] += now - t
        return now

    t1 = time.perf_counter()
    schedule = list(range(L - 1)) + list(range(L - 2, -1, -1))
    for _ in range(n_sweeps):
        for n_, k in enumerate(schedule):
            move_right = n_ < L - 1
            tp = time.perf_counter()
            th, layt = form_theta(k)
            tp = mark("theta", tp)
            e, it = ex.ground(Lenv[k], Wd[k], Wd[k + 1], Renv[k + 2], th, mps.bonds[k],
                              mps.bonds[k + 2], d, qw[k], qw[k + 2], W[k].shape[3], precision,
                              lanczos_tol, lanczos_max_iter)
            tp = mark("lanczos", tp)
            iters += it
            energy_step = e
            disc = do_split(k, th, layt, move_right, chi_max, eps_local)
            tp = mark("split", tp)
            max_disc = max(max_disc, disc)
            if move_right:
                Lenv[k + 1] = env_left(k, Lenv[k])
            else:
                Renv[k + 1] = env_right(k + 1, Renv[k + 2])
            mark("env", tp)
            steps += 1
    ex.sync()
    t_sweep = time.perf_counter() - t1
    # float64 <psi|H|psi> through the chain (the centre is at site 0)
    t2 = time.perf_counter()
    Lk = Lenv[0]
    for k in range(L):
        Lk = env_left(k, Lk)
    h = float(ex.download(Lk, 1)[0])
    norm2 = ex.norm2(mps.A[0], mps.layout(0).size)
    t_energy = time.perf_counter() - t2
    return {"energy": h / norm2, "last_step_energy": energy_step, "max_discarded": max_disc,
            "lanczos_iters": iters, "steps": steps, "max_chi": max(b.dim for b in mps.bonds),
            "setup_seconds": t_setup, "sweep_seconds": t_sweep, "energy_seconds": t_energy,
            "phase_seconds": phase if phase_timing else None}
