"""The two Lanczos drivers, the host loop and the CUDA graph whose while-node
repeats the recorded step on the device, run the same kernels on the same
data: energies, step counts, residuals and Ritz vectors must be bit-identical,
for every precision, the projected (excited-state) and U(1) forms, the
iteration cap and the sweeps built on them. Each case is also checked
against the oracle where that adds something (the graph must not be merely
self-consistent)."""
import numpy as np
import pytest

from oracle import dmrg as od
from oracle import u1 as ou1
from paper_1703_00387_gb300 import binding as B
from paper_1703_00387_gb300 import hamiltonians, inputs

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
    c.set_lanczos_mode("auto")
    c.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _xxz_operator(L, k, chi, seed):
    W = hamiltonians.xxz(L, 1.0, 1.0, 0.0)
    mps = od.right_canonicalize(inputs.random_mps(L, 2, chi, seed=seed))
    Renv = od.build_right_envs(W, mps)
    Lenv = np.ones((1, 1, 1))
    for j in range(k):
        chl, d, chr_ = mps[j].shape
        Q, Rm = np.linalg.qr(mps[j].reshape(chl * d, chr_))
        mps[j] = Q.reshape(chl, d, Q.shape[1])
        mps[j + 1] = np.tensordot(Rm, mps[j + 1], axes=([1], [0]))
        Lenv = od.env_left(Lenv, mps[j], W[j])
    theta = np.tensordot(mps[k], mps[k + 1], axes=([2], [0]))
    return Lenv, W[k], W[k + 1], Renv[k + 2], theta


def _both(ctx, run):
    """run() -> (result tuple, output tensor); once per driver, after one
    untimed run (the first product of a size class times the GEMM tile
    widths, launches that neither driver repeats)."""
    run()
    torch.cuda.synchronize()
    out = {}
    for mode in ("host", "graph"):
        ctx.set_lanczos_mode(mode)
        n0 = B.osmps_kernel_launches()
        res, t = run()
        torch.cuda.synchronize()
        out[mode] = (res, t.clone(), B.osmps_kernel_launches() - n0)
    ctx.set_lanczos_mode("auto")
    return out


# (L, k, chi, seed): n = 4 chi_l chi_r from 196 to ~40 000, ragged tails
CASES = [(12, 5, 32, 2), (14, 6, 100, 4), (9, 4, 7, 6)]


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32x3", "fp64emu"])
@pytest.mark.parametrize("case", CASES)
def test_graph_driver_is_bit_identical_to_host_loop(ctx, prec, case):
    L, k, chi, seed = case
    Lh, W1, W2, Rh, theta = _xxz_operator(L, k, chi, seed)
    ops = [dev(x) for x in (Lh, W1, W2, Rh)]
    tol = 1e-12 if prec in ("fp64", "fp64emu") else 1e-6

    def run():
        th = dev(theta)
        r = B.osmps_lanczos_ground(ctx, *ops, th, max_iter=100, tol=tol, precision=prec)
        return r, th

    out = _both(ctx, run)
    (eh, ih, rh, okh), th_h, nh = out["host"]
    (eg, ig, rg, okg), th_g, ng = out["graph"]
    assert (eh, ih, rh, okh) == (eg, ig, rg, okg)
    assert torch.equal(th_h, th_g)
    # the same kernels per step on both drivers; the graph adds only its
    # loop-entry kernel
    assert ng - nh == 1
    # and the pair is the oracle's ground state
    mv = lambda x: od.heff_apply(Lh, W1, W2, Rh, x)
    e_ref, _, _, _ = od.lanczos_ground(mv, theta, 100, 1e-12)
    assert okg
    assert abs(eg - e_ref) <= (1e-10 if prec in ("fp64", "fp64emu") else 1e-5) * abs(e_ref)


@pytest.mark.parametrize("max_iter", [1, 2, 3, 7])
def test_graph_driver_iteration_cap(ctx, max_iter):
    Lh, W1, W2, Rh, theta = _xxz_operator(10, 4, 16, seed=3)
    ops = [dev(x) for x in (Lh, W1, W2, Rh)]

    def run():
        th = dev(theta)
        r = B.osmps_lanczos_ground(ctx, *ops, th, max_iter=max_iter, tol=1e-15, precision="fp64")
        return r, th

    out = _both(ctx, run)
    assert out["host"][0] == out["graph"][0]
    assert torch.equal(out["host"][1], out["graph"][1])
    e, it, res, ok = out["graph"][0]
    assert not ok and it == max_iter
    assert abs(torch.linalg.norm(out["graph"][1]).item() - 1.0) < 1e-12
    # the Ritz value of an m-step Krylov space from the oracle's own Lanczos
    mv = lambda x: od.heff_apply(Lh, W1, W2, Rh, x)
    e_ref, _, it_ref, _ = od.lanczos_ground(mv, theta, max_iter, 0.0)
    assert it_ref == max_iter
    assert abs(e - e_ref) <= 1e-11 * abs(e_ref)


def test_graph_driver_exhausted_krylov_space(ctx):
    # n = 8: the Krylov space is the whole space after at most 8 steps
    Lh, W1, W2, Rh, theta = _xxz_operator(4, 0, 2, seed=8)
    n = theta.size
    assert n <= 8
    ops = [dev(x) for x in (Lh, W1, W2, Rh)]

    def run():
        th = dev(theta)
        r = B.osmps_lanczos_ground(ctx, *ops, th, max_iter=100, tol=0.0, precision="fp64")
        return r, th

    out = _both(ctx, run)
    assert out["host"][0] == out["graph"][0]
    assert torch.equal(out["host"][1], out["graph"][1])
    e, it, res, ok = out["graph"][0]
    H = np.stack([od.heff_apply(Lh, W1, W2, Rh, np.eye(n)[c].reshape(theta.shape)).ravel()
                  for c in range(n)], axis=1)
    assert ok and it <= n
    assert abs(e - np.linalg.eigvalsh(H)[0]) <= 1e-12 * np.abs(H).max() * n


@pytest.mark.parametrize("k", [1, 3])
def test_graph_driver_projected(ctx, k):
    Lh, W1, W2, Rh, theta = _xxz_operator(12, 5, 24, seed=5)
    n = theta.size
    P = dev(np.random.default_rng(7).standard_normal((k, n)))
    ops = [dev(x) for x in (Lh, W1, W2, Rh)]

    def run():
        th = dev(theta)
        r = B.osmps_lanczos_ground_projected(ctx, *ops, th, P, max_iter=150, tol=1e-11,
                                             precision="fp64")
        return r, th

    out = _both(ctx, run)
    assert out["host"][0] == out["graph"][0]
    assert torch.equal(out["host"][1], out["graph"][1])
    v = out["graph"][1].cpu().numpy().ravel()
    Pn = P.cpu().numpy()
    assert np.abs(Pn @ v).max() <= 1e-10 * np.abs(Pn).max() * np.sqrt(n)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_graph_driver_u1(ctx, prec):
    from oracle import mpo as ompo
    from paper_1703_00387_gb300 import u1 as pu1
    Lc, N, nmax, chi_sec = 6, 6, 2, 2  # the operator of test_gpu_u1's Lanczos case
    d = nmax + 1
    sectors = []
    for kk in range(Lc + 1):
        qs = list(range(max(0, N - (Lc - kk) * nmax), min(N, kk * nmax) + 1))
        sectors.append((qs, [1 if kk in (0, Lc) else chi_sec] * len(qs)))
    q = [ou1.index_charges(*s) for s in sectors]
    A = [inputs.random_dense((len(q[kk]), d, len(q[kk + 1])), 10 + kk) * ou1.mps_mask(q[kk], q[kk + 1], d)
         for kk in range(Lc)]
    Wo = ompo.bose_hubbard_mpo(Lc, 1.0, 4.0, nmax)
    Le = np.ones((1, 1, 1))
    for kk in range(2):
        Le = od.env_left(Le, A[kk], Wo[kk])
    Re = np.ones((1, 1, 1))
    for kk in range(Lc - 1, 3, -1):
        Re = od.env_right(Re, A[kk], Wo[kk])
    Wp = hamiltonians.bose_hubbard(Lc, 1.0, 4.0, nmax)
    qp = pu1.channel_charges(Wp)
    op = pu1.U1Operator(ctx, sectors[2], sectors[4], d, d, Wp[2], Wp[3], qp[2], qp[4])
    mt = ou1.theta_mask(q[2], q[4], d, d)
    th0 = pu1.pack(inputs.random_dense(mt.shape, 5), op.m_theta)
    args = (dev(pu1.pack(Le, op.m_L)), dev(Wp[2]), dev(Wp[3]), dev(pu1.pack(Re, op.m_R)))

    def run():
        th = dev(th0)
        r = B.osmps_lanczos_ground_u1(ctx, op.plan, *args, th, max_iter=200, tol=1e-9,
                                      precision=prec)
        return r, th

    out = _both(ctx, run)
    op.close()
    assert out["host"][0] == out["graph"][0]
    assert torch.equal(out["host"][1], out["graph"][1])
    E0 = np.linalg.eigvalsh(ou1.sector_heff_matrix(Le, Wo[2], Wo[3], Re, mt))[0]
    assert abs(out["graph"][0][0] - E0) <= 1e-5 * abs(E0)


@pytest.mark.parametrize("prec,refine", [("fp64", 0), ("bf16x3", 1)])
def test_graph_driver_sweeps(ctx, prec, refine):
    W = hamiltonians.ising(12, 1.0, 1.0)
    mps0 = inputs.random_mps(12, 2, 32, seed=0)
    res = {}
    for mode in ("host", "graph"):
        ctx.set_lanczos_mode(mode)
        mpo = B.MPO(ctx, W)
        mps = B.MPS(ctx, mps0, chi_cap=32)
        p = B.sweep_params(32, 2, prec, lanczos_tol=1e-12, lanczos_max_iter=100,
                           refine_sweeps=refine)
        st = B.osmps_sweep(ctx, mps, mpo, p)
        res[mode] = (st["energy"], st["lanczos_iters"], [t.copy() for t in mps.tensors()])
        mps.close()
        mpo.close()
    ctx.set_lanczos_mode("auto")
    assert res["host"][0] == res["graph"][0]
    assert res["host"][1] == res["graph"][1]
    for a, b in zip(res["host"][2], res["graph"][2]):
        assert np.array_equal(a, b)


def test_graph_cache_replay_growth_and_eviction(ctx):
    # 20 shapes in growing size (each grows the workspace, so every cached
    # graph's addresses go stale), more than the 16 graphs a context keeps;
    # every solve runs twice in graph mode (record, then replay) and once in
    # the host loop, then the first shapes again (evicted or stale).
    cases = [(10, 4, chi, 20 + chi) for chi in range(3, 23)]
    ops = {}
    for case in cases + cases[:4]:
        L, k, chi, seed = case
        if case not in ops:
            Lh, W1, W2, Rh, theta = _xxz_operator(L, k, chi, seed)
            ops[case] = ([dev(x) for x in (Lh, W1, W2, Rh)], theta)
        o, theta = ops[case]
        got = []
        for mode in ("graph", "graph", "host"):
            ctx.set_lanczos_mode(mode)
            th = dev(theta)
            r = B.osmps_lanczos_ground(ctx, *o, th, max_iter=60, tol=1e-12, precision="bf16x3")
            got.append((r, th))
        ctx.set_lanczos_mode("auto")
        for r, th in got[1:]:
            assert r == got[0][0]
            assert torch.equal(th, got[0][1])


def test_lanczos_mode_is_validated(ctx):
    with pytest.raises(B.OsmpsError) as e:
        ctx.set_lanczos_mode(3)
    assert e.value.status == 1
    with pytest.raises(B.OsmpsError):
        ctx.set_lanczos_mode(-1)
