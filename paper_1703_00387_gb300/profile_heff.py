"""Small driver for profiler runs, with seeded inputs and under 2 GB of
device memory:

* repeated H_eff.theta products (and optionally one full two-site step) at a
  given bond dimension; --identity gives L and R the unit-matrix channels of
  a canonical MPS;
* --lanczos-solve: one 20-step Lanczos solve on a symmetric operator, after 3
  untimed solves, between the profiler's start and stop (for
  `ncu --profile-from-start off`);
* --u1: 3 products of the U(1) block-sparse H_eff.theta of the Bose-Hubbard
  workload (L=64, N=64, d=5, w=4, chi=512 per bond, sites 31 and 32), after
  3 untimed ones, between the profiler's start and stop;
* --tdvp: one two-site TDVP step (XXZ, L --tdvp-L, chi --chi, dt 0.05) from a
  random MPS right-canonicalised on the GPU, after one untimed step, between
  the profiler's start and stop.

    python -m paper_1703_00387_gb300.profile_heff --chi 1024 --prec bf16x3 --reps 3
    python -m paper_1703_00387_gb300.profile_heff --chi 1024 --prec bf16x3 --reps 3 --identity
    python -m paper_1703_00387_gb300.profile_heff --chi 1024 --step
    python -m paper_1703_00387_gb300.profile_heff --lanczos-solve --chi 32 --lanczos-mode host
    python -m paper_1703_00387_gb300.profile_heff --u1
    python -m paper_1703_00387_gb300.profile_heff --tdvp --tdvp-L 32 --chi 64
"""
import argparse
import time

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--chi", type=int, default=1024)
    ap.add_argument("--d", type=int, default=2)
    ap.add_argument("--w", type=int, default=5)
    ap.add_argument("--prec", default="bf16x3")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--step", action="store_true",
                    help="also run theta formation + Lanczos + split + env update once")
    ap.add_argument("--lanczos-solve", action="store_true")
    ap.add_argument("--lanczos-mode", default="auto", choices=["auto", "host", "graph"])
    ap.add_argument("--u1", action="store_true")
    ap.add_argument("--tdvp", action="store_true")
    ap.add_argument("--tdvp-L", type=int, default=32)
    ap.add_argument("--autotune", action="store_true",
                    help="let the tcgen05 GEMMs pick their tile width by timing (off by default: "
                         "timings under a profiler are distorted; 256 columns)")
    ap.add_argument("--identity", action="store_true",
                    help="environments of a canonical MPS: L's last and R's first channel the "
                         "unit matrix (left out of the GEMMs, with identity skipping 'always')")
    args = ap.parse_args()
    if args.lanczos_solve:
        return lanczos_solve(args)
    if args.u1:
        return u1_products(args)
    if args.tdvp:
        return tdvp_step(args)

    import torch
    from paper_1703_00387_gb300 import binding as B
    from paper_1703_00387_gb300 import hamiltonians, inputs

    dev = torch.device("cuda:0")
    ctx = B.Context(0)
    ctx.set_autotune(args.autotune)
    chi, d, w = args.chi, args.d, args.w
    W = hamiltonians.xxz(8, 1.0, 1.0, 0.0)[3] if (d, w) == (2, 5) else \
        np.random.default_rng(3).standard_normal((w, d, d, w))
    Lh = inputs.random_symmetric_env(chi, w, seed=1)
    Rh = inputs.random_symmetric_env(chi, w, seed=2)
    if args.identity:
        Lh[:, w - 1, :] = np.eye(chi)
        Rh[:, 0, :] = np.eye(chi)
        ctx.set_identity_skip("always")
    th = np.random.default_rng(3).standard_normal((chi, d, d, chi))
    L, Wt, R, x = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (Lh, W, Rh, th))
    y = torch.empty_like(x)
    for _ in range(args.reps):
        B.osmps_heff_apply(ctx, L, Wt, Wt, R, x, y, precision=args.prec)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B.osmps_heff_apply(ctx, L, Wt, Wt, R, x, y, precision=args.prec)
    torch.cuda.synchronize()
    print(f"heff_apply chi={chi} {args.prec}: {1e3 * (time.perf_counter() - t0):.3f} ms")
    if args.step:
        A1 = torch.from_numpy(np.random.default_rng(4).standard_normal((chi, d, chi))).to(dev)
        A2 = torch.from_numpy(np.random.default_rng(5).standard_normal((chi, d, chi))).to(dev)
        B.osmps_theta_form(ctx, A1, A2, x)
        B.osmps_lanczos_ground(ctx, L, Wt, Wt, R, x, max_iter=20, tol=1e-10, precision=args.prec)
        a1 = torch.empty(chi * d * chi, dtype=torch.float64, device=dev)
        a2 = torch.empty(chi * d * chi, dtype=torch.float64, device=dev)
        chn, _, _, _ = B.osmps_split(ctx, x, a1, a2, 1, chi, 1e-14, precision=args.prec)
        Lo = torch.empty(chn * w * chn, dtype=torch.float64, device=dev)
        B.osmps_env_update(ctx, 0, L, a1[: chi * d * chn].view(chi, d, chn), Wt,
                           Lo.view(chn, w, chn), precision=args.prec)
        torch.cuda.synchronize()
        print("step done, chi_new", chn)
    ctx.close()


def lanczos_solve(args):
    import torch
    from paper_1703_00387_gb300 import binding as B
    from paper_1703_00387_gb300 import inputs

    chi = args.chi
    Lh, W1, W2, Rh, th = inputs.random_heff_operands(chi, 2, 2, chi, 5, 5, 5, seed=1)
    # symmetric H_eff: environments symmetric in (bra, ket), MPO tensors in (t, s)
    Lh = 0.5 * (Lh + Lh.transpose(2, 1, 0))
    Rh = 0.5 * (Rh + Rh.transpose(2, 1, 0))
    W1 = 0.5 * (W1 + W1.transpose(0, 2, 1, 3))
    W2 = 0.5 * (W2 + W2.transpose(0, 2, 1, 3))
    ctx = B.Context(0)
    ctx.set_lanczos_mode(args.lanczos_mode)
    ops = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (Lh, W1, W2, Rh)]
    t0 = torch.from_numpy(th).cuda()
    for _ in range(3):
        B.osmps_lanczos_ground(ctx, *ops, t0.clone(), max_iter=20, tol=1e-15, precision=args.prec)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    r = B.osmps_lanczos_ground(ctx, *ops, t0.clone(), max_iter=20, tol=1e-15, precision=args.prec)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print("lanczos solve", r)
    ctx.close()


def u1_products(args):
    import torch
    from paper_1703_00387_gb300 import binding as B
    from paper_1703_00387_gb300 import hamiltonians, inputs
    from paper_1703_00387_gb300 import u1 as pu1

    ctx = B.Context(0)
    dev = torch.device("cuda:0")
    W = hamiltonians.bose_hubbard(64, 1.0, 4.0, 4)
    q = pu1.channel_charges(W)
    left = inputs.u1_sector_profile(31.0, total=512, width=8.0)
    right = inputs.u1_sector_profile(33.0, total=512, width=8.0)
    op = pu1.U1Operator(ctx, left, right, 5, 5, W[31], W[32], q[31], q[33])
    pl = op.plan
    t = [torch.from_numpy(inputs.random_dense((n,), seed)).to(dev)
         for n, seed in ((pl.n_L, 1), (pl.n_R, 2), (pl.n_theta, 3))]
    W1, W2 = (torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (W[31], W[32]))
    y = torch.empty_like(t[2])
    B.osmps_u1_heff_prepare(ctx, pl, t[0], W1, W2, t[1], precision=args.prec)
    for _ in range(3):
        B.osmps_u1_heff_apply(ctx, pl, t[2], y)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    for _ in range(3):
        B.osmps_u1_heff_apply(ctx, pl, t[2], y)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print("u1 products done, n_theta", pl.n_theta)
    op.close()
    ctx.close()


def tdvp_step(args):
    import torch
    from paper_1703_00387_gb300 import binding as B
    from paper_1703_00387_gb300 import hamiltonians, inputs

    ctx = B.Context(0)
    L, chi = args.tdvp_L, args.chi
    mpo = B.MPO(ctx, hamiltonians.xxz(L, 1.0, 1.0, 0.0))
    mps = B.MPS(ctx, inputs.random_mps(L, 2, chi, seed=21), chi_cap=chi)
    B.osmps_mps_canonicalize(ctx, mps, mpo, 0, precision="fp64")
    start = [t.astype(np.complex128) for t in mps.tensors()]
    mps.close()
    warm, _, _, _ = B.osmps_tdvp_evolve(ctx, mpo, start, 0.05, 1, chi_max=chi, krylov_tol=1e-10,
                                        precision=args.prec)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    _, e, _, st = B.osmps_tdvp_evolve(ctx, mpo, warm, 0.05, 1, chi_max=chi, krylov_tol=1e-10,
                                      precision=args.prec)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print("tdvp step", st, e)
    mpo.close()
    ctx.close()


if __name__ == "__main__":
    main()
