"""Small driver for profiler runs: repeated H_eff.theta products (and
optionally one full two-site step) at a given bond dimension, with seeded
inputs and under 2 GB of device memory.

    python -m paper_1703_00387_gb300.profile_heff --chi 1024 --prec bf16x3 --reps 3
    python -m paper_1703_00387_gb300.profile_heff --chi 1024 --step
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
    args = ap.parse_args()

    import torch
    from paper_1703_00387_gb300 import binding as B
    from paper_1703_00387_gb300 import hamiltonians, inputs

    dev = torch.device("cuda:0")
    ctx = B.Context(0)
    chi, d, w = args.chi, args.d, args.w
    W = hamiltonians.xxz(8, 1.0, 1.0, 0.0)[3] if (d, w) == (2, 5) else \
        np.random.default_rng(3).standard_normal((w, d, d, w))
    Lh = inputs.random_symmetric_env(chi, w, seed=1)
    Rh = inputs.random_symmetric_env(chi, w, seed=2)
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


if __name__ == "__main__":
    main()
