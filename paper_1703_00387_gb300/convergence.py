"""The paper's convergence loop around the sweeps (Sec. 3.4, convergence
parameters): inner sweeps with the variance checked after each, and after
every block of inner sweeps (one outer sweep) the local tolerance lowered by
Eq. linearExtrap, eps_local' = eps_local * eps_V / V. Host orchestration of
library calls (osmps_sweep, osmps_variance); all arithmetic is in the library.

Readings (the paper states the target as "variance tolerance 1e-12,
effectively L x 1e-12 for the whole system"): the state is converged when its
whole-chain variance V <= L eps_V; the initial local tolerance is
eps_V / (4 L) (the paper's default); the update uses Eq. linearExtrap as
printed, with V the whole-chain variance.
"""
from . import binding as B


def ground_state(ctx, mps, mpo, chi_max, eps_var=1e-12, n_inner=2, n_outer=4,
                 precision="fp64", lanczos_tol=1e-12, lanczos_max_iter=100, refine_sweeps=0):
    """Returns dict(energy, variance, converged, sweeps, history, eps_local)."""
    L = mps.L
    eps_local = eps_var / (4 * L)
    history = []
    E = V = None
    for outer in range(n_outer):
        for inner in range(n_inner):
            p = B.sweep_params(chi_max, 1, precision, eps_local=eps_local, lanczos_tol=lanczos_tol,
                               lanczos_max_iter=lanczos_max_iter, refine_sweeps=refine_sweeps)
            st = B.osmps_sweep(ctx, mps, mpo, p, record_steps=False)
            E, V = B.osmps_variance(ctx, mps, mpo)
            history.append(dict(outer=outer, inner=inner, energy=E, variance=V, eps_local=eps_local,
                                max_chi=st["max_chi"], max_discarded=st["max_discarded"]))
            if V <= L * eps_var:
                return dict(energy=E, variance=V, converged=True, sweeps=len(history),
                            history=history, eps_local=eps_local)
        if V > 0:
            eps_local = eps_local * eps_var / V  # Eq. linearExtrap
    return dict(energy=E, variance=V, converged=False, sweeps=len(history), history=history,
                eps_local=eps_local)
