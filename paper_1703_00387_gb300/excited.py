"""Excited-state search (Sec. 4.1, eMPS): the two-site variational sweeps with
the Lagrange multipliers of Eq. emps_lagrange, i.e. every local Lanczos
search restricted to the orthogonal complement of the lower eigenstates'
two-site blocks in the current basis.

Host orchestration of library calls: theta formation, the projected Lanczos
(osmps_lanczos_ground_projected), the split, the environment updates of H
and of the overlaps with every lower state. The state starts from the
library's canonical form (osmps_mps_canonicalize); all arithmetic is in the
library.
"""
import numpy as np
import torch

from . import binding as B


def _dev(x, device):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=device)


def excited_state(ctx, W, lower, init, chi_max, n_sweeps=4, precision="fp64", lanczos_tol=1e-12,
                  lanczos_max_iter=100, eps_local=-1.0):
    """W: MPO site tensors (host arrays); lower: list of lower eigenstates, each a
    list of site tensors (host arrays); init: starting MPS tensors (host).
    Returns dict(energy, tensors (host), overlaps (with each lower state),
    step_energies)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    L = len(W)
    if eps_local < 0:
        eps_local = 1e-12 / (4 * L)
    h = B.MPS(ctx, init, chi_cap=chi_max)
    hm = B.MPO(ctx, W)
    B.osmps_mps_canonicalize(ctx, h, hm, 0)  # right-canonical from site 1, centre at 0
    A = [_dev(t, dev) for t in h.tensors()]
    h.close()
    Wd = [_dev(w, dev) for w in W]
    Bs = [[_dev(t, dev) for t in st] for st in lower]
    # environments: Lenv[k] covers sites < k, Renv[k] sites >= k
    Lenv = [None] * (L + 1)
    Renv = [None] * (L + 1)
    Lenv[0] = torch.ones((1, 1, 1), dtype=torch.float64, device=dev)
    Renv[L] = torch.ones((1, 1, 1), dtype=torch.float64, device=dev)
    OL = [[None] * (L + 1) for _ in Bs]
    OR = [[None] * (L + 1) for _ in Bs]
    for j in range(len(Bs)):
        OL[j][0] = torch.ones((1, 1), dtype=torch.float64, device=dev)
        OR[j][L] = torch.ones((1, 1), dtype=torch.float64, device=dev)

    def grow_right(k):  # Renv[k] and OR[.][k] from site k
        a = A[k]
        Renv[k] = torch.empty((a.shape[0], W[k].shape[0], a.shape[0]), dtype=torch.float64, device=dev)
        B.osmps_env_update(ctx, 1, Renv[k + 1], a, Wd[k], Renv[k], precision="fp64")
        for j, st in enumerate(Bs):
            OR[j][k] = torch.empty((a.shape[0], st[k].shape[0]), dtype=torch.float64, device=dev)
            B.osmps_overlap_env_update(ctx, 1, OR[j][k + 1], a, st[k], OR[j][k])

    def grow_left(k):  # Lenv[k + 1] and OL[.][k + 1] from site k
        a = A[k]
        Lenv[k + 1] = torch.empty((a.shape[2], W[k].shape[3], a.shape[2]), dtype=torch.float64, device=dev)
        B.osmps_env_update(ctx, 0, Lenv[k], a, Wd[k], Lenv[k + 1], precision="fp64")
        for j, st in enumerate(Bs):
            OL[j][k + 1] = torch.empty((a.shape[2], st[k].shape[2]), dtype=torch.float64, device=dev)
            B.osmps_overlap_env_update(ctx, 0, OL[j][k], a, st[k], OL[j][k + 1])

    for k in range(L - 1, 1, -1):
        grow_right(k)
    energies = []
    schedule = [(i, 1) for i in range(L - 1)] + [(i, 0) for i in range(L - 2, -1, -1)]
    for _ in range(n_sweeps):
        for i, move_right in schedule:
            a1, a2 = A[i], A[i + 1]
            chi_l, d1, chi_m = a1.shape
            _, d2, chi_r = a2.shape
            theta = torch.empty((chi_l, d1, d2, chi_r), dtype=torch.float64, device=dev)
            B.osmps_theta_form(ctx, a1, a2, theta)
            P = None
            if Bs:
                P = torch.empty((len(Bs), chi_l * d1 * d2 * chi_r), dtype=torch.float64, device=dev)
                for j, st in enumerate(Bs):
                    B.osmps_projected_state(ctx, OL[j][i], st[i], st[i + 1], OR[j][i + 2],
                                            P[j].view(chi_l, d1, d2, chi_r))
            e, _, _, _ = B.osmps_lanczos_ground_projected(ctx, Lenv[i], Wd[i], Wd[i + 1], Renv[i + 2],
                                                          theta, P, max_iter=lanczos_max_iter,
                                                          tol=lanczos_tol, precision=precision)
            energies.append(e)
            cap = min(chi_l * d1, d2 * chi_r)
            o1 = torch.empty(chi_l * d1 * cap, dtype=torch.float64, device=dev)
            o2 = torch.empty(cap * d2 * chi_r, dtype=torch.float64, device=dev)
            chn, _, _, _ = B.osmps_split(ctx, theta, o1, o2, move_right, chi_max, eps_local)
            A[i] = o1[: chi_l * d1 * chn].view(chi_l, d1, chn).clone()
            A[i + 1] = o2[: chn * d2 * chi_r].view(chn, d2, chi_r).clone()
            if move_right:
                grow_left(i)
            else:
                grow_right(i + 1)
    torch.cuda.synchronize()
    tensors = [a.cpu().numpy() for a in A]
    # energy of the final state and its overlaps with the lower states
    h = B.MPS(ctx, tensors, chi_cap=chi_max)
    E = B.osmps_energy(ctx, h, hm)
    h.close()
    hm.close()
    overlaps = []
    for st in Bs:
        o = torch.ones((1, 1), dtype=torch.float64, device=dev)
        for k in range(L):
            nxt = torch.empty((A[k].shape[2], st[k].shape[2]), dtype=torch.float64, device=dev)
            B.osmps_overlap_env_update(ctx, 0, o, A[k], st[k], nxt)
            o = nxt
        overlaps.append(float(o.cpu().numpy().ravel()[0]))
    return dict(energy=E, tensors=tensors, overlaps=overlaps, step_energies=energies)
