"""Seeded synthetic inputs shared by the tests and the benchmark.

This module draws random numbers and fixes shapes; it holds none of the
method's arithmetic (no canonicalisation, no contraction, no MPO algebra).
Both the GPU library and the CPU oracle receive the arrays it returns.

Recipes (all float64, ``numpy.random.default_rng(seed)``):

* ``random_mps``: site tensors A[chi_k, d, chi_{k+1}] with entries N(0, 1),
  drawn site 1 ... L, each in C order; bond dimensions
  chi_k = min(d^k, d^(L-k), chi_init).
* ``random_heff_operands``: L, W1, W2, R, theta with N(0, 1) entries, for
  matvec parity tests at arbitrary (ragged) shapes.
* ``random_symmetric_env``: E[a2, w, a] with N(0, 1) entries, symmetrised in
  (a2, a).
* ``random_couplings``: site-dependent XXZ couplings J_i ~ U[0.8, 1.2] for the
  L-1 bonds, then fields h_i ~ U[-0.5, 0.5] for the L sites.
* ``chain_batch``: a batch of independent chain specifications (model, L,
  chi_max, g or delta) drawn as in the batched-chains workload.
"""
import numpy as np


def bond_dims(L, d, chi_init):
    return [int(min(d ** k, d ** (L - k), chi_init)) for k in range(L + 1)]


def random_mps(L, d, chi_init, seed=0):
    rng = np.random.default_rng(seed)
    chi = bond_dims(L, d, chi_init)
    return [rng.standard_normal((chi[k], d, chi[k + 1])) for k in range(L)]


def random_heff_operands(chi_l, d1, d2, chi_r, wl, wm, wr, seed=0):
    rng = np.random.default_rng(seed)
    Lenv = rng.standard_normal((chi_l, wl, chi_l))
    W1 = rng.standard_normal((wl, d1, d1, wm))
    W2 = rng.standard_normal((wm, d2, d2, wr))
    Renv = rng.standard_normal((chi_r, wr, chi_r))
    theta = rng.standard_normal((chi_l, d1, d2, chi_r))
    return Lenv, W1, W2, Renv, theta


def random_env_operands(chi_l, d, chi_r, w_in, w_out, side, seed=0):
    """(env_in, A, W) for an environment update. side 0 grows L (env_in is
    [chi_l, w_in, chi_l], output [chi_r, w_out, chi_r]); side 1 grows R
    (env_in is [chi_r, w_in, chi_r], output [chi_l, w_out, chi_l])."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((chi_l, d, chi_r))
    if side == 0:
        env = rng.standard_normal((chi_l, w_in, chi_l))
        W = rng.standard_normal((w_in, d, d, w_out))
    else:
        env = rng.standard_normal((chi_r, w_in, chi_r))
        W = rng.standard_normal((w_out, d, d, w_in))
    return env, A, W


def random_symmetric_env(chi, w, seed=0):
    """Environment-shaped tensor E[a2, w, a] with N(0, 1) entries, symmetrised
    in (a2, a) for every channel so that an effective Hamiltonian built from it
    is symmetric (timing inputs for a single two-site step)."""
    rng = np.random.default_rng(seed)
    E = rng.standard_normal((chi, w, chi))
    return 0.5 * (E + E.transpose(2, 1, 0))


def random_couplings(L, seed=0):
    rng = np.random.default_rng(seed)
    J = rng.uniform(0.8, 1.2, size=L - 1)
    h = rng.uniform(-0.5, 0.5, size=L)
    return J, h


def chain_batch(n_chains=64, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_chains):
        model = "tfi" if rng.random() < 0.5 else "xxz"
        L = int(rng.integers(16, 129))
        chi_max = int(rng.choice([32, 64, 128, 256]))
        param = float(rng.uniform(0.5, 1.5))
        out.append(dict(model=model, L=L, chi_max=chi_max, param=param))
    return out


def u1_sector_profile(n_bar, total=512, width=8.0):
    """Sector charges and sizes of one bond for the U(1) Bose-Hubbard workload:
    sizes proportional to exp(-(n - n_bar)^2 / width), n integer, keeping the
    n whose share rounds to at least half a state, each at least 1, the
    largest adjusted so that the sizes sum to `total`."""
    n = np.arange(int(np.floor(n_bar - 6 * np.sqrt(width))), int(np.ceil(n_bar + 6 * np.sqrt(width))) + 1)
    p = np.exp(-(n - n_bar) ** 2 / width)
    p = p / p.sum()
    keep = total * p >= 0.5
    n, p = n[keep], p[keep] / p[keep].sum()
    chi = np.maximum(1, np.rint(total * p).astype(np.int64))
    chi[np.argmax(chi)] += total - chi.sum()
    return n.astype(np.int64), chi


def random_dense(shape, seed=0):
    return np.random.default_rng(seed).standard_normal(shape)
