"""torch.autograd.Function wrappers around the library's gradient calls.

* ``heff_apply(theta, W1, W2, L, R, ctx, precision)``: y = H_eff theta
  (Sec. 3.4, Fig. LanczosMPS) with gradients for theta, W1 and W2 from
  ``osmps_heff_backward``. L and R are constants here (an error is raised if
  they require a gradient).
* ``CouplingEnergy``: E(p) = <psi|H(p)|psi> / <psi|psi> for a fixed MPS and
  an MPO that is affine in the couplings p (Eq. mpo), with dE/dp from
  ``osmps_energy_grad`` (dE/dW for every site) and ``osmps_coupling_grad``
  (the chain rule through the coupling basis dW/dp). At a ground state
  these are the Hellmann-Feynman derivatives of the ground energy.

All arithmetic runs in the library; this module only allocates outputs and
routes cotangents.
"""
import numpy as np
import torch

from . import binding


class _HeffApply(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta, W1, W2, L, R, ctx, precision):
        theta, W1, W2 = theta.contiguous(), W1.contiguous(), W2.contiguous()
        y = torch.empty_like(theta)
        binding.osmps_heff_apply(ctx, L, W1, W2, R, theta, y, precision=precision)
        fctx.save_for_backward(theta, W1, W2, L, R)
        fctx.octx, fctx.precision = ctx, precision
        return y

    @staticmethod
    def backward(fctx, gy):
        theta, W1, W2, L, R = fctx.saved_tensors
        need = fctx.needs_input_grad
        gt = torch.empty_like(theta) if need[0] else None
        g1 = torch.empty_like(W1) if need[1] else None
        g2 = torch.empty_like(W2) if need[2] else None
        if gt is not None or g1 is not None or g2 is not None:
            binding.osmps_heff_backward(fctx.octx, L, W1, W2, R, theta, gy.contiguous(), gt, g1,
                                        g2, precision=fctx.precision)
        return gt, g1, g2, None, None, None, None


def heff_apply(theta, W1, W2, L, R, ctx, precision="fp64"):
    """Differentiable H_eff theta (float64 CUDA tensors in the library's layouts)."""
    if L.requires_grad or R.requires_grad:
        raise NotImplementedError("heff_apply: gradients with respect to L or R are not provided")
    return _HeffApply.apply(theta, W1, W2, L, R, ctx, precision)


class _CouplingEnergyFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, params, model):
        p = params.detach().to("cpu", torch.float64).numpy().copy()
        model._load(p)
        E = binding.osmps_energy(model.ctx, model.mps, model.mpo)
        fctx.model, fctx.p, fctx.dtype = model, p, params.dtype
        return torch.tensor(E, dtype=torch.float64, device=params.device)

    @staticmethod
    def backward(fctx, gE):
        model = fctx.model
        model._load(fctx.p)
        g_par = model.coupling_grad()
        return (g_par * gE).to(fctx.dtype), None


class CouplingEnergy:
    """E(p) for a fixed MPS and an affine MPO W(p) = W_0 + sum_j p_j B_j.

    ``build(p)`` returns the site tensors for the coupling vector p (numpy);
    ``basis`` = (row_ptr, col, val), the B_j in compressed sparse rows over
    the concatenated site tensors. ``checkpoint_every`` > 1 keeps only every
    such right environment during the gradient pass and rebuilds the rest."""

    def __init__(self, ctx, mps, build, basis, checkpoint_every=0, precision="fp64emu"):
        self.ctx, self.mps, self.build = ctx, mps, build
        self.checkpoint_every, self.precision = int(checkpoint_every), precision
        dev = torch.device("cuda", torch.cuda.current_device())
        row_ptr, col, val = basis
        self.row_ptr = torch.as_tensor(np.asarray(row_ptr, dtype=np.int64), device=dev)
        self.col = torch.as_tensor(np.asarray(col, dtype=np.int64), device=dev)
        self.val = torch.as_tensor(np.asarray(val, dtype=np.float64), device=dev)
        self.n_par = self.row_ptr.numel() - 1
        self.mpo = None
        self._p = None
        self.energy = None
        self.norm = None

    def _load(self, p):
        if self._p is not None and np.array_equal(self._p, p):
            return
        W = self.build(p)
        if self.mpo is None:
            self.mpo = binding.MPO(self.ctx, W)
        else:
            self.mpo.set(W)
        self._p = p.copy()

    def weight_grad(self):
        """dE/dW for the loaded couplings (flat, sites concatenated)."""
        gW = torch.empty(self.mpo.n_params, dtype=torch.float64, device=self.val.device)
        self.energy, self.norm = binding.osmps_energy_grad(
            self.ctx, self.mps, self.mpo, gW, checkpoint_every=self.checkpoint_every,
            precision=self.precision)
        return gW

    def coupling_grad(self):
        """dE/dp for the loaded couplings."""
        gW = self.weight_grad()
        g = torch.empty(self.n_par, dtype=torch.float64, device=gW.device)
        return binding.osmps_coupling_grad(self.ctx, self.row_ptr, self.col, self.val, gW, g)

    def __call__(self, params):
        if params.numel() != self.n_par:
            raise ValueError(f"CouplingEnergy: {params.numel()} couplings, basis has {self.n_par}")
        return _CouplingEnergyFn.apply(params, self)


def xxz_energy(ctx, mps, L, delta=1.0, checkpoint_every=0, precision="fp64emu"):
    """CouplingEnergy for the XXZ chain with couplings (J_0..J_{L-2}, h_0..h_{L-1})."""
    from . import hamiltonians
    _, row_ptr, col, val = hamiltonians.xxz_coupling_basis(L, delta)

    def build(p):
        return hamiltonians.xxz(L, p[:L - 1], delta, p[L - 1:])

    return CouplingEnergy(ctx, mps, build, (row_ptr, col, val), checkpoint_every, precision)
