"""GPU gradients against the FP64 oracle (oracle.grad), finite differences
and the free-fermion Hellmann-Feynman derivatives.

Bars: g_theta is H_eff^T gy computed in the requested precision, so it takes
the forward product's bars (1e-12 for float64, 1e-5 for bf16x3 and
tf32x3). The MPO-tensor gradients are
float64-accurate in every precision: 1e-12 norm-wise. Every quantity is
linear in the varied tensor, so a central difference with step 1e-6 is exact
up to rounding: its error is about eps * |f| / 1e-6 = 2e-10 |f|."""
import numpy as np
import pytest

from oracle import dmrg as od
from oracle import exact, grad as og, mpo as ompo
from paper_1703_00387_gb300 import binding as B
from paper_1703_00387_gb300 import hamiltonians, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_THETA = {"fp64": 1e-12, "bf16x3": 1e-5, "tf32x3": 1e-5, "fp64emu": 1e-12}
TOL_W = 1e-12


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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


SHAPES = [
    (5, 2, 2, 7, 3, 3, 3),        # single tile
    (130, 2, 2, 70, 5, 5, 5),     # ragged tiles in every GEMM dimension
    (64, 2, 2, 64, 1, 5, 5),      # left boundary (wl = 1)
    (200, 2, 2, 256, 5, 5, 1),    # right boundary (wr = 1)
    (40, 3, 3, 33, 14, 14, 14),   # AKLT-sized MPO (w = 14, d = 3)
    (48, 5, 5, 40, 4, 4, 4),      # Bose-Hubbard local dimension d = 5
]


def _vjp_gpu(ctx, ops, gy, prec, want=(True, True, True)):
    Lh, W1, W2, Rh, th = ops
    t = [dev(x) for x in (Lh, W1, W2, Rh, th)]
    g = dev(gy)
    gt = torch.empty_like(t[4]) if want[0] else None
    g1 = torch.empty_like(t[1]) if want[1] else None
    g2 = torch.empty_like(t[2]) if want[2] else None
    B.osmps_heff_backward(ctx, t[0], t[1], t[2], t[3], t[4], g, gt, g1, g2, precision=prec)
    torch.cuda.synchronize()
    return [None if x is None else x.cpu().numpy() for x in (gt, g1, g2)]


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32x3", "fp64emu"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_heff_backward_parity(ctx, prec, shape):
    ops = inputs.random_heff_operands(*shape, seed=sum(shape) + 1)
    gy = np.random.default_rng(sum(shape)).standard_normal(ops[4].shape)
    ref = og.heff_vjp(*ops, gy)
    gt, g1, g2 = _vjp_gpu(ctx, ops, gy, prec)
    assert rel(gt, ref[0]) <= TOL_THETA[prec]
    assert rel(g1, ref[1]) <= TOL_W
    assert rel(g2, ref[2]) <= TOL_W


@pytest.mark.parametrize("prec", ["fp64emu", "bf16x3", "fp64"])
def test_heff_backward_differentiation_size(ctx, prec):
    """chi_l = chi_r = 256, d = 2, w = 5 (the XXZ differentiation workload)."""
    ops = inputs.random_heff_operands(256, 2, 2, 256, 5, 5, 5, seed=256)
    gy = np.random.default_rng(257).standard_normal(ops[4].shape)
    ref = og.heff_vjp(*ops, gy)
    gt, g1, g2 = _vjp_gpu(ctx, ops, gy, prec)
    assert rel(gt, ref[0]) <= (1e-5 if prec == "bf16x3" else 1e-12)
    assert rel(g1, ref[1]) <= TOL_W
    assert rel(g2, ref[2]) <= TOL_W


def test_heff_backward_partial_outputs(ctx):
    ops = inputs.random_heff_operands(33, 2, 2, 31, 5, 5, 5, seed=4)
    gy = np.random.default_rng(5).standard_normal(ops[4].shape)
    ref = og.heff_vjp(*ops, gy)
    gt, g1, g2 = _vjp_gpu(ctx, ops, gy, "fp64", want=(True, False, False))
    assert g1 is None and g2 is None and rel(gt, ref[0]) <= 1e-12
    _, g1, _ = _vjp_gpu(ctx, ops, gy, "fp64", want=(False, True, False))
    assert rel(g1, ref[1]) <= TOL_W
    _, _, g2 = _vjp_gpu(ctx, ops, gy, "fp64emu", want=(False, False, True))
    assert rel(g2, ref[2]) <= TOL_W


def test_heff_backward_transpose_identity(ctx):
    """<gy, H theta> = <H^T gy, theta> on the device path alone."""
    ops = inputs.random_heff_operands(70, 2, 2, 90, 5, 5, 5, seed=12)
    gy = np.random.default_rng(13).standard_normal(ops[4].shape)
    t = [dev(x) for x in ops]
    y = torch.empty_like(t[4])
    B.osmps_heff_apply(ctx, *t, y, precision="fp64")
    gt, _, _ = _vjp_gpu(ctx, ops, gy, "fp64", want=(True, False, False))
    lhs = float(np.vdot(gy, y.cpu().numpy()))
    rhs = float(np.vdot(gt, ops[4]))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(gy) * np.linalg.norm(y.cpu().numpy())


def test_heff_backward_errors(ctx):
    ops = inputs.random_heff_operands(8, 2, 2, 8, 5, 5, 5, seed=1)
    t = [dev(x) for x in ops]
    g = torch.empty_like(t[4])
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_heff_backward(ctx, t[0], t[1], t[2], t[3], t[4], g, g, None, None)
    assert e.value.status == B.EINVAL
    with pytest.raises(B.OsmpsError) as e:  # weight gradients need theta
        B.osmps_heff_backward(ctx, t[0], t[1], t[2], t[3], None, g, None, torch.empty_like(t[1]), None)
    assert e.value.status == B.EINVAL
    big = inputs.random_heff_operands(6, 5, 5, 6, 14, 14, 14, seed=2)   # w * d = 70 > 64
    tb = [dev(x) for x in big]
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_heff_backward(ctx, *tb, torch.empty_like(tb[4]), None, torch.empty_like(tb[1]), None)
    assert e.value.status == B.EUNSUPPORTED


def test_autograd_heff_finite_differences(ctx):
    """torch.autograd through heff_apply against central differences (step
    1e-6) of the float64 GPU forward and against the oracle's VJP."""
    from paper_1703_00387_gb300.autograd import heff_apply
    ops = inputs.random_heff_operands(40, 2, 2, 36, 5, 5, 5, seed=21)
    gy = np.random.default_rng(22).standard_normal(ops[4].shape)
    Lt, W1, W2, Rt, th = [dev(x) for x in ops]
    gyt = dev(gy)
    th.requires_grad_(True)
    W1.requires_grad_(True)
    W2.requires_grad_(True)
    f = (heff_apply(th, W1, W2, Lt, Rt, ctx, "fp64") * gyt).sum()
    f.backward()
    ref = og.heff_vjp(*ops, gy)
    assert rel(th.grad.cpu().numpy(), ref[0]) <= 1e-12
    assert rel(W1.grad.cpu().numpy(), ref[1]) <= 1e-12
    assert rel(W2.grad.cpu().numpy(), ref[2]) <= 1e-12
    rng = np.random.default_rng(23)
    h = 1e-6
    with torch.no_grad():
        for x in (th, W1, W2):
            v = dev(rng.standard_normal(tuple(x.shape)))
            x.add_(h * v)
            fp = (heff_apply(th, W1, W2, Lt, Rt, ctx, "fp64") * gyt).sum().item()
            x.sub_(2 * h * v)
            fm = (heff_apply(th, W1, W2, Lt, Rt, ctx, "fp64") * gyt).sum().item()
            x.add_(h * v)
            fd = (fp - fm) / (2 * h)
            an = float((x.grad * v).sum())
            assert abs(fd - an) <= 1e-8 * max(1.0, abs(f.item()))


def _mps_handle(ctx, tensors):
    return B.MPS(ctx, tensors, chi_cap=max(t.shape[2] for t in tensors))


@pytest.mark.parametrize("every", [0, 3, 8])
@pytest.mark.parametrize("prec", ["fp64", "fp64emu"])
def test_energy_grad_parity(ctx, prec, every):
    L = 8
    J, h = inputs.random_couplings(L, seed=7)
    W = ompo.xxz_mpo(L, J, 0.9, h)
    tensors = inputs.random_mps(L, 2, 8, seed=8)   # neither canonical nor normalised
    E_ref, gW_ref = og.energy_grad_W(W, tensors)
    mps = _mps_handle(ctx, tensors)
    mpo = B.MPO(ctx, hamiltonians.xxz(L, J, 0.9, h))
    gW = torch.empty(mpo.n_params, dtype=torch.float64, device="cuda:0")
    E, nrm = B.osmps_energy_grad(ctx, mps, mpo, gW, checkpoint_every=every, precision=prec)
    assert abs(E - E_ref) <= 1e-12 * abs(E_ref)
    assert abs(nrm - od.mps_norm2(tensors)) <= 1e-12 * nrm
    ref = np.concatenate([g.ravel() for g in gW_ref])
    assert rel(gW.cpu().numpy(), ref) <= 1e-12
    mps.close()
    mpo.close()


def test_energy_grad_checkpointing_is_exact(ctx):
    """Rebuilding right environments from checkpoints repeats the same
    arithmetic: the gradients agree bit for bit."""
    L = 20
    J, h = inputs.random_couplings(L, seed=9)
    mps = _mps_handle(ctx, inputs.random_mps(L, 2, 32, seed=10))
    mpo = B.MPO(ctx, hamiltonians.xxz(L, J, 1.0, h))
    out = []
    for every in (0, 4, 7, 20):
        gW = torch.empty(mpo.n_params, dtype=torch.float64, device="cuda:0")
        E, _ = B.osmps_energy_grad(ctx, mps, mpo, gW, checkpoint_every=every)
        out.append((E, gW.cpu().numpy()))
    for E, g in out[1:]:
        assert E == out[0][0]
        assert np.array_equal(g, out[0][1])
    mps.close()
    mpo.close()


def test_energy_grad_errors(ctx):
    L = 6
    mps = _mps_handle(ctx, inputs.random_mps(L, 2, 4, seed=1))
    mpo = B.MPO(ctx, hamiltonians.xxz(L))
    gW = torch.empty(mpo.n_params + 1, dtype=torch.float64, device="cuda:0")
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_energy_grad(ctx, mps, mpo, gW)
    assert e.value.status == B.ESHAPE
    gW = torch.empty(mpo.n_params, dtype=torch.float64, device="cuda:0")
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_energy_grad(ctx, mps, mpo, gW, precision="bf16x3")
    assert e.value.status == B.EINVAL
    mps.close()
    mpo.close()


def test_coupling_grad_bad_index(ctx):
    gW = torch.zeros(10, dtype=torch.float64, device="cuda:0")
    rp = torch.tensor([0, 1, 2], dtype=torch.int64, device="cuda:0")
    col = torch.tensor([3, 10], dtype=torch.int64, device="cuda:0")   # 10 is out of range
    val = torch.ones(2, dtype=torch.float64, device="cuda:0")
    g = torch.empty(2, dtype=torch.float64, device="cuda:0")
    with pytest.raises(B.OsmpsError) as e:
        B.osmps_coupling_grad(ctx, rp, col, val, gW, g)
    assert e.value.status == B.EINVAL


def test_coupling_energy_autograd_matches_oracle_and_fd(ctx):
    from paper_1703_00387_gb300.autograd import xxz_energy
    L = 10
    J, h = inputs.random_couplings(L, seed=11)
    tensors = inputs.random_mps(L, 2, 16, seed=12)
    mps = _mps_handle(ctx, tensors)
    model = xxz_energy(ctx, mps, L, delta=0.8)
    p = torch.tensor(np.concatenate([J, h]), dtype=torch.float64, device="cuda:0", requires_grad=True)
    E = model(p)
    E.backward()
    W = ompo.xxz_mpo(L, J, 0.8, h)
    E_ref, gW = og.energy_grad_W(W, tensors)
    dJ, dh = og.xxz_coupling_grads(gW, L, J, 0.8, h)
    assert abs(E.item() - E_ref) <= 1e-12 * abs(E_ref)
    np.testing.assert_allclose(p.grad.cpu().numpy(), np.concatenate([dJ, dh]), rtol=0, atol=1e-12)
    # central differences of the oracle energy, step 1e-6 (E is linear in every coupling)
    for j in (0, L - 2, L - 1, 2 * L - 2):
        q = np.concatenate([J, h])
        q[j] += 1e-6
        Ep = od.mps_energy(ompo.xxz_mpo(L, q[:L - 1], 0.8, q[L - 1:]), tensors)
        q[j] -= 2e-6
        Em = od.mps_energy(ompo.xxz_mpo(L, q[:L - 1], 0.8, q[L - 1:]), tensors)
        assert abs((Ep - Em) / 2e-6 - float(p.grad[j])) <= 1e-8
    mps.close()


def test_hellmann_feynman_xx_ground_state(ctx):
    """Site-dependent XX chain: the GPU ground state (exact bond dimension)
    and the GPU coupling gradient reproduce the free-fermion derivatives."""
    from paper_1703_00387_gb300.autograd import xxz_energy
    L = 10
    J, h = inputs.random_couplings(L, seed=0)
    mps = B.MPS(ctx, inputs.random_mps(L, 2, 32, seed=1), chi_cap=32)
    mpo = B.MPO(ctx, hamiltonians.xxz(L, J, 0.0, h))
    B.osmps_sweep(ctx, mps, mpo, B.sweep_params(32, 3, "fp64", lanczos_tol=1e-13))
    mpo.close()
    model = xxz_energy(ctx, mps, L, delta=0.0)
    p = torch.tensor(np.concatenate([J, h]), dtype=torch.float64, device="cuda:0", requires_grad=True)
    model(p).backward()
    dJ, dh = exact.xx_free_fermion_gradients(J, h)
    np.testing.assert_allclose(p.grad.cpu().numpy(), np.concatenate([dJ, dh]), rtol=0, atol=1e-8)
    mps.close()


def test_differentiation_workload_full_size(ctx):
    """XXZ L = 64, chi = 256, J_i in [0.8, 1.2], h_i in [-0.5, 0.5]: every
    dE/dW_k and dE/dp against the oracle, with checkpointed environments."""
    from paper_1703_00387_gb300.autograd import xxz_energy
    L = 64
    J, h = inputs.random_couplings(L, seed=5)
    # the couplings enter as float32: the oracle takes the same rounded values
    J = J.astype(np.float32).astype(np.float64)
    h = h.astype(np.float32).astype(np.float64)
    tensors = inputs.random_mps(L, 2, 256, seed=5)
    E_ref, gW_ref = og.energy_grad_W(ompo.xxz_mpo(L, J, 1.0, h), tensors)
    dJ, dh = og.xxz_coupling_grads(gW_ref, L, J, 1.0, h)
    mps = _mps_handle(ctx, tensors)
    model = xxz_energy(ctx, mps, L, delta=1.0, checkpoint_every=8)
    p = torch.tensor(np.concatenate([J, h]), dtype=torch.float32, device="cuda:0", requires_grad=True)
    E = model(p)
    E.backward()
    assert p.grad.dtype == torch.float32
    assert abs(model.energy - E_ref) <= 1e-12 * max(1.0, abs(E_ref))
    gW = model.weight_grad().cpu().numpy()
    assert rel(gW, np.concatenate([g.ravel() for g in gW_ref])) <= 1e-12
    g64 = model.coupling_grad().cpu().numpy()
    np.testing.assert_allclose(g64, np.concatenate([dJ, dh]), rtol=0, atol=1e-12)
    mps.close()
