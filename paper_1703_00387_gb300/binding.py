"""Thin ctypes binding of libosmps (C ABI in include/osmps.h).

Functions keep the C names. Device tensors are torch float64 CUDA tensors
(contiguous); dimensions are read from their shapes, and every call is
argument marshalling only: the arithmetic runs in the library's kernels.
There is no fallback: if the library is missing or a call fails, an
``OsmpsError`` is raised.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libosmps.so")

PRECISION = {"fp64": 0, "bf16x3": 1, "tf32x3": 2, "fp64emu": 3}
STATUS = {0: "OSMPS_OK", 1: "OSMPS_EINVAL", 2: "OSMPS_ESHAPE", 3: "OSMPS_ENOMEM", 4: "OSMPS_ECUDA",
          5: "OSMPS_ENOCONV", 6: "OSMPS_ETIMEOUT", 7: "OSMPS_ENAN", 8: "OSMPS_EUNSUPPORTED"}
EINVAL, ESHAPE, ENOMEM, ECUDA, ENOCONV, ETIMEOUT, ENAN, EUNSUPPORTED = range(1, 9)

_c = ctypes
_i64 = _c.c_int64
_vp = _c.c_void_p
_dp = _c.POINTER(_c.c_double)


class OsmpsError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class SweepParams(_c.Structure):
    _fields_ = [("chi_max", _i64), ("eps_local", _c.c_double), ("lanczos_tol", _c.c_double),
                ("lanczos_max_iter", _c.c_int), ("n_sweeps", _c.c_int), ("precision", _c.c_int),
                ("refine_sweeps", _c.c_int)]


class SweepStats(_c.Structure):
    _fields_ = [("energy", _c.c_double), ("last_step_energy", _c.c_double),
                ("max_discarded", _c.c_double), ("entropy_center", _c.c_double),
                ("max_chi", _i64), ("steps", _i64), ("lanczos_iters", _i64),
                ("nonconverged", _i64), ("seconds", _c.c_double), ("setup_seconds", _c.c_double),
                ("sweep_seconds", _c.c_double), ("energy_seconds", _c.c_double),
                ("step_energies", _dp), ("step_iters", _c.POINTER(_i64))]


class StepStats(_c.Structure):
    _fields_ = [("energy", _c.c_double), ("resid", _c.c_double), ("discarded", _c.c_double),
                ("entropy", _c.c_double), ("chi_new", _i64), ("iters", _c.c_int),
                ("converged", _c.c_int)]


class TdvpParams(_c.Structure):
    _fields_ = [("dt", _c.c_double), ("n_steps", _c.c_int), ("chi_max", _i64),
                ("eps_local", _c.c_double), ("krylov_tol", _c.c_double),
                ("krylov_max_iter", _c.c_int), ("precision", _c.c_int)]


class TdvpStats(_c.Structure):
    _fields_ = [("energy", _dp), ("norm", _dp), ("max_chi", _i64), ("max_krylov", _c.c_int),
                ("krylov_calls", _i64), ("krylov_vectors", _i64), ("nonconverged", _i64),
                ("max_discarded", _c.c_double), ("seconds", _c.c_double)]


# osmps_gemm_term / osmps_gemm_out as NumPy record types (same field order and
# 8-byte fields, so an array of records is the C array)
GEMM_TERM_DTYPE = np.dtype([("A", np.uint64), ("sam", np.int64), ("sak", np.int64), ("B", np.uint64),
                            ("sbk", np.int64), ("sbn", np.int64), ("K", np.int64), ("alpha", np.float64)])
GEMM_OUT_DTYPE = np.dtype([("C", np.uint64), ("scm", np.int64), ("scn", np.int64), ("M", np.int64),
                           ("N", np.int64), ("beta", np.float64), ("term_begin", np.int64),
                           ("term_count", np.int64)])


class CopyDesc(_c.Structure):
    _fields_ = [("src", _vp), ("dst", _vp), ("rows", _i64), ("cols", _i64), ("srs", _i64),
                ("scs", _i64), ("drs", _i64), ("alpha", _c.c_double)]


class U1Desc(_c.Structure):
    _fields_ = [("n_left", _i64), ("q_left", _c.POINTER(_i64)), ("chi_left", _c.POINTER(_i64)),
                ("n_right", _i64), ("q_right", _c.POINTER(_i64)), ("chi_right", _c.POINTER(_i64)),
                ("d1", _i64), ("d2", _i64), ("wl", _i64), ("wm", _i64), ("wr", _i64),
                ("q_wl", _c.POINTER(_i64)), ("q_wr", _c.POINTER(_i64))]


_LIB = None

_SIGS = {
    "osmps_last_error": (_c.c_char_p, []),
    "osmps_status_string": (_c.c_char_p, [_c.c_int]),
    "osmps_ctx_create": (_c.c_int, [_c.c_int, _c.c_size_t, _c.POINTER(_vp)]),
    "osmps_ctx_destroy": (_c.c_int, [_vp]),
    "osmps_ctx_workspace_bytes": (_c.c_size_t, [_vp]),
    "osmps_ctx_set_eig_solver": (_c.c_int, [_vp, _c.c_int]),
    "osmps_ctx_set_lanczos_mode": (_c.c_int, [_vp, _c.c_int]),
    "osmps_ctx_set_identity_skip": (_c.c_int, [_vp, _c.c_int]),
    "osmps_ctx_set_autotune": (_c.c_int, [_vp, _c.c_int]),
    "osmps_ctx_tuning_count": (_i64, [_vp]),
    "osmps_ctx_tuning_entry": (_c.c_int, [_vp, _i64, _c.POINTER(_i64), _c.POINTER(_c.c_int),
                                          _c.POINTER(_c.c_float)]),
    "osmps_ctx_set_tuning": (_c.c_int, [_vp, _c.POINTER(_i64), _c.c_int]),
    "osmps_profile_enable": (_c.c_int, [_vp, _c.c_int]),
    "osmps_profile_read": (_c.c_int, [_vp, _c.c_int, _c.POINTER(_i64), _dp, _dp, _dp]),
    "osmps_kernel_launches": (_i64, []),
    "osmps_heff_apply": (_c.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp] + [_i64] * 7 + [_c.c_int, _vp]),
    "osmps_heff_apply_noalloc": (_c.c_int, [_vp, _vp, _vp, _vp, _vp, _vp] + [_i64] * 7 + [_vp]),
    "osmps_dgemm_emu": (_c.c_int, [_vp, _vp, _vp, _vp, _i64, _i64, _i64, _vp]),
    "osmps_sytrd": (_c.c_int, [_vp, _vp, _i64, _vp, _vp, _vp, _vp]),
    "osmps_selftest_wait_timeout": (_c.c_int, [_vp, _c.c_int, _c.c_double, _vp]),
    "osmps_selftest_convert": (_c.c_int, [_vp, _vp, _vp, _vp, _vp, _i64, _vp]),
    "osmps_selftest_bf16": (_c.c_int, [_vp, _vp, _vp, _vp, _i64, _vp]),
    "osmps_gemm_grouped": (_c.c_int, [_vp, _vp, _i64, _vp, _i64, _vp]),
    "osmps_copy_list": (_c.c_int, [_vp, _c.POINTER(CopyDesc), _i64, _vp]),
    "osmps_sym_eig_top": (_c.c_int, [_vp, _vp, _i64, _i64, _dp, _vp, _vp]),
    "osmps_vec_norm2": (_c.c_int, [_vp, _vp, _i64, _dp, _vp]),
    "osmps_env_update": (_c.c_int, [_vp, _c.c_int, _vp, _vp, _vp, _vp] + [_i64] * 5 + [_c.c_int, _vp]),
    "osmps_lanczos_ground": (_c.c_int, [_vp, _vp, _vp, _vp, _vp, _vp] + [_i64] * 7 +
                             [_c.c_int, _c.c_double, _c.c_int, _dp, _c.POINTER(_c.c_int), _dp, _vp]),
    "osmps_lanczos_ground_projected": (_c.c_int, [_vp] * 7 + [_c.c_int] + [_i64] * 7 +
                                       [_c.c_int, _c.c_double, _c.c_int, _dp, _c.POINTER(_c.c_int),
                                        _dp, _vp]),
    "osmps_heff_expm": (_c.c_int, [_vp] * 6 + [_i64] * 7 +
                        [_c.c_double, _c.c_int, _c.c_double, _c.c_int, _c.POINTER(_c.c_int), _dp,
                         _vp]),
    "osmps_split_complex": (_c.c_int, [_vp, _vp, _vp, _vp] + [_i64] * 4 +
                            [_c.c_int, _i64, _c.c_double, _c.POINTER(_i64), _dp, _dp, _dp,
                             _c.c_int, _vp]),
    "osmps_tdvp_evolve": (_c.c_int, [_vp, _vp, _c.POINTER(_i64), _c.POINTER(_dp), _vp,
                                     _c.POINTER(_i64), _c.POINTER(_dp), _vp, _vp]),
    "osmps_overlap_env_update": (_c.c_int, [_vp, _c.c_int, _vp, _vp, _vp, _vp] + [_i64] * 5 + [_vp]),
    "osmps_projected_state": (_c.c_int, [_vp] * 6 + [_i64] * 7 + [_vp]),
    "osmps_theta_form": (_c.c_int, [_vp, _vp, _vp, _vp] + [_i64] * 5 + [_vp]),
    "osmps_split": (_c.c_int, [_vp, _vp, _vp, _vp] + [_i64] * 4 +
                    [_c.c_int, _i64, _c.c_double, _c.POINTER(_i64), _dp, _dp, _dp, _c.c_int, _vp]),
    "osmps_mps_create": (_c.c_int, [_vp, _i64, _c.POINTER(_i64), _c.POINTER(_i64), _c.POINTER(_dp),
                                    _i64, _c.POINTER(_vp)]),
    "osmps_mps_destroy": (_c.c_int, [_vp]),
    "osmps_mps_bond_dims": (_c.c_int, [_vp, _c.POINTER(_i64)]),
    "osmps_mps_get_tensor": (_c.c_int, [_vp, _i64, _dp]),
    "osmps_mps_device_tensor": (_vp, [_vp, _i64]),
    "osmps_mpo_create": (_c.c_int, [_vp, _i64, _c.POINTER(_i64), _c.POINTER(_i64), _c.POINTER(_dp),
                                    _c.POINTER(_vp)]),
    "osmps_mpo_destroy": (_c.c_int, [_vp]),
    "osmps_mps_canonicalize": (_c.c_int, [_vp, _vp, _vp, _i64, _c.c_int, _vp]),
    "osmps_sweep_step": (_c.c_int, [_vp, _vp, _vp, _i64, _c.c_int, _c.POINTER(SweepParams),
                                    _c.POINTER(StepStats), _vp]),
    "osmps_sweep": (_c.c_int, [_vp, _vp, _vp, _c.POINTER(SweepParams), _c.POINTER(SweepStats), _vp]),
    "osmps_energy": (_c.c_int, [_vp, _vp, _vp, _dp, _vp]),
    "osmps_variance": (_c.c_int, [_vp, _vp, _vp, _dp, _dp, _vp]),
    "osmps_mpo_set": (_c.c_int, [_vp, _c.POINTER(_dp)]),
    "osmps_heff_backward": (_c.c_int, [_vp] + [_vp] * 9 + [_i64] * 7 + [_c.c_int, _vp]),
    "osmps_energy_grad": (_c.c_int, [_vp, _vp, _vp, _vp, _i64, _i64, _c.c_int, _dp, _dp, _vp]),
    "osmps_coupling_grad": (_c.c_int, [_vp, _i64, _vp, _vp, _vp, _i64, _vp, _i64, _vp, _vp]),
    "osmps_u1_heff_create": (_c.c_int, [_vp, _c.POINTER(U1Desc), _c.POINTER(_vp)]),
    "osmps_u1_heff_destroy": (_c.c_int, [_vp]),
    "osmps_u1_heff_sizes": (_c.c_int, [_vp, _c.POINTER(_i64), _c.POINTER(_i64), _c.POINTER(_i64), _dp]),
    "osmps_u1_heff_stage_sizes": (_c.c_int, [_vp, _c.POINTER(_i64), _c.POINTER(_i64), _c.POINTER(_i64)]),
    "osmps_heff_apply_u1": (_c.c_int, [_vp, _vp] + [_vp] * 6 + [_c.c_int, _vp]),
    "osmps_u1_heff_prepare": (_c.c_int, [_vp, _vp] + [_vp] * 4 + [_c.c_int, _vp]),
    "osmps_u1_heff_apply": (_c.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "osmps_lanczos_ground_u1": (_c.c_int, [_vp, _vp] + [_vp] * 5 + [_c.c_int, _c.c_double, _c.c_int,
                                                                     _dp, _c.POINTER(_c.c_int), _dp, _vp]),
    "osmps_sweep_batch": (_c.c_int, [_c.POINTER(_vp), _c.c_int, _c.POINTER(_vp), _c.POINTER(_vp),
                                     _c.POINTER(SweepParams), _i64, _c.POINTER(SweepStats),
                                     _c.POINTER(_c.c_int)]),
}


def lib():
    """Load libosmps.so (built in-tree by ``build.build()``); raise if absent."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise OsmpsError(4, f"{LIB_PATH} is missing: build it with paper_1703_00387_gb300.build")
        handle = _c.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = handle
    return _LIB


def exported_symbols():
    return list(_SIGS)


def _check(status, allow=()):
    if status != 0 and status not in allow:
        raise OsmpsError(status, lib().osmps_last_error().decode(errors="replace"))
    return status


def _prec(p):
    return PRECISION[p] if isinstance(p, str) else int(p)


def _dev(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return _vp(t.data_ptr())


def _devc(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.complex128:
        raise TypeError(f"{name} must be a complex128 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return _vp(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        return _vp(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _vp(stream)
    return _vp(stream.cuda_stream)


class Context:
    """Owns an osmps_ctx (workspace, cuSOLVER handle, error flags) on one device."""

    def __init__(self, device=0, ws_bytes=0):
        self.ptr = _vp()
        _check(lib().osmps_ctx_create(int(device), int(ws_bytes), _c.byref(self.ptr)))
        self.device = device

    def set_eig_solver(self, solver):
        """'auto', 'cusolver' or 'tridiag' (the split's float64 eigensolver)."""
        code = {"auto": 0, "cusolver": 1, "tridiag": 2}[solver] if isinstance(solver, str) else int(solver)
        _check(lib().osmps_ctx_set_eig_solver(self.ptr, code))

    def set_lanczos_mode(self, mode):
        """'auto', 'host' or 'graph': how Lanczos drives its steps (a host loop
        reading the stopping decision after every step, or one CUDA graph
        whose while-node repeats the recorded step on the device)."""
        code = {"auto": 0, "host": 1, "graph": 2}[mode] if isinstance(mode, str) else int(mode)
        _check(lib().osmps_ctx_set_lanczos_mode(self.ptr, code))

    def set_identity_skip(self, mode):
        """'off', 'solver' (default) or 'always': when the split-precision
        H_eff.theta leaves unit-matrix environment channels out of its GEMMs."""
        code = {"off": 0, "solver": 1, "always": 2}[mode] if isinstance(mode, str) else int(mode)
        _check(lib().osmps_ctx_set_identity_skip(self.ptr, code))

    def set_autotune(self, on):
        """Measure the tcgen05 GEMM tile width per size class on first use (True,
        the default) or always use 256 columns (False)."""
        _check(lib().osmps_ctx_set_autotune(self.ptr, 1 if on else 0))

    def tuning(self):
        """The tile-width table: list of dicts (key, width, us at 256/128/64)."""
        out = []
        for i in range(int(lib().osmps_ctx_tuning_count(self.ptr))):
            key = (_i64 * 6)()
            w = _c.c_int()
            us = (_c.c_float * 3)()
            _check(lib().osmps_ctx_tuning_entry(self.ptr, i, key, _c.byref(w), us))
            out.append({"key": [int(k) for k in key], "width": w.value,
                        "us": {"256": us[0], "128": us[1], "64": us[2]}})
        return out

    def set_tuning(self, key, width):
        """Set the tile width of a size class (key: 6 integers, as in tuning())."""
        k = (_i64 * 6)(*[int(x) for x in key])
        _check(lib().osmps_ctx_set_tuning(self.ptr, k, int(width)))

    def workspace_bytes(self):
        return int(lib().osmps_ctx_workspace_bytes(self.ptr))

    def close(self):
        if self.ptr:
            lib().osmps_ctx_destroy(self.ptr)
            self.ptr = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


KERNEL = {"gemm_tc": 0, "gemm_f64": 1, "gemm_emu": 2, "sytrd_panel": 3, "u1_wstep": 4}


def osmps_profile_enable(ctx, enable=True):
    _check(lib().osmps_profile_enable(ctx.ptr, 1 if enable else 0))


def osmps_profile_read(ctx, kernel):
    """Returns dict(launches, ms, flops, tensor_flops) since the last enable."""
    n = _i64()
    ms, f, tf = _c.c_double(), _c.c_double(), _c.c_double()
    _check(lib().osmps_profile_read(ctx.ptr, KERNEL[kernel] if isinstance(kernel, str) else int(kernel),
                                    _c.byref(n), _c.byref(ms), _c.byref(f), _c.byref(tf)))
    return dict(launches=n.value, ms=ms.value, flops=f.value, tensor_flops=tf.value)


def osmps_kernel_launches():
    return int(lib().osmps_kernel_launches())


def osmps_heff_apply(ctx, L, W1, W2, R, theta, y, precision="bf16x3", stream=None):
    chi_l, d1, d2, chi_r = theta.shape
    wl, wm, wr = W1.shape[0], W1.shape[3], W2.shape[3]
    _check(lib().osmps_heff_apply(ctx.ptr, _dev(L, "L"), _dev(W1, "W1"), _dev(W2, "W2"),
                                  _dev(R, "R"), _dev(theta, "theta"), _dev(y, "y"), chi_l, d1, d2,
                                  chi_r, wl, wm, wr, _prec(precision), _stream(stream)))
    return y


def osmps_heff_apply_noalloc(L, W1, W2, R, theta, y, stream=None):
    """Float64 H_eff.theta through the allocation-free entry point (no context;
    fixed 32 MiB scratch inside the library, shared by all calls).

    The library runs on the device current on the calling thread and reads
    every operand with the dimensions taken from theta, W1 and W2, so the
    operands are checked here first: all on the current device, and L, R,
    W1, W2 and y of the shapes those dimensions imply."""
    import torch
    chi_l, d1, d2, chi_r = theta.shape
    wl, wm, wr = W1.shape[0], W1.shape[3], W2.shape[3]
    cur = torch.cuda.current_device()
    for name, t in (("L", L), ("W1", W1), ("W2", W2), ("R", R), ("theta", theta), ("y", y)):
        if not t.is_cuda or t.device.index != cur:
            raise ValueError(f"{name} is on {t.device}, not on the current device cuda:{cur}")
    want = {"L": (chi_l, wl, chi_l), "R": (chi_r, wr, chi_r), "W1": (wl, d1, d1, wm),
            "W2": (wm, d2, d2, wr), "y": (chi_l, d1, d2, chi_r)}
    for name, t in (("L", L), ("R", R), ("W1", W1), ("W2", W2), ("y", y)):
        if tuple(t.shape) != want[name]:
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {want[name]}")
    _check(lib().osmps_heff_apply_noalloc(_dev(L, "L"), _dev(W1, "W1"), _dev(W2, "W2"),
                                          _dev(R, "R"), _dev(theta, "theta"), _dev(y, "y"), chi_l,
                                          d1, d2, chi_r, wl, wm, wr, _stream(stream)))
    return y


def osmps_dgemm_emu(ctx, A, B, C, stream=None):
    """C = A @ B in float64 accuracy on the bf16 tensor cores (error-free slices)."""
    M, K = A.shape
    K2, N = B.shape
    assert K == K2 and tuple(C.shape) == (M, N)
    _check(lib().osmps_dgemm_emu(ctx.ptr, _dev(A, "A"), _dev(B, "B"), _dev(C, "C"), M, N, K,
                                 _stream(stream)))
    return C


def osmps_env_update(ctx, side, env_in, A, W, env_out, precision="bf16x3", stream=None):
    chi_l, d, chi_r = A.shape
    if side == 0:
        w_in, w_out = W.shape[0], W.shape[3]
    else:
        w_in, w_out = W.shape[3], W.shape[0]
    _check(lib().osmps_env_update(ctx.ptr, int(side), _dev(env_in, "env_in"), _dev(A, "A"),
                                  _dev(W, "W"), _dev(env_out, "env_out"), chi_l, d, chi_r, w_in,
                                  w_out, _prec(precision), _stream(stream)))
    return env_out


def osmps_lanczos_ground(ctx, L, W1, W2, R, theta, max_iter=100, tol=1e-12, precision="fp64",
                         stream=None, allow_noconv=True):
    """Returns (energy, iterations, residual estimate, converged)."""
    chi_l, d1, d2, chi_r = theta.shape
    wl, wm, wr = W1.shape[0], W1.shape[3], W2.shape[3]
    e = _c.c_double()
    it = _c.c_int()
    res = _c.c_double()
    st = lib().osmps_lanczos_ground(ctx.ptr, _dev(L, "L"), _dev(W1, "W1"), _dev(W2, "W2"),
                                    _dev(R, "R"), _dev(theta, "theta"), chi_l, d1, d2, chi_r, wl,
                                    wm, wr, int(max_iter), float(tol), _prec(precision),
                                    _c.byref(e), _c.byref(it), _c.byref(res), _stream(stream))
    _check(st, allow=(ENOCONV,) if allow_noconv else ())
    return e.value, it.value, res.value, st == 0


def osmps_heff_expm(ctx, L, W1, W2, R, theta, tau, max_iter=40, tol=1e-12, precision="fp64",
                    stream=None, allow_noconv=True):
    """theta <- exp(-i tau H_eff) theta in place by the Krylov propagator.
    L, R, theta are complex128 tensors (L[a2,w,a], R[c2,w,c], theta[a,s1,s2,c]),
    W1, W2 float64. Returns (Krylov vectors used, error estimate, converged)."""
    chi_l, d1, d2, chi_r = theta.shape
    wl, wm, wr = W1.shape[0], W1.shape[3], W2.shape[3]
    it = _c.c_int()
    err = _c.c_double()
    st = lib().osmps_heff_expm(ctx.ptr, _devc(L, "L"), _dev(W1, "W1"), _dev(W2, "W2"),
                               _devc(R, "R"), _devc(theta, "theta"), chi_l, d1, d2, chi_r, wl,
                               wm, wr, float(tau), int(max_iter), float(tol), _prec(precision),
                               _c.byref(it), _c.byref(err), _stream(stream))
    _check(st, allow=(ENOCONV,) if allow_noconv else ())
    return it.value, err.value, st == 0


def osmps_split_complex(ctx, theta, A1, A2, move_right, chi_max, eps_local, precision="fp64",
                        stream=None):
    """Complex split (complex128 CUDA tensors). Returns (chi_new, discarded,
    entropy, lam2 numpy array); A1/A2 are flat buffers as for osmps_split."""
    chi_l, d1, d2, chi_r = theta.shape
    n = min(chi_l * d1, d2 * chi_r)
    lam2 = np.zeros(n)
    chn = _i64()
    disc = _c.c_double()
    ent = _c.c_double()
    _check(lib().osmps_split_complex(ctx.ptr, _devc(theta, "theta"), _devc(A1, "A1"),
                                     _devc(A2, "A2"), chi_l, d1, d2, chi_r, int(move_right),
                                     int(chi_max), float(eps_local), _c.byref(chn),
                                     _c.byref(disc), _c.byref(ent),
                                     lam2.ctypes.data_as(_dp), _prec(precision), _stream(stream)))
    return chn.value, disc.value, ent.value, lam2


def osmps_tdvp_evolve(ctx, mpo, tensors, dt, n_steps, chi_max, eps_local=0.0, krylov_tol=1e-12,
                      krylov_max_iter=40, precision="fp64", stream=None):
    """Two-site TDVP real-time evolution of a complex MPS given as host arrays
    tensors[k] (chi_k, d_k, chi_{k+1}) with sites 1..L-1 right-canonical.
    Returns (evolved tensors as complex128 numpy arrays, energies, norms, stats)."""
    L = len(tensors)
    if L != mpo.L:
        raise ValueError(f"osmps_tdvp_evolve: {L} site tensors for an MPO of {mpo.L} sites")
    ts = [np.ascontiguousarray(t, dtype=np.complex128) for t in tensors]
    for k, t in enumerate(ts):
        if t.ndim != 3 or t.shape[1] != mpo.shapes[k][1]:
            raise ValueError(f"osmps_tdvp_evolve: site {k} has shape {t.shape}, physical "
                             f"dimension {mpo.shapes[k][1]} expected")
        if k + 1 < L and t.shape[2] != ts[k + 1].shape[0]:
            raise ValueError(f"osmps_tdvp_evolve: bond {k + 1} differs between sites {k} and {k + 1}")
    chi_in = (_i64 * (L + 1))(*([t.shape[0] for t in ts] + [ts[-1].shape[2]]))
    ins = (_dp * L)(*[t.ctypes.data_as(_dp) for t in ts])
    d = [t.shape[1] for t in ts]
    left = [1]
    for k in range(L):
        left.append(min(left[-1] * d[k], 1 << 30))
    right = [1] * (L + 1)
    for k in range(L - 1, -1, -1):
        right[k] = min(right[k + 1] * d[k], 1 << 30)
    cap = [min(chi_max, left[k], right[k]) for k in range(L + 1)]
    outs = [np.zeros(cap[k] * d[k] * cap[k + 1], dtype=np.complex128) for k in range(L)]
    outp = (_dp * L)(*[o.ctypes.data_as(_dp) for o in outs])
    chi_out = (_i64 * (L + 1))()
    energy = np.zeros(max(n_steps, 1))
    norm = np.zeros(max(n_steps, 1))
    st = TdvpStats()
    st.energy = energy.ctypes.data_as(_dp)
    st.norm = norm.ctypes.data_as(_dp)
    prm = TdvpParams(float(dt), int(n_steps), int(chi_max), float(eps_local), float(krylov_tol),
                     int(krylov_max_iter), _prec(precision))
    _check(lib().osmps_tdvp_evolve(ctx.ptr, mpo.ptr, chi_in, ins, _c.byref(prm), chi_out, outp,
                                   _c.byref(st), _stream(stream)))
    res = [outs[k][: chi_out[k] * d[k] * chi_out[k + 1]].reshape(chi_out[k], d[k], chi_out[k + 1])
           for k in range(L)]
    stats = {f: getattr(st, f) for f, _ in TdvpStats._fields_ if f not in ("energy", "norm")}
    return res, energy[:n_steps], norm[:n_steps], stats


def osmps_theta_form(ctx, A1, A2, theta, stream=None):
    chi_l, d1, chi_m = A1.shape
    _, d2, chi_r = A2.shape
    _check(lib().osmps_theta_form(ctx.ptr, _dev(A1, "A1"), _dev(A2, "A2"), _dev(theta, "theta"),
                                  chi_l, d1, chi_m, d2, chi_r, _stream(stream)))
    return theta


def osmps_split(ctx, theta, A1, A2, move_right, chi_max, eps_local, precision="fp64", stream=None):
    """Returns (chi_new, discarded, entropy, lam2 numpy array). A1/A2 are flat
    buffers large enough for the largest possible chi_new; reshape them to
    (chi_l, d1, chi_new) / (chi_new, d2, chi_r)."""
    chi_l, d1, d2, chi_r = theta.shape
    n = min(chi_l * d1, d2 * chi_r)
    lam2 = np.zeros(n)
    chn = _i64()
    disc = _c.c_double()
    ent = _c.c_double()
    _check(lib().osmps_split(ctx.ptr, _dev(theta, "theta"), _dev(A1, "A1"), _dev(A2, "A2"), chi_l,
                             d1, d2, chi_r, int(move_right), int(chi_max), float(eps_local),
                             _c.byref(chn), _c.byref(disc), _c.byref(ent),
                             lam2.ctypes.data_as(_dp), _prec(precision), _stream(stream)))
    return chn.value, disc.value, ent.value, lam2


class MPS:
    """Device-resident MPS handle (osmps_mps)."""

    def __init__(self, ctx, tensors, chi_cap):
        tensors = [np.ascontiguousarray(t, dtype=np.float64) for t in tensors]
        self.ctx = ctx
        self.L = len(tensors)
        d = (_i64 * self.L)(*[t.shape[1] for t in tensors])
        chi = (_i64 * (self.L + 1))(*([t.shape[0] for t in tensors] + [tensors[-1].shape[2]]))
        self._keep = tensors
        ptrs = (_dp * self.L)(*[t.ctypes.data_as(_dp) for t in tensors])
        self.ptr = _vp()
        _check(lib().osmps_mps_create(ctx.ptr, self.L, d, chi, ptrs, int(chi_cap), _c.byref(self.ptr)))
        self.d = [t.shape[1] for t in tensors]
        self._keep = None

    def bond_dims(self):
        out = (_i64 * (self.L + 1))()
        _check(lib().osmps_mps_bond_dims(self.ptr, out))
        return list(out)

    def tensor(self, k):
        chi = self.bond_dims()
        out = np.empty((chi[k], self.d[k], chi[k + 1]))
        _check(lib().osmps_mps_get_tensor(self.ptr, int(k), out.ctypes.data_as(_dp)))
        return out

    def tensors(self):
        return [self.tensor(k) for k in range(self.L)]

    def close(self):
        if self.ptr:
            lib().osmps_mps_destroy(self.ptr)
            self.ptr = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MPO:
    """Device-resident MPO handle (osmps_mpo); W[k] has shape (w_k, d, d, w_{k+1})."""

    def __init__(self, ctx, W):
        W = [np.ascontiguousarray(x, dtype=np.float64) for x in W]
        self.ctx = ctx
        self.L = len(W)
        d = (_i64 * self.L)(*[x.shape[1] for x in W])
        w = (_i64 * (self.L + 1))(*([x.shape[0] for x in W] + [W[-1].shape[3]]))
        ptrs = (_dp * self.L)(*[x.ctypes.data_as(_dp) for x in W])
        self.ptr = _vp()
        _check(lib().osmps_mpo_create(ctx.ptr, self.L, d, w, ptrs, _c.byref(self.ptr)))
        self.shapes = [x.shape for x in W]

    def set(self, W):
        """Overwrite the site tensors with new values of the same shapes."""
        W = [np.ascontiguousarray(x, dtype=np.float64) for x in W]
        if [x.shape for x in W] != self.shapes:
            raise ValueError("MPO.set: shapes differ from the handle's")
        ptrs = (_dp * self.L)(*[x.ctypes.data_as(_dp) for x in W])
        _check(lib().osmps_mpo_set(self.ptr, ptrs))

    @property
    def n_params(self):
        """Number of values in the concatenated site tensors."""
        return int(sum(np.prod(sh) for sh in self.shapes))

    def close(self):
        if self.ptr:
            lib().osmps_mpo_destroy(self.ptr)
            self.ptr = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sweep_params(chi_max, n_sweeps=1, precision="fp64", eps_local=-1.0, lanczos_tol=1e-12,
                 lanczos_max_iter=100, refine_sweeps=0):
    return SweepParams(int(chi_max), float(eps_local), float(lanczos_tol), int(lanczos_max_iter),
                       int(n_sweeps), _prec(precision), int(refine_sweeps))


def osmps_mps_canonicalize(ctx, mps, mpo, center, precision="fp64", stream=None):
    _check(lib().osmps_mps_canonicalize(ctx.ptr, mps.ptr, mpo.ptr, int(center), _prec(precision),
                                        _stream(stream)))


def osmps_sweep_step(ctx, mps, mpo, k, move_right, params, stream=None):
    out = StepStats()
    _check(lib().osmps_sweep_step(ctx.ptr, mps.ptr, mpo.ptr, int(k), int(move_right),
                                  _c.byref(params), _c.byref(out), _stream(stream)))
    return {f: getattr(out, f) for f, _ in StepStats._fields_}


def osmps_sweep(ctx, mps, mpo, params, stream=None, record_steps=True):
    stats = SweepStats()
    nsteps = 2 * (mps.L - 1) * (params.n_sweeps + params.refine_sweeps)
    if record_steps:
        energies = np.zeros(max(nsteps, 1))
        iters = np.zeros(max(nsteps, 1), dtype=np.int64)
        stats.step_energies = energies.ctypes.data_as(_dp)
        stats.step_iters = iters.ctypes.data_as(_c.POINTER(_i64))
    _check(lib().osmps_sweep(ctx.ptr, mps.ptr, mpo.ptr, _c.byref(params), _c.byref(stats),
                             _stream(stream)))
    out = {f: getattr(stats, f) for f, _ in SweepStats._fields_ if not f.startswith("step_")}
    if record_steps:
        out["step_energies"] = energies[:nsteps]
        out["step_iters"] = iters[:nsteps]
    return out


def osmps_energy(ctx, mps, mpo, stream=None):
    e = _c.c_double()
    _check(lib().osmps_energy(ctx.ptr, mps.ptr, mpo.ptr, _c.byref(e), _stream(stream)))
    return e.value


def _opt(t, name):
    return _vp(0) if t is None else _dev(t, name)


def osmps_heff_backward(ctx, L, W1, W2, R, theta, gy, gtheta=None, gW1=None, gW2=None,
                        precision="fp64", stream=None):
    """Vector-Jacobian product of H_eff.theta: fills whichever of gtheta, gW1,
    gW2 are given (shapes of theta, W1, W2)."""
    chi_l, d1, d2, chi_r = gy.shape
    wl, wm, wr = W1.shape[0], W1.shape[3], W2.shape[3]
    _check(lib().osmps_heff_backward(ctx.ptr, _dev(L, "L"), _dev(W1, "W1"), _dev(W2, "W2"),
                                     _dev(R, "R"), _opt(theta, "theta"), _dev(gy, "gy"),
                                     _opt(gtheta, "gtheta"), _opt(gW1, "gW1"), _opt(gW2, "gW2"),
                                     chi_l, d1, d2, chi_r, wl, wm, wr, _prec(precision),
                                     _stream(stream)))


def osmps_energy_grad(ctx, mps, mpo, gW, checkpoint_every=0, precision="fp64emu", stream=None):
    """E and dE/dW (written into the flat device tensor gW, sites concatenated).
    Returns (energy, <psi|psi>)."""
    e = _c.c_double()
    n = _c.c_double()
    _check(lib().osmps_energy_grad(ctx.ptr, mps.ptr, mpo.ptr, _dev(gW, "gW"), gW.numel(),
                                   int(checkpoint_every), _prec(precision), _c.byref(e),
                                   _c.byref(n), _stream(stream)))
    return e.value, n.value


def osmps_coupling_grad(ctx, row_ptr, col, val, gW, g_par, stream=None):
    """g_par[p] = sum over row p of the CSR basis of val * gW[col] (int64 row_ptr
    and col, float64 val, all CUDA tensors)."""
    import torch
    for t, nm in ((row_ptr, "row_ptr"), (col, "col")):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int64 and t.is_contiguous()):
            raise TypeError(f"{nm} must be a contiguous int64 CUDA tensor")
    _check(lib().osmps_coupling_grad(ctx.ptr, g_par.numel(), _vp(row_ptr.data_ptr()),
                                     _vp(col.data_ptr()), _dev(val, "val"), col.numel(),
                                     _dev(gW, "gW"), gW.numel(), _dev(g_par, "g_par"),
                                     _stream(stream)))
    return g_par


def osmps_sweep_batch(ctxs, mps_list, mpo_list, params_list):
    """Sweeps of many chains at once: one host thread, context and stream per
    entry of ctxs. Returns (list of per-chain stats dicts, list of statuses);
    raises on the first failure."""
    n = len(mps_list)
    assert len(mpo_list) == n and len(params_list) == n
    cs = (_vp * len(ctxs))(*[c.ptr for c in ctxs])
    ms = (_vp * n)(*[m.ptr for m in mps_list])
    hs = (_vp * n)(*[h.ptr for h in mpo_list])
    ps = (SweepParams * n)(*params_list)
    st = (SweepStats * n)()
    cst = (_c.c_int * n)()
    status = lib().osmps_sweep_batch(cs, len(ctxs), ms, hs, ps, n, st, cst)
    stats = [{f: getattr(x, f) for f, _ in SweepStats._fields_ if not f.startswith("step_")}
             for x in st]
    if status != 0:
        err = OsmpsError(status, lib().osmps_last_error().decode(errors="replace"))
        err.chain_status = list(cst)
        raise err
    return stats, list(cst)


def _i64arr(x):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.int64))
    return a, a.ctypes.data_as(_c.POINTER(_i64))


class U1Heff:
    """Block plan of the U(1)-symmetric H_eff (osmps_u1_heff): sectors of the
    left and right bond (charges and sizes, in index order), local dims and
    the charges of the MPO channels on the two outer MPO bonds."""

    def __init__(self, ctx, q_left, chi_left, q_right, chi_right, d1, d2, wl, wm, wr, q_wl, q_wr):
        self.ctx = ctx
        keep = [_i64arr(v) for v in (q_left, chi_left, q_right, chi_right, q_wl, q_wr)]
        self._keep = keep
        desc = U1Desc(len(keep[0][0]), keep[0][1], keep[1][1], len(keep[2][0]), keep[2][1],
                      keep[3][1], int(d1), int(d2), int(wl), int(wm), int(wr), keep[4][1], keep[5][1])
        self.ptr = _vp()
        _check(lib().osmps_u1_heff_create(ctx.ptr, _c.byref(desc), _c.byref(self.ptr)))
        nt, nl, nr, fl = _i64(), _i64(), _i64(), _c.c_double()
        _check(lib().osmps_u1_heff_sizes(self.ptr, _c.byref(nt), _c.byref(nl), _c.byref(nr),
                                         _c.byref(fl)))
        self.n_theta, self.n_L, self.n_R, self.flops = nt.value, nl.value, nr.value, fl.value
        t1, a4, ny = _i64(), _i64(), _i64()
        _check(lib().osmps_u1_heff_stage_sizes(self.ptr, _c.byref(t1), _c.byref(a4), _c.byref(ny)))
        # intermediates: stage-1 output entries, W-step output entries, stage-4 output entries
        self.n_T1, self.n_A4, self.n_Y = t1.value, a4.value, ny.value

    def close(self):
        if self.ptr:
            lib().osmps_u1_heff_destroy(self.ptr)
            self.ptr = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def osmps_heff_apply_u1(ctx, plan, L, W1, W2, R, theta, y, precision="bf16x3", stream=None):
    """y = H_eff theta on packed block-sparse vectors (see U1Heff)."""
    for t, n, name in ((L, plan.n_L, "L"), (R, plan.n_R, "R"), (theta, plan.n_theta, "theta"),
                       (y, plan.n_theta, "y")):
        if t.numel() != n:
            raise ValueError(f"{name} has {t.numel()} entries, the plan expects {n}")
    _check(lib().osmps_heff_apply_u1(ctx.ptr, plan.ptr, _dev(L, "L"), _dev(W1, "W1"), _dev(W2, "W2"),
                                     _dev(R, "R"), _dev(theta, "theta"), _dev(y, "y"),
                                     _prec(precision), _stream(stream)))
    return y


def osmps_u1_heff_prepare(ctx, plan, L, W1, W2, R, precision="bf16x3", stream=None):
    _check(lib().osmps_u1_heff_prepare(ctx.ptr, plan.ptr, _dev(L, "L"), _dev(W1, "W1"),
                                       _dev(W2, "W2"), _dev(R, "R"), _prec(precision),
                                       _stream(stream)))


def osmps_u1_heff_apply(ctx, plan, theta, y, stream=None):
    _check(lib().osmps_u1_heff_apply(ctx.ptr, plan.ptr, _dev(theta, "theta"), _dev(y, "y"),
                                     _stream(stream)))
    return y


def osmps_lanczos_ground_u1(ctx, plan, L, W1, W2, R, theta, max_iter=100, tol=1e-12,
                            precision="bf16x3", stream=None, allow_noconv=True):
    """Returns (energy, iterations, residual estimate, converged)."""
    e, it, res = _c.c_double(), _c.c_int(), _c.c_double()
    st = lib().osmps_lanczos_ground_u1(ctx.ptr, plan.ptr, _dev(L, "L"), _dev(W1, "W1"),
                                       _dev(W2, "W2"), _dev(R, "R"), _dev(theta, "theta"),
                                       int(max_iter), float(tol), _prec(precision), _c.byref(e),
                                       _c.byref(it), _c.byref(res), _stream(stream))
    _check(st, allow=(ENOCONV,) if allow_noconv else ())
    return e.value, it.value, res.value, st == 0


def osmps_sytrd(ctx, A, d, e, tau, stream=None):
    """Householder tridiagonalisation of the symmetric A (overwritten, dsytrd layout)."""
    n = A.shape[0]
    _check(lib().osmps_sytrd(ctx.ptr, _dev(A, "A"), n, _dev(d, "d"), _dev(e, "e"), _dev(tau, "tau"),
                             _stream(stream)))


def osmps_selftest_wait_timeout(ctx, which, limit_us=2000.0, stream=None):
    """Make one bounded device wait run out on purpose (which = 0: an mbarrier
    wait in a kernel holding tensor memory; 1: a grid barrier one block never
    reaches). Raises OsmpsError(ETIMEOUT) when the wait gave up, as it should."""
    _check(lib().osmps_selftest_wait_timeout(ctx.ptr, int(which), float(limit_us), _stream(stream)))


def osmps_selftest_convert(ctx, x64, x32, stream=None):
    """(float32 of x64, float64 of x32) by the library's integer-field
    conversions (device tensors of equal length)."""
    import torch
    if not (isinstance(x32, torch.Tensor) and x32.is_cuda and x32.dtype == torch.float32
            and x32.is_contiguous()) or x32.numel() != x64.numel():
        raise TypeError("x32 must be a contiguous float32 CUDA tensor as long as x64")
    y32 = torch.empty(x64.numel(), dtype=torch.float32, device=x64.device)
    y64 = torch.empty(x32.numel(), dtype=torch.float64, device=x32.device)
    _check(lib().osmps_selftest_convert(ctx.ptr, _dev(x64, "x64"), _vp(y32.data_ptr()),
                                        _vp(x32.data_ptr()), _dev(y64, "y64"), x64.numel(),
                                        _stream(stream)))
    return y32, y64


def osmps_selftest_bf16(ctx, x, stream=None):
    """(integer-field, CUDA) bf16 roundings of the float64 device tensor x as
    int16 tensors of raw bit patterns."""
    import torch
    yi = torch.empty(x.numel(), dtype=torch.int16, device=x.device)
    yh = torch.empty(x.numel(), dtype=torch.int16, device=x.device)
    _check(lib().osmps_selftest_bf16(ctx.ptr, _dev(x, "x"), _vp(yi.data_ptr()), _vp(yh.data_ptr()),
                                     x.numel(), _stream(stream)))
    return yi, yh


def osmps_gemm_grouped(ctx, outs, terms, stream=None):
    """Grouped float64 products of strided device views in one launch: outs
    (GEMM_OUT_DTYPE records), terms (GEMM_TERM_DTYPE records); per output
    C = sum over its terms of alpha A B + beta C."""
    outs = np.ascontiguousarray(outs, dtype=GEMM_OUT_DTYPE)
    terms = np.ascontiguousarray(terms, dtype=GEMM_TERM_DTYPE)
    _check(lib().osmps_gemm_grouped(ctx.ptr, outs.ctypes.data if len(outs) else None, len(outs),
                                    terms.ctypes.data if len(terms) else None, len(terms),
                                    _stream(stream)))


def osmps_copy_list(ctx, descs, stream=None):
    """Run a list of scaled strided 2-D copies (CopyDesc tuples) in one launch."""
    arr = (CopyDesc * len(descs))(*[d if isinstance(d, CopyDesc) else CopyDesc(*d) for d in descs])
    _check(lib().osmps_copy_list(ctx.ptr, arr, len(descs), _stream(stream)))


def osmps_sym_eig_top(ctx, G, nev, Y, stream=None):
    """Largest nev eigenpairs of the symmetric device matrix G (n x n, float64,
    overwritten): returns the eigenvalues (ascending, numpy); Y (nev x n) gets
    the eigenvectors as rows."""
    n = G.shape[0]
    ev = np.zeros(int(nev))
    _check(lib().osmps_sym_eig_top(ctx.ptr, _dev(G, "G"), n, int(nev), ev.ctypes.data_as(_dp),
                                   _dev(Y, "Y"), _stream(stream)))
    return ev


def osmps_vec_norm2(ctx, x, stream=None):
    out = _c.c_double()
    _check(lib().osmps_vec_norm2(ctx.ptr, _dev(x, "x"), x.numel(), _c.byref(out), _stream(stream)))
    return out.value


def osmps_variance(ctx, mps, mpo, stream=None):
    """(E, V) of the MPS, V = <(H - E)^2>."""
    e, v = _c.c_double(), _c.c_double()
    _check(lib().osmps_variance(ctx.ptr, mps.ptr, mpo.ptr, _c.byref(e), _c.byref(v), _stream(stream)))
    return e.value, v.value


def osmps_lanczos_ground_projected(ctx, L, W1, W2, R, theta, P, max_iter=100, tol=1e-12,
                                   precision="fp64", stream=None, allow_noconv=True):
    """Lanczos in the orthogonal complement of the rows of P (k x n, or None)."""
    chi_l, d1, d2, chi_r = theta.shape
    wl, wm, wr = W1.shape[0], W1.shape[3], W2.shape[3]
    k = 0 if P is None else P.shape[0]
    e, it, res = _c.c_double(), _c.c_int(), _c.c_double()
    st = lib().osmps_lanczos_ground_projected(
        ctx.ptr, _dev(L, "L"), _dev(W1, "W1"), _dev(W2, "W2"), _dev(R, "R"), _dev(theta, "theta"),
        _vp(0) if P is None else _dev(P, "P"), k, chi_l, d1, d2, chi_r, wl, wm, wr, int(max_iter),
        float(tol), _prec(precision), _c.byref(e), _c.byref(it), _c.byref(res), _stream(stream))
    _check(st, allow=(ENOCONV,) if allow_noconv else ())
    return e.value, it.value, res.value, st == 0


def osmps_overlap_env_update(ctx, side, env_in, A, Bk, env_out, stream=None):
    chi_l, d, chi_r = A.shape
    chik_l, _, chik_r = Bk.shape
    _check(lib().osmps_overlap_env_update(ctx.ptr, int(side), _dev(env_in, "env_in"), _dev(A, "A"),
                                          _dev(Bk, "Bk"), _dev(env_out, "env_out"), chi_l, d, chi_r,
                                          chik_l, chik_r, _stream(stream)))
    return env_out


def osmps_projected_state(ctx, OL, B1, B2, OR, v, stream=None):
    chi_l, d1, d2, chi_r = v.shape
    chik_l, _, chik_m = B1.shape
    chik_r = B2.shape[2]
    _check(lib().osmps_projected_state(ctx.ptr, _dev(OL, "OL"), _dev(B1, "B1"), _dev(B2, "B2"),
                                       _dev(OR, "OR"), _dev(v, "v"), chi_l, d1, d2, chi_r, chik_l,
                                       chik_m, chik_r, _stream(stream)))
    return v
