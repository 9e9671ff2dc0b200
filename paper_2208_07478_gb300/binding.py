"""Thin ctypes binding of the CCGF C ABI (include/ccgf.h).

Argument marshalling only: every step of the computation runs in libccgf.so.
Arrays are passed by pointer: torch tensors (host or CUDA) or numpy arrays
(host). Complex arrays must be complex128 and C-contiguous. ``load()`` raises
when the compiled library is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libccgf.so")

CCGF_OK, CCGF_NOT_CONVERGED = 0, 1
CCGF_ERR_INVALID_ARG, CCGF_ERR_OOM, CCGF_ERR_CUDA, CCGF_ERR_NAN, CCGF_ERR_TIMEOUT = -1, -2, -3, -4, -5
FP64, FP32, TF32X3, FP64_TC = 0, 1, 2, 3
IP, EA, BOTH = 1, 2, 3


class System(C.Structure):
    _fields_ = [("kmesh", C.c_int * 3), ("nocc", C.c_int), ("nvir", C.c_int), ("naux", C.c_int),
                ("mo_energy", C.c_void_p), ("L", C.c_void_p), ("t1", C.c_void_p), ("t2", C.c_void_p),
                ("l1", C.c_void_p), ("l2", C.c_void_p), ("inputs_on_device", C.c_int)]


class Options(C.Structure):
    _fields_ = [("prec", C.c_int), ("tol", C.c_double), ("restart_m", C.c_int), ("max_iter", C.c_int),
                ("max_refine", C.c_int), ("omega_chunk", C.c_int), ("device_wait_timeout_ms", C.c_double),
                ("warm_start", C.c_int), ("kpoint", C.c_int), ("orbital_first", C.c_int), ("orbital_count", C.c_int),
                ("direct_terms", C.c_int), ("refine_prec", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("rhs_solved", C.c_longlong), ("inner_iterations", C.c_longlong),
                ("fp64_sigma_calls", C.c_longlong), ("lowp_sigma_calls", C.c_longlong),
                ("max_rel_residual", C.c_double), ("sigma_ms", C.c_double), ("total_ms", C.c_double),
                ("kernel_launches", C.c_longlong), ("warm_columns", C.c_longlong), ("warm_fallbacks", C.c_longlong),
                ("warm_val_loss", C.c_double), ("warm_val_loss_baseline", C.c_double),
                ("warm_rel_residual", C.c_double), ("warm_rel_residual_net", C.c_double),
                ("warm_rel_residual_base", C.c_double), ("restart_used", C.c_longlong),
                ("columns_per_batch", C.c_longlong), ("vector_ms", C.c_double), ("vector_bytes", C.c_double),
                ("refine_ms", C.c_double), ("vector_flops", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


EXPORTS = ["ccgf_default_options", "ccgf_build_intermediates", "ccgf_dims", "ccgf_sigma_ip", "ccgf_sigma_ea",
           "ccgf_rhs", "ccgf_left", "ccgf_solve_gf", "ccgf_sigma_profile", "ccgf_sigma_step_name", "ccgf_sigma_ip_noalloc", "ccgf_launch_count",
           "ccgf_set_autotune", "ccgf_sigma_step_kernel", "ccgf_tensor_wait_selftest", "ccgf_inject_alloc_failure",
           "ccgf_spectral_function", "ccgf_self_energy_correction", "ccgf_solve_gf_mor",
           "ccgf_train_warmstart", "ccgf_mlp_param_count", "ccgf_mlp_forward", "ccgf_mlp_loss_grad", "ccgf_destroy",
           "ccgf_status_string", "ccgf_last_error"]

_lib = None


def load(path: str | None = None):
    """Load libccgf.so (raises FileNotFoundError / OSError when absent)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise FileNotFoundError(f"{p} is missing: run __graft_entry__.build() (the CUDA library is required)")
    lib = C.CDLL(p)
    vp, i, ll, d = C.c_void_p, C.c_int, C.c_longlong, C.c_double
    lib.ccgf_default_options.argtypes = [C.POINTER(Options)]
    lib.ccgf_default_options.restype = None
    lib.ccgf_build_intermediates.argtypes = [C.POINTER(System), C.POINTER(Options), vp, C.POINTER(vp)]
    lib.ccgf_build_intermediates.restype = i
    lib.ccgf_dims.argtypes = [vp, C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(ll), C.POINTER(ll)]
    lib.ccgf_dims.restype = i
    for name in ("ccgf_sigma_ip", "ccgf_sigma_ea"):
        getattr(lib, name).argtypes = [vp, i, ll, vp, vp, i, vp]
        getattr(lib, name).restype = i
    for name in ("ccgf_rhs", "ccgf_left"):
        getattr(lib, name).argtypes = [vp, i, i, i, vp, vp]
        getattr(lib, name).restype = i
    lib.ccgf_solve_gf.argtypes = [vp, i, i, vp, d, C.POINTER(Options), vp, i, C.POINTER(Stats), vp]
    lib.ccgf_solve_gf.restype = i
    lib.ccgf_sigma_profile.argtypes = [vp, i, i, ll, vp, vp, i, vp, i, C.POINTER(d), C.POINTER(d), C.POINTER(i)]
    lib.ccgf_sigma_profile.restype = i
    lib.ccgf_sigma_step_name.argtypes = [vp, i, i, i]
    lib.ccgf_sigma_step_name.restype = C.c_char_p
    lib.ccgf_sigma_ip_noalloc.argtypes = [vp, i, ll, vp, vp, vp]
    lib.ccgf_sigma_ip_noalloc.restype = i
    lib.ccgf_train_warmstart.argtypes = [vp, i, i, vp, d, C.POINTER(Options), i, ll, d, C.c_uint, C.POINTER(d),
                                         C.POINTER(Stats), vp]
    lib.ccgf_train_warmstart.restype = i
    lib.ccgf_mlp_param_count.argtypes = [i, i]
    lib.ccgf_mlp_param_count.restype = ll
    lib.ccgf_mlp_forward.argtypes = [i, i, ll, vp, vp, i, vp, vp]
    lib.ccgf_mlp_forward.restype = i
    lib.ccgf_mlp_loss_grad.argtypes = [i, i, ll, vp, vp, vp, i, C.POINTER(d), vp, vp]
    lib.ccgf_mlp_loss_grad.restype = i
    lib.ccgf_launch_count.argtypes = [vp]
    lib.ccgf_launch_count.restype = ll
    lib.ccgf_tensor_wait_selftest.argtypes = [C.c_double, vp]
    lib.ccgf_tensor_wait_selftest.restype = C.c_int
    lib.ccgf_solve_gf_mor.argtypes = [vp, i, i, vp, i, vp, d, C.POINTER(Options), vp, i, C.POINTER(Stats), vp]
    lib.ccgf_solve_gf_mor.restype = i
    lib.ccgf_self_energy_correction.argtypes = [i, i, i, i, vp, vp, vp, vp, vp, vp]
    lib.ccgf_self_energy_correction.restype = i
    lib.ccgf_spectral_function.argtypes = [i, i, i, vp, vp, vp, vp, vp]
    lib.ccgf_spectral_function.restype = i
    lib.ccgf_inject_alloc_failure.argtypes = [C.c_longlong]
    lib.ccgf_inject_alloc_failure.restype = None
    lib.ccgf_set_autotune.argtypes = [C.c_int]
    lib.ccgf_set_autotune.restype = None
    lib.ccgf_sigma_step_kernel.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int]
    lib.ccgf_sigma_step_kernel.restype = C.c_int
    lib.ccgf_destroy.argtypes = [vp]
    lib.ccgf_destroy.restype = None
    lib.ccgf_status_string.argtypes = [i]
    lib.ccgf_status_string.restype = C.c_char_p
    lib.ccgf_last_error.argtypes = []
    lib.ccgf_last_error.restype = C.c_char_p
    if path is None:
        _lib = lib
    return lib


class CCGFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"status {status}: {msg}")
        self.status = status


def _check(status, allow_not_converged=False):
    if status == CCGF_OK or (allow_not_converged and status == CCGF_NOT_CONVERGED):
        return status
    lib = load()
    raise CCGFError(status, lib.ccgf_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(type(a))


def _stream_ptr(stream):
    if stream is None:
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def default_options(**kw) -> Options:
    o = Options()
    load().ccgf_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Handle:
    """Owns a ccgf_handle; the arrays of ``system`` are copied during the build."""

    def __init__(self, ptr, keepalive=()):
        self.ptr = ptr
        self._keep = keepalive

    def close(self):
        if self.ptr:
            load().ccgf_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self):
        return int(load().ccgf_launch_count(self.ptr))

    def step_kernel(self, sector, kshift, step, prec):
        """Kernel chosen for a plan step (see ccgf_sigma_step_kernel)."""
        return int(load().ccgf_sigma_step_kernel(self.ptr, sector, kshift, step, prec))

    def dims(self):
        nk, o, v = C.c_int(), C.c_int(), C.c_int()
        dip, dea = C.c_longlong(), C.c_longlong()
        _check(load().ccgf_dims(self.ptr, C.byref(nk), C.byref(o), C.byref(v), C.byref(dip), C.byref(dea)))
        return dict(nk=nk.value, nocc=o.value, nvir=v.value, dim_ip=dip.value, dim_ea=dea.value)


def build_intermediates(kmesh, nocc, nvir, naux, mo_energy, L, t1, t2, l1=None, l2=None, *, on_device=False,
                        options=None, stream=None) -> Handle:
    s = System()
    s.kmesh[:] = list(kmesh)
    s.nocc, s.nvir, s.naux = nocc, nvir, naux
    arrs = [mo_energy, L, t1, t2, l1, l2]
    for a in arrs:
        if isinstance(a, np.ndarray):
            assert a.flags["C_CONTIGUOUS"]
    s.mo_energy, s.L, s.t1, s.t2 = _ptr(mo_energy), _ptr(L), _ptr(t1), _ptr(t2)
    s.l1, s.l2 = _ptr(l1), _ptr(l2)
    s.inputs_on_device = 1 if on_device else 0
    h = C.c_void_p()
    opt = options or default_options()
    _check(load().ccgf_build_intermediates(C.byref(s), C.byref(opt), _stream_ptr(stream), C.byref(h)))
    return Handle(h.value)


def sigma_ip(h: Handle, kshift, x, y, prec=FP64, stream=None):
    nvec = x.shape[0] if x.ndim == 2 else 1
    return _check(load().ccgf_sigma_ip(h.ptr, kshift, nvec, _ptr(x), _ptr(y), prec, _stream_ptr(stream)))


def sigma_ea(h: Handle, kshift, x, y, prec=FP64, stream=None):
    nvec = x.shape[0] if x.ndim == 2 else 1
    return _check(load().ccgf_sigma_ea(h.ptr, kshift, nvec, _ptr(x), _ptr(y), prec, _stream_ptr(stream)))


def set_autotune(enable: bool):
    """Measured kernel choice per contraction on (default) or off (model defaults); process-wide."""
    load().ccgf_set_autotune(1 if enable else 0)


KERNEL_TC_TMA, KERNEL_TC_REG, KERNEL_TC_BULK = 100, 101, 102


def tensor_wait_selftest(limit_ms=50.0, stream=None):
    """Status of ccgf_tensor_wait_selftest (CCGF_ERR_TIMEOUT when the bounded wait gave up as designed)."""
    return int(load().ccgf_tensor_wait_selftest(float(limit_ms), _stream_ptr(stream)))


def spectral_function(G, dos, G_minus=None, dos_total=None, stream=None):
    """ccgf_spectral_function on device tensors: G [nk][nomega][nmo][nmo] complex128, dos [nk][nomega] float64."""
    nk, nomega, nmo = G.shape[0], G.shape[1], G.shape[2]
    return _check(load().ccgf_spectral_function(nk, nomega, nmo, _ptr(G), _ptr(G_minus), _ptr(dos), _ptr(dos_total),
                                                _stream_ptr(stream)))


def self_energy_correction(V, G_gw, G_gw_cas, G_cc_cas, G_out, stream=None):
    """ccgf_self_energy_correction on device tensors (complex128): V [nk][nmo][nact], G_gw / G_out
    [nk][nomega][nmo][nmo], G_gw_cas / G_cc_cas [nk][nomega][nact][nact]."""
    nk, nomega, nmo = G_gw.shape[0], G_gw.shape[1], G_gw.shape[2]
    nact = V.shape[2]
    return _check(load().ccgf_self_energy_correction(nk, nomega, nmo, nact, _ptr(V), _ptr(G_gw), _ptr(G_gw_cas),
                                                     _ptr(G_cc_cas), _ptr(G_out), _stream_ptr(stream)))


def inject_alloc_failure(after):
    """ccgf_inject_alloc_failure: make the library's allocations fail after `after` more (-1 resets)."""
    load().ccgf_inject_alloc_failure(int(after))


def sigma_ip_noalloc(h: Handle, kshift, x, y, stream=None):
    """ccgf_sigma_ip_noalloc: FP64 IP sigma using only the library's static device workspace."""
    nvec = x.shape[0] if x.ndim == 2 else 1
    return _check(load().ccgf_sigma_ip_noalloc(h.ptr, kshift, nvec, _ptr(x), _ptr(y), _stream_ptr(stream)))


def train_warmstart(h: Handle, sectors, omega_train, eta, *, options=None, steps=400, rows=65536, lr=2e-3, seed=1,
                    stream=None):
    """Solve the training frequencies and train the warm-start network; returns (final loss, stats dict)."""
    om = np.ascontiguousarray(np.asarray(omega_train, dtype=np.float64))
    st = Stats()
    loss = C.c_double()
    opt = options or default_options()
    _check(load().ccgf_train_warmstart(h.ptr, sectors, len(om), om.ctypes.data, float(eta), C.byref(opt), steps, rows,
                                       lr, seed, C.byref(loss), C.byref(st), _stream_ptr(stream)))
    return loss.value, st.as_dict()


def mlp_param_count(F, H):
    return int(load().ccgf_mlp_param_count(F, H))


def mlp_forward(F, H, theta, X, Y, bf16=True, stream=None):
    return _check(load().ccgf_mlp_forward(F, H, X.shape[0], _ptr(theta), _ptr(X), 1 if bf16 else 0, _ptr(Y),
                                          _stream_ptr(stream)))


def mlp_loss_grad(F, H, theta, X, T, grad, bf16=True, stream=None):
    loss = C.c_double()
    _check(load().ccgf_mlp_loss_grad(F, H, X.shape[0], _ptr(theta), _ptr(X), _ptr(T), 1 if bf16 else 0, C.byref(loss),
                                     _ptr(grad), _stream_ptr(stream)))
    return loss.value


def sigma_profile(h: Handle, sector, kshift, x, y, prec=FP64, stream=None, max_steps=64):
    """One sigma call with per-step device times; returns [(name, ms, flops, kernel)] with kernel
    the choice code of ccgf_sigma_step_kernel (-1 for steps that are not contractions)."""
    nvec = x.shape[0] if x.ndim == 2 else 1
    ms = (C.c_double * max_steps)()
    fl = (C.c_double * max_steps)()
    n = C.c_int()
    lib = load()
    _check(lib.ccgf_sigma_profile(h.ptr, sector, kshift, nvec, _ptr(x), _ptr(y), prec, _stream_ptr(stream), max_steps,
                                  ms, fl, C.byref(n)))
    return [(lib.ccgf_sigma_step_name(h.ptr, sector, kshift, k).decode(), ms[k], fl[k],
             int(lib.ccgf_sigma_step_kernel(h.ptr, sector, kshift, k, prec))) for k in range(min(n.value, max_steps))]


def rhs(h: Handle, sector, K, p, out, stream=None):
    return _check(load().ccgf_rhs(h.ptr, sector, K, p, _ptr(out), _stream_ptr(stream)))


def left(h: Handle, sector, K, p, out, stream=None):
    return _check(load().ccgf_left(h.ptr, sector, K, p, _ptr(out), _stream_ptr(stream)))


def solve_gf_mor(h: Handle, sectors, omega_mor, omega, eta, G_out, *, options=None, on_device=False, stream=None):
    """Model-order-reduction G on the grid `omega` from solves at `omega_mor`; returns (status, stats dict)."""
    om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64))
    omm = np.ascontiguousarray(np.asarray(omega_mor, dtype=np.float64))
    st = Stats()
    opt = options or default_options()
    status = load().ccgf_solve_gf_mor(h.ptr, sectors, len(omm), omm.ctypes.data, len(om), om.ctypes.data, float(eta),
                                      C.byref(opt), _ptr(G_out), 1 if on_device else 0, C.byref(st), _stream_ptr(stream))
    _check(status, allow_not_converged=True)
    return status, st.as_dict()


def solve_gf(h: Handle, sectors, omega, eta, G_out, *, options=None, on_device=False, stream=None):
    """Returns (status, stats dict); status may be NOT_CONVERGED (G written)."""
    om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64))
    st = Stats()
    opt = options or default_options()
    status = load().ccgf_solve_gf(h.ptr, sectors, len(om), om.ctypes.data, float(eta), C.byref(opt), _ptr(G_out),
                                  1 if on_device else 0, C.byref(st), _stream_ptr(stream))
    _check(status, allow_not_converged=True)
    return status, st.as_dict()
