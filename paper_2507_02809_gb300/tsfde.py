"""Thin ctypes binding of libtsfde (include/tsfde.h).

Only argument marshalling lives here: every step of the solve runs in the CUDA
library.  Functions carry the C names; arrays are torch tensors (float64,
contiguous; CUDA tensors for the device-only calls) or, for ``tsfde_setup``
and ``tsfde_gmres_solve``, host numpy arrays / CPU tensors as well.  If the
shared library is missing or no GPU is present the calls raise: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_size_t, c_void_p

import numpy as np

TSFDE_OK = 0
TSFDE_NOT_CONVERGED = 1
TSFDE_EINVAL = -1
TSFDE_ENOMEM = -2
TSFDE_ECUDA = -3
TSFDE_EBREAKDOWN = -4
TSFDE_EUNSUPPORTED = -5
TSFDE_ETIMEOUT = -6

PREC_FP64 = 0
PREC_MIXED = 1
SIDE_LEFT = 0
SIDE_RIGHT = 1
SIDE_FLEXIBLE = 2
BLOCK_SOLVE = 0    # block_solver: P_{n,S}, diagonal blocks solved to inner_tol (Sec. 5.1)
BLOCK_TAU = 1      # T_{n,S}: tau(B_n) blocks, one sine-transform solve each (Remark 1)
BLOCK_STRANG = 2   # S_{n,S}: Strang circulant blocks, one Fourier solve each (Remark 1)


class TsfdeGrid(ctypes.Structure):
    _fields_ = [("d", c_int), ("n", c_int), ("length", c_double), ("S", c_int), ("T", c_double)]


class TsfdeOpts(ctypes.Structure):
    _fields_ = [("precision", c_int), ("side", c_int), ("restart", c_int), ("max_iters", c_int),
                ("tol", c_double), ("inner_tol", c_double), ("inner_tol_mixed", c_double),
                ("pcg_iters", c_int), ("pcg_max", c_int), ("refine_max", c_int), ("coeff_K", c_int),
                ("graphs", c_int), ("persistent", c_int), ("warm_start", c_int), ("fused_cg", c_int),
                ("inner_tol_corr", c_double), ("block_solver", c_int), ("spin_limit", ctypes.c_longlong),
                ("warm_start_mixed", c_int), ("grid_ctas", c_int)]


class TsfdeInfo(ctypes.Structure):
    _fields_ = [("iters", c_int), ("restarts", c_int), ("converged", c_int), ("relres_est", c_double),
                ("relres_true", c_double), ("seconds", c_double), ("precond_failures", c_int),
                ("history", POINTER(c_double)), ("history_cap", c_int), ("history_len", c_int)]


class TsfdeProfileStats(ctypes.Structure):
    _fields_ = [("precond_count", ctypes.c_longlong), ("precond_ms", c_double),
                ("matvec_count", ctypes.c_longlong), ("matvec_ms", c_double),
                ("fp64_block_residuals", ctypes.c_longlong), ("pcg_iterations", ctypes.c_longlong),
                ("flops_bapply", c_double), ("flops_tau", c_double), ("flops_timesum", c_double),
                ("bytes_matvec", c_double), ("launches", ctypes.c_longlong),
                ("graph_kernels", ctypes.c_longlong), ("precond_apps_total", ctypes.c_longlong),
                ("phase_ms", c_double * 12),
                ("phase_count", ctypes.c_longlong * 12),
                ("orth_count", ctypes.c_longlong), ("orth_ms", c_double), ("orth_bytes", c_double),
                ("batch_graph_builds", ctypes.c_longlong), ("batch_graph_replays", ctypes.c_longlong),
                ("batch_graph_error", ctypes.c_char * 96), ("guess_fallbacks", ctypes.c_longlong)]


EXPORTS = ("tsfde_default_opts", "tsfde_setup", "tsfde_set_opts", "tsfde_rhs", "tsfde_matvec",
           "tsfde_precond_apply", "tsfde_gmres_solve", "tsfde_device_bytes", "tsfde_destroy",
           "tsfde_status_string", "tsfde_last_error", "tsfde_profile", "tsfde_profile_read",
           "tsfde_matvec_1d_noalloc", "tsfde_matvec_transpose", "tsfde_precond_apply_transpose",
           "tsfde_adjoint", "tsfde_precond_apply_batch", "tsfde_gmres_solve_batch", "tsfde_direct_solve",
           "tsfde_spectral_bidiag", "tsfde_spectral_arnoldi", "tsfde_solve")

_lib = None


def library_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libtsfde.so")


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libtsfde.so (built by paper_2507_02809_gb300.build) and declare the ABI."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or library_path()
    if not os.path.exists(p):
        raise RuntimeError("libtsfde.so not found at %s: build it first (python -c 'import __graft_entry__ as g; "
                           "g.build()')" % p)
    lib = ctypes.CDLL(p)
    lib.tsfde_default_opts.argtypes = [POINTER(TsfdeOpts)]
    lib.tsfde_default_opts.restype = None
    lib.tsfde_setup.argtypes = [POINTER(c_void_p), POINTER(TsfdeGrid), c_double, c_double, c_double,
                                c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, POINTER(TsfdeOpts), c_void_p]
    lib.tsfde_setup.restype = c_int
    lib.tsfde_set_opts.argtypes = [c_void_p, POINTER(TsfdeOpts)]
    lib.tsfde_set_opts.restype = c_int
    lib.tsfde_rhs.argtypes = [c_void_p, c_void_p]
    lib.tsfde_rhs.restype = c_int
    lib.tsfde_matvec.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.tsfde_matvec.restype = c_int
    lib.tsfde_precond_apply.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.tsfde_precond_apply.restype = c_int
    lib.tsfde_gmres_solve.argtypes = [c_void_p, c_void_p, POINTER(TsfdeInfo)]
    lib.tsfde_gmres_solve.restype = c_int
    lib.tsfde_matvec_transpose.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.tsfde_matvec_transpose.restype = c_int
    lib.tsfde_precond_apply_transpose.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.tsfde_precond_apply_transpose.restype = c_int
    lib.tsfde_adjoint.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_double), c_void_p, c_void_p,
                                  POINTER(TsfdeInfo)]
    lib.tsfde_adjoint.restype = c_int
    lib.tsfde_solve.argtypes = [c_void_p, c_void_p, c_void_p, POINTER(TsfdeInfo)]
    lib.tsfde_solve.restype = c_int
    lib.tsfde_spectral_bidiag.argtypes = [c_void_p, c_int, c_int, c_void_p, POINTER(c_double), POINTER(c_double)]
    lib.tsfde_spectral_bidiag.restype = c_int
    lib.tsfde_spectral_arnoldi.argtypes = [c_void_p, c_int, c_int, c_void_p, POINTER(c_double), POINTER(c_int)]
    lib.tsfde_spectral_arnoldi.restype = c_int
    lib.tsfde_direct_solve.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    lib.tsfde_direct_solve.restype = c_int
    lib.tsfde_precond_apply_batch.argtypes = [c_int, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_void_p)]
    lib.tsfde_precond_apply_batch.restype = c_int
    lib.tsfde_gmres_solve_batch.argtypes = [c_int, POINTER(c_void_p), POINTER(c_void_p), POINTER(TsfdeInfo)]
    lib.tsfde_gmres_solve_batch.restype = c_int
    lib.tsfde_device_bytes.argtypes = [c_void_p]
    lib.tsfde_device_bytes.restype = c_size_t
    lib.tsfde_destroy.argtypes = [c_void_p]
    lib.tsfde_destroy.restype = None
    lib.tsfde_status_string.argtypes = [c_int]
    lib.tsfde_status_string.restype = c_char_p
    lib.tsfde_matvec_1d_noalloc.argtypes = [c_int, c_int, c_double, c_double, c_double, c_double, c_double,
                                            c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.tsfde_matvec_1d_noalloc.restype = c_int
    lib.tsfde_profile.argtypes = [c_void_p, c_int]
    lib.tsfde_profile.restype = c_int
    lib.tsfde_profile_read.argtypes = [c_void_p, POINTER(TsfdeProfileStats)]
    lib.tsfde_profile_read.restype = c_int
    lib.tsfde_last_error.argtypes = []
    lib.tsfde_last_error.restype = c_char_p
    if path is None:
        _lib = lib
    return lib


class TsfdeError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = "%s: %s (%s)" % (where, lib.tsfde_status_string(status).decode(), lib.tsfde_last_error().decode())
        super().__init__(msg)
        self.status = status


def _check(status: int, where: str, allow_not_converged: bool = False) -> int:
    if status == TSFDE_OK or (allow_not_converged and status == TSFDE_NOT_CONVERGED):
        return status
    raise TsfdeError(status, where)


def _ptr(a) -> int:
    """Address of a contiguous float64 torch tensor or numpy array."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("need a C-contiguous float64 array")
        return a.ctypes.data
    import torch
    if not isinstance(a, torch.Tensor):
        raise TypeError("need a torch tensor or numpy array")
    if a.dtype != torch.float64 or not a.is_contiguous():
        raise TypeError("need a contiguous float64 tensor")
    return a.data_ptr()


def _dev_ptr(a) -> int:
    import torch
    if not (isinstance(a, torch.Tensor) and a.is_cuda):
        raise TypeError("this call takes CUDA tensors")
    return _ptr(a)


def tsfde_default_opts(**overrides) -> TsfdeOpts:
    o = TsfdeOpts()
    load().tsfde_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def tsfde_setup(d: int, n: int, length: float, S: int, T: float, beta: float, omega: float, alpha: float,
                gamma1, gamma2, q, rho, mu, opts: TsfdeOpts | None = None, stream: int | None = None) -> int:
    """Returns the opaque handle (an int).  Arrays: [S*N], [S*N], [S], [N], [N] float64."""
    lib = load()
    g = TsfdeGrid(d, n, length, S, T)
    h = c_void_p()
    st = c_void_p(stream if stream is not None else _current_stream())
    status = lib.tsfde_setup(ctypes.byref(h), ctypes.byref(g), beta, omega, alpha, _ptr(gamma1), _ptr(gamma2),
                             _ptr(q), _ptr(rho), _ptr(mu), ctypes.byref(opts) if opts is not None else None, st)
    _check(status, "tsfde_setup")
    return h.value


def tsfde_set_opts(h: int, opts: TsfdeOpts) -> None:
    _check(load().tsfde_set_opts(h, ctypes.byref(opts)), "tsfde_set_opts")


def tsfde_rhs(h: int, z) -> None:
    _check(load().tsfde_rhs(h, _dev_ptr(z)), "tsfde_rhs")


def tsfde_matvec(h: int, y, z) -> None:
    _check(load().tsfde_matvec(h, _dev_ptr(y), _dev_ptr(z)), "tsfde_matvec")


def tsfde_precond_apply(h: int, r, y) -> int:
    return _check(load().tsfde_precond_apply(h, _dev_ptr(r), _dev_ptr(y)), "tsfde_precond_apply",
                  allow_not_converged=True)


def tsfde_matvec_transpose(h: int, lam, z) -> None:
    _check(load().tsfde_matvec_transpose(h, _dev_ptr(lam), _dev_ptr(z)), "tsfde_matvec_transpose")


def tsfde_precond_apply_transpose(h: int, r, lam) -> int:
    return _check(load().tsfde_precond_apply_transpose(h, _dev_ptr(r), _dev_ptr(lam)),
                  "tsfde_precond_apply_transpose", allow_not_converged=True)


def _info_dict(status: int, info: TsfdeInfo) -> dict:
    return dict(status=status, iters=info.iters, restarts=info.restarts, converged=bool(info.converged),
                relres_est=info.relres_est, relres_true=info.relres_true, seconds=info.seconds,
                precond_failures=info.precond_failures)


def tsfde_adjoint(h: int, y, ybar, lam=None, dmu=None, dgamma2=None, want_alpha: bool = True) -> dict:
    """A^T lam = ybar and the misfit gradients (arrays: float64 [U], [U], [U], [N], [S*N], host or
    device; lam / dmu / dgamma2 may be None).  Returns the adjoint solve's info plus "dalpha"."""
    info = TsfdeInfo()
    da = c_double(0.0)
    want_alpha = want_alpha and y is not None
    status = load().tsfde_adjoint(h, _ptr(y) if y is not None else None, _ptr(ybar),
                                  _ptr(lam) if lam is not None else None,
                                  ctypes.byref(da) if want_alpha else None,
                                  _ptr(dmu) if dmu is not None else None,
                                  _ptr(dgamma2) if dgamma2 is not None else None, ctypes.byref(info))
    _check(status, "tsfde_adjoint", allow_not_converged=True)
    out = _info_dict(status, info)
    out["dalpha"] = da.value if want_alpha else None
    return out


def tsfde_direct_solve(h: int, v, f=None, F=None) -> int:
    """v [S*N] <- the direct problem's levels for the source q(t) f(x) (f [N]) or F [S*N]."""
    if (f is None) == (F is None):
        raise ValueError("give exactly one of f, F")
    return _check(load().tsfde_direct_solve(h, _ptr(f) if f is not None else None,
                                            _ptr(F) if F is not None else None, _ptr(v)),
                  "tsfde_direct_solve", allow_not_converged=True)


def tsfde_solve(h: int, z, y) -> dict:
    """A y = z for a given z by the handle's preconditioned GMRES; y: initial guess in, solution out."""
    info = TsfdeInfo()
    status = load().tsfde_solve(h, _ptr(z), _ptr(y), ctypes.byref(info))
    _check(status, "tsfde_solve", allow_not_converged=True)
    return _info_dict(status, info)


def tsfde_spectral_bidiag(h: int, which: int, k: int, u0):
    """Golub-Kahan bidiagonalisation of M = A (which 0) or P^-1 A (1): returns (alpha, beta)."""
    alpha = np.zeros(k)
    beta = np.zeros(k)
    _check(load().tsfde_spectral_bidiag(h, which, k, _ptr(u0), alpha.ctypes.data_as(POINTER(c_double)),
                                        beta.ctypes.data_as(POINTER(c_double))), "tsfde_spectral_bidiag")
    return alpha, beta


def tsfde_spectral_arnoldi(h: int, which: int, k: int, v0):
    """Arnoldi on M = A (which 0) or P^-1 A (1): returns (H [(k+1) x k], steps)."""
    H = np.zeros((k, k + 1))   # column-major (k+1) x k: row i of this array is column i
    steps = ctypes.c_int(0)
    _check(load().tsfde_spectral_arnoldi(h, which, k, _ptr(v0), H.ctypes.data_as(POINTER(c_double)),
                                         ctypes.byref(steps)), "tsfde_spectral_arnoldi")
    return H.T.copy(), steps.value


def _ptr_array(vals):
    arr = (c_void_p * len(vals))()
    for i, v in enumerate(vals):
        arr[i] = v
    return arr


def tsfde_precond_apply_batch(handles, rs, ys) -> int:
    """y_i = P_i^-1 r_i for all handles in one launch (CUDA tensors)."""
    k = len(handles)
    status = load().tsfde_precond_apply_batch(k, _ptr_array(handles), _ptr_array([_dev_ptr(r) for r in rs]),
                                              _ptr_array([_dev_ptr(y) for y in ys]))
    return _check(status, "tsfde_precond_apply_batch", allow_not_converged=True)


def tsfde_gmres_solve_batch(handles, ys) -> list:
    """Solve every instance in lockstep, preconditioner applications batched; ys: [U_i] float64,
    host or device.  Returns the infos as dicts."""
    k = len(handles)
    infos = (TsfdeInfo * k)()
    status = load().tsfde_gmres_solve_batch(k, _ptr_array(handles), _ptr_array([_ptr(y) for y in ys]), infos)
    _check(status, "tsfde_gmres_solve_batch", allow_not_converged=True)
    return [_info_dict(status if status < 0 else (0 if infos[i].converged else 1), infos[i]) for i in range(k)]


def tsfde_gmres_solve(h: int, y, history_cap: int = 0) -> dict:
    """Solve in place; y: [U] float64, host or device.  Returns the info as a dict."""
    info = TsfdeInfo()
    hist = None
    if history_cap > 0:
        hist = (c_double * history_cap)()
        info.history = ctypes.cast(hist, POINTER(c_double))
        info.history_cap = history_cap
    status = load().tsfde_gmres_solve(h, _ptr(y), ctypes.byref(info))
    _check(status, "tsfde_gmres_solve", allow_not_converged=True)
    out = _info_dict(status, info)
    if hist is not None:
        out["history"] = [hist[i] for i in range(info.history_len)]
    return out


def tsfde_matvec_1d_noalloc(n: int, S: int, length: float, T: float, beta: float, omega: float, alpha: float,
                            gamma1, gamma2, q, y, z, stream: int | None = None) -> None:
    """z = A y for d = 1 with no device allocation (all arrays CUDA tensors)."""
    st = c_void_p(stream if stream is not None else _current_stream())
    _check(load().tsfde_matvec_1d_noalloc(n, S, length, T, beta, omega, alpha, _dev_ptr(gamma1), _dev_ptr(gamma2),
                                          _dev_ptr(q), _dev_ptr(y), _dev_ptr(z), st),
           "tsfde_matvec_1d_noalloc", "tsfde_matvec_transpose", "tsfde_precond_apply_transpose",
           "tsfde_adjoint", "tsfde_precond_apply_batch", "tsfde_gmres_solve_batch", "tsfde_direct_solve",
           "tsfde_spectral_bidiag", "tsfde_spectral_arnoldi", "tsfde_solve")


def tsfde_profile(h: int, enable) -> None:
    """enable: False/0 off, True/1 event timing, 2 event timing + timeline."""
    _check(load().tsfde_profile(h, int(enable)), "tsfde_profile")


def tsfde_profile_read(h: int) -> dict:
    st = TsfdeProfileStats()
    _check(load().tsfde_profile_read(h, ctypes.byref(st)), "tsfde_profile_read")
    out = {}
    for name, _ in TsfdeProfileStats._fields_:
        v = getattr(st, name)
        if name in ("phase_ms", "phase_count"):
            v = list(v)
        elif name == "batch_graph_error":
            v = v.decode(errors="replace")
        out[name] = v
    return out


def tsfde_device_bytes(h: int) -> int:
    return int(load().tsfde_device_bytes(h))


def tsfde_destroy(h: int) -> None:
    if h:
        load().tsfde_destroy(h)


def _current_stream() -> int:
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


class Solver:
    """Owns one handle; built from a workload object (``workloads.Workload``) or keywords."""

    def __init__(self, w, opts: TsfdeOpts | None = None, stream: int | None = None):
        self.d = len(w.ns)
        self.n = int(w.ns[0])
        self.S = int(w.S)
        self.N = self.n ** self.d
        self.U = (self.S + 1) * self.N
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
                for a in (w.gamma1, w.gamma2, w.q, w.rho, w.mu)]
        self.handle = tsfde_setup(self.d, self.n, float(w.length), self.S, float(w.T), float(w.beta),
                                  float(w.omega), float(w.alpha), *arrs, opts=opts, stream=stream)

    def rhs(self, z):
        tsfde_rhs(self.handle, z)

    def matvec(self, y, z):
        tsfde_matvec(self.handle, y, z)

    def precond_apply(self, r, y):
        return tsfde_precond_apply(self.handle, r, y)

    def solve(self, y, history_cap: int = 0) -> dict:
        return tsfde_gmres_solve(self.handle, y, history_cap)

    def solve_rhs(self, z, y) -> dict:
        return tsfde_solve(self.handle, z, y)

    def direct_solve(self, v, f=None, F=None):
        return tsfde_direct_solve(self.handle, v, f=f, F=F)

    def matvec_transpose(self, lam, z):
        tsfde_matvec_transpose(self.handle, lam, z)

    def precond_apply_transpose(self, r, lam):
        return tsfde_precond_apply_transpose(self.handle, r, lam)

    def adjoint(self, y, ybar, lam=None, dmu=None, dgamma2=None) -> dict:
        return tsfde_adjoint(self.handle, y, ybar, lam, dmu, dgamma2)

    def profile(self, enable):
        tsfde_profile(self.handle, enable)

    def profile_read(self) -> dict:
        return tsfde_profile_read(self.handle)

    def set_opts(self, opts: TsfdeOpts):
        tsfde_set_opts(self.handle, opts)

    def close(self):
        if self.handle:
            tsfde_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
