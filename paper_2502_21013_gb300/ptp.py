"""ctypes binding of libptp.so (argument marshalling only).

Every method maps one-to-one onto a C entry point of include/ptp.h with the
same name minus the `ptp_` prefix.  Host-pointer entry points take and return
numpy arrays; `_dev` entry points take torch CUDA tensors (device memory and
the stream come from PyTorch; all arithmetic runs in the library's kernels).
There is no fallback: if libptp.so is missing or fails to load, importing
this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libptp.so")

PTP_OK, PTP_EINVAL, PTP_ECUDA, PTP_ENOTCONV, PTP_ENAN, PTP_ESTATE, PTP_ENOMEM = 0, -1, -2, -3, -4, -5, -6
PTP_FP64, PTP_MIXED = 0, 1
PTP_PREC_JACOBI, PTP_PREC_GMG = 0, 1
PTP_COARSE_VCYCLES, PTP_COARSE_DFT = 0, 1
PTP_BATCH_MERGED, PTP_BATCH_BRANCHES, PTP_BATCH_AUTO = 0, 1, 2


class Opts(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double), ("max_outer", ctypes.c_int), ("precision", ctypes.c_int),
        ("time_levels", ctypes.c_int), ("coarse_steps", ctypes.c_int), ("vcycles", ctypes.c_int),
        ("pre_smooth", ctypes.c_int), ("post_smooth", ctypes.c_int), ("omega_t", ctypes.c_double),
        ("pcg_iters", ctypes.c_int), ("spatial_prec", ctypes.c_int), ("gmg_smooth", ctypes.c_int),
        ("gmg_omega", ctypes.c_double), ("coarse_tol", ctypes.c_double), ("coarse_max_it", ctypes.c_int),
        ("use_graph", ctypes.c_int), ("check_every", ctypes.c_int), ("coarse_cycles", ctypes.c_int),
        ("coarse_solver", ctypes.c_int), ("dft_max_it", ctypes.c_int), ("init_tol", ctypes.c_double),
        ("init_static", ctypes.c_int), ("newton_eta", ctypes.c_double), ("krylov_dim", ctypes.c_int),
        ("stencil", ctypes.c_int), ("k1_fused", ctypes.c_int),
        ("coarse_direct", ctypes.c_int), ("fuse_coarse", ctypes.c_int),
        ("fuse_update", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [
        ("outer_iterations", ctypes.c_int), ("converged", ctypes.c_int), ("res0", ctypes.c_double),
        ("res_final", ctypes.c_double), ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
        ("residual_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int64), ("time_levels", ctypes.c_int),
        ("spatial_levels", ctypes.c_int), ("init_ms", ctypes.c_double), ("init_iterations", ctypes.c_int),
        ("inner_iterations", ctypes.c_int), ("omega_t", ctypes.c_double), ("post_smooth", ctypes.c_int),
        ("kappa_min", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PtpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ptp error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2502_21013_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    pI, pD = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    sig = {
        "ptp_default_opts": (None, [ctypes.POINTER(Opts)]),
        "ptp_version": (ctypes.c_char_p, []),
        "ptp_abi_sizes": (None, [ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
        "ptp_create": (I, [ctypes.POINTER(P), I]),
        "ptp_destroy": (None, [P]),
        "ptp_last_error": (ctypes.c_char_p, [P]),
        "ptp_set_stream": (I, [P, P]),
        "ptp_set_mesh": (I, [P, I, P, I, P, P]),
        "ptp_set_structured": (I, [P, I, I, D, D, D, D]),
        "ptp_set_materials": (I, [P, P, P, D, D, D, D]),
        "ptp_set_sources": (I, [P, I, P, P, P]),
        "ptp_set_time": (I, [P, D, I]),
        "ptp_setup": (I, [P, ctypes.POINTER(Opts)]),
        "ptp_sizes": (I, [P, pI, pI, pI, pI]),
        "ptp_info": (I, [P, ctypes.POINTER(ctypes.c_int64), I]),
        "ptp_source": (I, [P, P]),
        "ptp_source_dev": (I, [P, P]),
        "ptp_residual": (I, [P, P, P, pD]),
        "ptp_residual_dev": (I, [P, P, P, pD]),
        "ptp_residual_noalloc_dev": (I, [P, P, P, P]),
        "ptp_apply_shifted_dev": (I, [P, I, P, P]),
        "ptp_apply_shifted_f32_dev": (I, [P, I, P, P]),
        "ptp_periodic_apply_dev": (I, [P, I, P, P]),
        "ptp_periodic_residual_f32_dev": (I, [P, I, P, P, P]),
        "ptp_spatial_solve_dev": (I, [P, I, P, P, D, I, pI]),
        "ptp_spatial_solve_f32_dev": (I, [P, I, P, P, D, I, pI]),
        "ptp_periodic_solve_dev": (I, [P, ctypes.POINTER(Opts), P, P, I, pD]),
        "ptp_solve": (I, [P, ctypes.POINTER(Opts), P, P, ctypes.POINTER(Stats)]),
        "ptp_solve_dev": (I, [P, ctypes.POINTER(Opts), P, P, ctypes.POINTER(Stats)]),
        "ptp_static_solve": (I, [P, ctypes.POINTER(Opts), P, ctypes.POINTER(Stats)]),
        "ptp_set_law_exp": (I, [P, P]),
        "ptp_newton_solve": (I, [P, ctypes.POINTER(Opts), P, P, ctypes.POINTER(Stats)]),
        "ptp_newton_solve_dev": (I, [P, ctypes.POINTER(Opts), P, P, ctypes.POINTER(Stats)]),
        "ptp_jacobian_apply_dev": (I, [P, P, P, P]),
        "ptp_set_khat": (I, [P, P]),
        "ptp_static_solve_dev": (I, [P, ctypes.POINTER(Opts), P, ctypes.POINTER(Stats)]),
        "ptp_loss_dev": (I, [P, P, pD]),
        "ptp_autotune": (I, [P, pI, pD]),
        "ptp_batch_create": (I, [ctypes.POINTER(P), I]),
        "ptp_batch_destroy": (None, [P]),
        "ptp_batch_last_error": (ctypes.c_char_p, [P]),
        "ptp_batch_add": (I, [P, P]),
        "ptp_batch_size": (I, [P]),
        "ptp_batch_solve": (I, [P, ctypes.POINTER(Opts), P, pI]),
        "ptp_batch_result_dev": (I, [P, I, P]),
        "ptp_batch_set_mode": (I, [P, I]),
        "ptp_batch_set_groups": (I, [P, I]),
        "ptp_batch_plan_info": (I, [P, ctypes.POINTER(ctypes.c_int64), pI, pI]),
        "ptp_adjoint_gradient_dev": (I, [P, ctypes.POINTER(Opts), P, pD, pD, pD, P, ctypes.POINTER(Stats)]),
        "ptp_adjoint_gradient": (I, [P, ctypes.POINTER(Opts), P, pD, pD, pD, P, ctypes.POINTER(Stats)]),
        "ptp_probe_fma": (I, [I, I, pD]),
        "ptp_probe_recip_dev": (I, [I, P, P, ctypes.c_int64, P]),
        "ptp_time_cycle_rho": (I, [pI, I, D, I, I, D, pD]),
        "ptp_choose_time_smoother": (I, [pI, I, D, I, I, D, pI, pD, pD]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    so, ss = ctypes.c_size_t(), ctypes.c_size_t()
    lib.ptp_abi_sizes(ctypes.byref(so), ctypes.byref(ss))
    if so.value != ctypes.sizeof(Opts) or ss.value != ctypes.sizeof(Stats):
        raise ImportError(f"libptp.so struct sizes ({so.value}, {ss.value}) do not match the binding "
                          f"({ctypes.sizeof(Opts)}, {ctypes.sizeof(Stats)}): rebuild the library")
    return lib


lib = _load()

EXPORTED = [
    "ptp_default_opts", "ptp_version", "ptp_abi_sizes", "ptp_create", "ptp_destroy", "ptp_last_error", "ptp_set_stream",
    "ptp_set_mesh", "ptp_set_structured", "ptp_set_materials", "ptp_set_law_exp", "ptp_set_khat",
    "ptp_set_sources", "ptp_set_time",
    "ptp_setup", "ptp_sizes", "ptp_info", "ptp_source", "ptp_source_dev", "ptp_residual", "ptp_residual_dev",
    "ptp_residual_noalloc_dev",
    "ptp_apply_shifted_dev", "ptp_apply_shifted_f32_dev", "ptp_periodic_apply_dev", "ptp_periodic_residual_f32_dev", "ptp_spatial_solve_dev",
    "ptp_spatial_solve_f32_dev", "ptp_periodic_solve_dev", "ptp_solve", "ptp_solve_dev",
    "ptp_static_solve", "ptp_static_solve_dev", "ptp_newton_solve", "ptp_newton_solve_dev",
    "ptp_jacobian_apply_dev",
    "ptp_loss_dev", "ptp_adjoint_gradient_dev", "ptp_adjoint_gradient", "ptp_autotune",
    "ptp_batch_create", "ptp_batch_destroy", "ptp_batch_last_error", "ptp_batch_add", "ptp_batch_size",
    "ptp_batch_solve", "ptp_batch_result_dev", "ptp_batch_set_mode", "ptp_batch_set_groups", "ptp_batch_plan_info", "ptp_probe_fma", "ptp_probe_recip_dev",
    "ptp_time_cycle_rho", "ptp_choose_time_smoother",
]


def time_cycle_rho(Nl, kappa0, pre, post, omega):
    """Model spectral radius of the V(pre, post) time cycle (ptp_time_cycle_rho; host only)."""
    arr = (ctypes.c_int * len(Nl))(*[int(v) for v in Nl])
    r = ctypes.c_double()
    rc = lib.ptp_time_cycle_rho(arr, len(Nl), float(kappa0), int(pre), int(post), float(omega), ctypes.byref(r))
    if rc != PTP_OK:
        raise PtpError(rc, "ptp_time_cycle_rho: bad arguments")
    return r.value


def choose_time_smoother(Nl, kappa_min, pre=1, post=-1, omega=0.0):
    """(post, omega, rho) that the automatic time smoother takes (ptp_choose_time_smoother; host only)."""
    arr = (ctypes.c_int * len(Nl))(*[int(v) for v in Nl])
    q, w, r = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    rc = lib.ptp_choose_time_smoother(arr, len(Nl), float(kappa_min), int(pre), int(post), float(omega),
                                      ctypes.byref(q), ctypes.byref(w), ctypes.byref(r))
    if rc != PTP_OK:
        raise PtpError(rc, "ptp_choose_time_smoother: bad arguments")
    return q.value, w.value, r.value


def probe_fma(device=0, fp64=True):
    """Measured FMA rate of the device in TFLOP/s (ptp_probe_fma)."""
    r = ctypes.c_double()
    rc = lib.ptp_probe_fma(int(device), 1 if fp64 else 0, ctypes.byref(r))
    if rc != PTP_OK:
        raise PtpError(rc, "ptp_probe_fma failed")
    return r.value


def probe_recip_dev(d, out, stream=None):
    """out = 1/d by the residual kernels' Newton reciprocal (ptp_probe_recip_dev)."""
    rc = lib.ptp_probe_recip_dev(d.device.index or 0, _dev_ptr(d, "float64"), _dev_ptr(out, "float64", d.numel()),
                                 d.numel(), ctypes.c_void_p(stream or 0))
    if rc != PTP_OK:
        raise PtpError(rc, "ptp_probe_recip_dev failed")


def default_opts(**kw) -> Opts:
    o = Opts()
    lib.ptp_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _np(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t, dtype_name, count=None):
    """Device address of a contiguous CUDA tensor of the given dtype; `count`
    (when known) is the number of elements the library reads or writes."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("_dev entry points take CUDA tensors")
    if count is not None and t.numel() != count:
        raise PtpError(PTP_EINVAL, f"expected a tensor of {count} elements, got {t.numel()}")
    if not t.is_cuda:
        raise TypeError("_dev entry points take CUDA tensors")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"expected {dtype_name}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """One solver context (ptp_create ... ptp_destroy)."""

    def __init__(self, device: int = 0):
        self._h = ctypes.c_void_p()
        rc = lib.ptp_create(ctypes.byref(self._h), int(device))
        if rc != PTP_OK:
            raise PtpError(rc, "ptp_create failed")
        self.device = device
        self._n_tri = None    # triangles of the mesh last set, for the array-length checks
        self._sizes = None    # (n_free, N, n_tri, time levels) after a successful ptp_setup

    def _count(self, level=0):
        """Values of a space-time block on time level `level` (N >> level
        steps: every coarsening halves an even step count), or None before
        setup or for a level out of range (the library then reports the error)."""
        if self._sizes is None:
            return None
        n, N, _, levels = self._sizes
        level = int(level)
        if not 0 <= level < levels:
            return None
        return n * (N >> level)

    def _nN(self):
        """(n_free, N) of the set-up problem."""
        n, N, _, _ = self._sizes if self._sizes is not None else self.sizes()
        return n, N

    def _host_in(self, a, name):
        a, pa = _np(a, np.float64)
        count = self._count()
        if count is not None and a.size != count:
            raise PtpError(PTP_EINVAL, f"{name}: expected {count} values, got {a.size}")
        return a, pa

    def _need_len(self, name, a, shape):
        """The per-element arrays are read with the mesh's triangle count by
        the library, so their lengths are checked here first."""
        if tuple(a.shape) != tuple(shape):
            raise PtpError(PTP_EINVAL, f"{name}: expected shape {tuple(shape)}, got {tuple(a.shape)}")

    def close(self):
        if self._h:
            lib.ptp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != PTP_OK and rc not in allow:
            raise PtpError(rc, lib.ptp_last_error(self._h).decode())
        return rc

    # ---- problem definition ----
    def set_stream(self, stream_ptr: int | None):
        self._sizes = None
        return self._check(lib.ptp_set_stream(self._h, ctypes.c_void_p(stream_ptr or 0)))

    def set_mesh(self, xy, tri, dirichlet):
        self._sizes = None
        xy, pxy = _np(xy, np.float64)
        tri, ptri = _np(tri, np.int32)
        dr, pdr = _np(dirichlet, np.uint8)
        if xy.ndim != 2 or xy.shape[1] != 2 or tri.ndim != 2 or tri.shape[1] != 3:
            raise PtpError(PTP_EINVAL, "set_mesh: xy must be (n_nodes, 2) and tri (n_tri, 3)")
        self._need_len("set_mesh dirichlet", dr, (xy.shape[0],))
        rc = self._check(lib.ptp_set_mesh(self._h, xy.shape[0], pxy, tri.shape[0], ptri, pdr))
        self._n_tri = tri.shape[0]
        return rc

    def set_structured(self, nx, ny, x0, y0, x1, y1):
        self._sizes = None
        rc = self._check(lib.ptp_set_structured(self._h, nx, ny, x0, y0, x1, y1))
        self._n_tri = 2 * (int(nx) - 1) * (int(ny) - 1)
        return rc

    def set_materials(self, sigma_e, nonlinear_e, nu_min, nu_max, s_sat, nu_linear):
        self._sizes = None
        s, ps = _np(sigma_e, np.float64)
        nl, pnl = _np(nonlinear_e, np.uint8)
        if self._n_tri is not None:
            self._need_len("set_materials sigma_e", s, (self._n_tri,))
            self._need_len("set_materials nonlinear_e", nl, (self._n_tri,))
        return self._check(lib.ptp_set_materials(self._h, ps, pnl, nu_min, nu_max, s_sat, nu_linear))

    def set_law_exp(self, abcd):
        self._sizes = None
        if abcd is None:
            return self._check(lib.ptp_set_law_exp(self._h, None))
        a, pa = _np(abcd, np.float64)
        if self._n_tri is not None:
            self._need_len("set_law_exp abcd", a, (self._n_tri, 4))
        return self._check(lib.ptp_set_law_exp(self._h, pa))

    def set_khat(self, khat_e):
        self._sizes = None
        if khat_e is None:
            return self._check(lib.ptp_set_khat(self._h, None))
        k, pk = _np(khat_e, np.float64)
        if self._n_tri is not None:
            self._need_len("set_khat khat_e", k, (self._n_tri,))
        return self._check(lib.ptp_set_khat(self._h, pk))

    def set_sources(self, coil_of_elem, amp, phase):
        self._sizes = None
        c, pc = _np(coil_of_elem, np.int32)
        a, pa = _np(amp, np.float64)
        ph, pph = _np(phase, np.float64)
        if a.ndim != 1:
            raise PtpError(PTP_EINVAL, "set_sources: amp must be one-dimensional")
        self._need_len("set_sources phase", ph, a.shape)
        if self._n_tri is not None and a.shape[0] > 0:
            self._need_len("set_sources coil_of_elem", c, (self._n_tri,))
        return self._check(lib.ptp_set_sources(self._h, a.shape[0], pc, pa, pph))

    def set_time(self, T, N):
        self._sizes = None
        return self._check(lib.ptp_set_time(self._h, float(T), int(N)))

    def setup(self, opts: Opts | None = None):
        self.opts = opts if opts is not None else default_opts()
        self._sizes = None
        rc = self._check(lib.ptp_setup(self._h, ctypes.byref(self.opts)))
        self._sizes = self.sizes()
        return rc

    def sizes(self):
        v = [ctypes.c_int() for _ in range(4)]
        self._check(lib.ptp_sizes(self._h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    INFO_KEYS = ("n_free", "N", "n_tri", "n_iron", "iron_incidences", "lin_nnz", "mass_nnz", "op_nnz",
                 "spatial_levels", "time_levels", "n_coils", "row_block", "st_tile", "st_waves")

    def autotune(self):
        b, us = ctypes.c_int(), ctypes.c_double()
        self._check(lib.ptp_autotune(self._h, ctypes.byref(b), ctypes.byref(us)))
        return b.value, us.value

    def info(self):
        buf = (ctypes.c_int64 * len(self.INFO_KEYS))()
        m = lib.ptp_info(self._h, buf, len(self.INFO_KEYS))
        if m < 0:
            self._check(m)
        return {k: int(buf[i]) for i, k in enumerate(self.INFO_KEYS[:m])}

    # ---- hot path, host pointers ----
    @staticmethod
    def _check_out(U, count):
        """A caller's output array must be a writable C-contiguous float64
        block of `count` values: the library writes it in place."""
        if (not isinstance(U, np.ndarray) or U.dtype != np.float64 or not U.flags.c_contiguous
                or not U.flags.writeable or U.size != count):
            raise PtpError(PTP_EINVAL, f"output: expected a writable C-contiguous float64 array of {count} values")

    def source(self):
        n, N = self._nN()
        F = np.empty((n, N))
        self._check(lib.ptp_source(self._h, F.ctypes.data_as(ctypes.c_void_p)))
        return F

    def residual(self, U):
        U, pU = self._host_in(U, "residual U")
        R = np.empty_like(U)
        nrm = ctypes.c_double()
        self._check(lib.ptp_residual(self._h, pU, R.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nrm)))
        return R, nrm.value

    def solve(self, opts: Opts | None = None, U0=None, U_out=None):
        n, N = self._nN()
        o = opts if opts is not None else self.opts
        U = U_out if U_out is not None else np.empty((n, N))
        self._check_out(U, n * N)
        p0 = None
        if U0 is not None:
            U0, p0 = self._host_in(U0, "solve U0")
        st = Stats()
        rc = lib.ptp_solve(self._h, ctypes.byref(o), p0, U.ctypes.data_as(ctypes.c_void_p), ctypes.byref(st))
        self._check(rc, allow=(PTP_ENOTCONV,))
        return U, st, rc

    def static_solve(self, opts: Opts | None = None, U_out=None):
        """Initialisation of Section 4: U with K(u^n) = f^n for every step (host array)."""
        n, N = self._nN()
        o = opts if opts is not None else self.opts
        U = U_out if U_out is not None else np.empty((n, N))
        self._check_out(U, n * N)
        st = Stats()
        rc = lib.ptp_static_solve(self._h, ctypes.byref(o), U.ctypes.data_as(ctypes.c_void_p), ctypes.byref(st))
        self._check(rc, allow=(PTP_ENOTCONV,))
        return U, st, rc

    # ---- hot path, device pointers (torch CUDA tensors) ----
    def source_dev(self, F):
        return self._check(lib.ptp_source_dev(self._h, _dev_ptr(F, "float64", self._count())))

    def residual_dev(self, U, R=None, want_norm=True):
        """R = F - A(U) on the device; returns ||R|| (synchronising) or None."""
        nrm = ctypes.c_double()
        n = self._count()
        pR = _dev_ptr(R, "float64", n) if R is not None else None
        self._check(lib.ptp_residual_dev(self._h, _dev_ptr(U, "float64", n), pR,
                                         ctypes.byref(nrm) if want_norm else None))
        return nrm.value if want_norm else None

    def apply_shifted_dev(self, level, X, Y):
        n = self._count(level)
        if X.dtype.is_floating_point and X.element_size() == 4:
            return self._check(lib.ptp_apply_shifted_f32_dev(self._h, level, _dev_ptr(X, "float32", n),
                                                             _dev_ptr(Y, "float32", n)))
        return self._check(lib.ptp_apply_shifted_dev(self._h, level, _dev_ptr(X, "float64", n),
                                                     _dev_ptr(Y, "float64", n)))

    def periodic_apply_dev(self, level, X, Y):
        n = self._count(level)
        return self._check(lib.ptp_periodic_apply_dev(self._h, level, _dev_ptr(X, "float64", n),
                                                      _dev_ptr(Y, "float64", n)))

    def periodic_residual_f32_dev(self, level, X, B, R):
        n = self._count(level)
        return self._check(lib.ptp_periodic_residual_f32_dev(self._h, level, _dev_ptr(X, "float32", n),
                                                             _dev_ptr(B, "float32", n), _dev_ptr(R, "float32", n)))

    def spatial_solve_dev(self, level, B, X, tol, max_it):
        it = ctypes.c_int()
        n = self._count(level)
        if B.element_size() == 4:
            self._check(lib.ptp_spatial_solve_f32_dev(self._h, level, _dev_ptr(B, "float32", n),
                                                      _dev_ptr(X, "float32", n), tol, max_it, ctypes.byref(it)))
        else:
            self._check(lib.ptp_spatial_solve_dev(self._h, level, _dev_ptr(B, "float64", n),
                                                  _dev_ptr(X, "float64", n), tol, max_it, ctypes.byref(it)))
        return it.value

    def periodic_solve_dev(self, B, X, cycles, opts: Opts | None = None):
        rel = ctypes.c_double()
        o = ctypes.byref(opts) if opts is not None else None
        n = self._count()
        self._check(lib.ptp_periodic_solve_dev(self._h, o, _dev_ptr(B, "float64", n), _dev_ptr(X, "float64", n),
                                               int(cycles), ctypes.byref(rel)))
        return rel.value

    def solve_dev(self, U, opts: Opts | None = None, U0=None):
        o = opts if opts is not None else self.opts
        st = Stats()
        n = self._count()
        p0 = _dev_ptr(U0, "float64", n) if U0 is not None else None
        rc = lib.ptp_solve_dev(self._h, ctypes.byref(o), p0, _dev_ptr(U, "float64", n), ctypes.byref(st))
        self._check(rc, allow=(PTP_ENOTCONV,))
        return st, rc


def _newton_solve(ctx, opts=None, U0=None):
    """Newton's method (M2); returns (U, stats, rc) with U a host array."""
    n, N = ctx._nN()
    o = opts if opts is not None else ctx.opts
    U = np.empty((n, N))
    p0 = None
    if U0 is not None:
        U0, p0 = ctx._host_in(U0, "newton_solve U0")
    st = Stats()
    rc = lib.ptp_newton_solve(ctx._h, ctypes.byref(o), p0, U.ctypes.data_as(ctypes.c_void_p), ctypes.byref(st))
    ctx._check(rc, allow=(PTP_ENOTCONV,))
    return U, st, rc


def _newton_solve_dev(ctx, U, opts=None, U0=None):
    o = opts if opts is not None else ctx.opts
    st = Stats()
    n = ctx._count()
    p0 = _dev_ptr(U0, "float64", n) if U0 is not None else None
    rc = lib.ptp_newton_solve_dev(ctx._h, ctypes.byref(o), p0, _dev_ptr(U, "float64", n), ctypes.byref(st))
    ctx._check(rc, allow=(PTP_ENOTCONV,))
    return st, rc


def _jacobian_apply_dev(ctx, U, V, Y):
    n = ctx._count()
    return ctx._check(lib.ptp_jacobian_apply_dev(ctx._h, _dev_ptr(U, "float64", n), _dev_ptr(V, "float64", n),
                                                 _dev_ptr(Y, "float64", n)))


Context.newton_solve = _newton_solve
Context.newton_solve_dev = _newton_solve_dev
Context.jacobian_apply_dev = _jacobian_apply_dev


def _static_solve_dev(ctx, U, opts=None):
    o = opts if opts is not None else ctx.opts
    st = Stats()
    rc = lib.ptp_static_solve_dev(ctx._h, ctypes.byref(o), _dev_ptr(U, "float64", ctx._count()), ctypes.byref(st))
    ctx._check(rc, allow=(PTP_ENOTCONV,))
    return st, rc


Context.static_solve_dev = _static_solve_dev


def _loss_dev(ctx, U):
    J = ctypes.c_double()
    ctx._check(lib.ptp_loss_dev(ctx._h, _dev_ptr(U, "float64", ctx._count()), ctypes.byref(J)))
    return J.value


def _adjoint_gradient_dev(ctx, U, opts=None):
    """(J, dJ/damp [n_coils], dJ/d(nu_min, nu_max, s_sat) [3], dJ/dsigma [n_tri] (CUDA), stats, rc)."""
    import torch
    info = ctx.info()
    J = ctypes.c_double()
    damp = (ctypes.c_double * max(1, info["n_coils"]))()
    dnu = (ctypes.c_double * 3)()
    dsig = torch.empty(info["n_tri"], dtype=torch.float64, device=U.device)
    st = Stats()
    o = opts if opts is not None else ctx.opts
    rc = lib.ptp_adjoint_gradient_dev(ctx._h, ctypes.byref(o), _dev_ptr(U, "float64", ctx._count()),
                                      ctypes.byref(J), damp, dnu,
                                      _dev_ptr(dsig, "float64"), ctypes.byref(st))
    ctx._check(rc, allow=(PTP_ENOTCONV,))
    return J.value, [damp[k] for k in range(info["n_coils"])], [dnu[k] for k in range(3)], dsig, st, rc


Context.loss_dev = _loss_dev
Context.adjoint_gradient_dev = _adjoint_gradient_dev


class Batch:
    """Many set-up contexts advanced by one graph launch per fixed-point step
    (ptp_batch_*).  Keeps references to its contexts."""

    def __init__(self, device: int = 0):
        self._h = ctypes.c_void_p()
        rc = lib.ptp_batch_create(ctypes.byref(self._h), int(device))
        if rc != PTP_OK:
            raise PtpError(rc, "ptp_batch_create failed")
        self.contexts = []

    def _check(self, rc, allow=()):
        if rc != PTP_OK and rc not in allow:
            raise PtpError(rc, lib.ptp_batch_last_error(self._h).decode())
        return rc

    def add(self, ctx: Context):
        self._check(lib.ptp_batch_add(self._h, ctx._h))
        self.contexts.append(ctx)

    def solve(self, opts: Opts):
        K = len(self.contexts)
        stats = (Stats * K)()
        nconv = ctypes.c_int()
        rc = lib.ptp_batch_solve(self._h, ctypes.byref(opts), stats, ctypes.byref(nconv))
        self._check(rc, allow=(PTP_ENOTCONV,))
        return [stats[i] for i in range(K)], nconv.value, rc

    def set_mode(self, mode):
        self._check(lib.ptp_batch_set_mode(self._h, int(mode)))

    def set_groups(self, groups):
        self._check(lib.ptp_batch_set_groups(self._h, int(groups)))

    def plan_info(self):
        """(kernels per batched step, instances merged, merged launches)."""
        lps, mi, ml = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
        self._check(lib.ptp_batch_plan_info(self._h, ctypes.byref(lps), ctypes.byref(mi), ctypes.byref(ml)))
        return lps.value, mi.value, ml.value

    def result_dev(self, i, U):
        i = int(i)
        n = self.contexts[i]._count() if 0 <= i < len(self.contexts) else None
        return self._check(lib.ptp_batch_result_dev(self._h, i, _dev_ptr(U, "float64", n)))

    def close(self):
        if self._h:
            lib.ptp_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def load_problem(ctx: Context, prob, structured: bool = True):
    """Pass a problem description (mesh, materials, sources, time) to the
    library.  `prob` is any object with the attributes of workloads.Problem.
    When `structured` and the problem carries its grid, the library builds the
    same uniform mesh itself and enables geometric multigrid."""
    if structured and getattr(prob, "grid", None) is not None:
        ctx.set_structured(*prob.grid)
    else:
        ctx.set_mesh(prob.xy, prob.tri, prob.dirichlet)
    ctx.set_materials(prob.sigma_e, prob.nonlinear_e, prob.nu_min, prob.nu_max, prob.s_sat, prob.nu_linear)
    ctx.set_law_exp(getattr(prob, "law_abcd", None))
    ctx.set_khat(getattr(prob, "khat_e", None))
    ctx.set_sources(prob.coil_of_elem, prob.amp, prob.phase)
    ctx.set_time(prob.T, prob.N)
