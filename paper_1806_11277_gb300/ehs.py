"""Thin ctypes binding of libehs.so (include/ehs.h).

Argument marshalling only: every step of the solver runs in the CUDA
library.  Vectors are torch tensors on the GPU (complex128 or complex64) in
the slot layout of include/ehs.h, shaped (items, d+1, [n_z,] n_y, n_x);
the solves also accept host numpy arrays.  There is no CPU fallback: if the
library cannot be loaded, importing a Solver raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libehs.so")

EHS_C128, EHS_C64 = 0, 1
EHS_PRECOND_MG, EHS_PRECOND_DD = 0, 1
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_NOCONV", 5: "ERR_BREAKDOWN",
          6: "ERR_TIMEOUT", 7: "ERR_NONFINITE", 8: "ERR_UNSUPPORTED"}


class Problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double), ("omega", C.c_double),
                ("omegas", C.c_void_p), ("nmedia", C.c_int), ("lam", C.c_void_p), ("mu", C.c_void_p), ("rho", C.c_void_p),
                ("abl_cells", C.c_int), ("abl_max", C.c_double), ("gamma_add", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("levels", C.c_int), ("alpha", C.c_double), ("w", C.c_double * 8),
                ("wp_ratio", C.c_double), ("nu_pre", C.c_int), ("nu_post", C.c_int),
                ("cycle", C.c_int), ("restart", C.c_int), ("maxit", C.c_int), ("tol", C.c_double),
                ("precond", C.c_int), ("prec", C.c_int), ("nrhs", C.c_int), ("dd", C.c_int * 3),
                ("dd_overlap", C.c_int), ("dd_pad", C.c_int), ("dd_abl_max", C.c_double),
                ("coef_half", C.c_int),
                ("vanka_full", C.c_int),
                ("coarse_dd", C.c_int * 3),
                ("coarse_dd_overlap", C.c_int),
                ("coarse_fmt", C.c_int),
                ("coarse_persist", C.c_int),
                ("ortho", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("relres", C.c_double), ("converged", C.c_int)]


EXPORTS = ["ehs_default_opts", "ehs_create", "ehs_destroy", "ehs_op_apply", "ehs_smooth",
           "ehs_vcycle", "ehs_dd_precond", "ehs_fgmres_solve", "ehs_adjoint_solve", "ehs_items",
           "ehs_level_len", "ehs_level_dims", "ehs_sync", "ehs_kernel_launches", "ehs_last_error",
           "ehs_fine_smooth_noalloc", "ehs_gradient", "ehs_coarse_solve", "ehs_coarse_dims",
           "ehs_coarse_local_apply", "ehs_coarse_local_add", "ehs_residual_restrict", "ehs_prolong_add"]

_lib = None


def load(path=LIB_PATH):
    """Load libehs.so and declare its signatures; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libehs.so not built at {path}: run __graft_entry__.build() "
                           "or python -m paper_1806_11277_gb300.build")
    lib = C.CDLL(path)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    lib.ehs_default_opts.argtypes = [C.POINTER(Opts)]
    lib.ehs_default_opts.restype = None
    lib.ehs_create.argtypes = [C.POINTER(Problem), C.POINTER(Opts), vp, C.POINTER(vp)]
    lib.ehs_destroy.argtypes = [vp]
    lib.ehs_op_apply.argtypes = [vp, i, i, i, vp, vp]
    lib.ehs_smooth.argtypes = [vp, i, i, i, vp, vp]
    lib.ehs_vcycle.argtypes = [vp, i, vp, vp]
    lib.ehs_dd_precond.argtypes = [vp, i, vp, vp]
    lib.ehs_fgmres_solve.argtypes = [vp, vp, vp, C.POINTER(SolveInfo)]
    lib.ehs_adjoint_solve.argtypes = [vp, vp, vp, C.POINTER(SolveInfo)]
    lib.ehs_items.argtypes = [vp]
    lib.ehs_level_len.argtypes = [vp, i]
    lib.ehs_level_len.restype = C.c_longlong
    lib.ehs_level_dims.argtypes = [vp, i, C.POINTER(C.c_int * 3)]
    lib.ehs_sync.argtypes = [vp]
    lib.ehs_kernel_launches.argtypes = []
    lib.ehs_kernel_launches.restype = C.c_longlong
    lib.ehs_last_error.argtypes = [vp]
    lib.ehs_last_error.restype = C.c_char_p
    lib.ehs_fine_smooth_noalloc.argtypes = [C.POINTER(Problem), i, d, d, d, i, i, vp, vp, vp]
    lib.ehs_gradient.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.ehs_coarse_solve.argtypes = [vp, i, vp, vp]
    lib.ehs_coarse_dims.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), vp]
    lib.ehs_coarse_local_apply.argtypes = [vp, i, i, vp, vp]
    lib.ehs_coarse_local_add.argtypes = [vp, i, i, vp, vp]
    lib.ehs_residual_restrict.argtypes = [vp, i, i, vp, vp, vp]
    lib.ehs_prolong_add.argtypes = [vp, i, i, vp, vp]
    for name in EXPORTS:
        getattr(lib, name)
    _lib = lib
    return lib


class EhsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def default_opts(**kw):
    o = Opts()
    load().ehs_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "w":
            for j, x in enumerate(v):
                o.w[j] = x
        elif k in ("dd", "coarse_dd"):
            arr = getattr(o, k)
            for j, x in enumerate(v):
                arr[j] = x
        else:
            setattr(o, k, v)
    return o


def _ptr(t):
    if hasattr(t, "data_ptr"):
        assert t.is_contiguous()
        return C.c_void_p(t.data_ptr())
    assert isinstance(t, np.ndarray) and t.flags["C_CONTIGUOUS"]
    return C.c_void_p(t.ctypes.data)


class Solver:
    """One context: media, hierarchy and workspaces on the current CUDA device."""

    def __init__(self, lam, mu, rho, omega, h=1.0, abl_cells=10, abl_max=1.0,
                 gamma_add=0.01 * math.pi, opts=None, stream=None, **kw):
        """lam, mu, rho: arrays of shape (nmedia, [n_z,] n_y, n_x)."""
        lib = load()
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        if lam.ndim not in (3, 4) or lam.shape != mu.shape or lam.shape != rho.shape:
            raise ValueError("media must have shape (nmedia, [n_z,] n_y, n_x)")
        self.nmedia = lam.shape[0]
        self.shape = lam.shape[1:]
        self.dim = len(self.shape)
        p = Problem()
        p.dim = self.dim
        n = list(reversed(self.shape)) + [1] * (3 - self.dim)
        for k in range(3):
            p.n[k] = n[k]
        om = np.ascontiguousarray(np.broadcast_to(np.asarray(omega, dtype=np.float64), (self.nmedia,)))
        self._omegas = om
        p.h, p.omega, p.nmedia = h, float(om[0]), self.nmedia
        p.omegas = om.ctypes.data
        p.lam, p.mu, p.rho = lam.ctypes.data, mu.ctypes.data, rho.ctypes.data
        p.abl_cells, p.abl_max, p.gamma_add = abl_cells, abl_max, gamma_add
        self.opts = opts if opts is not None else default_opts(**kw)
        self.stream = stream
        sp = C.c_void_p(stream) if stream else None
        ctx = C.c_void_p()
        st = lib.ehs_create(C.byref(p), C.byref(self.opts), sp, C.byref(ctx))
        if st != 0:
            raise EhsError(st, lib.ehs_last_error(None).decode())
        self.ctx = ctx
        self.lib = lib
        self.items = lib.ehs_items(ctx)

    def _check(self, st):
        if st != 0:
            raise EhsError(st, self.lib.ehs_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.ehs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def level_shape(self, level):
        n = (C.c_int * 3)()
        self._check(self.lib.ehs_level_dims(self.ctx, level, C.byref(n)))
        dims = [n[0], n[1], n[2]][:self.dim]
        return (self.items, self.dim + 1) + tuple(reversed(dims))

    def op_apply(self, x, y, level=0, shifted=False, prec=None):
        prec = _prec_of(x) if prec is None else prec
        self._check(self.lib.ehs_op_apply(self.ctx, level, int(shifted), prec, _ptr(x), _ptr(y)))

    def smooth(self, b, x, level=0, nsweeps=1, prec=None):
        prec = _prec_of(x) if prec is None else prec
        self._check(self.lib.ehs_smooth(self.ctx, level, nsweeps, prec, _ptr(b), _ptr(x)))

    def vcycle(self, b, x, prec=None):
        prec = _prec_of(x) if prec is None else prec
        self._check(self.lib.ehs_vcycle(self.ctx, prec, _ptr(b), _ptr(x)))

    def residual_restrict(self, b, x, rc, level=0, prec=None):
        """rc = P_l^T (b - K_l x)."""
        prec = _prec_of(x) if prec is None else prec
        self._check(self.lib.ehs_residual_restrict(self.ctx, level, prec, _ptr(b), _ptr(x), _ptr(rc)))

    def prolong_add(self, ec, x, level=0, prec=None):
        """x += P_l ec."""
        prec = _prec_of(x) if prec is None else prec
        self._check(self.lib.ehs_prolong_add(self.ctx, level, prec, _ptr(ec), _ptr(x)))

    def coarse_solve(self, b, x, prec=None):
        prec = _prec_of(x) if prec is None else prec
        self._check(self.lib.ehs_coarse_solve(self.ctx, prec, _ptr(b), _ptr(x)))

    def coarse_dims(self):
        """(nsub, nloc, sizes) of the coarsest local solves (nsub = 1: exact solve)."""
        ns, nl = C.c_int(), C.c_int()
        self._check(self.lib.ehs_coarse_dims(self.ctx, C.byref(ns), C.byref(nl), None))
        sizes = (C.c_int * ns.value)()
        self._check(self.lib.ehs_coarse_dims(self.ctx, C.byref(ns), C.byref(nl), sizes))
        return ns.value, nl.value, list(sizes)

    def coarse_local_apply(self, colour, r_loc, z_loc, prec=None):
        prec = _prec_of(z_loc) if prec is None else prec
        self._check(self.lib.ehs_coarse_local_apply(self.ctx, prec, colour, _ptr(r_loc), _ptr(z_loc)))

    def coarse_local_add(self, colour, r_loc, x, prec=None):
        prec = _prec_of(x) if prec is None else prec
        self._check(self.lib.ehs_coarse_local_add(self.ctx, prec, colour, _ptr(r_loc), _ptr(x)))

    def dd_precond(self, r, z, prec=EHS_C64):
        self._check(self.lib.ehs_dd_precond(self.ctx, prec, _ptr(r), _ptr(z)))

    def _solve(self, fn, q, u, raise_noconv):
        info = (SolveInfo * self.items)()
        st = fn(self.ctx, _ptr(q), _ptr(u), info)
        if st != 0 and (raise_noconv or st not in (4, 5)):
            self._check(st)
        return [dict(iters=i.iters, relres=i.relres, converged=bool(i.converged)) for i in info]

    def fgmres_solve(self, q, u, raise_noconv=True):
        return self._solve(self.lib.ehs_fgmres_solve, q, u, raise_noconv)

    def adjoint_solve(self, g, w, raise_noconv=True):
        return self._solve(self.lib.ehs_adjoint_solve, g, w, raise_noconv)

    def gradient(self, x, w, out=None):
        """(g_lambda, g_mu, g_rho): -Re(w^H dK/dm x) per cell, summed over each medium's rhs.
        x, w: complex128 CUDA tensors of all items; returns float64 CUDA tensors
        of shape (nmedia, *grid)."""
        import torch
        if out is None:
            out = [torch.empty((self.nmedia,) + tuple(self.shape), dtype=torch.float64, device=x.device)
                   for _ in range(3)]
        self._check(self.lib.ehs_gradient(self.ctx, _ptr(x), _ptr(w), _ptr(out[0]), _ptr(out[1]),
                                          _ptr(out[2])))
        return out

    def sync(self):
        self._check(self.lib.ehs_sync(self.ctx))


def _prec_of(t):
    name = str(t.dtype)
    if "complex64" in name:
        return EHS_C64
    if "complex128" in name:
        return EHS_C128
    raise TypeError(f"vectors must be complex64 or complex128, got {t.dtype}")


def kernel_launches():
    return int(load().ehs_kernel_launches())


def solver_for(medium, **kw):
    """Solver for a synth.Medium (or a list of media of one shape)."""
    meds = medium if isinstance(medium, (list, tuple)) else [medium]
    m0 = meds[0]
    lam = np.stack([m.lam for m in meds])
    mu = np.stack([m.mu for m in meds])
    rho = np.stack([m.rho for m in meds])
    return Solver(lam, mu, rho, [m.omega for m in meds], m0.h, m0.abl_cells, **kw)
