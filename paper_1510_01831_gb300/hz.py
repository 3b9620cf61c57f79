"""Thin ctypes binding of libhz (include/hz.h): argument marshalling only.

Every function keeps the C name.  Arrays are numpy complex128 (host pointers)
or, for contexts created with ``device_ptrs=True``, contiguous torch
complex128 CUDA tensors (device pointers).  Statuses other than HZ_OK raise
:class:`HzError`; HZ_ENOTCONV is reported through the returned stats instead
(``stats.converged == False``) because the best iterate is still written.

The library must have been built (``paper_1510_01831_gb300.build.build()``);
loading fails loudly otherwise -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

HZ_OK, HZ_EINVAL, HZ_ENOMEM, HZ_ECUDA, HZ_ESTATE, HZ_ENOTCONV, HZ_ETIMEOUT, HZ_ESINGULAR = range(8)
HZ_FP64, HZ_MIXED = 0, 1
HZ_PGS, HZ_PJAC, HZ_PNONE = 0, 1, 2
HZ_GMRES, HZ_BICGSTAB = 0, 1
HZ_INNER_LU, HZ_INNER_NESTED = 0, 1
STATUS_NAMES = ["HZ_OK", "HZ_EINVAL", "HZ_ENOMEM", "HZ_ECUDA", "HZ_ESTATE", "HZ_ENOTCONV", "HZ_ETIMEOUT",
                "HZ_ESINGULAR"]

# every entry point declared in include/hz.h
EXPORTS = ["hz_default_opts", "hz_setup", "hz_factor", "hz_update_model", "hz_solve", "hz_solve_group", "hz_gradient", "hz_adjoint", "hz_traces", "hz_reconstruct", "hz_cell_solve",
           "hz_layer_green", "hz_apply_M", "hz_precond", "hz_residual", "hz_residual_noalloc",
           "hz_check_timeout", "hz_set_device_ptrs", "hz_set_time_kernels", "hz_device_bytes", "hz_destroy", "hz_last_error"]


class HzError(RuntimeError):
    def __init__(self, status: int, msg: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")
        self.status = status


class HzOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("precond", ctypes.c_int), ("restart", ctypes.c_int),
                ("max_it", ctypes.c_int), ("tol", ctypes.c_double), ("refine_tol", ctypes.c_double),
                ("max_refine", ctypes.c_int), ("pml_C", ctypes.c_double),
                ("layer_rows", ctypes.POINTER(ctypes.c_int)), ("cell_cols", ctypes.POINTER(ctypes.c_int)),
                ("device_ptrs", ctypes.c_int), ("stream", ctypes.c_void_p), ("time_kernels", ctypes.c_int),
                ("krylov", ctypes.c_int), ("autotune", ctypes.c_int), ("tensor_cores", ctypes.c_int),
                ("rhs_lanes", ctypes.c_int), ("wait_ms", ctypes.c_double), ("inner", ctypes.c_int),
                ("compress", ctypes.c_double), ("inner_tol", ctypes.c_double)]


class HzStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("refinements", ctypes.c_int), ("gmres_resid", ctypes.c_double),
                ("resid", ctypes.c_double), ("t_total_ms", ctypes.c_double), ("t_local_ms", ctypes.c_double),
                ("t_gmres_ms", ctypes.c_double), ("t_recon_ms", ctypes.c_double), ("t_resid_ms", ctypes.c_double),
                ("gpu_launches", ctypes.c_int), ("kt_launches", ctypes.c_int * 3), ("kt_ms", ctypes.c_double * 3),
                ("kt_bytes", ctypes.c_double * 3), ("kt_flops", ctypes.c_double * 3),
                ("inner_iterations", ctypes.c_int), ("compress_rank", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        for k in ("kt_launches", "kt_ms", "kt_bytes", "kt_flops"):
            d[k] = list(d[k])
        d["converged"] = getattr(self, "converged", True)
        return d


_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load libhz.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libhz is not built ({path} missing); run paper_1510_01831_gb300.build.build()")
            L = ctypes.CDLL(path)
            vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            P = ctypes.POINTER
            L.hz_default_opts.argtypes = [P(HzOpts)]
            L.hz_default_opts.restype = None
            L.hz_setup.argtypes = [P(vp), vp, i, i, d, d, i, i, i, P(HzOpts)]
            L.hz_factor.argtypes = [vp]
            L.hz_update_model.argtypes = [vp, vp, P(i)]
            L.hz_solve.argtypes = [vp, vp, i, vp, P(HzStats)]
            L.hz_solve_group.argtypes = [P(vp), i, P(vp), i, P(vp), P(HzStats)]
            L.hz_gradient.argtypes = [vp, vp, i, vp, vp, i, P(d), vp, vp, P(HzStats)]
            L.hz_adjoint.argtypes = [vp, vp, vp, i, vp, vp, P(HzStats)]
            L.hz_traces.argtypes = [vp, vp, i, vp]
            L.hz_reconstruct.argtypes = [vp, vp, vp, i, vp]
            L.hz_cell_solve.argtypes = [vp, i, i, vp, i, vp]
            L.hz_layer_green.argtypes = [vp, i, vp, i, i, vp]
            L.hz_apply_M.argtypes = [vp, vp, i, vp]
            L.hz_precond.argtypes = [vp, i, vp, i, vp]
            L.hz_residual.argtypes = [vp, vp, vp, i, vp]
            L.hz_residual_noalloc.argtypes = [vp, vp, vp, i, vp]
            L.hz_residual_noalloc.restype = ctypes.c_int
            L.hz_check_timeout.argtypes = [vp]
            L.hz_check_timeout.restype = ctypes.c_int
            L.hz_set_device_ptrs.argtypes = [vp, i]
            L.hz_set_device_ptrs.restype = ctypes.c_int
            L.hz_set_time_kernels.argtypes = [vp, i]
            L.hz_set_time_kernels.restype = ctypes.c_int
            L.hz_device_bytes.argtypes = [vp]
            L.hz_device_bytes.restype = ctypes.c_longlong
            L.hz_destroy.argtypes = [vp]
            L.hz_destroy.restype = None
            L.hz_last_error.argtypes = [vp]
            L.hz_last_error.restype = ctypes.c_char_p
            for name in ("hz_setup", "hz_factor", "hz_solve", "hz_solve_group", "hz_gradient", "hz_adjoint", "hz_traces", "hz_reconstruct", "hz_cell_solve", "hz_layer_green",
                         "hz_apply_M", "hz_precond", "hz_residual"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def _check(st: int, ctx) -> None:
    if st != HZ_OK:
        msg = load().hz_last_error(ctx).decode(errors="replace")
        raise HzError(st, msg)


def _ptr(a, device: bool):
    """Data pointer of a numpy array (host) or torch tensor (device)."""
    if device:
        if not hasattr(a, "data_ptr") or not a.is_cuda or not a.is_contiguous():
            raise TypeError("device_ptrs context expects contiguous CUDA tensors")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or not a.flags.c_contiguous:
        raise TypeError("host context expects C-contiguous numpy arrays")
    return ctypes.c_void_p(a.ctypes.data)


def hz_default_opts() -> HzOpts:
    o = HzOpts()
    load().hz_default_opts(ctypes.byref(o))
    return o


class Context:
    """Owns one hz_ctx (one medium, one frequency)."""

    def __init__(self, m, n_x, n_z, omega, h, n_pml, L, C, precision=HZ_FP64, precond=HZ_PGS, tol=0.0,
                 refine_tol=1e-8, max_refine=6, restart=30, max_it=200, pml_C=0.0, layer_rows=None,
                 cell_cols=None, device_ptrs=False, stream=None, time_kernels=False, tensor_cores=True, krylov=0, autotune=False,
                 rhs_lanes=1, wait_ms=0.0, inner=HZ_INNER_LU, inner_tol=0.0, compress=None):
        self._ctx = None
        lib = load()
        o = hz_default_opts()
        o.precision, o.precond, o.tol = precision, precond, tol
        o.refine_tol, o.max_refine, o.restart, o.max_it, o.pml_C = refine_tol, max_refine, restart, max_it, pml_C
        self._rows = self._cols = None
        if layer_rows is not None:
            self._rows = (ctypes.c_int * L)(*[int(v) for v in layer_rows])
            o.layer_rows = ctypes.cast(self._rows, ctypes.POINTER(ctypes.c_int))
        if cell_cols is not None:
            self._cols = (ctypes.c_int * C)(*[int(v) for v in cell_cols])
            o.cell_cols = ctypes.cast(self._cols, ctypes.POINTER(ctypes.c_int))
        o.device_ptrs = 1 if device_ptrs else 0
        o.stream = ctypes.c_void_p(stream) if stream else None
        o.time_kernels = 1 if time_kernels else 0
        o.tensor_cores = int(tensor_cores)  # False / True / 2 (cell solves and batched products)
        o.krylov = int(krylov)
        o.autotune = 1 if autotune else 0
        o.rhs_lanes = int(rhs_lanes)
        if wait_ms > 0:
            o.wait_ms = float(wait_ms)
        o.inner = int(inner)
        o.inner_tol = float(inner_tol)
        if compress is not None:  # None: the library default (1e-8 in mixed precision, dense in FP64)
            o.compress = float(compress)
        m = np.ascontiguousarray(m, dtype=np.float64)
        if m.shape != (n_z + 2 * n_pml, n_x + 2 * n_pml):
            raise ValueError(f"m has shape {m.shape}, expected {(n_z + 2 * n_pml, n_x + 2 * n_pml)}")
        h_ = ctypes.c_void_p()
        st = lib.hz_setup(ctypes.byref(h_), m.ctypes.data, n_x, n_z, float(omega), float(h), n_pml, L, C,
                          ctypes.byref(o))
        _check(st, None)
        self._ctx = h_
        self.device = bool(device_ptrs)
        self.n_x, self.n_z, self.n_pml, self.L, self.C = n_x, n_z, n_pml, L, C
        self.NX, self.NZ = n_x + 2 * n_pml, n_z + 2 * n_pml
        self.rows = list(layer_rows) if layer_rows is not None else [
            n_z // L + (1 if i < n_z % L else 0) for i in range(L)]
        self.cols = list(cell_cols) if cell_cols is not None else [
            n_x // C + (1 if i < n_x % C else 0) for i in range(C)]

    # -- lifecycle --
    def close(self):
        if self._ctx is not None:
            load().hz_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _alloc(self, shape, dtype=np.complex128, like=None):
        if self.device:
            import torch
            tdt = torch.complex128 if dtype == np.complex128 else torch.float64
            dev = like.device if like is not None else torch.device("cuda")
            return torch.empty(shape, dtype=tdt, device=dev)
        return np.empty(shape, dtype=dtype)

    def _in(self, a, dtype=np.complex128):
        if self.device:
            return a.contiguous()
        return np.ascontiguousarray(a, dtype=dtype)

    # -- calls --
    def hz_factor(self):
        _check(load().hz_factor(self._ctx), self._ctx)

    def hz_update_model(self, m_new) -> int:
        """Replace the medium (host array, extended grid) and re-factor the touched layers; returns their count."""
        m_new = np.ascontiguousarray(m_new, dtype=np.float64)
        if m_new.shape != (self.NZ, self.NX):
            raise ValueError(f"m_new has shape {m_new.shape}, expected {(self.NZ, self.NX)}")
        n = ctypes.c_int(0)
        _check(load().hz_update_model(self._ctx, m_new.ctypes.data, ctypes.byref(n)), self._ctx)
        return n.value

    def hz_solve(self, f, u=None):
        f = self._in(f)
        B = f.shape[0]
        if u is None:
            u = self._alloc(tuple(f.shape), like=f)
        s = HzStats()
        st = load().hz_solve(self._ctx, _ptr(f, self.device), B, _ptr(u, self.device), ctypes.byref(s))
        if st == HZ_ENOTCONV:
            s.converged = False
        else:
            _check(st, self._ctx)
        return u, s

    def hz_gradient(self, f, d, rec_idx):
        f = self._in(f)
        d = self._in(d)
        rec = self._in(rec_idx, np.int32) if not self.device else rec_idx.contiguous()
        B = f.shape[0]
        grad = self._alloc((self.NZ, self.NX), np.float64, like=f)
        u = self._alloc(tuple(f.shape), like=f)
        J = ctypes.c_double()
        s = HzStats()
        st = load().hz_gradient(self._ctx, _ptr(f, self.device), B, _ptr(d, self.device), _ptr(rec, self.device),
                                int(rec.shape[0]), ctypes.byref(J), _ptr(grad, self.device), _ptr(u, self.device),
                                ctypes.byref(s))
        if st == HZ_ENOTCONV:
            s.converged = False
        else:
            _check(st, self._ctx)
        return J.value, grad, u, s

    def hz_adjoint(self, u, gu, want_grad_f=True):
        """(grad_m, grad_f, stats) for a loss with gradient gu = dL/dRe(u) + i dL/dIm(u)."""
        u, gu = self._in(u), self._in(gu)
        B = u.shape[0]
        grad_m = self._alloc((self.NZ, self.NX), np.float64, like=u)
        grad_f = self._alloc(tuple(u.shape), like=u) if want_grad_f else None
        s = HzStats()
        st = load().hz_adjoint(self._ctx, _ptr(u, self.device), _ptr(gu, self.device), B, _ptr(grad_m, self.device),
                               _ptr(grad_f, self.device) if grad_f is not None else None, ctypes.byref(s))
        if st == HZ_ENOTCONV:
            s.converged = False
        else:
            _check(st, self._ctx)
        return grad_m, grad_f, s

    def hz_traces(self, u):
        """Interface traces [B][L-1][2][NX] of the fields u [B][NZ][NX] (a solve's checkpoint)."""
        u = self._in(u)
        B = u.shape[0]
        tr = self._alloc((B, self.L - 1, 2, self.NX), like=u)
        _check(load().hz_traces(self._ctx, _ptr(u, self.device), B, _ptr(tr, self.device)), self._ctx)
        return tr

    def hz_reconstruct(self, f, tr):
        """Fields u [B][NZ][NX] from their sources f and interface traces tr."""
        f, tr = self._in(f), self._in(tr)
        B = f.shape[0]
        u = self._alloc(tuple(f.shape), like=f)
        _check(load().hz_reconstruct(self._ctx, _ptr(f, self.device), _ptr(tr, self.device), B,
                                     _ptr(u, self.device)), self._ctx)
        return u

    def hz_cell_solve(self, l, c, g):
        g = self._in(g)
        x = self._alloc(tuple(g.shape), like=g)
        _check(load().hz_cell_solve(self._ctx, l, c, _ptr(g, self.device), g.shape[0], _ptr(x, self.device)),
               self._ctx)
        return x

    def hz_layer_green(self, l, tr, in_mask=3):
        tr = self._in(tr)
        out = self._alloc(tuple(tr.shape), like=tr)
        _check(load().hz_layer_green(self._ctx, l, _ptr(tr, self.device), in_mask, tr.shape[0],
                                     _ptr(out, self.device)), self._ctx)
        return out

    def hz_apply_M(self, x):
        x = self._in(x)
        y = self._alloc(tuple(x.shape), like=x)
        _check(load().hz_apply_M(self._ctx, _ptr(x, self.device), x.shape[0], _ptr(y, self.device)), self._ctx)
        return y

    def hz_precond(self, which, x):
        x = self._in(x)
        y = self._alloc(tuple(x.shape), like=x)
        _check(load().hz_precond(self._ctx, which, _ptr(x, self.device), x.shape[0], _ptr(y, self.device)),
               self._ctx)
        return y

    def hz_residual(self, u, f):
        u, f = self._in(u), self._in(f)
        B = f.shape[0]
        r = self._alloc((B,), np.float64, like=f)
        _check(load().hz_residual(self._ctx, _ptr(u, self.device), _ptr(f, self.device), B, _ptr(r, self.device)),
               self._ctx)
        return r

    def hz_residual_noalloc(self, u, f, res):
        """Allocation-free residual: u, f, res must be CUDA tensors (res: float64 [B]).
        Enqueued on the context's stream; no device memory is allocated."""
        for a in (u, f, res):
            if not (hasattr(a, "data_ptr") and a.is_cuda and a.is_contiguous()):
                raise TypeError("hz_residual_noalloc expects contiguous CUDA tensors")
        _check(load().hz_residual_noalloc(self._ctx, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                          int(f.shape[0]), ctypes.c_void_p(res.data_ptr())), self._ctx)
        return res

    def hz_check_timeout(self) -> int:
        """Run the timeout check (a bounded device wait that nothing completes); returns
        the status (HZ_ETIMEOUT when the timeout path works) without raising."""
        return load().hz_check_timeout(self._ctx)

    def last_error(self) -> str:
        return load().hz_last_error(self._ctx).decode(errors="replace")

    def hz_set_device_ptrs(self, device: bool):
        _check(load().hz_set_device_ptrs(self._ctx, 1 if device else 0), self._ctx)
        self.device = bool(device)

    def hz_set_time_kernels(self, on: bool):
        _check(load().hz_set_time_kernels(self._ctx, 1 if on else 0), self._ctx)

    def hz_device_bytes(self) -> int:
        return int(load().hz_device_bytes(self._ctx))


def hz_solve_group(ctxs, fs, us=None):
    """Solve the G problems ctxs[i] H u_i = fs[i] together (one batch size B for
    all; each context on its own stream for overlap).  Returns (us, stats)."""
    G = len(ctxs)
    if G < 1 or len(fs) != G:
        raise ValueError("need one source array per context")
    fs = [c._in(f) for c, f in zip(ctxs, fs)]
    B = fs[0].shape[0]
    if any(f.shape[0] != B for f in fs):
        raise ValueError("every member needs the same batch size B")
    if us is None:
        us = [c._alloc(tuple(f.shape), like=f) for c, f in zip(ctxs, fs)]
    vp = ctypes.c_void_p
    hs = (vp * G)(*[c._ctx for c in ctxs])
    fp = (vp * G)(*[_ptr(f, c.device) for c, f in zip(ctxs, fs)])
    up = (vp * G)(*[_ptr(u, c.device) for c, u in zip(ctxs, us)])
    sts = (HzStats * G)()
    st = load().hz_solve_group(hs, G, fp, B, up, sts)
    stats = [sts[i] for i in range(G)]
    if st == HZ_ENOTCONV:
        for s in stats:
            s.converged = False
    else:
        _check(st, ctxs[0]._ctx)
    return us, stats
