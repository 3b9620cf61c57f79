"""CPU FP64 oracle for the nested polarized-traces Helmholtz solver.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_1510_01831_gb300``) and never imports it.

Layers of the oracle:

* ``hz_oracle.c`` (compiled on first use with gcc): the discrete operator of
  Appendix A and a banded LU with partial pivoting.  ``solve`` is the plain
  definition u = H^{-1} f that the nested method reproduces exactly
  (Sections 2-3: the SIE and polarized reformulations are exact).
* this module: the decomposition into layers and cells, the local Green's
  integrals of Section 2.3 written through the identity of Appendix C, the
  polarized system of Section 3 and its preconditioners, the inner nested
  polarized traces of Section 4.2 (a layer solved over its cells by the same
  functions on its swapped-axes box), the block-LU sweeps of the inner SIE and
  their compressed (low-rank) form (Sections 4.2.2, 4.3), and the misfit
  gradient.  Every operator is applied through explicit local solves; no
  operator is precomputed or compressed.

Readings of the paper taken where it is ambiguous (each is listed with its
reason in the design notes of the repository):

R2  PML nodes and profile: nodes x_k = k h, interior k = 1..n, PML
    k = -p+1..0 and n+1..n+p, Dirichlet beyond; sigma from the distance past
    [0, (n+1) h].
R3  Local problems (layers, cells) are boxes with their own p-point PML
    built by the same rule, with m extended by its boundary row/column.
R4  Green's integrals are defined by the forcing terms of Appendix C,
    eq. (pde_GRF_real): no h factors.
R5  Interface k carries (a = last row of layer k, b = first row of layer k+1).
R6  The extended system jump_1..jump_4 with jump_4 read as defining the
    down-going trace at row n+1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hz_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libhz_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile hz_oracle.c into oracle/_build/libhz_oracle.so (gcc, OpenMP)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    cmd = ["gcc", "-O3", "-fPIC", "-shared", "-fopenmp", "-fcx-limited-range",
           "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Box(ctypes.Structure):
    _fields_ = [("nxi", ctypes.c_int), ("nzi", ctypes.c_int), ("p", ctypes.c_int),
                ("omega", ctypes.c_double), ("h", ctypes.c_double), ("C", ctypes.c_double),
                ("m", ctypes.POINTER(ctypes.c_double))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Box)
            lib.hzo_factor.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
            lib.hzo_factor.restype = ctypes.c_void_p
            lib.hzo_factor_ordered.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            lib.hzo_factor_ordered.restype = ctypes.c_void_p
            lib.hzo_solve.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
            lib.hzo_solve.restype = ctypes.c_int
            lib.hzo_free.argtypes = [ctypes.c_void_p]
            lib.hzo_apply.argtypes = [P, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            lib.hzo_entry.argtypes = [P, ctypes.c_long, ctypes.c_long,
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            lib.hzo_alpha.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]
            lib.hzo_stencil.argtypes = [P, ctypes.c_void_p]
            _lib = lib
    return _lib


def default_pml_C(m: np.ndarray) -> float:
    """sigma amplitude giving exp(-2C/(3c)) = 1e-6 continuum reflection at c_max (R2)."""
    c_max = float(np.max(1.0 / np.sqrt(m)))
    return 1.5 * c_max * np.log(1e6)


class Box:
    """A rectangular problem: interior nxi x nzi, p-point PML on all sides (Appendix A)."""

    def __init__(self, m: np.ndarray, nxi: int, nzi: int, p: int, omega: float, h: float, C: float):
        self.m = np.ascontiguousarray(m, dtype=np.float64)
        assert self.m.shape == (nzi + 2 * p, nxi + 2 * p), (self.m.shape, nxi, nzi, p)
        self.nxi, self.nzi, self.p = nxi, nzi, p
        self.omega, self.h, self.C = float(omega), float(h), float(C)
        self._c = _Box(nxi, nzi, p, self.omega, self.h, self.C,
                       self.m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))

    @property
    def shape(self):
        return self.m.shape

    @property
    def N(self):
        return self.m.size

    def apply(self, u: np.ndarray) -> np.ndarray:
        """H u for u of shape (..., NZ, NX)."""
        lib = _load()
        u = np.ascontiguousarray(u, dtype=np.complex128)
        lead = u.shape[:-2]
        uu = u.reshape(-1, self.N)
        out = np.empty_like(uu)
        lib.hzo_apply(ctypes.byref(self._c), uu.shape[0], uu.ctypes.data, out.ctypes.data)
        return out.reshape(lead + self.shape)

    def entry(self, row: int, col: int) -> complex:
        lib = _load()
        re, im = ctypes.c_double(), ctypes.c_double()
        lib.hzo_entry(ctypes.byref(self._c), row, col, ctypes.byref(re), ctypes.byref(im))
        return complex(re.value, im.value)

    def alpha(self, axis: int, pos) -> np.ndarray:
        """alpha_x (axis 0) or alpha_z (axis 1) at array positions `pos` (may be +-0.5)."""
        lib = _load()
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        re = np.empty_like(pos)
        im = np.empty_like(pos)
        lib.hzo_alpha(ctypes.byref(self._c), axis, pos.size, pos.ctypes.data,
                      re.ctypes.data, im.ctypes.data)
        return re + 1j * im

    def dense(self) -> np.ndarray:
        """The full matrix (tiny boxes only), built from single entries."""
        N = self.N
        A = np.zeros((N, N), dtype=np.complex128)
        eye = np.zeros((1,) + self.shape, dtype=np.complex128)
        for j in range(N):
            eye.reshape(-1)[:] = 0
            eye.reshape(-1)[j] = 1
            A[:, j] = self.apply(eye).reshape(-1)
        return A

    def factor(self, order: int = 0) -> "Factor":
        """order 0: smaller band width; 1: x fastest; 2: z fastest."""
        return Factor(self, order)

    def stencil(self) -> np.ndarray:
        """The five coefficient planes (5, NZ, NX) of the operator: couplings to
        (z-1, x), (z, x-1), the node itself, (z, x+1), (z+1, x); zero beyond
        the extended grid."""
        out = np.empty((5,) + self.shape, dtype=np.complex128)
        _load().hzo_stencil(ctypes.byref(self._c), out.ctypes.data)
        return out

    def factor_rows(self, keep_every: int = 1, rows: int | None = None) -> "RowBlockFactor":
        """Block-tridiagonal elimination over grid rows (see RowBlockFactor)."""
        return RowBlockFactor(self, keep_every, rows)


class Factor:
    """Banded LU (partial pivoting) of a Box's operator."""

    def __init__(self, box: Box, order: int = 0):
        lib = _load()
        self.box = box
        info = ctypes.c_int(0)
        self._h = lib.hzo_factor_ordered(ctypes.byref(box._c), order, ctypes.byref(info))
        if not self._h:
            raise MemoryError("oracle factor: allocation failed")
        if info.value != 0:
            raise np.linalg.LinAlgError(f"oracle factor: zero pivot at column {info.value - 1}")

    def solve(self, f: np.ndarray, trans: bool = False) -> np.ndarray:
        """H^{-1} f (or H^{-T} f) for f of shape (..., NZ, NX)."""
        lib = _load()
        f = np.array(f, dtype=np.complex128, order="C", copy=True)
        lead = f.shape[:-2]
        ff = f.reshape(-1, self.box.N)
        rc = lib.hzo_solve(self._h, ff.shape[0], ff.ctypes.data, 1 if trans else 0)
        if rc != 0:
            raise MemoryError("oracle solve: allocation failed")
        return ff.reshape(lead + self.box.shape)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().hzo_free(h)
            self._h = None


class RowBlockFactor:
    """u = H^{-1} f by block-tridiagonal elimination over the grid rows, the
    direct solve for grids whose pivoted band LU does not fit in memory.

    With the unknowns of one grid row z as a block, the operator of Appendix A
    is block tridiagonal: H = tridiag(A_z, D_z, C_z) with D_z the tridiagonal
    (x-coupling) block of row z and A_z, C_z the diagonal couplings to rows
    z-1 and z+1.  Block Gaussian elimination without block pivoting:
        S_0 = D_0,   S_z = D_z - A_z S_{z-1}^{-1} C_{z-1},
        y_0 = f_0,   y_z = f_z - A_z S_{z-1}^{-1} y_{z-1},
        u_last = S_last^{-1} y_last,   u_z = S_z^{-1} (y_z - C_z u_{z+1}),
    each Schur block S_z factored by LAPACK's LU with partial pivoting
    (scipy.linalg.lu_factor, a library primitive).  Storage: NZ factors of
    NX x NX.  keep_every = k > 1 keeps every k-th factor only and recomputes
    the others a segment at a time when a solve needs them (the same
    arithmetic from the same inputs; 1/k of the memory, up to three times the
    factorization work).  rows = r eliminates only the leading r grid rows,
    i.e. solves the leading principal r x r block system of H (every row of
    the elimination costs the same, so this times a bounded sample of it).
    """

    def __init__(self, box: Box, keep_every: int = 1, rows: int | None = None):
        import scipy.linalg as sl
        self._sl = sl
        self.box = box
        st = box.stencil()
        self.NZ, self.NX = box.shape
        if rows is not None:
            self.NZ = max(1, min(int(rows), self.NZ))
        self.A, self.Cp = st[0], st[4]          # couplings of row z to rows z-1 and z+1
        self.lo, self.di, self.up = st[1], st[2], st[3]
        self.k = max(1, int(keep_every))
        self.lu = [None] * self.NZ
        f = None
        for z in range(self.NZ):
            f = sl.lu_factor(self._S(z, f), check_finite=False)
            if z % self.k == 0:
                self.lu[z] = f

    def _S(self, z, f_prev):
        """Schur block S_z from the LU factors of S_{z-1}."""
        NX = self.NX
        S = np.zeros((NX, NX), dtype=np.complex128)
        i = np.arange(NX)
        S[i, i] = self.di[z]
        S[i[1:], i[:-1]] = self.lo[z][1:]
        S[i[:-1], i[1:]] = self.up[z][:-1]
        if z > 0:
            X = self._sl.lu_solve(f_prev, np.diag(self.Cp[z - 1]), check_finite=False)
            S -= self.A[z][:, None] * X
        return S

    def _segment(self, z0):
        """Factors of rows z0 .. z0+k-1, recomputed from the kept factor of row z0."""
        out = {z0: self.lu[z0]}
        f = self.lu[z0]
        for z in range(z0 + 1, min(z0 + self.k, self.NZ)):
            f = self._sl.lu_factor(self._S(z, f), check_finite=False)
            out[z] = f
        return out

    def solve(self, f: np.ndarray) -> np.ndarray:
        """H^{-1} f for f of shape (..., NZ, NX)."""
        sl, NZ, NX, k = self._sl, self.NZ, self.NX, self.k
        lead = f.shape[:-2]
        F = np.asarray(f, dtype=np.complex128).reshape((-1,) + f.shape[-2:])[:, :NZ, :]
        Y = np.empty((NZ, NX, F.shape[0]), dtype=np.complex128)
        seg = {}

        def fac(z):
            nonlocal seg
            if k == 1:
                return self.lu[z]
            if z not in seg:
                seg = self._segment((z // k) * k)
            return seg[z]
        for z in range(NZ):
            y = F[:, z, :].T.copy()
            if z > 0:
                y -= self.A[z][:, None] * sl.lu_solve(fac(z - 1), Y[z - 1], check_finite=False)
            Y[z] = y
        U = np.empty_like(Y)
        for z in range(NZ - 1, -1, -1):
            r = Y[z] if z == NZ - 1 else Y[z] - self.Cp[z][:, None] * U[z + 1]
            U[z] = sl.lu_solve(fac(z), r, check_finite=False)
        return np.ascontiguousarray(np.transpose(U, (2, 0, 1))).reshape(lead + (NZ, NX))


def relative_residual(box: Box, u: np.ndarray, f: np.ndarray) -> np.ndarray:
    """||H u - f||_2 / ||f||_2 per right-hand side (plain definition)."""
    r = box.apply(u) - f
    lead = f.shape[:-2]
    r = r.reshape(lead + (-1,))
    ff = f.reshape(lead + (-1,))
    return np.linalg.norm(r, axis=-1) / np.linalg.norm(ff, axis=-1)


# --------------------------------------------------------------------------
# Decomposition (Sections 2 and 4): L layers of interior rows, C cells of
# interior columns; every local problem is a Box with its own PML (R3).
# --------------------------------------------------------------------------

class Decomposition:
    def __init__(self, m, n_x, n_z, p, omega, h, C_pml, L, C, layer_rows=None, cell_cols=None):
        self.m = np.asarray(m, dtype=np.float64)
        self.n_x, self.n_z, self.p = n_x, n_z, p
        self.omega, self.h, self.C_pml = float(omega), float(h), float(C_pml)
        self.L, self.C = L, C
        self.rows = list(layer_rows) if layer_rows is not None else _split(n_z, L)
        self.cols = list(cell_cols) if cell_cols is not None else _split(n_x, C)
        assert sum(self.rows) == n_z and len(self.rows) == L
        assert sum(self.cols) == n_x and len(self.cols) == C
        self.s = np.concatenate([[0], np.cumsum(self.rows)]).astype(int)
        self.t = np.concatenate([[0], np.cumsum(self.cols)]).astype(int)
        self.NX, self.NZ = n_x + 2 * p, n_z + 2 * p
        self.box = Box(self.m, n_x, n_z, p, omega, h, C_pml)
        self._layer_fac = {}

    # R3: the layer's medium, extended by its first/last row into its own PML
    def layer_medium(self, l: int) -> np.ndarray:
        p, n = self.p, self.rows[l]
        idx = self.s[l] + np.arange(n + 2 * p)
        if l > 0:
            idx = np.maximum(idx, self.s[l] + p)
        if l < self.L - 1:
            idx = np.minimum(idx, self.s[l] + n + p - 1)
        return self.m[idx, :]

    def layer_box(self, l: int) -> Box:
        return Box(self.layer_medium(l), self.n_x, self.rows[l], self.p, self.omega, self.h, self.C_pml)

    def cell_medium(self, l: int, c: int) -> np.ndarray:
        p, w = self.p, self.cols[c]
        ml = self.layer_medium(l)
        idx = self.t[c] + np.arange(w + 2 * p)
        if c > 0:
            idx = np.maximum(idx, self.t[c] + p)
        if c < self.C - 1:
            idx = np.minimum(idx, self.t[c] + w + p - 1)
        return ml[:, idx]

    def cell_box(self, l: int, c: int) -> Box:
        return Box(self.cell_medium(l, c), self.cols[c], self.rows[l], self.p, self.omega, self.h, self.C_pml)

    def layer_factor(self, l: int) -> Factor:
        if l not in self._layer_fac:
            self._layer_fac[l] = self.layer_box(l).factor()
        return self._layer_fac[l]

    # array index of local row r (node number) in layer l's box
    def lrow(self, r: int) -> int:
        return r + self.p - 1

    # global array row index of layer l's local node row r
    def grow(self, l: int, r: int) -> int:
        return self.s[l] + r + self.p - 1

    def owned_rows(self, l: int):
        """Local array rows of layer l that belong to it in the global grid."""
        p, n = self.p, self.rows[l]
        lo = 0 if l == 0 else p
        hi = n + 2 * p if l == self.L - 1 else n + p
        return lo, hi

    # Appendix C forcing: sources on local rows 0,1,n,n+1 from traces at the
    # same rows: -d_n H_{n,n+1} u_{n+1} + d_{n+1} H_{n+1,n} u_n - d_1 H_{1,0} u_0 + d_0 H_{0,1} u_1
    def interface_source(self, l: int, t0, t1, tn, tn1) -> np.ndarray:
        box = self.layer_box(l)
        NX, n = self.NX, self.rows[l]
        shp = np.broadcast(t0, t1, tn, tn1).shape[:-1]
        g = np.zeros(shp + box.shape, dtype=np.complex128)
        r0, r1, rn, rn1 = self.lrow(0), self.lrow(1), self.lrow(n), self.lrow(n + 1)
        H01 = np.array([box.entry(r0 * NX + x, r1 * NX + x) for x in range(NX)])
        H10 = np.array([box.entry(r1 * NX + x, r0 * NX + x) for x in range(NX)])
        Hnn1 = np.array([box.entry(rn * NX + x, rn1 * NX + x) for x in range(NX)])
        Hn1n = np.array([box.entry(rn1 * NX + x, rn * NX + x) for x in range(NX)])
        g[..., r0, :] += H01 * t1
        g[..., r1, :] += -H10 * t0
        g[..., rn1, :] += Hn1n * tn
        g[..., rn, :] += -Hnn1 * tn1
        return g

    def layer_source(self, l: int, f: np.ndarray) -> np.ndarray:
        """f restricted to layer l (its owned rows), on the layer's box."""
        p, n = self.p, self.rows[l]
        g = np.zeros(f.shape[:-2] + (n + 2 * p, self.NX), dtype=np.complex128)
        lo, hi = self.owned_rows(l)
        g[..., lo:hi, :] = f[..., self.s[l] + lo:self.s[l] + hi, :]
        return g

    def green(self, l: int, t0, t1, tn, tn1, f=None, full=False):
        """Local Green's integrals of layer l (R4): the field of the Appendix C
        forcing built from traces at local rows (0, 1, n, n+1), plus the Newton
        potential of f if given.  Returns samples at rows (0, 1, n, n+1), shape
        (..., 4, NX), or the whole local field if full=True."""
        g = self.interface_source(l, t0, t1, tn, tn1)
        if f is not None:
            g = g + self.layer_source(l, f)
        v = self.layer_factor(l).solve(g)
        if full:
            return v
        n = self.rows[l]
        rows = [self.lrow(0), self.lrow(1), self.lrow(n), self.lrow(n + 1)]
        return v[..., rows, :]

    def traces(self, u: np.ndarray) -> np.ndarray:
        """Interface traces of a global field: (..., L-1, 2, NX) with (a, b) rows (R5)."""
        out = []
        for k in range(self.L - 1):
            a = self.grow(k, self.rows[k])
            out.append(np.stack([u[..., a, :], u[..., a + 1, :]], axis=-2))
        return np.stack(out, axis=-3)


def _split(n, parts):
    base, rem = divmod(n, parts)
    return [base + (1 if i < rem else 0) for i in range(parts)]


# --------------------------------------------------------------------------
# Polarized system (Section 3, eqs. jump_1..jump_4; reading R6).
# Unknown layout x[..., k, c, :] with k = interface 0..L-2 and components
# c = (d_a, d_b, u_a, u_b): down-going and up-going parts of the traces at the
# last row of layer k (a) and the first row of layer k+1 (b).
# --------------------------------------------------------------------------

DA, DB, UA, UB = 0, 1, 2, 3


def polarized_rhs(D: Decomposition, f: np.ndarray) -> np.ndarray:
    """Right-hand side from the Newton potentials (matrix-free solver, lines 2-7)."""
    L = D.L
    z = np.zeros(f.shape[:-2] + (D.NX,), dtype=np.complex128)
    out = np.zeros(f.shape[:-2] + (L - 1, 4, D.NX), dtype=np.complex128)
    for l in range(L):
        s = D.green(l, z, z, z, z, f=f)
        if l < L - 1:
            out[..., l, DA, :] = s[..., 2, :]
            out[..., l, DB, :] = s[..., 3, :]
        if l > 0:
            out[..., l - 1, UA, :] = s[..., 0, :]
            out[..., l - 1, UB, :] = s[..., 1, :]
    return out


def apply_M(D: Decomposition, x: np.ndarray) -> np.ndarray:
    """The polarized operator M (equations jump_1..jump_4 moved to the left)."""
    L = D.L
    out = np.zeros_like(x)
    z = np.zeros(x.shape[:-3] + (D.NX,), dtype=np.complex128)
    d = x[..., DA:DB + 1, :]
    u = x[..., UA:UB + 1, :]
    for l in range(L):
        if l < L - 1:   # rows n, n+1 of layer l: jump_2 and jump_4
            top = (d[..., l - 1, :, :] + u[..., l - 1, :, :]) if l > 0 else None
            t0, t1 = (top[..., 0, :], top[..., 1, :]) if top is not None else (z, z)
            s = D.green(l, t0, t1, u[..., l, 0, :], u[..., l, 1, :])
            out[..., l, DA, :] = d[..., l, 0, :] + u[..., l, 0, :] - s[..., 2, :]
            out[..., l, DB, :] = d[..., l, 1, :] - s[..., 3, :]
        if l > 0:       # rows 0, 1 of layer l: jump_3 and jump_1
            bot = (u[..., l, :, :] + d[..., l, :, :]) if l < L - 1 else None
            bn, bn1 = (bot[..., 0, :], bot[..., 1, :]) if bot is not None else (z, z)
            t = D.green(l, d[..., l - 1, 0, :], d[..., l - 1, 1, :], bn, bn1)
            out[..., l - 1, UA, :] = u[..., l - 1, 0, :] - t[..., 0, :]
            out[..., l - 1, UB, :] = u[..., l - 1, 1, :] + d[..., l - 1, 1, :] - t[..., 1, :]
    return out


def sweep_down(D: Decomposition, v: np.ndarray) -> np.ndarray:
    """(D_down)^{-1} v (Alg. downwardsSweep): v, result shaped (..., L-1, 2, NX)."""
    L = D.L
    z = np.zeros(v.shape[:-3] + (D.NX,), dtype=np.complex128)
    d = np.array(v, copy=True)
    for k in range(1, L - 1):
        s = D.green(k, d[..., k - 1, 0, :], d[..., k - 1, 1, :], z, z)
        d[..., k, 0, :] += s[..., 2, :]
        d[..., k, 1, :] += s[..., 3, :]
    return d


def sweep_up(D: Decomposition, v: np.ndarray) -> np.ndarray:
    """(D_up)^{-1} v (Alg. upwardsSweep)."""
    L = D.L
    z = np.zeros(v.shape[:-3] + (D.NX,), dtype=np.complex128)
    u = np.array(v, copy=True)
    for k in range(L - 3, -1, -1):
        s = D.green(k + 1, z, z, u[..., k + 1, 0, :], u[..., k + 1, 1, :])
        u[..., k, 0, :] += s[..., 0, :]
        u[..., k, 1, :] += s[..., 1, :]
    return u


def reflections(D: Decomposition, d: np.ndarray) -> np.ndarray:
    """L d (Alg. upwardsReflections): the d-columns of jump_1 / jump_3."""
    L = D.L
    z = np.zeros(d.shape[:-3] + (D.NX,), dtype=np.complex128)
    out = np.zeros_like(d)
    for k in range(L - 1):
        bn, bn1 = (d[..., k + 1, 0, :], d[..., k + 1, 1, :]) if k + 1 < L - 1 else (z, z)
        t = D.green(k + 1, d[..., k, 0, :], d[..., k, 1, :], bn, bn1)
        out[..., k, 0, :] = -t[..., 0, :]
        out[..., k, 1, :] = d[..., k, 1, :] - t[..., 1, :]
    return out


def precond_gs(D: Decomposition, v: np.ndarray) -> np.ndarray:
    """Gauss-Seidel preconditioner, eq. (preconditioner_GS)."""
    d = sweep_down(D, v[..., DA:DB + 1, :])
    u = sweep_up(D, v[..., UA:UB + 1, :] - reflections(D, d))
    return np.concatenate([d, u], axis=-2)


def precond_jac(D: Decomposition, v: np.ndarray) -> np.ndarray:
    """Jacobi preconditioner, eq. (preconditioner_Jac)."""
    return np.concatenate([sweep_down(D, v[..., DA:DB + 1, :]),
                           sweep_up(D, v[..., UA:UB + 1, :])], axis=-2)


def gmres(apply_A, b: np.ndarray, apply_P=None, tol=1e-10, maxit=200):
    """Right-preconditioned GMRES (MGS Arnoldi, no restart) on one vector, in
    the flexible form (Saad 1993): the preconditioned directions z_j are kept
    and x = sum y_j z_j, so a preconditioner that changes between applications
    (inexact inner solves) is admissible.

    Returns (x, iterations, residual history)."""
    shape = b.shape
    bv = b.reshape(-1)
    beta = np.linalg.norm(bv)
    P = apply_P if apply_P is not None else (lambda y: y)
    V = [bv / beta]
    Z = []
    H = np.zeros((maxit + 1, maxit), dtype=np.complex128)
    hist = [1.0]
    y = np.zeros(0)
    for j in range(maxit):
        z = P(V[j].reshape(shape)).reshape(-1)
        Z.append(z)
        w = apply_A(z.reshape(shape)).reshape(-1)
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        e1 = np.zeros(j + 2, dtype=np.complex128)
        e1[0] = beta
        y, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)
        res = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y) / beta
        hist.append(res)
        if res <= tol or H[j + 1, j] == 0:
            break
        V.append(w / H[j + 1, j])
    x = sum(yi * zi for yi, zi in zip(y, Z))
    return x.reshape(shape), len(hist) - 1, hist


def reconstruct(D: Decomposition, f: np.ndarray, tr: np.ndarray) -> np.ndarray:
    """Volume from the traces (matrix-free solver, lines 10-18)."""
    u = np.zeros(f.shape, dtype=np.complex128)
    z = np.zeros(f.shape[:-2] + (D.NX,), dtype=np.complex128)
    for l in range(D.L):
        t0, t1 = (tr[..., l - 1, 0, :], tr[..., l - 1, 1, :]) if l > 0 else (z, z)
        tn, tn1 = (tr[..., l, 0, :], tr[..., l, 1, :]) if l < D.L - 1 else (z, z)
        v = D.green(l, t0, t1, tn, tn1, f=f, full=True)
        lo, hi = D.owned_rows(l)
        u[..., D.s[l] + lo:D.s[l] + hi, :] = v[..., lo:hi, :]
    return u


# --------------------------------------------------------------------------
# Inner nested polarized traces (Section 4.2): a layer's local problem solved
# by the method of polarized traces over its cells (GMRES on the cells'
# polarized system, preconditioned by the Gauss-Seidel sweeps over the cells)
# instead of a direct factorization.  The layer box with its axes swapped is a
# problem of the same form -- the operator of Appendix A treats both axes
# alike, and the cells extend the layer's medium by the rule R3 just as the
# layers extend the global one -- so the cells are the layers of that problem
# and the functions above apply to it unchanged.
# --------------------------------------------------------------------------

def layer_inner_decomposition(D: Decomposition, l: int) -> Decomposition:
    """Layer l of D with x and z swapped: its C cells become the layers."""
    return Decomposition(D.layer_medium(l).T, D.rows[l], D.n_x, D.p, D.omega, D.h, D.C_pml, D.C, 1,
                         layer_rows=D.cols)


def nested_layer_solve(DT: Decomposition, g: np.ndarray, tol: float = 1e-10, precond=None, maxit: int = 200):
    """v = (H^l)^{-1} g for the layer whose swapped-axes decomposition is DT
    (g, v on the layer's box, (..., n_l + 2p, NX)).  Returns (v, iterations)."""
    gT = np.swapaxes(g, -1, -2)
    if DT.L == 1:
        return DT.layer_factor(0).solve(gT).swapaxes(-1, -2), 0
    P = precond if precond is not None else precond_gs
    b = polarized_rhs(DT, gT)
    x, its, _ = gmres(lambda y: apply_M(DT, y), b, lambda y: P(DT, y), tol=tol, maxit=maxit)
    tr = x[..., DA:DB + 1, :] + x[..., UA:UB + 1, :]  # interface traces = down + up (R6)
    return np.swapaxes(reconstruct(DT, gT, tr), -1, -2), its


class NestedDecomposition(Decomposition):
    """The decomposition with every layer solve done by the inner nested
    polarized traces to relative tolerance tol_inner (the nested method of
    Section 4: outer polarized traces over layers, inner over cells)."""

    def __init__(self, *args, tol_inner: float = 1e-10, **kw):
        super().__init__(*args, **kw)
        self.tol_inner = tol_inner
        self.inner_iterations = []
        self._inner = {}

    def inner(self, l: int) -> Decomposition:
        if l not in self._inner:
            self._inner[l] = layer_inner_decomposition(self, l)
        return self._inner[l]

    def green(self, l: int, t0, t1, tn, tn1, f=None, full=False):
        g = self.interface_source(l, t0, t1, tn, tn1)
        if f is not None:
            g = g + self.layer_source(l, f)
        v, its = nested_layer_solve(self.inner(l), g, self.tol_inner)
        self.inner_iterations.append(its)
        if full:
            return v
        n = self.rows[l]
        rows = [self.lrow(0), self.lrow(1), self.lrow(n), self.lrow(n + 1)]
        return v[..., rows, :]


# --------------------------------------------------------------------------
# Receiver misfit and its gradient (adjoint-state; not in the paper).
# --------------------------------------------------------------------------

def misfit_gradient(box: Box, f: np.ndarray, d: np.ndarray, rec_idx: np.ndarray, fac: Factor | None = None):
    """J = 1/2 sum_s ||R u_s - d_s||^2 with H u_s = f_s, and dJ/dm on the grid.

    H depends on m only through -omega^2 m u, so
    dJ/dm_i = omega^2 sum_s Re(lambda_{s,i} u_{s,i}) with H^T lambda_s = R^T conj(r_s).
    """
    fac = fac or box.factor()
    u = fac.solve(f)
    B = f.shape[0]
    uf = u.reshape(B, -1)
    r = uf[:, rec_idx] - d
    J = 0.5 * float(np.sum(np.abs(r) ** 2))
    g = np.zeros_like(uf)
    # R^T conj(r): a node listed twice as a receiver takes both residuals
    np.add.at(g, (np.arange(B)[:, None], np.asarray(rec_idx)[None, :]), np.conj(r))
    lam = fac.solve(g.reshape(f.shape), trans=True).reshape(B, -1)
    grad = box.omega ** 2 * np.sum(np.real(lam * uf), axis=0)
    return J, grad.reshape(box.shape), u


# ---------------------------------------------------------------------------
# Block-LU sweeps of a layer's inner SIE (Section 4.2.2) and their compressed
# form (the compression of the inner operators to a tolerance eps, Section 4.3).
# The inner unknowns of interface j are written x_j; with W_j the inverted
# diagonal Schur block, h_j = W_j g_j, P_j the sub-diagonal and V_j the
# super-diagonal factor, the two sweeps are
#     y_0 = h_0,  y_j = h_j + P_j y_{j-1};   x_{J-1} = y_{J-1},  x_j = y_j + V_j x_{j+1}.

def inner_block_lu(P, V, h):
    """The two sweeps above.  P[j] (j >= 1), V[j] (j <= J-2): (n x n); h: (J, n, B)."""
    J = len(h)
    y = [None] * J
    y[0] = h[0].copy()
    for j in range(1, J):
        y[j] = h[j] + P[j] @ y[j - 1]
    x = [None] * J
    x[J - 1] = y[J - 1]
    for j in range(J - 2, -1, -1):
        x[j] = y[j] + V[j] @ x[j + 1]
    return np.array(x)


def lowrank(A, eps):
    """A ~ Q Bf with orthonormal Q and the smallest rank whose relative Frobenius
    error is <= eps (truncated SVD: the optimal low-rank form for that norm)."""
    U, s, Vh = np.linalg.svd(A, full_matrices=False)
    tail = np.sqrt(np.cumsum((s ** 2)[::-1]))[::-1]  # tail[k] = ||s[k:]||
    total = tail[0] if len(s) else 0.0
    r = len(s)
    for k in range(len(s)):
        if tail[k] <= eps * total:
            r = k
            break
    r = max(r, 1)
    return U[:, :r], s[:r, None] * Vh[:r]


def inner_block_lu_lowrank(QP, BP, QV, BV, h):
    """The same sweeps with P_j = QP_j BP_j and V_j = QV_j BV_j, carried on the
    r-vectors t_j = BP_j y_{j-1} and s_j = BV_j x_{j+1}:
        t_1 = BP_1 h_0,  t_{j+1} = BP_{j+1} (h_j + QP_j t_j);
        s_{J-2} = BV_{J-2} (h_{J-1} + QP_{J-1} t_{J-1}),  s_{j-1} = BV_{j-1} (h_j + QP_j t_j + QV_j s_j);
        x_j = h_j + QP_j t_j + QV_j s_j   (t_0 = 0, s_{J-1} = 0)."""
    J = len(h)
    y = [None] * J
    y[0] = h[0]
    for j in range(1, J):
        t = BP[j] @ y[j - 1]
        y[j] = h[j] + QP[j] @ t
    x = [None] * J
    x[J - 1] = y[J - 1]
    for j in range(J - 2, -1, -1):
        s = BV[j] @ x[j + 1]
        x[j] = y[j] + QV[j] @ s
    return np.array(x)
