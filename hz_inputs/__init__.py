"""Seeded synthetic inputs shared by the oracle and the GPU path.

This module holds no arithmetic of the solver: it only draws media (squared
slowness m = 1/c^2 on the PML-extended grid), partitions, sources and
receiver data layouts.  Both the CPU oracle (``oracle/``) and the CUDA path
(``paper_1510_01831_gb300``) receive these arrays as plain inputs.

Grid convention (Appendix A of the paper): nodes x_p = p*h, interior
p = 1..n_x, PML nodes p = -n_pml+1..0 and n_x+1..n_x+n_pml; arrays are
row-major ``[n_z + 2 n_pml][n_x + 2 n_pml]`` (x fastest).  Interior column
p sits at array index ``p + n_pml - 1``.

The paper's media (BP2004, Marmousi2) are not available; the generators
below stand in for them with smooth random and layered-faulted velocity
models of the sizes the paper's tables use.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import ndimage


@dataclasses.dataclass
class Problem:
    """One Helmholtz problem instance on the PML-extended grid."""
    name: str
    m: np.ndarray           # (n_z+2p, n_x+2p) float64 squared slowness
    n_x: int
    n_z: int
    n_pml: int
    h: float
    omega: float
    L: int
    C: int
    layer_rows: list | None = None   # interior rows per layer (None = uniform)
    cell_cols: list | None = None    # interior columns per cell (None = uniform)

    @property
    def shape_ext(self):
        return (self.n_z + 2 * self.n_pml, self.n_x + 2 * self.n_pml)


def uniform_split(n: int, parts: int) -> list[int]:
    """Split n points into `parts` nearly equal contiguous pieces."""
    base, rem = divmod(n, parts)
    return [base + (1 if i < rem else 0) for i in range(parts)]


def random_split(n: int, lo: int, hi: int, seed: int) -> list[int]:
    """Uneven partition: widths drawn uniformly in [lo, hi] until they sum to n.

    The last piece absorbs the remainder; if it would fall below `lo` it is
    merged with its neighbour (and the merged piece split evenly if above hi).
    """
    rng = np.random.default_rng(seed)
    out: list[int] = []
    left = n
    while left > hi:
        w = int(rng.integers(lo, hi + 1))
        if left - w < lo:
            w = left - lo
        out.append(w)
        left -= w
    out.append(left)
    return out


def omega_for_ppw(c_min: float, h: float, ppw: float) -> float:
    """Angular frequency with `ppw` grid points per wavelength at speed c_min."""
    return 2.0 * math.pi * c_min / (ppw * h)


def smooth_random_velocity(n_x: int, n_z: int, n_pml: int, seed: int,
                           corr_pts: float = 20.0, c_lo: float = 1.5,
                           c_hi: float = 4.5) -> np.ndarray:
    """Gaussian-smoothed white noise on the extended grid, mapped to [c_lo, c_hi].

    The Gaussian filter has standard deviation corr_pts/sqrt(2) grid points
    (covariance length corr_pts).  Returns the velocity c.
    """
    rng = np.random.default_rng(seed)
    shape = (n_z + 2 * n_pml, n_x + 2 * n_pml)
    w = rng.standard_normal(shape)
    s = ndimage.gaussian_filter(w, sigma=corr_pts / math.sqrt(2.0), mode="reflect")
    s = (s - s.min()) / (s.max() - s.min())
    return c_lo + (c_hi - c_lo) * s


def layered_faulted_velocity(n_x: int, n_z: int, n_pml: int, seed: int,
                             n_layers: int = 12, c_top: float = 1.5,
                             c_bot: float = 5.5) -> np.ndarray:
    """Layered medium: interfaces are sums of 3 sinusoids, two dip-slip faults.

    Velocity increases with depth from c_top to c_bot (linear trend with a
    +-0.1 jitter per layer).  Each fault is a line at 60+-10 degrees dip; the
    hanging wall is shifted down by 2-5 % of the depth.
    """
    rng = np.random.default_rng(seed)
    NZ, NX = n_z + 2 * n_pml, n_x + 2 * n_pml
    x = (np.arange(NX) - n_pml + 1) / (n_x + 1)        # 0..1 across the interior
    zbar = np.linspace(0, 1, n_layers + 1)[1:-1]        # mean interface depths
    thick = 1.0 / n_layers
    ifaces = []
    for zi in zbar:
        z = np.full(NX, zi)
        for _ in range(3):
            a = rng.uniform(0, 0.3 * thick) / 3.0
            k = int(rng.integers(1, 7))
            ph = rng.uniform(0, 2 * math.pi)
            z = z + a * np.sin(2 * math.pi * k * x + ph)
        ifaces.append(z)
    speeds = np.linspace(c_top, c_bot, n_layers) + rng.uniform(-0.1, 0.1, n_layers)
    speeds = np.clip(speeds, c_top, c_bot)
    zz = ((np.arange(NZ) - n_pml + 1) / (n_z + 1))[:, None] * np.ones((1, NX))
    xx = np.ones((NZ, 1)) * x[None, :]

    def label(zq):
        lab = np.zeros(zq.shape, dtype=np.int64)
        for zi in ifaces:
            lab += (zq > zi[None, :]).astype(np.int64)
        return lab

    zq = zz.copy()
    for _ in range(2):
        dip = math.radians(60.0 + rng.uniform(-10, 10))
        x0 = rng.uniform(0.25, 0.75)
        off = rng.uniform(0.02, 0.05)
        # hanging wall: points to the right of the fault line x = x0 + z/tan(dip)
        hang = xx > (x0 + zz / math.tan(dip))
        zq = np.where(hang, zq - off, zq)
    return speeds[label(zq)]


def gaussian_source(n_x: int, n_z: int, n_pml: int, h: float,
                    x0: float, z0: float, sigma: float) -> np.ndarray:
    """exp(-|x-x0|^2/(2 sigma^2)) / (2 pi sigma^2) at interior nodes (0 in the PML)."""
    NZ, NX = n_z + 2 * n_pml, n_x + 2 * n_pml
    f = np.zeros((NZ, NX), dtype=np.complex128)
    p = np.arange(1, n_x + 1) * h
    q = np.arange(1, n_z + 1) * h
    Q, P = np.meshgrid(q, p, indexing="ij")
    g = np.exp(-((P - x0) ** 2 + (Q - z0) ** 2) / (2 * sigma ** 2)) / (2 * math.pi * sigma ** 2)
    f[n_pml:n_pml + n_z, n_pml:n_pml + n_x] = g
    return f


def point_source_columns(n_x: int, B: int) -> np.ndarray:
    """Interior column numbers p (1-based) of B evenly spaced sources."""
    return np.array([int(math.floor((s + 0.5) * n_x / B)) + 1 for s in range(B)])


def point_sources_row(n_x: int, n_z: int, n_pml: int, h: float, B: int,
                      row: int = 1) -> np.ndarray:
    """B discrete Diracs e_s/h^2 on interior row `row`, evenly spaced in x.

    Returns a complex128 array (B, n_z+2p, n_x+2p).
    """
    NZ, NX = n_z + 2 * n_pml, n_x + 2 * n_pml
    f = np.zeros((B, NZ, NX), dtype=np.complex128)
    iz = row + n_pml - 1
    for s, p in enumerate(point_source_columns(n_x, B)):
        f[s, iz, p + n_pml - 1] = 1.0 / (h * h)
    return f


def random_sources(shape_ext, n_pml: int, B: int, seed: int) -> np.ndarray:
    """Dense complex random sources supported in the interior (0 in the PML)."""
    rng = np.random.default_rng(seed)
    NZ, NX = shape_ext
    f = np.zeros((B, NZ, NX), dtype=np.complex128)
    sl = (slice(None), slice(n_pml, NZ - n_pml), slice(n_pml, NX - n_pml))
    inner = f[sl]
    f[sl] = rng.standard_normal(inner.shape) + 1j * rng.standard_normal(inner.shape)
    return f


def receivers_top_row(n_x: int, n_pml: int, row: int = 1) -> np.ndarray:
    """Flat indices (into the extended grid) of every interior node of `row`."""
    NX = n_x + 2 * n_pml
    iz = row + n_pml - 1
    return np.array([iz * NX + (p + n_pml - 1) for p in range(1, n_x + 1)], dtype=np.int32)


def gaussian_blob(shape_ext, n_pml: int, h: float, radius_pts: float) -> np.ndarray:
    """exp(-r^2/(2 (radius h)^2)) centred on the extended grid."""
    NZ, NX = shape_ext
    zc, xc = (NZ - 1) / 2.0, (NX - 1) / 2.0
    Z, X = np.meshgrid(np.arange(NZ) - zc, np.arange(NX) - xc, indexing="ij")
    return np.exp(-(X ** 2 + Z ** 2) / (2.0 * radius_pts ** 2))


# --------------------------------------------------------------------------
# The five workloads (constant, smooth random, layered-faulted, batched
# multi-frequency with uneven cells, adjoint gradient), plus scaled twins.
# --------------------------------------------------------------------------

def constant_medium(n: int = 128, n_pml: int = 10, L: int = 4, C: int = 4,
                    ppw: float = 10.0) -> Problem:
    """m = 1 on [0,1]^2 with an n x n interior grid, h = 1/(n+1)."""
    h = 1.0 / (n + 1)
    m = np.ones((n + 2 * n_pml, n + 2 * n_pml))
    return Problem("constant", m, n, n, n_pml, h, omega_for_ppw(1.0, h, ppw), L, C)


def smooth_random(n: int = 1024, n_pml: int = 20, L: int = 16, C: int = 16,
                  seed: int = 2, ppw: float = 10.0, corr_pts: float = 20.0,
                  n_z: int | None = None) -> Problem:
    """Smooth random medium, c in [1.5, 4.5], correlation length corr_pts*h."""
    nz = n if n_z is None else n_z
    h = 1.0 / (n + 1)
    c = smooth_random_velocity(n, nz, n_pml, seed, corr_pts=corr_pts)
    return Problem("smooth_random", 1.0 / c ** 2, n, nz, n_pml, h,
                   omega_for_ppw(1.5, h, ppw), L, C)


def layered_faulted(n_x: int = 2000, n_z: int = 4000, n_pml: int = 30, L: int = 40,
                    C: int = 20, seed: int = 3, ppw: float = 8.0) -> Problem:
    h = 1.0 / (n_x + 1)
    c = layered_faulted_velocity(n_x, n_z, n_pml, seed)
    return Problem("layered_faulted", 1.0 / c ** 2, n_x, n_z, n_pml, h,
                   omega_for_ppw(1.5, h, ppw), L, C)


def uneven_multifreq(n: int = 512, n_pml: int = 20, seed: int = 4,
                     part_seed: int = 40, ppw_list=(6.0, 8.0, 10.0),
                     lo: int = 24, hi: int = 64) -> list[Problem]:
    h = 1.0 / (n + 1)
    c = smooth_random_velocity(n, n, n_pml, seed)
    rows = random_split(n, lo, hi, part_seed)
    cols = random_split(n, lo, hi, part_seed + 1)
    out = []
    for ppw in ppw_list:
        out.append(Problem(f"uneven_ppw{ppw:g}", 1.0 / c ** 2, n, n, n_pml, h,
                           omega_for_ppw(1.5, h, ppw), len(rows), len(cols),
                           layer_rows=rows, cell_cols=cols))
    return out


def gradient_case(n: int = 512, n_pml: int = 20, L: int = 8, C: int = 8,
                  seed: int = 5, ppw: float = 10.0, blob_pts: float = 30.0):
    """Background m0 and the perturbed m_true = m0 (1 + 0.05 blob)."""
    p0 = smooth_random(n, n_pml, L, C, seed=seed, ppw=ppw)
    blob = gaussian_blob(p0.shape_ext, n_pml, p0.h, blob_pts)
    m_true = p0.m * (1.0 + 0.05 * blob)
    return p0, m_true
