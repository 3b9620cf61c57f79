"""FP32 cell chain for panels of at most 16 right-hand sides (SIMT, the form the
2000 x 4000 workload takes: 160-column cells, 16 sources) against the oracle's
cell solve, at cell widths of one, two and three 64-row chunks, an odd width
(a K tail and an odd W row length), and batches of 1, 13 (ragged) and 16
columns; 17 columns take the general kernel and must agree with it.

Tolerance: the FP32 chain reaches ~1e-6 against the oracle on these cells
(2 nz' - 1 dependent steps of FP32 products); the bar is 2e-6, as for the
general SIMT kernel."""
import numpy as np
import pytest

import hz_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

hz = pytest.importorskip("paper_1510_01831_gb300.hz")


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


# (n, n_pml, L, C): cell widths 62 (one chunk), 113 (odd), 160 (three chunks: 64, 64, 32), 172
@pytest.mark.parametrize("n,p,L,C", [(100, 6, 4, 2), (101, 6, 2, 1), (200, 30, 2, 2), (224, 30, 2, 2)])
@pytest.mark.parametrize("B", [1, 13, 16])
def test_cell_solve_16_columns(n, p, L, C, B):
    pb = I.smooth_random(n, n_pml=p, L=L, C=C, seed=61, ppw=8, corr_pts=10, n_z=min(n, 120))
    C_pml = O.default_pml_C(pb.m)
    D = O.Decomposition(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml, pb.L, pb.C)
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=hz.HZ_MIXED,
                     pml_C=C_pml, tensor_cores=False)
    ctx.hz_factor()
    rng = np.random.default_rng(62)
    for l, c in ((0, 0), (L - 1, C - 1)):
        box = D.cell_box(l, c)
        g = rng.standard_normal((B,) + box.shape) + 1j * rng.standard_normal((B,) + box.shape)
        ax = box.alpha(0, np.arange(box.shape[1]))
        az = box.alpha(1, np.arange(box.shape[0]))
        ref = box.factor().solve(g * (az[:, None] * ax[None, :]))
        x = ctx.hz_cell_solve(l, c, g)
        assert _rel(x, ref) < 2e-6, (box.shape, B)
    ctx.close()


def test_16_and_17_columns_agree():
    pb = I.smooth_random(200, n_pml=30, L=2, C=2, seed=63, ppw=8, corr_pts=10, n_z=100)
    C_pml = O.default_pml_C(pb.m)
    D = O.Decomposition(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml, pb.L, pb.C)
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=hz.HZ_MIXED,
                     pml_C=C_pml, tensor_cores=False)
    ctx.hz_factor()
    box = D.cell_box(1, 0)
    rng = np.random.default_rng(64)
    g = rng.standard_normal((17,) + box.shape) + 1j * rng.standard_normal((17,) + box.shape)
    x17 = ctx.hz_cell_solve(1, 0, g)          # general kernel
    x16 = ctx.hz_cell_solve(1, 0, g[:16])     # 16-column kernel
    ctx.close()
    # each kernel is within 2e-6 of the oracle (its own FP32 rounding order), so the two
    # differ by at most the sum of their bars
    assert _rel(x16, x17[:16]) < 4e-6
