"""Tensor-core cell solve (tcgen05, 3xTF32 split) against the SIMT FP32 cell
solve and the oracle, at cell widths that exercise a padded K (62 -> 64
columns) and a partial last K chunk (104 columns), with right-hand-side tails.

Tolerance of the cell solve: the SIMT FP32 chain reaches ~8e-7 against the
oracle; the tensor-core chain ~6e-6 (measured 2.4e-6 at 62 columns and 6.3e-6
at 104 columns): each step's accumulators take ~13 truncating additions of
K = 8 partial products and the 2nz'-1 steps of the chain compound them.  The
bar is 2e-5; the full solve after FP64 refinement keeps the 1e-5 bar."""
import numpy as np
import pytest

import hz_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

hz = pytest.importorskip("paper_1510_01831_gb300.hz")


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _ctx(pb, C_pml, tc):
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=hz.HZ_MIXED,
                     pml_C=C_pml, tensor_cores=tc)
    ctx.hz_factor()
    return ctx


# B > 32 takes the 64-column form of the kernel where its panel fits in shared memory
# (cells up to 104 columns), else the 32-column form (115 columns): B = 40 and 70 leave
# ragged tails
@pytest.mark.parametrize("n,p,L,C,B", [(100, 6, 4, 2, 5), (128, 20, 2, 2, 40), (100, 20, 2, 2, 70),
                                       (150, 20, 2, 2, 70)])
def test_cell_solve_tensor_vs_simt_and_oracle(n, p, L, C, B):
    pb = I.smooth_random(n, n_pml=p, L=L, C=C, seed=31, ppw=8, corr_pts=10)
    C_pml = O.default_pml_C(pb.m)
    D = O.Decomposition(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml, pb.L, pb.C)
    tc, simt = _ctx(pb, C_pml, True), _ctx(pb, C_pml, False)
    rng = np.random.default_rng(32)
    for l, c in ((0, 0), (L - 1, C - 1)):
        box = D.cell_box(l, c)
        g = rng.standard_normal((B,) + box.shape) + 1j * rng.standard_normal((B,) + box.shape)
        ax = box.alpha(0, np.arange(box.shape[1]))
        az = box.alpha(1, np.arange(box.shape[0]))
        ref = box.factor().solve(g * (az[:, None] * ax[None, :]))
        xt = tc.hz_cell_solve(l, c, g)
        xs = simt.hz_cell_solve(l, c, g)
        assert _rel(xt, ref) < 2e-5
        assert _rel(xs, ref) < 2e-6
        assert _rel(xt, xs) < 2e-5
    tc.close()
    simt.close()


def test_full_solve_with_tensor_core_cells():
    pb = I.smooth_random(128, n_pml=20, L=2, C=2, seed=33, ppw=8, corr_pts=10)
    C_pml = O.default_pml_C(pb.m)
    f = I.point_sources_row(pb.n_x, pb.n_z, pb.n_pml, pb.h, 40)
    box = O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml)
    ref = box.factor().solve(f)
    ctx = _ctx(pb, C_pml, True)
    u, st = ctx.hz_solve(f)
    u2, _ = ctx.hz_solve(f)
    ctx.close()
    assert _rel(u, ref) < 1e-5
    assert st.resid < 1e-8
    assert np.all(O.relative_residual(box, u, f) < 1e-8)
    assert _rel(u2, u) < 1e-12


# The batched F / E / S products on the tensor cores (3xTF32, accumulators
# drained into FP32 registers every 16 columns of K) against the SIMT FP32
# products and the oracle, through the layer application, the polarized
# operator and the Gauss-Seidel preconditioner.  B = 5 leaves a ragged
# right-hand-side tile and takes split-K; B = 70 spans two 64-wide tiles.
# Measured: both forms ~1e-6 against the oracle; the bar is 1e-5.
@pytest.mark.parametrize("B", [5, 70])
def test_batched_products_tensor_vs_simt_and_oracle(B):
    pb = I.smooth_random(128, n_pml=20, L=3, C=2, seed=34, ppw=8, corr_pts=10)
    C_pml = O.default_pml_C(pb.m)
    D = O.Decomposition(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml, pb.L, pb.C)
    tc, simt = _ctx(pb, C_pml, 2), _ctx(pb, C_pml, False)
    rng = np.random.default_rng(35)
    tr = rng.standard_normal((B, 4, D.NX)) + 1j * rng.standard_normal((B, 4, D.NX))
    x = rng.standard_normal((B, D.L - 1, 4, D.NX)) + 1j * rng.standard_normal((B, D.L - 1, 4, D.NX))
    refs = {"green": D.green(1, tr[:, 0], tr[:, 1], tr[:, 2], tr[:, 3]), "M": O.apply_M(D, x),
            "gs": O.precond_gs(D, x)}
    outs = []
    for ctx in (tc, simt):
        outs.append({"green": ctx.hz_layer_green(1, tr, 3), "M": ctx.hz_apply_M(x), "gs": ctx.hz_precond(0, x)})
        ctx.close()
    for k, ref in refs.items():
        assert _rel(outs[0][k], ref) < 1e-5, k
        assert _rel(outs[1][k], ref) < 1e-5, k
        assert _rel(outs[0][k], outs[1][k]) < 1e-5, k
