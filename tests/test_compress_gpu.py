"""Compressed-block LU (hz_opts.compress; Section 4.2.2 with the compression of
Section 4.3) against the oracle and the dense factors.

The inner block-LU factors P_j, V_j are the cell's Green's function between
its two sides; in low-rank form (adaptive randomized range finder to a
relative Frobenius tolerance eps) the inner sweeps run on r-vectors.

- a layer's Green's integrals at eps = 1e-12 agree with the oracle's direct
  layer solve to 1e-9 (the FP64 component bar of the dense factors);
- their distance to the dense-factor result grows with eps and stays within
  a modest multiple of it (eps 1e-4 ... 1e-10), so the compression is in
  effect and controlled;
- the Gauss-Seidel preconditioner at eps = 1e-8 within 1e-6 of the oracle's;
- whole solves at the paper's eps = 1e-8 meet the 1e-8 (FP64) and 1e-5
  (mixed) bars against the oracle's global solve, on an uneven partition too.
"""
import numpy as np
import pytest

import hz_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

hz = pytest.importorskip("paper_1510_01831_gb300.hz")


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def case():
    pb = I.smooth_random(120, n_pml=6, L=3, C=5, seed=91, ppw=8, corr_pts=8, n_z=72)
    C_pml = O.default_pml_C(pb.m)
    D = O.Decomposition(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml, pb.L, pb.C)
    return pb, C_pml, D


def _ctx(pb, C_pml, eps, precision=None, **kw):
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, pml_C=C_pml,
                     precision=hz.HZ_FP64 if precision is None else precision, compress=eps, **kw)
    ctx.hz_factor()
    return ctx


def _tr(D, B, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B, 4, D.NX)) + 1j * rng.standard_normal((B, 4, D.NX))


def test_layer_green_tight_tolerance_matches_oracle(case):
    pb, C_pml, D = case
    tr = _tr(D, 3, 92)
    ctx = _ctx(pb, C_pml, 1e-12)
    for l in range(pb.L):
        out = ctx.hz_layer_green(l, tr, 3)
        ref = D.green(l, tr[:, 0], tr[:, 1], tr[:, 2], tr[:, 3])
        assert _rel(out, ref) < 1e-9, l
    ctx.close()


def test_error_follows_the_tolerance(case):
    pb, C_pml, D = case
    tr = _tr(D, 3, 93)
    dense = _ctx(pb, C_pml, 0.0)
    ref = dense.hz_layer_green(1, tr, 3)
    dense.close()
    errs = {}
    for eps in (1e-4, 1e-7, 1e-10):
        ctx = _ctx(pb, C_pml, eps)
        errs[eps] = _rel(ctx.hz_layer_green(1, tr, 3), ref)
        ctx.close()
    assert errs[1e-4] > 1e-8             # a loose tolerance visibly truncates: the low-rank path is in use
    assert errs[1e-4] > errs[1e-7] > errs[1e-10]
    for eps, e in errs.items():
        assert e < 100 * eps, (eps, e)


def test_gauss_seidel_preconditioner(case):
    pb, C_pml, D = case
    B = 2
    rng = np.random.default_rng(94)
    x = rng.standard_normal((B, pb.L - 1, 4, D.NX)) + 1j * rng.standard_normal((B, pb.L - 1, 4, D.NX))
    ctx = _ctx(pb, C_pml, 1e-8)
    y = ctx.hz_precond(0, np.ascontiguousarray(x))
    ctx.close()
    assert _rel(y, O.precond_gs(D, x)) < 1e-6


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-8), ("mixed", 1e-5)])
def test_full_solve_at_the_papers_tolerance(case, precision, bar):
    pb, C_pml, D = case
    f = I.random_sources(pb.shape_ext, pb.n_pml, 4, 95)
    ref = D.box.factor().solve(f)
    ctx = _ctx(pb, C_pml, 1e-8, hz.HZ_FP64 if precision == "fp64" else hz.HZ_MIXED)
    u, st = ctx.hz_solve(f)
    ctx.close()
    assert _rel(u, ref) < bar and st.resid < 1e-8


def test_uneven_partition_mixed():
    pb = I.smooth_random(110, n_pml=6, L=3, C=4, seed=96, ppw=8, corr_pts=8, n_z=64)
    rows, cols = [20, 26, 18], [30, 22, 33, 25]
    C_pml = O.default_pml_C(pb.m)
    f = I.random_sources(pb.shape_ext, pb.n_pml, 3, 97)
    ref = O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml).factor().solve(f)
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, pml_C=C_pml, precision=hz.HZ_MIXED,
                     compress=1e-8, layer_rows=rows, cell_cols=cols)
    ctx.hz_factor()
    u, st = ctx.hz_solve(f)
    ctx.close()
    assert _rel(u, ref) < 1e-5 and st.resid < 1e-8
