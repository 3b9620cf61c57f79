"""Sweep steps of the compressed-block LU through the per-cell composites
(P2 = E W F + S, P1 = STW F, P3 = E UX; the step is out += P2 in, ac = P1 in,
ts = LAM ac, out += P3 ts) against the oracle's sweeps and reflections
(Alg. downwardsSweep, Alg. upwardsSweep, Alg. upwardsReflections; Section
4.2.2 with the compression of Section 4.3), and the polarized operator (Alg.
applyM).  The reflections and the operator apply every layer at once with four
input rows and the r-vector chain between the products.

The composites are the same linear map regrouped and formed in FP64, so at a
tight compression tolerance (eps = 1e-12) the FP64 sweeps match the oracle to
the FP64 component bar (1e-9); mixed precision rounds the composites once to
FP32 and is held to 1e-5.  The partition is uneven (cells of different owned
widths, edge cells owning the global PML) and has several layers, so that the
input range of every cell kind (first, interior, last) and every sweep step is
exercised; a local model update rewrites one layer's composites in place."""
import numpy as np
import pytest

import hz_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

hz = pytest.importorskip("paper_1510_01831_gb300.hz")


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


ROWS, COLS = [18, 22, 16, 20, 24], [26, 31, 20, 33]


@pytest.fixture(scope="module")
def case():
    pb = I.smooth_random(110, n_pml=6, L=5, C=4, seed=71, ppw=8, corr_pts=8, n_z=100)
    C_pml = O.default_pml_C(pb.m)
    D = O.Decomposition(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml, pb.L, pb.C,
                        layer_rows=ROWS, cell_cols=COLS)
    return pb, C_pml, D


def _ctx(pb, C_pml, eps, precision):
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, pml_C=C_pml, precision=precision,
                     compress=eps, layer_rows=ROWS, cell_cols=COLS)
    ctx.hz_factor()
    return ctx


def _x(D, B, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B, D.L - 1, 4, D.NX)) + 1j * rng.standard_normal((B, D.L - 1, 4, D.NX))


@pytest.mark.parametrize("precision,eps,bar", [(hz.HZ_FP64, 1e-12, 1e-9), (hz.HZ_MIXED, 1e-8, 1e-5)])
def test_sweeps_match_the_oracle(case, precision, eps, bar):
    pb, C_pml, D = case
    x = _x(D, 3, 72)
    ctx = _ctx(pb, C_pml, eps, precision)
    down = ctx.hz_precond(2, x)
    up = ctx.hz_precond(3, x)
    refl = ctx.hz_precond(4, x)
    gs = ctx.hz_precond(0, x)
    ctx.close()
    ref_down = np.concatenate([O.sweep_down(D, x[..., 0:2, :]), x[..., 2:4, :]], axis=-2)
    ref_up = np.concatenate([x[..., 0:2, :], O.sweep_up(D, x[..., 2:4, :])], axis=-2)
    ref_refl = np.concatenate([np.zeros_like(x[..., 0:2, :]), O.reflections(D, x[..., 0:2, :])], axis=-2)
    assert _rel(down, ref_down) < bar
    assert _rel(up, ref_up) < bar
    assert _rel(refl, ref_refl) < bar
    assert _rel(gs, O.precond_gs(D, x)) < bar


@pytest.mark.parametrize("precision,eps,bar", [(hz.HZ_FP64, 1e-12, 1e-9), (hz.HZ_MIXED, 1e-8, 1e-5)])
def test_polarized_operator_matches_the_oracle(case, precision, eps, bar):
    # both input sets of every layer (4 input rows each) in one 2B-wide application
    pb, C_pml, D = case
    x = _x(D, 3, 74)
    ctx = _ctx(pb, C_pml, eps, precision)
    y = ctx.hz_apply_M(x)
    ctx.close()
    assert _rel(y, O.apply_M(D, x)) < bar


@pytest.mark.parametrize("B", [2, 16])
def test_persistent_sweeps(case, B, monkeypatch):
    # with HZ_PERSIST=1, even batches of <= 16 columns run each sweep as one persistent
    # launch (phases separated by grid barriers)
    pb, C_pml, D = case
    x = _x(D, B, 75)
    monkeypatch.setenv("HZ_PERSIST", "1")
    ctx = _ctx(pb, C_pml, 1e-8, hz.HZ_MIXED)
    down = ctx.hz_precond(2, x)
    up = ctx.hz_precond(3, x)
    gs = ctx.hz_precond(0, x)
    gs2 = ctx.hz_precond(0, x)
    ctx.close()
    ref_down = np.concatenate([O.sweep_down(D, x[..., 0:2, :]), x[..., 2:4, :]], axis=-2)
    ref_up = np.concatenate([x[..., 0:2, :], O.sweep_up(D, x[..., 2:4, :])], axis=-2)
    assert _rel(down, ref_down) < 1e-5
    assert _rel(up, ref_up) < 1e-5
    assert _rel(gs, O.precond_gs(D, x)) < 1e-5
    assert _rel(gs2, gs) < 1e-12  # repeatable: split-K slices are added in a fixed order


def test_persistent_solve_matches_and_launches_less(case, monkeypatch):
    pb, C_pml, D = case
    f = I.random_sources(pb.shape_ext, pb.n_pml, 4, 76)
    monkeypatch.setenv("HZ_PERSIST", "1")
    ctx = _ctx(pb, C_pml, 1e-8, hz.HZ_MIXED)
    u1, st1 = ctx.hz_solve(f)
    ctx.close()
    monkeypatch.setenv("HZ_PERSIST", "0")
    ctx = _ctx(pb, C_pml, 1e-8, hz.HZ_MIXED)
    u0, st0 = ctx.hz_solve(f)
    ctx.close()
    assert st1.gpu_launches < st0.gpu_launches  # the sweeps ran as single launches
    assert st1.resid < 1e-8 and st0.resid < 1e-8
    assert _rel(u1, u0) < 1e-6


def test_local_update_rewrites_the_composites(case):
    pb, C_pml, D = case
    m1 = pb.m.copy()
    z0 = pb.n_pml + ROWS[0] + ROWS[1] + 5       # inside layer 2
    x0 = pb.n_pml + COLS[0] + 4                 # inside cell 1
    m1[z0:z0 + 4, x0:x0 + 4] *= 1.07
    D1 = O.Decomposition(m1, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml, pb.L, pb.C,
                         layer_rows=ROWS, cell_cols=COLS)
    x = _x(D, 2, 73)
    ctx = _ctx(pb, C_pml, 1e-12, hz.HZ_FP64)
    ctx.hz_update_model(m1)
    gs = ctx.hz_precond(0, x)
    ctx.close()
    assert _rel(gs, O.precond_gs(D1, x)) < 1e-9
