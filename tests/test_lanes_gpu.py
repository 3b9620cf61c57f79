"""Right-hand-side lanes (opts.rhs_lanes): the batch is solved as equal groups
in lockstep on separate streams over one factorization.  Each group's solve is
the same algorithm on a sub-batch, so the result meets the same bars as the
one-group solve (mixed precision: relative error against the oracle within
1e-5, FP64 residual within 1e-8) and the groups agree with the one-group solve
to the solver tolerance.  A batch that the lane count does not divide is
solved as one group.  The gradient runs its forward and adjoint solves through
the same path."""
import numpy as np
import pytest

import hz_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

hz = pytest.importorskip("paper_1510_01831_gb300.hz")


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _setup(lanes, precision=hz.HZ_MIXED):
    pb = I.smooth_random(96, n_pml=8, L=4, C=2, seed=41, ppw=8, corr_pts=10)
    C_pml = O.default_pml_C(pb.m)
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=precision,
                     pml_C=C_pml, rhs_lanes=lanes)
    ctx.hz_factor()
    box = O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml)
    return pb, ctx, box


@pytest.mark.parametrize("precision", [hz.HZ_MIXED, hz.HZ_FP64])
@pytest.mark.parametrize("lanes,B", [(2, 8), (4, 8), (2, 5)])
def test_lanes_match_oracle_and_one_group(precision, lanes, B):
    pb, ctx, box = _setup(lanes, precision)
    f = I.random_sources(pb.shape_ext, pb.n_pml, B, 42)
    ref = box.factor().solve(f)
    u, st = ctx.hz_solve(f)
    ctx.close()
    pb1, ctx1, _ = _setup(1, precision)
    u1, _ = ctx1.hz_solve(f)
    ctx1.close()
    assert st.resid < 1e-8
    assert np.all(O.relative_residual(box, u, f) < 1e-8)
    assert _rel(u, ref) < (1e-5 if precision == hz.HZ_MIXED else 1e-8)
    assert _rel(u, u1) < (1e-5 if precision == hz.HZ_MIXED else 1e-8)


def test_lanes_repeat_and_device_bytes():
    pb, ctx, box = _setup(2)
    f = I.random_sources(pb.shape_ext, pb.n_pml, 8, 43)
    b0 = ctx.hz_device_bytes()
    u, _ = ctx.hz_solve(f)
    b1 = ctx.hz_device_bytes()
    u2, st = ctx.hz_solve(f)
    ctx.close()
    assert b1 > b0  # the lane's workspaces count towards the context
    assert _rel(u2, u) < 1e-12
    assert st.gpu_launches > 0


def test_gradient_with_lanes_matches_one_group():
    pb, ctx, box = _setup(2)
    B, n_rec = 4, 30
    rng = np.random.default_rng(44)
    f = I.random_sources(pb.shape_ext, pb.n_pml, B, 45)
    rec = rng.choice(pb.shape_ext[0] * pb.shape_ext[1], n_rec, replace=False).astype(np.int32)
    d = rng.standard_normal((B, n_rec)) + 1j * rng.standard_normal((B, n_rec))
    J2, g2 = ctx.hz_gradient(f, d, rec)[:2]
    ctx.close()
    pb1, ctx1, _ = _setup(1)
    J1, g1 = ctx1.hz_gradient(f, d, rec)[:2]
    ctx1.close()
    assert abs(J2 - J1) <= 1e-6 * abs(J1)
    assert _rel(g2, g1) < 1e-5
