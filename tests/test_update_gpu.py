"""Local model update (hz_update_model; the paper's Conclusion: a locally
updated medium needs only a local modification of the method).  The reference
is the factorization of the new medium from scratch: a context updated in
place must solve exactly as a fresh context factored with the new medium (the
same kernels on the same data: agreement to 1e-12), and both must match the
oracle's direct solve of the new medium.  The layer count re-factored is the
number of layers whose cells read a changed value: cells read their layer's
interior rows (plus the outer PML rows at the top and bottom of the grid)."""
import numpy as np
import pytest

import hz_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

hz = pytest.importorskip("paper_1510_01831_gb300.hz")

N_, P_, L_, C_ = 96, 8, 4, 3


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _problem():
    pb = I.smooth_random(N_, n_pml=P_, L=L_, C=C_, seed=51, ppw=8, corr_pts=10)
    return pb, O.default_pml_C(pb.m)


def _ctx(pb, m, C_pml, precision, tc=True):
    ctx = hz.Context(m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=precision, pml_C=C_pml,
                     tensor_cores=tc)
    ctx.hz_factor()
    return ctx


def _blob(m, z0, z1, x0, x1, scale):
    m1 = m.copy()
    m1[z0:z1, x0:x1] *= scale
    return m1


@pytest.mark.parametrize("precision,tc", [(hz.HZ_FP64, True), (hz.HZ_MIXED, True), (hz.HZ_MIXED, 2)])
def test_update_equals_fresh_factorization(precision, tc):
    pb, C_pml = _problem()
    # layer 1 owns interior rows [P + 24, P + 48) of the extended grid (24 rows per layer)
    m1 = _blob(pb.m, P_ + 30, P_ + 40, 40, 52, 1.3)
    f = I.random_sources(pb.shape_ext, pb.n_pml, 4, 52)
    ctx = _ctx(pb, pb.m, C_pml, precision, tc)
    u0, _ = ctx.hz_solve(f)
    n = ctx.hz_update_model(m1)
    u1, st = ctx.hz_solve(f)
    ctx.close()
    fresh = _ctx(pb, m1, C_pml, precision, tc)
    u_ref, _ = fresh.hz_solve(f)
    fresh.close()
    box = O.Box(m1, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml)
    assert n == 1
    assert _rel(u1, u_ref) < 1e-12
    assert _rel(u1, box.factor().solve(f)) < (1e-8 if precision == hz.HZ_FP64 else 1e-5)
    assert np.all(O.relative_residual(box, u1, f) < 1e-8)
    assert _rel(u1, u0) > 1e-3  # the medium did change the field


def test_update_counts_touched_layers_and_keeps_context_on_errors():
    pb, C_pml = _problem()
    ctx = _ctx(pb, pb.m, C_pml, hz.HZ_MIXED)
    f = I.random_sources(pb.shape_ext, pb.n_pml, 2, 53)
    u0, _ = ctx.hz_solve(f)
    assert ctx.hz_update_model(pb.m) == 0  # same medium: nothing to do
    u_same, _ = ctx.hz_solve(f)
    assert _rel(u_same, u0) < 1e-12
    # a change in the bottom PML rows: only the last layer reads them
    m_pml = _blob(pb.m, pb.m.shape[0] - 3, pb.m.shape[0], 10, 30, 1.1)
    assert ctx.hz_update_model(m_pml) == 1
    # a change straddling the boundary between layers 1 and 2 touches both
    m_two = _blob(m_pml, P_ + 44, P_ + 52, 60, 70, 0.9)
    assert ctx.hz_update_model(m_two) == 2
    bad = m_two.copy()
    bad[5, 5] = np.nan
    with pytest.raises(hz.HzError):
        ctx.hz_update_model(bad)
    bad[5, 5] = -1.0
    with pytest.raises(hz.HzError):
        ctx.hz_update_model(bad)
    u2, st = ctx.hz_solve(f)  # still the factorization of m_two
    ctx.close()
    box = O.Box(m_two, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml)
    assert st.resid < 1e-8
    assert _rel(u2, box.factor().solve(f)) < 1e-5


def test_inversion_loop_gradient_after_update():
    """The gradient after a local update is the gradient of the new medium."""
    pb, C_pml = _problem()
    B, n_rec = 2, 40
    rng = np.random.default_rng(54)
    f = I.random_sources(pb.shape_ext, pb.n_pml, B, 55)
    rec = rng.choice(pb.m.size, n_rec, replace=False).astype(np.int32)
    d = rng.standard_normal((B, n_rec)) + 1j * rng.standard_normal((B, n_rec))
    m1 = _blob(pb.m, P_ + 5, P_ + 15, 20, 30, 1.2)
    ctx = _ctx(pb, pb.m, C_pml, hz.HZ_FP64)
    ctx.hz_update_model(m1)
    J1, g1 = ctx.hz_gradient(f, d, rec)[:2]
    ctx.close()
    fresh = _ctx(pb, m1, C_pml, hz.HZ_FP64)
    J2, g2 = fresh.hz_gradient(f, d, rec)[:2]
    fresh.close()
    assert abs(J1 - J2) <= 1e-12 * abs(J2)
    assert _rel(g1, g2) < 1e-12
