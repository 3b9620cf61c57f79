"""The five workloads (exact where the oracle finishes in seconds, scaled twins
otherwise) against the CPU oracle, through the C ABI.

- constant medium 128 x 128 + 10 PML, L = C = 4, Gaussian source, FP64, GMRES
  tolerance 1e-10 (the exact small workload);
- layered-faulted medium (12 layers, sinusoidal interfaces, two dip-slip
  faults), mixed precision, L = 10 x C = 5: a 160 x 320 twin of the
  2000 x 4000 workload;
- smooth random medium with uneven layers and cells (24-64 points) at three
  frequencies (6, 8, 10 points per wavelength): a 192 x 192 twin;
- receiver misfit gradient with receivers on every node of the first row:
  a 96 x 96 twin against the oracle gradient.
At every size the FP64 residual of the Appendix A operator is checked too.
"""
import math

import numpy as np
import pytest

import hz_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

hz = pytest.importorskip("paper_1510_01831_gb300.hz")


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _oracle(pb, C_pml, f):
    box = O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml)
    return box, box.factor().solve(f)


def test_constant_medium_gaussian_source():
    pb = I.constant_medium(128, n_pml=10, L=4, C=4, ppw=10.0)
    assert abs(pb.omega - 2 * math.pi * 129 / 10) < 1e-9
    f = I.gaussian_source(pb.n_x, pb.n_z, pb.n_pml, pb.h, 0.5, 0.5, 2 * pb.h)[None]
    C_pml = O.default_pml_C(pb.m)
    box, ref = _oracle(pb, C_pml, f)
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=hz.HZ_FP64,
                     tol=1e-10, pml_C=C_pml)
    ctx.hz_factor()
    u, st = ctx.hz_solve(f)
    ctx.close()
    assert _rel(u, ref) < 1e-8
    assert st.gmres_resid <= 1e-10
    assert O.relative_residual(box, u, f)[0] < 1e-8


def test_layered_faulted_twin_mixed():
    pb = I.layered_faulted(n_x=160, n_z=320, n_pml=10, L=10, C=5, seed=3, ppw=8.0)
    c = 1.0 / np.sqrt(pb.m)
    assert 1.5 - 1e-9 <= c.min() and c.max() <= 5.5 + 1e-9
    f = np.zeros((4,) + pb.shape_ext, complex)
    cols = I.point_source_columns(pb.n_x, 4)
    for s, p in enumerate(cols):
        f[s, pb.n_pml, p + pb.n_pml - 1] = 1 / pb.h ** 2
    C_pml = O.default_pml_C(pb.m)
    box, ref = _oracle(pb, C_pml, f)
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=hz.HZ_MIXED,
                     pml_C=C_pml)
    ctx.hz_factor()
    u, st = ctx.hz_solve(f)
    ctx.close()
    for b in range(4):
        assert _rel(u[b], ref[b]) < 1e-5
    assert st.resid < 1e-8
    assert np.all(O.relative_residual(box, u, f) < 1e-8)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_uneven_multifrequency_twin(k):
    probs = I.uneven_multifreq(n=192, n_pml=10, seed=4, part_seed=40)
    pb = probs[k]
    assert len(set(pb.layer_rows)) > 1 and len(set(pb.cell_cols)) > 1
    assert min(pb.layer_rows + pb.cell_cols) >= 24 and max(pb.layer_rows + pb.cell_cols) <= 64
    f = I.point_sources_row(pb.n_x, pb.n_z, pb.n_pml, pb.h, 6)
    C_pml = O.default_pml_C(pb.m)
    box, ref = _oracle(pb, C_pml, f)
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=hz.HZ_MIXED,
                     pml_C=C_pml, layer_rows=pb.layer_rows, cell_cols=pb.cell_cols)
    ctx.hz_factor()
    u, st = ctx.hz_solve(f)
    ctx.close()
    assert _rel(u, ref) < 1e-5
    assert st.resid < 1e-8


def test_gradient_twin():
    p0, m_true = I.gradient_case(n=96, n_pml=10, L=4, C=4, seed=5, blob_pts=8)
    B = 6
    f = I.point_sources_row(p0.n_x, p0.n_z, p0.n_pml, p0.h, B)
    rec = I.receivers_top_row(p0.n_x, p0.n_pml)
    C_pml = O.default_pml_C(p0.m)
    d = O.Box(m_true, p0.n_x, p0.n_z, p0.n_pml, p0.omega, p0.h, C_pml).factor().solve(f).reshape(B, -1)[:, rec]
    box = O.Box(p0.m, p0.n_x, p0.n_z, p0.n_pml, p0.omega, p0.h, C_pml)
    J_ref, g_ref, _ = O.misfit_gradient(box, f, d, rec)
    for prec, tol in ((hz.HZ_FP64, 1e-7), (hz.HZ_MIXED, 1e-5)):
        ctx = hz.Context(p0.m, p0.n_x, p0.n_z, p0.omega, p0.h, p0.n_pml, p0.L, p0.C, precision=prec, pml_C=C_pml)
        ctx.hz_factor()
        J, g, u, st = ctx.hz_gradient(f, np.ascontiguousarray(d), rec.astype(np.int32))
        ctx.close()
        assert abs(J - J_ref) <= tol * abs(J_ref)
        assert _rel(g, g_ref) < 10 * tol


def test_uneven_rowless_cluster_ranks_wide_tiles():
    # Layers of 2nz' = 88..146 rows: with 16 CTAs per cluster the last CTA owns
    # no rows.  48 sources make the layer-parallel sweeps use 16-column tiles
    # and the single-layer sweeps 8-column tiles.  Repeated solves must agree.
    pb = I.uneven_multifreq(n=192, n_pml=10, seed=4, part_seed=40)[1]
    f = I.point_sources_row(pb.n_x, pb.n_z, pb.n_pml, pb.h, 48)
    C_pml = O.default_pml_C(pb.m)
    box, ref = _oracle(pb, C_pml, f)
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=hz.HZ_MIXED,
                     pml_C=C_pml, layer_rows=pb.layer_rows, cell_cols=pb.cell_cols)
    ctx.hz_factor()
    us = [ctx.hz_solve(f)[0] for _ in range(3)]
    ctx.close()
    for u in us:
        assert _rel(u, ref) < 1e-5
        assert np.all(O.relative_residual(box, u, f) < 1e-8)
    assert _rel(us[1], us[0]) < 1e-12 and _rel(us[2], us[0]) < 1e-12
