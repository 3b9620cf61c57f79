"""Parity at the full workload sizes, in the launch configuration the
benchmark times (mixed precision, 1e-8 refinement target).

Element by element against the oracle's direct solve (relative L2 error per
source: <= 1e-5 mixed, <= 1e-8 FP64):
- 1024 x 1024 + 20 PML, L = C = 16, 64 point sources on row 1 (smooth
  random), every source, both precisions, against the oracle's row-block
  elimination of the whole grid (19 GB of Schur factors on the host);
- the layered, faulted medium at 1000 x 2000 + 30 PML with L = 20 x C = 10:
  the 2000 x 4000 generator halved in each direction, so layers and cells
  keep the 100 x 100 shape of the full workload (the full grid's direct
  solve needs 275 GB of factors);
- 512 x 512 + 20 PML, uneven 24-64 point layers and cells, 6/8/10 points per
  wavelength, 256 sources each, solved as one group, every source.
At the full 2000 x 4000 size, through the FP64 residual ||H u - f|| / ||f||
of the GPU solution measured with the oracle's Appendix A operator.  For the
gradient workload (512 x 512, L = C = 8, 32 sources) the adjoint gradient
against central differences of the misfit at sampled nodes.
"""
import numpy as np
import pytest

import hz_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

hz = pytest.importorskip("paper_1510_01831_gb300.hz")
torch = pytest.importorskip("torch")


def _solve(pb, f, C_pml, precision=None, **kw):
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C,
                     precision=hz.HZ_MIXED if precision is None else precision, pml_C=C_pml, refine_tol=1e-8,
                     layer_rows=pb.layer_rows, cell_cols=pb.cell_cols, **kw)
    ctx.hz_factor()
    u, st = ctx.hz_solve(f)
    return ctx, u, st


def _rel_per_source(u, ref):
    d = (u - ref).reshape(u.shape[0], -1)
    return np.linalg.norm(d, axis=1) / np.linalg.norm(ref.reshape(u.shape[0], -1), axis=1)


def test_smooth1024_elementwise_against_oracle():
    pb = I.smooth_random(1024, n_pml=20, L=16, C=16, seed=2, ppw=10.0)
    f = I.point_sources_row(pb.n_x, pb.n_z, pb.n_pml, pb.h, 64)
    C_pml = O.default_pml_C(pb.m)
    box = O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml)
    ctx, u, st = _solve(pb, f, C_pml)
    ctx.close()
    res = O.relative_residual(box, u, f)
    assert np.all(res < 1e-8), res.max()
    assert abs(res.max() - st.resid) <= 1e-3 * st.resid + 1e-12  # the library's own FP64 residual agrees
    ctx, u64, st64 = _solve(pb, f, C_pml, precision=hz.HZ_FP64)
    ctx.close()
    ref = box.factor_rows().solve(f)
    e_mixed, e_fp64 = _rel_per_source(u, ref), _rel_per_source(u64, ref)
    print(f"\n1024^2 smooth, 64 sources: relative L2 vs oracle mixed max {e_mixed.max():.3e} "
          f"median {np.median(e_mixed):.3e} (residual {st.resid:.2e}); FP64 max {e_fp64.max():.3e}")
    assert np.all(e_mixed <= 1e-5), e_mixed.max()
    assert np.all(e_fp64 <= 1e-8), e_fp64.max()


def test_layered_faulted_twin_1000x2000_elementwise_against_oracle():
    pb = I.layered_faulted(n_x=1000, n_z=2000, n_pml=30, L=20, C=10, seed=3, ppw=8.0)
    assert pb.n_x // pb.C == 100 and pb.n_z // pb.L == 100   # the cells of the 2000 x 4000 workload
    f = I.point_sources_row(pb.n_x, pb.n_z, pb.n_pml, pb.h, 16)
    C_pml = O.default_pml_C(pb.m)
    box = O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml)
    ctx, u, st = _solve(pb, f, C_pml)
    ctx.close()
    ctx, u64, _ = _solve(pb, f, C_pml, precision=hz.HZ_FP64)
    ctx.close()
    ref = box.factor_rows().solve(f)
    e_mixed, e_fp64 = _rel_per_source(u, ref), _rel_per_source(u64, ref)
    print(f"\n1000x2000 layered twin, 16 sources: relative L2 vs oracle mixed max {e_mixed.max():.3e} "
          f"(residual {st.resid:.2e}); FP64 max {e_fp64.max():.3e}")
    assert np.all(e_mixed <= 1e-5), e_mixed.max()
    assert np.all(e_fp64 <= 1e-8), e_fp64.max()


def test_layered_faulted_2000x4000_residual():
    pb = I.layered_faulted(n_x=2000, n_z=4000, n_pml=30, L=40, C=20, seed=3, ppw=8.0)
    f = I.point_sources_row(pb.n_x, pb.n_z, pb.n_pml, pb.h, 16)
    C_pml = O.default_pml_C(pb.m)
    ctx, u, st = _solve(pb, f, C_pml)
    ctx.close()
    box = O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml)
    res = O.relative_residual(box, u, f)
    assert np.all(res < 1e-8), res.max()


def test_uneven_multifrequency_512_group_elementwise_against_oracle():
    probs = I.uneven_multifreq(n=512, n_pml=20, seed=4, part_seed=40)
    ctxs, fs, boxes = [], [], []
    for pb in probs:
        C_pml = O.default_pml_C(pb.m)
        f = I.point_sources_row(pb.n_x, pb.n_z, pb.n_pml, pb.h, 256)
        s = torch.cuda.Stream()
        ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=hz.HZ_MIXED,
                         pml_C=C_pml, layer_rows=pb.layer_rows, cell_cols=pb.cell_cols, stream=s.cuda_stream)
        ctx.hz_factor()
        ctxs.append(ctx)
        fs.append(f)
        boxes.append(O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml))
    us, sts = hz.hz_solve_group(ctxs, fs)
    for c in ctxs:
        c.close()
    for box, u, f, st in zip(boxes, us, fs, sts):
        res = O.relative_residual(box, u, f)
        assert np.all(res < 1e-8), res.max()
        e = _rel_per_source(u, box.factor_rows().solve(f))
        print(f"\n512^2 uneven, omega {box.omega:.1f}, 256 sources: relative L2 vs oracle max {e.max():.3e}")
        assert np.all(e <= 1e-5), e.max()


def test_gradient_512_against_central_differences():
    p0, m_true = I.gradient_case(n=512, n_pml=20, L=8, C=8, seed=5, blob_pts=30)
    B = 32
    f = I.point_sources_row(p0.n_x, p0.n_z, p0.n_pml, p0.h, B)
    rec = I.receivers_top_row(p0.n_x, p0.n_pml).astype(np.int32)
    C_pml = O.default_pml_C(p0.m)

    def ctx_for(m):
        ctx = hz.Context(m, p0.n_x, p0.n_z, p0.omega, p0.h, p0.n_pml, p0.L, p0.C, precision=hz.HZ_FP64,
                         pml_C=C_pml, tol=1e-12)
        ctx.hz_factor()
        return ctx
    ct = ctx_for(m_true)
    ut, _ = ct.hz_solve(f)
    ct.close()
    d = np.ascontiguousarray(ut.reshape(B, -1)[:, rec])
    c0 = ctx_for(p0.m)
    J0, g, _, _ = c0.hz_gradient(f, d, rec)
    c0.close()
    assert J0 > 0

    def J(m):
        c = ctx_for(m)
        u, _ = c.hz_solve(f)
        c.close()
        r = u.reshape(B, -1)[:, rec] - d
        return 0.5 * float(np.sum(np.abs(r) ** 2))
    NX = p0.n_x + 2 * p0.n_pml
    cz, cx = p0.n_pml + p0.n_z // 2, p0.n_pml + p0.n_x // 2  # blob centre and two nearby nodes
    for (iz, ix) in ((cz, cx), (cz - 40, cx + 25), (p0.n_pml + 60, cx - 100)):
        i = iz * NX + ix
        eps = 1e-4 * p0.m.reshape(-1)[i]
        mp, mm = p0.m.copy(), p0.m.copy()
        mp.reshape(-1)[i] += eps
        mm.reshape(-1)[i] -= eps
        fd = (J(mp) - J(mm)) / (2 * eps)
        gi = g.reshape(-1)[i]
        assert abs(gi - fd) <= 1e-4 * np.abs(g).max() + 1e-3 * abs(fd), (iz, ix, gi, fd)
