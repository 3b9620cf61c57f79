"""Adjoint entry point and the PyTorch autograd wrapper against the oracle."""
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
    pb = I.smooth_random(48, n_pml=5, L=3, C=2, seed=71, ppw=8, corr_pts=8, n_z=40)
    C_pml = O.default_pml_C(pb.m)
    box = O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml)
    return pb, C_pml, box, box.factor()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("mixed", 1e-5)])
def test_hz_adjoint_matches_oracle(case, precision, tol):
    pb, C_pml, box, fac = case
    B = 3
    f = I.random_sources(pb.shape_ext, pb.n_pml, B, 72)
    rng = np.random.default_rng(73)
    gu = rng.standard_normal(f.shape) + 1j * rng.standard_normal(f.shape)
    prec = hz.HZ_FP64 if precision == "fp64" else hz.HZ_MIXED
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=prec, pml_C=C_pml)
    ctx.hz_factor()
    u, _ = ctx.hz_solve(f)
    gm, gf, st = ctx.hz_adjoint(u, gu)
    ctx.close()
    uo = fac.solve(f)
    mu = fac.solve(np.conj(gu), trans=True)
    gm_ref = pb.omega ** 2 * np.sum(np.real(mu * uo), axis=0)
    assert _rel(gm, gm_ref) < tol
    assert _rel(gf, np.conj(mu)) < tol


def test_autograd_matches_finite_differences(case):
    torch = pytest.importorskip("torch")
    from paper_1510_01831_gb300 import torch_ops
    pb, C_pml, box, fac = case
    B = 2
    f = torch.from_numpy(I.point_sources_row(pb.n_x, pb.n_z, pb.n_pml, pb.h, B)).cuda()
    w = torch.from_numpy(np.random.default_rng(74).random(pb.shape_ext)).cuda()
    m = torch.from_numpy(pb.m.copy()).cuda().requires_grad_(True)
    op = torch_ops.HelmholtzOperator(m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, pml_C=C_pml)
    u = op(m, f)
    loss = (w * u.abs() ** 2).sum()
    loss.backward()
    g = m.grad.cpu().numpy()
    op.close()

    def J(mm):
        uu = O.Box(mm, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml).factor().solve(f.cpu().numpy())
        return float(np.sum(w.cpu().numpy() * np.abs(uu) ** 2))
    rng = np.random.default_rng(75)
    for i in rng.choice(pb.m.size, 6, replace=False):
        eps = 1e-6 * pb.m.reshape(-1)[i]
        mp, mm_ = pb.m.copy(), pb.m.copy()
        mp.reshape(-1)[i] += eps
        mm_.reshape(-1)[i] -= eps
        fd = (J(mp) - J(mm_)) / (2 * eps)
        assert abs(fd - g.reshape(-1)[i]) <= 1e-5 * np.abs(g).max() + 1e-4 * abs(fd)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_traces_reconstruct_roundtrip(case, precision, tol):
    # a field is recomputed from its source and its interface traces
    pb, C_pml, box, fac = case
    B = 3
    f = I.random_sources(pb.shape_ext, pb.n_pml, B, 76)
    prec = hz.HZ_FP64 if precision == "fp64" else hz.HZ_MIXED
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=prec, pml_C=C_pml)
    ctx.hz_factor()
    u, _ = ctx.hz_solve(f)
    tr = ctx.hz_traces(u)
    assert tr.shape == (B, pb.L - 1, 2, pb.n_x + 2 * pb.n_pml)
    # the traces are rows of u: last interior row of layer k, first of layer k+1
    rows = np.cumsum(ctx.rows)[:-1] + pb.n_pml  # first interior row of layers 1..L-1 (extended index)
    assert np.array_equal(tr[:, :, 1, :], u[:, rows, :])
    assert np.array_equal(tr[:, :, 0, :], u[:, rows - 1, :])
    u2 = ctx.hz_reconstruct(f, tr)
    # exact traces from the oracle give the oracle field
    uo = fac.solve(f)
    u3 = ctx.hz_reconstruct(f, np.ascontiguousarray(np.stack([uo[:, rows - 1, :], uo[:, rows, :]], axis=2)))
    ctx.close()
    assert _rel(u2, u) < tol
    assert _rel(u3, uo) < tol


def test_autograd_checkpoint_matches_stored_fields(case):
    torch = pytest.importorskip("torch")
    from paper_1510_01831_gb300 import torch_ops
    pb, C_pml, box, fac = case
    B = 3
    f0 = torch.from_numpy(I.random_sources(pb.shape_ext, pb.n_pml, B, 77)).cuda()
    w = torch.from_numpy(np.random.default_rng(78).random(pb.shape_ext)).cuda()
    grads = []
    for ck in (False, True):
        m = torch.from_numpy(pb.m.copy()).cuda().requires_grad_(True)
        f = f0.clone().requires_grad_(True)
        op = torch_ops.HelmholtzOperator(m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, pml_C=C_pml,
                                         checkpoint=ck)
        u = op(m, f)
        loss = (w * u.abs() ** 2).sum()
        loss.backward()
        grads.append((m.grad.cpu().numpy(), f.grad.cpu().numpy()))
        op.close()
    assert _rel(grads[1][0], grads[0][0]) < 1e-9
    assert _rel(grads[1][1], grads[0][1]) < 1e-9


def test_gradient_repeated_and_invalid_receivers(case):
    """Repeated receiver indices accumulate in the adjoint source (as in the
    oracle); out-of-range indices are rejected in both pointer modes before
    any kernel reads them."""
    torch = pytest.importorskip("torch")
    pb, C_pml, box, fac = case
    B = 2
    f = I.random_sources(pb.shape_ext, pb.n_pml, B, 79)
    top = I.receivers_top_row(pb.n_x, pb.n_pml).astype(np.int32)
    rec = np.concatenate([top, top[2:9], top[4:5]]).astype(np.int32)
    rng = np.random.default_rng(80)
    d = (rng.standard_normal((B, rec.size)) + 1j * rng.standard_normal((B, rec.size))) * 1e-3
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=hz.HZ_FP64,
                     pml_C=C_pml, tol=1e-12)
    ctx.hz_factor()
    J, g, _, _ = ctx.hz_gradient(f, d, rec)
    J_ref, g_ref, _ = O.misfit_gradient(box, f, d, rec, fac)
    assert abs(J - J_ref) <= 1e-9 * J_ref
    assert _rel(g, g_ref) < 1e-8
    bad = rec.copy()
    bad[3] = pb.m.size
    with pytest.raises(hz.HzError):
        ctx.hz_gradient(f, d, bad)
    ctx.hz_set_device_ptrs(True)
    fd_ = torch.from_numpy(f).cuda()
    dd_ = torch.from_numpy(d).cuda()
    Jd, gd, _, _ = ctx.hz_gradient(fd_, dd_, torch.from_numpy(rec).cuda())
    assert abs(Jd - J_ref) <= 1e-9 * J_ref
    assert _rel(gd.cpu().numpy(), g_ref) < 1e-8
    for v in (-1, pb.m.size):
        badd = torch.from_numpy(rec).cuda()
        badd[5] = v
        with pytest.raises(hz.HzError):
            ctx.hz_gradient(fd_, dd_, badd)
    ctx.close()
