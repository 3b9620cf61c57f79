"""The inner nested polarized traces on the GPU (Section 4.2; hz_opts.inner =
HZ_INNER_NESTED) against the oracle.

Every local solve of a layer goes through the layer's inner context: its box
with x and z swapped, whose layers are the cells, solved by FGMRES on the
cells' polarized traces with the Gauss-Seidel sweeps over the cells.

- one layer's Green's integrals (component entry point) against the oracle's
  direct layer solve, and against the oracle's own nested layer solve
  (tight inner tolerance: agreement to 1e-8);
- whole solves against the oracle's global direct solve: FP64 at the paper's
  inner tolerance 1e-6 inside the preconditioner (1e-8 bar; the polarized
  operator and the local solves of the Newton and reconstruction stages use
  tight inner solves), mixed precision (1e-5 bar);
- the outer iteration count with inexact inner solves stays within a few of
  the exact inner block LU's, and the inner solves report their iterations.
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
    pb = I.smooth_random(60, n_pml=5, L=3, C=3, seed=81, ppw=8, corr_pts=8, n_z=48)
    C_pml = O.default_pml_C(pb.m)
    D = O.Decomposition(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml, pb.L, pb.C)
    f = I.random_sources(pb.shape_ext, pb.n_pml, 3, 82)
    ref = D.box.factor().solve(f)
    return pb, C_pml, D, f, ref


def _ctx(pb, C_pml, **kw):
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, pml_C=C_pml,
                     inner=hz.HZ_INNER_NESTED, **kw)
    ctx.hz_factor()
    return ctx


@pytest.mark.parametrize("l,mask", [(0, 2), (1, 3), (2, 1)])
def test_nested_layer_green_matches_direct_and_oracle_nested(case, l, mask):
    pb, C_pml, D, f, ref = case
    B = 3
    rng = np.random.default_rng(83 + l)
    tr = rng.standard_normal((B, 4, D.NX)) + 1j * rng.standard_normal((B, 4, D.NX))
    if not (mask & 1):
        tr[:, 0:2] = 0
    if not (mask & 2):
        tr[:, 2:4] = 0
    ctx = _ctx(pb, C_pml, precision=hz.HZ_FP64)
    out = ctx.hz_layer_green(l, np.ascontiguousarray(tr), mask)
    ctx.close()
    direct = D.green(l, tr[:, 0], tr[:, 1], tr[:, 2], tr[:, 3])
    assert _rel(out, direct) < 1e-8
    # the oracle's nested layer solve (inner GMRES over the cells) gives the same samples
    ND = O.NestedDecomposition(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml, pb.L, pb.C, tol_inner=1e-11)
    nested = ND.green(l, tr[:, 0], tr[:, 1], tr[:, 2], tr[:, 3])
    assert _rel(out, nested) < 1e-8


def test_nested_solve_fp64_at_the_papers_inner_tolerance(case):
    pb, C_pml, D, f, ref = case
    ctx = _ctx(pb, C_pml, precision=hz.HZ_FP64, inner_tol=1e-6)
    u, st = ctx.hz_solve(f)
    ctx.close()
    exact = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, pml_C=C_pml, precision=hz.HZ_FP64)
    exact.hz_factor()
    ue, ste = exact.hz_solve(f)
    exact.close()
    assert _rel(u, ref) < 1e-8 and st.resid < 1e-8
    assert st.inner_iterations > 0
    assert st.iterations <= ste.iterations + 3, (st.iterations, ste.iterations)
    print(f"\nnested FP64: outer {st.iterations} its (exact inner LU: {ste.iterations}), "
          f"inner {st.inner_iterations} its, rel L2 {_rel(u, ref):.2e}")


def test_nested_solve_mixed(case):
    pb, C_pml, D, f, ref = case
    ctx = _ctx(pb, C_pml, precision=hz.HZ_MIXED)
    u, st = ctx.hz_solve(f)
    ctx.close()
    assert _rel(u, ref) < 1e-5 and st.resid < 1e-8


def test_nested_preconditioner_is_inexact_but_close(case):
    """P^GS through inner solves at 1e-6 differs from the exact one by about the
    inner tolerance, not more."""
    pb, C_pml, D, f, ref = case
    B = 2
    rng = np.random.default_rng(84)
    x = rng.standard_normal((B, pb.L - 1, 4, D.NX)) + 1j * rng.standard_normal((B, pb.L - 1, 4, D.NX))
    ctx = _ctx(pb, C_pml, precision=hz.HZ_FP64, inner_tol=1e-6)
    y = ctx.hz_precond(0, np.ascontiguousarray(x))
    ctx.close()
    y_ref = O.precond_gs(D, x)
    e = _rel(y, y_ref)
    assert 1e-12 < e < 1e-4, e
