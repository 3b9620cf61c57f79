"""The oracle's inner nested polarized traces (Section 4.2), pinned to what the
mathematics fixes: the operator of Appendix A is the same with the axes swapped
(exact, to roundoff), the nested layer solve reproduces the direct layer solve
to its GMRES tolerance, and the nested method as a whole (outer polarized
traces over layers, inner over cells) reproduces the direct global solve."""
import numpy as np
import pytest

import hz_inputs as I
import oracle as O


@pytest.fixture(scope="module")
def dec():
    pb = I.smooth_random(30, n_pml=4, L=3, C=3, seed=61, ppw=8, corr_pts=6, n_z=33)
    C_pml = O.default_pml_C(pb.m)
    return pb, C_pml


def test_swapped_axes_box_is_the_same_operator(dec):
    pb, C_pml = dec
    box = O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml)
    boxT = O.Box(pb.m.T.copy(), pb.n_z, pb.n_x, pb.n_pml, pb.omega, pb.h, C_pml)
    rng = np.random.default_rng(62)
    u = rng.standard_normal(box.shape) + 1j * rng.standard_normal(box.shape)
    Hu = box.apply(u)
    HTuT = boxT.apply(u.T.copy())
    assert np.linalg.norm(HTuT.T - Hu) <= 1e-13 * np.linalg.norm(Hu)
    # and therefore the same solution
    f = rng.standard_normal(box.shape) + 1j * rng.standard_normal(box.shape)
    v = box.factor().solve(f)
    vT = boxT.factor().solve(f.T.copy())
    assert np.linalg.norm(vT.T - v) <= 1e-11 * np.linalg.norm(v)


@pytest.mark.parametrize("l", [0, 1, 2])
def test_nested_layer_solve_matches_direct(dec, l):
    pb, C_pml = dec
    D = O.Decomposition(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml, pb.L, pb.C)
    rng = np.random.default_rng(63 + l)
    shp = D.layer_box(l).shape
    g = rng.standard_normal((2,) + shp) + 1j * rng.standard_normal((2,) + shp)
    ref = D.layer_factor(l).solve(g)
    v, its = O.nested_layer_solve(O.layer_inner_decomposition(D, l), g, tol=1e-11)
    assert np.linalg.norm(v - ref) <= 1e-8 * np.linalg.norm(ref)
    assert 1 <= its <= 30


def test_inner_gauss_seidel_beats_jacobi(dec):
    """The inner preconditioners keep the outer ordering: GS needs fewer
    iterations than Jacobi on a layer's cell system (Section 3.1)."""
    pb, C_pml = dec
    D = O.Decomposition(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml, pb.L, pb.C)
    DT = O.layer_inner_decomposition(D, 1)
    rng = np.random.default_rng(66)
    shp = D.layer_box(1).shape
    g = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    _, it_gs = O.nested_layer_solve(DT, g, tol=1e-10, precond=O.precond_gs)
    _, it_j = O.nested_layer_solve(DT, g, tol=1e-10, precond=O.precond_jac)
    assert it_gs < it_j


def test_nested_method_reproduces_global_solve(dec):
    pb, C_pml = dec
    D = O.NestedDecomposition(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml, pb.L, pb.C, tol_inner=1e-12)
    f = I.random_sources(pb.shape_ext, pb.n_pml, 1, 67)[0]
    ref = D.box.factor().solve(f)
    rhs = O.polarized_rhs(D, f)
    x, its, _ = O.gmres(lambda y: O.apply_M(D, y), rhs, lambda y: O.precond_gs(D, y), tol=1e-11, maxit=60)
    u = O.reconstruct(D, f, x[:, 0:2] + x[:, 2:4])
    assert np.linalg.norm(u - ref) <= 1e-8 * np.linalg.norm(ref)
    assert np.all(O.relative_residual(D.box, u, f) < 1e-9)
    assert len(D.inner_iterations) > 0 and max(D.inner_iterations) <= 30


def test_inexact_inner_solves_as_in_the_paper(dec):
    """The paper runs the nested method with inner solves to 1e-6 inside a
    flexible outer GMRES: the outer iteration count stays within two of the
    exact-inner count and the field is accurate to the inner tolerance's
    order."""
    pb, C_pml = dec
    f = I.random_sources(pb.shape_ext, pb.n_pml, 1, 68)[0]
    ref = O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml).factor().solve(f)
    out = {}
    for tol_inner in (1e-12, 1e-6):
        D = O.NestedDecomposition(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml, pb.L, pb.C,
                                  tol_inner=tol_inner)
        rhs = O.polarized_rhs(D, f)
        x, its, _ = O.gmres(lambda y: O.apply_M(D, y), rhs, lambda y: O.precond_gs(D, y), tol=1e-6, maxit=60)
        u = O.reconstruct(D, f, x[:, 0:2] + x[:, 2:4])
        out[tol_inner] = (its, np.linalg.norm(u - ref) / np.linalg.norm(ref), max(D.inner_iterations))
    assert out[1e-6][0] <= out[1e-12][0] + 2
    assert out[1e-6][1] <= 1e-4
    assert out[1e-6][2] < out[1e-12][2]  # looser inner solves take fewer inner iterations
