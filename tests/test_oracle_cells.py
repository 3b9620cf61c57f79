"""Pins of the oracle's cell boxes (Section 4: a layer split into cells, each
cell a local problem with its own artificial PML in x).

Every cell-solve parity test of the CUDA path takes its expected value from
``Decomposition.cell_box``; these tests pin that box against facts that do
not come from it:

* Appendix C at the cell level (Section 4.2): the cell's local solve, with
  the interface forcing built from the layer's own solution at the cell's
  boundary columns, reproduces that solution on the columns the cell owns and
  gives exactly zero at its columns 0 and w+1.  A cell box whose interior
  columns are shifted, whose artificial PML reaches into column 1/2 or w+1/2,
  or whose rows differ from the layer's (its z-PML included) fails this.
* the cell box is the layer box of the layer's swapped-axes decomposition
  with x and z exchanged (the reading under which the inner level is the
  outer method on the transposed layer), operator entry by entry.

Cases: interior, edge and corner cells of the top, a middle and the bottom
layer, on an uneven partition.
"""
import numpy as np
import pytest

import hz_inputs as I
import oracle as O


@pytest.fixture(scope="module")
def uneven():
    pb = I.smooth_random(37, n_pml=4, L=3, C=3, seed=71, ppw=8, corr_pts=6, n_z=29)
    rows, cols = [9, 12, 8], [10, 15, 12]
    D = O.Decomposition(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, O.default_pml_C(pb.m), 3, 3,
                        layer_rows=rows, cell_cols=cols)
    return D


def _owned_cols(D, c):
    """Array columns of cell c's box that belong to it in the layer (the outer
    PML columns go with the edge cells)."""
    p, w = D.p, D.cols[c]
    lo = 0 if c == 0 else p
    hi = w + 2 * p if c == D.C - 1 else w + p
    return lo, hi


def _cell_interface_source(cb, v_cols):
    """Appendix C forcing in x on the cell box cb from the layer field's values
    at the cell's local columns 0, 1, w, w+1 (v_cols[k]: a column of length
    nz'), with the cell's own couplings."""
    NZc, NXc = cb.shape
    w, p = cb.nxi, cb.p
    c0, c1, cw, cw1 = p - 1, p, w + p - 1, w + p   # array columns of local nodes 0, 1, w, w+1
    g = np.zeros(cb.shape, complex)
    for z in range(NZc):
        def H(a, b):
            return cb.entry(z * NXc + a, z * NXc + b)
        if v_cols[0] is not None:
            g[z, c0] += H(c0, c1) * v_cols[1][z]
            g[z, c1] += -H(c1, c0) * v_cols[0][z]
        if v_cols[2] is not None:
            g[z, cw1] += H(cw1, cw) * v_cols[2][z]
            g[z, cw] += -H(cw, cw1) * v_cols[3][z]
    return g


@pytest.mark.parametrize("l", [0, 1, 2])
@pytest.mark.parametrize("c", [0, 1, 2])
def test_cell_identity_reproduces_layer_solution(uneven, l, c):
    D = uneven
    lb = D.layer_box(l)
    rng = np.random.default_rng(100 + 3 * l + c)
    g = rng.standard_normal(lb.shape) + 1j * rng.standard_normal(lb.shape)
    v = lb.factor().solve(g)                         # the layer's own solution
    cb = D.cell_box(l, c)
    assert cb.shape == (lb.shape[0], D.cols[c] + 2 * D.p)
    p, w, t = D.p, D.cols[c], D.t[c]
    # cell array column j <-> layer array column t + j
    lo, hi = _owned_cols(D, c)
    src = np.zeros(cb.shape, complex)
    src[:, lo:hi] = g[:, t + lo:t + hi]
    left = (v[:, t + p - 1], v[:, t + p]) if c > 0 else (None, None)
    right = (v[:, t + w + p - 1], v[:, t + w + p]) if c < D.C - 1 else (None, None)
    src += _cell_interface_source(cb, (*left, *right))
    x = cb.factor().solve(src)
    ref = v[:, t + lo:t + hi]
    assert np.linalg.norm(x[:, lo:hi] - ref) <= 1e-12 * np.linalg.norm(ref)
    if c > 0:
        assert np.linalg.norm(x[:, p - 1]) <= 1e-12 * np.linalg.norm(ref)
        assert np.linalg.norm(x[:, :p - 1]) <= 1e-12 * np.linalg.norm(ref)  # artificial PML stays empty
    if c < D.C - 1:
        assert np.linalg.norm(x[:, w + p]) <= 1e-12 * np.linalg.norm(ref)
        assert np.linalg.norm(x[:, w + p + 1:]) <= 1e-12 * np.linalg.norm(ref)


def test_identity_fails_for_a_shifted_cell(uneven):
    """Negative control: the same construction on a cell box whose medium is
    shifted by one column does not reproduce the layer solution."""
    D = uneven
    l, c = 1, 1
    lb = D.layer_box(l)
    rng = np.random.default_rng(5)
    g = rng.standard_normal(lb.shape) + 1j * rng.standard_normal(lb.shape)
    v = lb.factor().solve(g)
    good = D.cell_box(l, c)
    bad = O.Box(np.roll(good.m, 1, axis=1), good.nxi, good.nzi, good.p, good.omega, good.h, good.C)
    p, w, t = D.p, D.cols[c], D.t[c]
    lo, hi = _owned_cols(D, c)
    src = np.zeros(bad.shape, complex)
    src[:, lo:hi] = g[:, t + lo:t + hi]
    src += _cell_interface_source(bad, (v[:, t + p - 1], v[:, t + p], v[:, t + w + p - 1], v[:, t + w + p]))
    x = bad.factor().solve(src)
    ref = v[:, t + lo:t + hi]
    assert np.linalg.norm(x[:, lo:hi] - ref) > 1e-6 * np.linalg.norm(ref)


@pytest.mark.parametrize("l", [0, 1, 2])
def test_cell_box_is_transposed_inner_layer_box(uneven, l):
    D = uneven
    DT = O.layer_inner_decomposition(D, l)
    rng = np.random.default_rng(40 + l)
    for c in range(D.C):
        cb, tb = D.cell_box(l, c), DT.layer_box(c)
        assert cb.shape == tb.shape[::-1]
        assert np.array_equal(cb.m, tb.m.T)
        u = rng.standard_normal((2,) + cb.shape) + 1j * rng.standard_normal((2,) + cb.shape)
        a = cb.apply(u)
        b = np.swapaxes(tb.apply(np.swapaxes(u, -1, -2)), -1, -2)
        assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(a)
