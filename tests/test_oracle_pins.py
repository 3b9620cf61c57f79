"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: library
routines, closed forms, the continuum Green's function, finite differences,
or structural statements of the paper.  A plausible slip in the oracle (a
dropped PML factor, a wrong sign of omega^2, a misplaced half-node alpha, a
transposed coupling, a bad pivot) fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy.special import hankel1

import hz_inputs as I
import oracle as O


def _box(pb, C=None):
    C = O.default_pml_C(pb.m) if C is None else C
    return O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C)


def _tiny(seed=1, n=20, nz=None, p=4):
    return I.smooth_random(n, n_pml=p, L=2, C=2, seed=seed, ppw=8, corr_pts=5, n_z=nz)


# ---------------------------------------------------------------- solver ---

@pytest.mark.parametrize("seed,n,nz", [(1, 20, 20), (2, 24, 17), (3, 15, 30)])
def test_manufactured_solution(seed, n, nz):
    """f = H u for a seeded random u is solved back to roundoff."""
    box = _box(_tiny(seed, n, nz))
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((3,) + box.shape) + 1j * rng.standard_normal((3,) + box.shape)
    f = box.apply(u)
    fac = box.factor()
    assert np.linalg.norm(fac.solve(f) - u) / np.linalg.norm(u) < 1e-11
    # transposed solve from the same factors
    A = box.dense()
    x = fac.solve(f, trans=True)
    res = A.T @ x.reshape(3, -1).T - f.reshape(3, -1).T
    assert np.linalg.norm(res) / np.linalg.norm(f) < 1e-12


def test_lu_matches_library_dense_solve():
    """Banded LU agrees with LAPACK's dense solve on the same matrix."""
    box = _box(_tiny(4, 18, 22))
    A = box.dense()
    rng = np.random.default_rng(4)
    f = rng.standard_normal(box.shape) + 1j * rng.standard_normal(box.shape)
    x_lib = np.linalg.solve(A, f.reshape(-1))
    x = box.factor().solve(f).reshape(-1)
    assert np.linalg.norm(x - x_lib) / np.linalg.norm(x_lib) < 1e-12


@pytest.mark.parametrize("n,nz,p,keep", [(30, 24, 4, 1), (17, 40, 3, 3), (64, 64, 8, 1), (40, 52, 6, 7)])
def test_row_block_elimination_matches_band_lu(n, nz, p, keep):
    """The block-tridiagonal (row-block) elimination used for grids whose band
    LU does not fit in memory agrees with the pivoted band LU and recovers a
    manufactured solution; with only every k-th Schur factor kept the
    recomputed segments give the same solution."""
    pb = I.smooth_random(n, n_pml=p, L=2, C=2, seed=n + nz, ppw=8, corr_pts=5, n_z=nz)
    box = _box(pb)
    st = box.stencil()
    rng = np.random.default_rng(n)
    u = rng.standard_normal((3,) + box.shape) + 1j * rng.standard_normal((3,) + box.shape)
    # the stencil planes are the operator's rows
    Hu = (st[2] * u
          + np.pad(st[0][1:] * u[:, :-1], ((0, 0), (1, 0), (0, 0)))
          + np.pad(st[4][:-1] * u[:, 1:], ((0, 0), (0, 1), (0, 0)))
          + np.pad(st[1][:, 1:] * u[:, :, :-1], ((0, 0), (0, 0), (1, 0)))
          + np.pad(st[3][:, :-1] * u[:, :, 1:], ((0, 0), (0, 0), (0, 1))))
    f = box.apply(u)
    assert np.linalg.norm(Hu - f) <= 1e-14 * np.linalg.norm(f)
    rb = box.factor_rows(keep)
    x = rb.solve(f)
    assert np.linalg.norm(x - u) <= 1e-11 * np.linalg.norm(u)
    g = I.random_sources(box.shape, p, 2, n)
    ref = box.factor().solve(g)
    assert np.linalg.norm(rb.solve(g) - ref) <= 1e-12 * np.linalg.norm(ref)


def test_pivoting_needed_case():
    """A zero leading diagonal entry (omega^2 m equal to the Laplacian diagonal)
    forces a row exchange; the factorization still solves exactly."""
    pb = _tiny(5, 12, 12, p=2)
    pb.m[0, 0] = 0.0
    box = O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, 0.0)
    d = box.entry(0, 0)
    pb.m[0, 0] = d.real / pb.omega ** 2
    box = O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, 0.0)
    assert abs(box.entry(0, 0)) < 1e-9 * abs(d)
    A = box.dense()
    rng = np.random.default_rng(5)
    f = rng.standard_normal(box.shape) + 0j
    x = box.factor().solve(f).reshape(-1)
    assert np.linalg.norm(A @ x - f.reshape(-1)) / np.linalg.norm(f) < 1e-10


# ------------------------------------------------------------- operator ---

def test_interior_stencil_exact_on_quadratics():
    """Away from the PML the operator is the textbook 5-point -Laplacian minus
    omega^2 m (Appendix A), exact on quadratic polynomials."""
    pb = _tiny(6, 16, 14, p=3)
    box = _box(pb)
    NZ, NX = box.shape
    k_x = np.arange(NX) - pb.n_pml + 1.0
    k_z = np.arange(NZ) - pb.n_pml + 1.0
    Z, X = np.meshgrid(k_z * pb.h, k_x * pb.h, indexing="ij")
    u = (X - 0.3) ** 2 + 3.0 * (Z - 0.1) ** 2 + 2.0 * X * Z + X + 0j
    lap = 2.0 + 6.0
    Hu = box.apply(u[None])[0]
    expect = -lap - pb.omega ** 2 * pb.m * u
    p = pb.n_pml
    sl = (slice(p, p + pb.n_z), slice(p, p + pb.n_x))
    err = np.abs(Hu[sl] - expect[sl]).max() / np.abs(expect[sl]).max()
    assert err < 1e-10


def test_dirichlet_laplacian_closed_form_eigenvalues():
    """With no absorption (C = 0) and m = 0 the operator is the Dirichlet
    5-point Laplacian on the whole extended grid: its eigenvalues are
    (4/h^2)(sin^2(j pi/(2(NX+1))) + sin^2(k pi/(2(NZ+1))))."""
    n, nz, p, h = 9, 7, 2, 0.1
    box = O.Box(np.zeros((nz + 2 * p, n + 2 * p)), n, nz, p, 3.0, h, 0.0)
    ev = np.sort(np.linalg.eigvals(box.dense()).real)
    NX, NZ = n + 2 * p, nz + 2 * p
    j = np.arange(1, NX + 1)
    k = np.arange(1, NZ + 1)
    lam = (4 / h ** 2) * (np.sin(j[:, None] * np.pi / (2 * (NX + 1))) ** 2
                          + np.sin(k[None, :] * np.pi / (2 * (NZ + 1))) ** 2)
    assert np.allclose(ev, np.sort(lam.reshape(-1)), rtol=1e-10, atol=1e-8)


def test_row_scaled_operator_is_complex_symmetric():
    """Dividing row (p,q) by alpha_x(p) alpha_z(q) gives a complex-symmetric
    matrix (the symmetric form of Appendix B, in finite differences).  This
    holds only if the half-node alphas sit on the couplings and the node
    alphas outside, as Appendix A prints."""
    pb = _tiny(7, 14, 12, p=4)
    box = _box(pb)
    A = box.dense()
    ax = box.alpha(0, np.arange(box.shape[1]))
    az = box.alpha(1, np.arange(box.shape[0]))
    D = (az[:, None] * ax[None, :]).reshape(-1)
    S = A / D[:, None]
    assert np.abs(S - S.T).max() <= 1e-13 * np.abs(S).max()
    # and the unscaled form is genuinely unsymmetric inside the PML
    assert np.abs(A - A.T).max() > 1e-6 * np.abs(A).max()
    # alpha is exactly 1 on the closed interior interval [0, (n+1)h]
    pos = np.arange(pb.n_pml - 1, pb.n_pml + pb.n_x + 0.25, 0.5)
    assert np.allclose(box.alpha(0, pos), 1.0)


def _hankel_err(n, C_scale=1.0):
    om = 2 * math.pi * 4
    h = 1.0 / (n + 1)
    p = int(round(0.25 / h))
    m = np.ones((n + 2 * p, n + 2 * p))
    box = O.Box(m, n, n, p, om, h, C_scale * O.default_pml_C(m))
    f = np.zeros(box.shape, complex)
    c = (n + 1) // 2 + p - 1
    f[c, c] = 1 / h ** 2
    u = box.factor().solve(f)
    X = (np.arange(box.shape[0]) - p + 1) * h
    ZZ, XX = np.meshgrid(X, X, indexing="ij")
    r = np.hypot(XX - 0.5, ZZ - 0.5)
    mask = (r >= 0.25) & (r <= 0.4) & (XX > 0.05) & (XX < 0.95) & (ZZ > 0.05) & (ZZ < 0.95)
    ex = 0.25j * hankel1(0, om * r[mask])
    return np.linalg.norm(u[mask] - ex) / np.linalg.norm(ex)


def test_constant_medium_converges_to_hankel_at_second_order():
    """Point source e_s/h^2 in m = 1: the discrete field tends to the outgoing
    continuum Green's function (i/4) H0^(1)(omega r) at O(h^2).  This pins the
    sign of omega^2, the 1/h^2 Dirac, the PML sign convention and absorption."""
    errs = [_hankel_err(n) for n in (31, 63, 127)]
    assert errs[2] < 0.015
    for e0, e1 in zip(errs[:-1], errs[1:]):
        assert 3.5 < e0 / e1 < 4.6
    # without absorption the box rings and the field is far from outgoing
    assert _hankel_err(63, C_scale=0.0) > 0.3


# ------------------------------------------------------------- gradient ---

def test_misfit_gradient_matches_central_differences():
    pb = _tiny(8, 16, 16, p=4)
    box = _box(pb)
    B = 2
    f = I.random_sources(box.shape, pb.n_pml, B, 8)
    rec = I.receivers_top_row(pb.n_x, pb.n_pml)
    rng = np.random.default_rng(8)
    d = rng.standard_normal((B, rec.size)) * 1e-3 + 0j
    J, g, _ = O.misfit_gradient(box, f, d, rec)
    idx = rng.choice(box.N, size=12, replace=False)
    for i in idx:
        eps = 1e-6 * max(abs(pb.m.reshape(-1)[i]), 1.0)
        Js = []
        for s in (+1, -1):
            m2 = pb.m.copy()
            m2.reshape(-1)[i] += s * eps
            b2 = O.Box(m2, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, box.C)
            Js.append(O.misfit_gradient(b2, f, d, rec)[0])
        fd = (Js[0] - Js[1]) / (2 * eps)
        assert abs(fd - g.reshape(-1)[i]) <= 1e-5 * np.abs(g).max() + 1e-4 * abs(fd)


def test_misfit_gradient_with_repeated_receivers():
    """A node listed twice as a receiver counts twice in J; the adjoint source
    R^T conj(r) must then carry both residuals (central differences of J)."""
    pb = _tiny(18, 14, 14, p=3)
    box = _box(pb)
    B = 2
    f = I.random_sources(box.shape, pb.n_pml, B, 18)
    top = I.receivers_top_row(pb.n_x, pb.n_pml)
    rec = np.concatenate([top, top[3:7], top[5:6]])   # four nodes twice, one three times
    rng = np.random.default_rng(18)
    d = (rng.standard_normal((B, rec.size)) + 1j * rng.standard_normal((B, rec.size))) * 1e-3
    J, g, _ = O.misfit_gradient(box, f, d, rec)
    for i in (rec[5], rec[0], box.N // 2):
        eps = 1e-6 * abs(pb.m.reshape(-1)[i])
        Js = []
        for s in (+1, -1):
            m2 = pb.m.copy()
            m2.reshape(-1)[i] += s * eps
            b2 = O.Box(m2, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, box.C)
            Js.append(O.misfit_gradient(b2, f, d, rec)[0])
        fd = (Js[0] - Js[1]) / (2 * eps)
        assert abs(fd - g.reshape(-1)[i]) <= 1e-5 * np.abs(g).max() + 1e-4 * abs(fd)


def test_adjoint_dot_product():
    """<H^{-1} a, b> = <a, H^{-T} b> (bilinear form)."""
    box = _box(_tiny(9, 14, 18))
    rng = np.random.default_rng(9)
    a = rng.standard_normal(box.shape) + 1j * rng.standard_normal(box.shape)
    b = rng.standard_normal(box.shape) + 1j * rng.standard_normal(box.shape)
    fac = box.factor()
    lhs = np.sum(fac.solve(a) * b)
    rhs = np.sum(a * fac.solve(b, trans=True))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# -------------------------------------------- decomposition and SIE ---

@pytest.fixture(scope="module")
def small_decomp():
    pb = I.smooth_random(30, n_pml=4, L=4, C=3, seed=11, ppw=8, corr_pts=6, n_z=36)
    D = O.Decomposition(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h,
                        O.default_pml_C(pb.m), pb.L, pb.C)
    f = I.random_sources(pb.shape_ext, pb.n_pml, 1, 12)[0]
    u = D.box.factor().solve(f)
    return D, f, u


def test_local_green_identity_reproduces_restriction(small_decomp):
    """Appendix C: each layer's solve with the interface forcing built from the
    global traces returns u on the layer's rows and 0 at its rows 0 and n+1."""
    D, f, u = small_decomp
    tr = D.traces(u)
    z = np.zeros(D.NX, complex)
    for l in range(D.L):
        t0, t1 = (tr[l - 1, 0], tr[l - 1, 1]) if l > 0 else (z, z)
        tn, tn1 = (tr[l, 0], tr[l, 1]) if l < D.L - 1 else (z, z)
        v = D.green(l, t0, t1, tn, tn1, f=f, full=True)
        lo, hi = D.owned_rows(l)
        ref = u[D.s[l] + lo:D.s[l] + hi]
        assert np.linalg.norm(v[lo:hi] - ref) <= 1e-12 * np.linalg.norm(ref)
        n = D.rows[l]
        if l > 0:
            assert np.linalg.norm(v[D.lrow(0)]) <= 1e-12 * np.linalg.norm(ref)
        if l < D.L - 1:
            assert np.linalg.norm(v[D.lrow(n + 1)]) <= 1e-12 * np.linalg.norm(ref)
    assert np.linalg.norm(O.reconstruct(D, f, tr) - u) <= 1e-12 * np.linalg.norm(u)


def _dense(op, shape):
    n = int(np.prod(shape))
    E = np.zeros((n,) + shape, complex)
    for j in range(n):
        E[j].reshape(-1)[j] = 1
    return op(E).reshape(n, n).T


def test_polarized_system_is_exact(small_decomp):
    """The extended system (jump_1..jump_4) has a unique solution whose
    down+up sum equals the true interface traces."""
    D, f, u = small_decomp
    rhs = O.polarized_rhs(D, f)
    M = _dense(lambda x: O.apply_M(D, x), rhs.shape)
    x = np.linalg.solve(M, rhs.reshape(-1)).reshape(rhs.shape)
    tr = D.traces(u)
    s = x[:, 0:2] + x[:, 2:4]
    assert np.linalg.norm(s - tr) <= 1e-11 * np.linalg.norm(tr)
    assert np.linalg.cond(M) < 1e4


def test_block_structure_and_sweeps(small_decomp):
    """D_down is block lower- and D_up block upper-triangular with identity
    diagonal blocks (Section 3); the sweeps invert them and the reflections
    apply L exactly."""
    D, f, u = small_decomp
    K, NX = D.L - 1, D.NX
    shp = (K, 4, NX)
    M = _dense(lambda x: O.apply_M(D, x), shp).reshape(K, 4, NX, K, 4, NX)
    Dd = M[:, 0:2, :, :, 0:2, :].reshape(2 * K * NX, 2 * K * NX)
    Du = M[:, 2:4, :, :, 2:4, :].reshape(2 * K * NX, 2 * K * NX)
    Lm = M[:, 2:4, :, :, 0:2, :].reshape(2 * K * NX, 2 * K * NX)
    b = 2 * NX
    for i in range(K):
        assert np.allclose(Dd[i * b:(i + 1) * b, i * b:(i + 1) * b], np.eye(b), atol=1e-12)
        assert np.allclose(Du[i * b:(i + 1) * b, i * b:(i + 1) * b], np.eye(b), atol=1e-12)
        for j in range(K):
            if j > i:
                assert np.abs(Dd[i * b:(i + 1) * b, j * b:(j + 1) * b]).max() == 0
            if j < i:
                assert np.abs(Du[i * b:(i + 1) * b, j * b:(j + 1) * b]).max() == 0
    rng = np.random.default_rng(13)
    v = rng.standard_normal((K, 2, NX)) + 1j * rng.standard_normal((K, 2, NX))
    vv = v.reshape(-1)
    assert np.allclose(O.sweep_down(D, v).reshape(-1), np.linalg.solve(Dd, vv), rtol=0, atol=1e-11 * np.abs(vv).max() * 10)
    assert np.allclose(O.sweep_up(D, v).reshape(-1), np.linalg.solve(Du, vv), rtol=0, atol=1e-11 * np.abs(vv).max() * 10)
    assert np.allclose(O.reflections(D, v).reshape(-1), Lm @ vv, rtol=0, atol=1e-11 * np.abs(vv).max() * 10)


def _golden_iterations():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_iterations.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    return np.array([[float(x) for x in r] for r in rows])


def test_gauss_seidel_beats_jacobi(small_decomp):
    """P^GS needs about half the GMRES iterations of P^Jac (Section 3.1 and
    the iteration table of Section 5, stored in tests/golden)."""
    D, f, u = small_decomp
    tab = _golden_iterations()
    paper_ratio = (tab[:, 5] / tab[:, 6]).max()
    assert 0.45 < paper_ratio <= 0.55
    rhs = O.polarized_rhs(D, f)
    A = lambda x: O.apply_M(D, x)
    _, it_gs, _ = O.gmres(A, rhs, lambda v: O.precond_gs(D, v), tol=1e-10, maxit=100)
    _, it_j, _ = O.gmres(A, rhs, lambda v: O.precond_jac(D, v), tol=1e-10, maxit=100)
    _, it_0, _ = O.gmres(A, rhs, None, tol=1e-10, maxit=100)
    assert it_gs <= 0.7 * it_j
    assert it_j < it_0
