"""Oracle pins of the inner block-LU sweeps and their compressed form (Section
4.2.2; the compression of Section 4.3), independent of the CUDA path:

- the two sweeps solve (I - Lo)(I - Up) x = h, Lo holding P_j below the block
  diagonal and Up holding V_j above it (checked against a dense LAPACK solve);
- with P_j = QP_j BP_j and V_j = QV_j BV_j exactly, the r-vector form equals the
  dense sweeps to roundoff;
- the truncated SVD meets its relative Frobenius tolerance with the smallest
  rank (Eckart-Young: one rank less misses it), and sweeps with factors
  truncated at eps stay within a modest multiple of eps of the exact ones."""
import numpy as np
import pytest

import oracle as O


def _rand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _factors(rng, J, n, decay):
    # P_j, V_j with singular values decaying like decay**k (inner Green's operators between
    # the two sides of a cell behave so), scaled to norm < 1 so that the sweeps are stable
    def mat():
        U, _ = np.linalg.qr(_rand(rng, n, n))
        V, _ = np.linalg.qr(_rand(rng, n, n))
        return 0.5 * (U * decay ** np.arange(n)) @ V.conj().T
    P = [None] + [mat() for _ in range(1, J)]
    V = [mat() for _ in range(J - 1)] + [None]
    return P, V


def test_sweeps_solve_the_block_bidiagonal_product():
    rng = np.random.default_rng(1)
    J, n, B = 5, 6, 3
    P, V = _factors(rng, J, n, 0.9)
    h = _rand(rng, J, n, B)
    x = O.inner_block_lu(P, V, h)
    I = np.eye(J * n, dtype=complex)
    Lo, Up = np.zeros_like(I), np.zeros_like(I)
    for j in range(1, J):
        Lo[j * n:(j + 1) * n, (j - 1) * n:j * n] = P[j]
    for j in range(J - 1):
        Up[j * n:(j + 1) * n, (j + 1) * n:(j + 2) * n] = V[j]
    ref = np.linalg.solve((I - Lo) @ (I - Up), h.reshape(J * n, B)).reshape(J, n, B)
    assert np.linalg.norm(x - ref) < 1e-12 * np.linalg.norm(ref)


def test_lowrank_form_equals_the_dense_sweeps():
    rng = np.random.default_rng(2)
    J, n, r, B = 6, 10, 4, 2
    QP = [None] + [np.linalg.qr(_rand(rng, n, r))[0] for _ in range(1, J)]
    BP = [None] + [0.3 * _rand(rng, r, n) for _ in range(1, J)]
    QV = [np.linalg.qr(_rand(rng, n, r))[0] for _ in range(J - 1)] + [None]
    BV = [0.3 * _rand(rng, r, n) for _ in range(J - 1)] + [None]
    P = [None] + [QP[j] @ BP[j] for j in range(1, J)]
    V = [QV[j] @ BV[j] for j in range(J - 1)] + [None]
    h = _rand(rng, J, n, B)
    dense = O.inner_block_lu(P, V, h)
    lr = O.inner_block_lu_lowrank(QP, BP, QV, BV, h)
    assert np.linalg.norm(lr - dense) < 1e-13 * np.linalg.norm(dense)


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_truncation_meets_the_tolerance_with_the_smallest_rank(eps):
    rng = np.random.default_rng(3)
    _, V = _factors(rng, 2, 40, 0.5)
    A = V[0]
    Q, Bf = O.lowrank(A, eps)
    r = Q.shape[1]
    assert np.allclose(Q.conj().T @ Q, np.eye(r), atol=1e-12)
    assert np.linalg.norm(A - Q @ Bf) <= eps * np.linalg.norm(A) * (1 + 1e-12)
    s = np.linalg.svd(A, compute_uv=False)
    assert np.sqrt(np.sum(s[r - 1:] ** 2)) > eps * np.linalg.norm(A)  # rank r - 1 would miss it
    assert r < 40


@pytest.mark.parametrize("eps", [1e-4, 1e-7, 1e-10])
def test_compressed_sweeps_stay_within_the_tolerance(eps):
    rng = np.random.default_rng(4)
    J, n, B = 6, 32, 3
    P, V = _factors(rng, J, n, 0.4)
    h = _rand(rng, J, n, B)
    exact = O.inner_block_lu(P, V, h)
    QP, BP, QV, BV = [None] * J, [None] * J, [None] * J, [None] * J
    for j in range(1, J):
        QP[j], BP[j] = O.lowrank(P[j], eps)
    for j in range(J - 1):
        QV[j], BV[j] = O.lowrank(V[j], eps)
    approx = O.inner_block_lu_lowrank(QP, BP, QV, BV, h)
    err = np.linalg.norm(approx - exact) / np.linalg.norm(exact)
    assert err < 10 * eps
    assert max(QP[j].shape[1] for j in range(1, J)) < n  # the compression is in effect
