"""Pins of the oracle's shifted operator and transfer function against closed
forms (not against the oracle's own formula)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import operator as op


def _sine_mode(N, j):
    h = 1.0 / (N + 1)
    x = np.arange(1, N + 1) * h
    return np.sin(j * np.pi * x), 4.0 / h**2 * np.sin(j * np.pi * h / 2) ** 2


@pytest.mark.parametrize("sigma", [3.0, 10.0 + 4.0j, -2.5j])
def test_laplacian_eigenpair_closed_form(sigma):
    """For A = -L2, E = I: (sigma I - A) u = (sigma + lambda) u with the
    closed-form sine eigenpairs of the Dirichlet 5-point Laplacian."""
    N = 13
    wl = W.laplace2d_siso(N=N)
    for (j, k) in [(1, 1), (2, 5), (13, 7)]:
        uj, lj = _sine_mode(N, j)
        uk, lk = _sine_mode(N, k)
        u = np.kron(uk, uj)            # row index i + N*j  ->  x fastest
        M = op.A_sigma(wl.A, wl.E, sigma)
        y = M @ u
        np.testing.assert_allclose(y, (sigma + lj + lk) * u, rtol=0, atol=1e-9 * abs(sigma + lj + lk))


def test_convdiff_interior_rowsums_and_diag_E():
    """Interior rows of the upwind convection-diffusion operator sum to zero
    (diffusion and the one-sided difference both annihilate constants), so
    (sigma E - A) 1 = sigma e at interior rows; boundary rows are larger."""
    N = 7
    wl = W.convdiff3d_siso(N=N)
    sigma = 2.0 + 1.0j
    y = op.A_sigma(wl.A, wl.E, sigma) @ np.ones(wl.n)
    idx = np.arange(wl.n)
    i, j, k = idx % N, (idx // N) % N, idx // (N * N)
    interior = (i > 0) & (i < N - 1) & (j > 0) & (j < N - 1) & (k > 0) & (k < N - 1)
    np.testing.assert_allclose(y[interior], sigma * wl.E[interior], rtol=1e-9, atol=1e-6)
    h = 1.0 / (N + 1)
    # the centre coefficient of the positive operator: 6/h^2 + 3 w/h, w = 10/sqrt 3
    assert np.allclose(-wl.A.diagonal(), 6 / h**2 + 3 * (10 / np.sqrt(3)) / h)


@pytest.mark.parametrize("e_kind", ["identity", "diag", "csr"])
def test_operator_dense_bruteforce(e_kind):
    """Entry-by-entry dense check of sigma E - A and its plain transpose."""
    wl = W.random_sparse_system(30, 0.15, seed=3, e_kind=e_kind)
    Ad = wl.A.toarray()
    if wl.E is None:
        Ed = np.eye(30)
    elif isinstance(wl.E, np.ndarray):
        Ed = np.diag(wl.E)
    else:
        Ed = wl.E.toarray()
    s = 1.5 - 0.25j
    ref = np.empty((30, 30), dtype=complex)
    for r in range(30):
        for c in range(30):
            ref[r, c] = s * Ed[r, c] - Ad[r, c]
    np.testing.assert_array_equal(op.A_sigma(wl.A, wl.E, s).toarray(), ref)
    np.testing.assert_array_equal(op.A_sigma(wl.A, wl.E, s, transpose=True).toarray(), ref.T)


def test_second_order_operator_eigenpair():
    """With M = m I and K's separable sine eigenvectors (27-point stencil,
    eigenvalue 27 - prod(1 + 2 cos theta)), s^2 M + s D + K acts as
    s^2 m + s (alpha m + beta lambda) + lambda."""
    nx, ny, nz = 5, 4, 3
    K = W.stencil27_3d(nx, ny, nz)
    m, alpha, beta, s = 1.7, 1e-3, 1e-4, 0.3 + 0.8j

    def mode(N, j):
        x = np.arange(1, N + 1) / (N + 1)
        return np.sin(j * np.pi * x), 1 + 2 * np.cos(j * np.pi / (N + 1))

    ux, ex = mode(nx, 2)
    uy, ey = mode(ny, 1)
    uz, ez = mode(nz, 3)
    u = np.kron(uz, np.kron(uy, ux))
    lam = 27 - ex * ey * ez
    np.testing.assert_allclose(K @ u, lam * u, atol=1e-12)
    M2 = op.A_sigma_2nd(K, np.full(K.shape[0], m), alpha, beta, s)
    np.testing.assert_allclose(M2 @ u, (s * s * m + s * (alpha * m + beta * lam) + lam) * u, atol=1e-11)


def test_transfer_function_diagonal_closed_form():
    """Diagonal SISO system: H(s) = sum_i c_i b_i / (s e_i - a_i)."""
    rng = np.random.default_rng(5)
    n = 12
    a = -rng.uniform(1, 10, n)
    e = rng.uniform(0.5, 1.5, n)
    b = rng.standard_normal((n, 1))
    c = rng.standard_normal((n, 1))
    A = sp.diags(a, format="csr")
    s = np.array([0.5j, 2 + 3j, 7.0])
    H = op.transfer_function(A, e, b, c, s)[:, 0, 0]
    ref = np.array([np.sum(c[:, 0] * b[:, 0] / (si * e - a)) for si in s])
    np.testing.assert_allclose(H, ref, rtol=1e-12)
    Hr = op.transfer_function_reduced(np.diag(a), np.diag(e), b, c, s)[:, 0, 0]
    np.testing.assert_allclose(Hr, ref, rtol=1e-12)
