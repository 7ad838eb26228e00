"""Pins of the oracle's right-preconditioned Krylov solvers (Sec. III.A, IV)
against dense LU, independently recomputed residuals and CG."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import operator as op
from oracle import spai, krylov


def _problem(sigma, N=14):
    wl = W.convdiff3d_siso(N=N)                        # nonsymmetric, E diagonal
    M = op.A_sigma(wl.A, wl.E, sigma)
    b = wl.B[:, 0].astype(M.dtype)
    return wl, M, b


@pytest.mark.parametrize("solver", ["bicgstab", "gmres"])
@pytest.mark.parametrize("sigma", [10.0, 30.0 + 15.0j])
@pytest.mark.parametrize("precond", [False, True])
def test_solution_matches_dense_lu(solver, sigma, precond):
    wl, M, b = _problem(sigma)
    P = None
    if precond:
        S = spai.spai_pattern(wl.A, wl.E)
        Pm = spai.spai(M, S)
        P = lambda x: Pm @ x  # noqa: E731
    f = krylov.bicgstab if solver == "bicgstab" else krylov.gmres
    x, it, rel, st = f(lambda v: M @ v, P, b, tol=1e-8, maxit=5000)
    assert st == krylov.STATUS_OK
    # residual recomputed independently with a dense product
    Md = M.toarray()
    r = b - Md @ x
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8 * 1.0001
    xref = krylov.dense_solve(M, b)
    kappa = np.linalg.cond(Md)
    assert np.linalg.norm(x - xref) / np.linalg.norm(xref) <= kappa * 1e-8


def test_preconditioner_reduces_iterations():
    wl, M, b = _problem(10.0, N=16)
    S = spai.spai_pattern(wl.A, wl.E)
    Pm = spai.spai(M, S)
    _, it0, _, st0 = krylov.bicgstab(lambda v: M @ v, None, b)
    _, it1, _, st1 = krylov.bicgstab(lambda v: M @ v, lambda v: Pm @ v, b)
    assert st0 == st1 == krylov.STATUS_OK
    assert it1 < it0


def test_symmetric_case_matches_cg():
    """Laplacian (SPD sigma I + L): BiCGSTAB and scipy CG agree."""
    wl = W.laplace2d_siso(N=20)
    M = op.A_sigma(wl.A, wl.E, 25.0)
    b = wl.B[:, 0]
    x, it, rel, st = krylov.bicgstab(lambda v: M @ v, None, b, tol=1e-10)
    xcg, info = spla.cg(M, b, rtol=1e-12, maxiter=10000)
    assert info == 0 and st == krylov.STATUS_OK
    np.testing.assert_allclose(x, xcg, rtol=0, atol=1e-8 * np.linalg.norm(xcg))


def test_maxit_gives_noconv_status():
    """Unpreconditioned Krylov on a hard shift stops at maxit with NOCONV
    (the paper's observation that unpreconditioned GMRES fails, Sec. IV)."""
    wl, M, b = _problem(1e-3, N=14)
    for f in (krylov.bicgstab, krylov.gmres):
        x, it, rel, st = f(lambda v: M @ v, None, b, tol=1e-12, maxit=5)
        assert st == krylov.STATUS_NOCONV and it == 5 and rel > 1e-12


def test_zero_rhs():
    wl, M, b = _problem(10.0, N=5)
    for f in (krylov.bicgstab, krylov.gmres):
        x, it, rel, st = f(lambda v: M @ v, None, np.zeros_like(b))
        assert it == 0 and st == krylov.STATUS_OK and not np.any(x)


def test_identity_preconditioned_by_exact_inverse_one_iteration():
    """With P = A^{-1} the preconditioned operator is I: BiCGSTAB converges
    in one iteration (a closed-form property of the right-preconditioned
    recurrence)."""
    rng = np.random.default_rng(1)
    n = 20
    Ad = rng.standard_normal((n, n)) + 8 * np.eye(n)
    M = sp.csr_matrix(Ad)
    Minv = np.linalg.inv(Ad)
    b = rng.standard_normal(n)
    x, it, rel, st = krylov.bicgstab(lambda v: M @ v, lambda v: Minv @ v, b, tol=1e-10)
    assert it == 1 and st == krylov.STATUS_OK


# ----------------------------------------------------------------------------
# block GMRES (several right-hand sides sharing one block Krylov space)
# ----------------------------------------------------------------------------
def _block_problem(sigma, p=3, N=9, seed=4):
    wl = W.convdiff3d_siso(N=N)
    M = op.A_sigma(wl.A, wl.E, sigma)
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((M.shape[0], p)).astype(M.dtype)
    return wl, M, B


@pytest.mark.parametrize("sigma", [10.0, 30.0 + 15.0j])
@pytest.mark.parametrize("precond", [False, True])
def test_block_gmres_matches_dense_lu(sigma, precond):
    wl, M, B = _block_problem(sigma)
    P = None
    if precond:
        Pm = spai.spai(M, spai.spai_pattern(wl.A, wl.E))
        P = lambda x: Pm @ x  # noqa: E731
    X, it, rel, st = krylov.block_gmres(lambda v: M @ v, P, B, tol=1e-10, m=12)
    assert st == krylov.STATUS_OK and np.all(rel <= 1e-10)
    Md = M.toarray()
    Xd = np.linalg.solve(Md, B)
    kappa = np.linalg.cond(Md)
    for c in range(B.shape[1]):
        assert np.linalg.norm(X[:, c] - Xd[:, c]) <= kappa * 2e-10 * np.linalg.norm(Xd[:, c])
        # the true residual is recomputed here, not taken from the solver
        assert np.linalg.norm(B[:, c] - Md @ X[:, c]) <= 1.001e-10 * np.linalg.norm(B[:, c])


def test_block_gmres_one_column_is_gmres():
    """p = 1: the block method is GMRES (QR of a single column = normalisation,
    the block least squares = the Givens least squares)."""
    wl, M, B = _block_problem(20.0 + 5.0j, p=1)
    X, itb, relb, _ = krylov.block_gmres(lambda v: M @ v, None, B, tol=1e-9, m=15)
    x, itg, relg, _ = krylov.gmres(lambda v: M @ v, None, B[:, 0], tol=1e-9, m=15)
    assert abs(itb - itg) <= 1
    np.testing.assert_allclose(X[:, 0], x, rtol=0, atol=1e-8 * np.linalg.norm(x))


def test_block_space_contains_each_columns_space():
    """Without restarts the block Krylov space of degree j contains every
    column's own Krylov space of degree j, so block GMRES needs no more
    iterations than the slowest column's GMRES, and (exact arithmetic) ends
    within ceil(n / p) block steps."""
    wl, M, B = _block_problem(5.0 + 2.0j, p=4, N=4)          # n = 64
    n, p = B.shape
    X, itb, rel, st = krylov.block_gmres(lambda v: M @ v, None, B, tol=1e-12, m=n)
    single = [krylov.gmres(lambda v: M @ v, None, B[:, c], tol=1e-12, m=n)[1] for c in range(p)]
    assert st == krylov.STATUS_OK
    assert itb <= max(single)
    assert itb <= -(-n // p)
