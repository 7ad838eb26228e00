"""GPU parity of block GMRES(m) (solver MOR_BGMRES: the right-hand sides of a
shift share one block Krylov space, the MIMO form of the shifted solves)
against the oracle's block GMRES, through the C ABI:

  * per-column true relative residual <= 1e-8, recomputed here in FP64;
  * solutions within kappa * 2e-8 of dense LU (kappa: the 2-norm condition
    number of the shifted matrix, computed densely);
  * block iterations (FP64) within 10% (+2) of the oracle's block GMRES with
    the same restart and preconditioner: the GPU orthogonalises by block CGS2
    and a rank-revealing CholQR2, the oracle by two passes of block modified
    Gram-Schmidt and Householder QR, both to working accuracy;
  * one right-hand side: the same iteration count as GMRES(m);
  * a block with two equal right-hand sides (rank-deficient residual block)
    converges in both columns (the dependent direction is deflated);
  * mixed precision (FP32 / complex64 block GMRES inside FP64 refinement)
    reaches the same FP64 residual.
"""
import numpy as np
import pytest

import paper_2003_12759_gb300 as mor
import workloads as W
from oracle import krylov as okry, operator as oop, spai as ospai

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    mor.load_library()
    hh = mor.mor_create(0)
    yield hh
    mor.mor_destroy(hh)


def _setup(h, N=10, p=4, seed=8):
    wl = W.convdiff3d_siso(N=N)
    mor.mor_set_system(h, wl.A, wl.B, wl.C, E_diag=wl.E)
    rng = np.random.default_rng(seed)
    R = rng.standard_normal((wl.n, p)) + 0j
    return wl, R


@pytest.mark.parametrize("sigma", [20.0 + 5.0j, 60.0])
@pytest.mark.parametrize("p", [4, 8])
def test_block_gmres_matches_oracle(h, sigma, p):
    wl, R = _setup(h, p=p)
    restart = 20
    mor.mor_build_precond(h, sigma, 0, mor.MOR_FP64)
    opts = mor.mor_default_opts(precision=mor.MOR_FP64, solver=mor.MOR_BGMRES, restart=restart)
    X, st, code = mor.mor_solve_shifts(h, [sigma] * p, 0, opts, R=R)
    assert code == mor.MOR_OK
    M = oop.A_sigma(wl.A, wl.E, sigma)
    Md = M.toarray()
    kappa = np.linalg.cond(Md)
    for c in range(p):
        rel = np.linalg.norm(R[:, c] - M @ X[:, c]) / np.linalg.norm(R[:, c])
        assert rel <= 1.001e-8 and st[c]["relres"] <= 1.001e-8, (c, rel)
    Xd = np.linalg.solve(Md, R)
    assert np.linalg.norm(X - Xd) <= kappa * 2e-8 * np.linalg.norm(Xd)
    P = ospai.spai(M, ospai.spai_pattern(wl.A, wl.E))
    _, it_o, rel_o, _ = okry.block_gmres(lambda v: M @ v, lambda v: P @ v, R, tol=1e-8, m=restart)
    it_g = max(x["iters"] for x in st)
    assert abs(it_g - it_o) <= 0.1 * it_o + 2, (it_g, it_o)


def test_block_gmres_one_column_is_gmres(h):
    wl, R = _setup(h, p=1)
    s = 30.0 + 2.0j
    mor.mor_build_precond(h, s, 0, mor.MOR_FP64)
    ob = mor.mor_default_opts(precision=mor.MOR_FP64, solver=mor.MOR_BGMRES, restart=15)
    og = mor.mor_default_opts(precision=mor.MOR_FP64, solver=mor.MOR_GMRES, restart=15)
    Xb, sb, _ = mor.mor_solve_shifts(h, [s], 0, ob, R=R)
    Xg, sg, _ = mor.mor_solve_shifts(h, [s], 0, og, R=R)
    assert abs(sb[0]["iters"] - sg[0]["iters"]) <= 2, (sb, sg)
    np.testing.assert_allclose(Xb, Xg, rtol=0, atol=1e-7 * np.abs(Xg).max())


def test_block_gmres_deflates_dependent_columns(h):
    wl, R = _setup(h, p=3)
    R[:, 2] = R[:, 0]                    # a repeated right-hand side
    s = 40.0
    mor.mor_build_precond(h, s, 0, mor.MOR_FP64)
    opts = mor.mor_default_opts(precision=mor.MOR_FP64, solver=mor.MOR_BGMRES, restart=20)
    X, st, code = mor.mor_solve_shifts(h, [s] * 3, 0, opts, R=R)
    assert code == mor.MOR_OK
    M = oop.A_sigma(wl.A, wl.E, s)
    for c in range(3):
        assert np.linalg.norm(R[:, c] - M @ X[:, c]) <= 1.001e-8 * np.linalg.norm(R[:, c])
    np.testing.assert_allclose(X[:, 2], X[:, 0], rtol=0, atol=1e-7 * np.abs(X[:, 0]).max())


def test_block_gmres_mixed_precision_and_mixed_shifts(h):
    """FP32 / complex64 block GMRES inside FP64 refinement; the columns of two
    shifts form two blocks (each with its own chain prefix)."""
    wl, R = _setup(h, p=6)
    s1, s2 = 15.0 + 3.0j, 90.0
    mor.mor_build_precond(h, s1, 0, mor.MOR_MIXED)
    mor.mor_update_precond(h, s2, 0)
    sig = [s1, s1, s1, s2, s2, s2]
    opts = mor.mor_default_opts(precision=mor.MOR_MIXED, solver=mor.MOR_BGMRES, restart=25)
    X, st, code = mor.mor_solve_shifts(h, sig, 0, opts, R=R)
    assert code == mor.MOR_OK
    for c in range(6):
        M = oop.A_sigma(wl.A, wl.E, sig[c])
        assert np.linalg.norm(R[:, c] - M @ X[:, c]) <= 1.001e-8 * np.linalg.norm(R[:, c]), c
