"""Full-size checks in the launch configuration that bench.py times.

  * The 100^3 convection-diffusion system of the default bench (n = 10^6,
    E diagonal, complex shifts; mixed precision, all shifts in one lock-step
    batch, CUDA graphs, autotuned storage format) on outputs the oracle can
    compute one at a time: operator rows at sampled indices (boundary rows
    included), SPAI and reuse-factor columns at sampled j (each column is one
    small least-squares problem), the true FP64 residual of every shifted
    solve, and, for the IRKA step, the Hermite interpolation conditions
    H(s_i) = H_r(s_i), H'(s_i) = H_r'(s_i) at every solved shift, which hold
    at any size (Sec. II), with H(s_i) = C^T v_i and H'(s_i) = -w_i^T E v_i
    from solves refined in FP64 to 1e-12.  A solve to 1e-8 moves H(s_i) by up to
    cond(A(s_i)) x 1e-8; the bar is 20 x the measured move of C^T v_i between
    the 1e-8 and the 1e-12 solves (at least 1e-7).
  * The 256-system uneven batch at full size (7.9M rows) on sampled systems:
    true residuals and agreement with a sparse direct solve.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import paper_2003_12759_gb300 as mor
import workloads as W
from oracle import operator as oop, spai as ospai

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    mor.load_library()
    hh = mor.mor_create(0)
    yield hh
    mor.mor_destroy(hh)


@pytest.fixture(scope="module")
def convdiff(h):
    wl = W.convdiff3d_siso()
    mor.mor_set_system(h, wl.A, wl.B, wl.C, E_diag=wl.E)
    return wl


def _sample_rows(n, rng, count=2000):
    edge = np.array([0, 1, 99, 100, 9999, 10000, n // 2, n - 10001, n - 101, n - 1])
    return np.unique(np.concatenate([edge, rng.choice(n, count, replace=False)]))


@pytest.mark.parametrize("precision", [mor.MOR_FP64, mor.MOR_MIXED])
def test_operator_rows_full_size(h, convdiff, precision):
    wl = convdiff
    rng = np.random.default_rng(11)
    sig = np.array([30.0, 45.0 + 20.0j, 90.0 + 5.0j, 200.0, 400.0 + 400.0j, 1e3 + 500j, 1e4])
    X = rng.standard_normal((wl.n, 7)) + 1j * rng.standard_normal((wl.n, 7))
    Y = mor.mor_apply_operator(h, sig, X, 0, precision)
    rows = _sample_rows(wl.n, rng)
    for c, s in enumerate(sig):
        Mr = oop.A_sigma(wl.A, wl.E, s)[rows]
        ref = Mr @ X[:, c]
        scale = abs(Mr) @ np.abs(X[:, c])
        tol = 1e-13 if precision == mor.MOR_FP64 else 2e-6
        assert np.all(np.abs(Y[rows, c] - ref) <= tol * scale), c


@pytest.mark.parametrize("transpose", [0, 1])
def test_spai_and_reuse_columns_full_size(h, convdiff, transpose):
    wl = convdiff
    s1, s2 = 12.0 + 3.0j, 20.0 - 1.0j
    mor.mor_build_precond(h, s1, transpose, mor.MOR_MIXED)
    mor.mor_update_precond(h, s2, transpose)
    rowptr, col = mor.mor_get_pattern(h, transpose)
    S = ospai.spai_pattern(wl.A, wl.E, transpose=bool(transpose))
    M1 = oop.A_sigma(wl.A, wl.E, s1, transpose=bool(transpose))
    M2 = oop.A_sigma(wl.A, wl.E, s2, transpose=bool(transpose))
    rng = np.random.default_rng(12 + transpose)
    js = np.unique(np.concatenate([[0, 1, 99, 9999, wl.n - 1], rng.choice(wl.n, 300, replace=False)]))
    refs = [ospai.column_least_squares(M1, sp.identity(wl.n, format="csr"), S, columns=js),
            ospai.column_least_squares(M2, M1, S, columns=js)]
    for idx in range(2):
        vals, _, _ = mor.mor_get_factor(h, transpose, idx)
        Pg = sp.csr_matrix((vals, col, rowptr), shape=(wl.n, wl.n)).tocsc()
        Po = sp.csc_matrix(refs[idx])
        for j in js:
            a = Pg[:, j].toarray().ravel()
            b = Po[:, j].toarray().ravel()
            assert np.linalg.norm(a - b) <= 2e-4 * np.linalg.norm(b), (idx, j)


def test_irka_step_full_size_solves_and_hermite(h, convdiff):
    wl = convdiff
    mor.mor_irka_reset(h)
    opts = mor.mor_default_opts()
    s0 = wl.shifts.copy()
    s1, rom, st = mor.mor_irka_step(h, s0, opts)
    assert st["max_relres"] <= 1.001e-8
    # the solved shifts of that step (one per conjugate pair, sorted) and the chains it left
    order = np.lexsort((-s0.imag, np.abs(s0.imag), s0.real))
    sol = s0[order][s0[order].imag >= 0]
    X, sx, code = mor.mor_solve_shifts(h, sol, 0, opts)
    Y, sy, code2 = mor.mor_solve_shifts(h, sol, 1, opts)
    assert code == mor.MOR_OK and code2 == mor.MOR_OK
    tight = mor.mor_default_opts(tol=1e-12, max_refine=30, maxit=100000)   # the same (mixed) chain
    X2, _, c3 = mor.mor_solve_shifts(h, sol, 0, tight)
    Y2, _, c4 = mor.mor_solve_shifts(h, sol, 1, tight)
    assert c3 == mor.MOR_OK and c4 == mor.MOR_OK
    E = sp.diags(wl.E)
    Ar, Er, Br, Cr = rom.arrays()
    for c, s in enumerate(sol):
        M = oop.A_sigma(wl.A, wl.E, s)
        assert np.linalg.norm(wl.B[:, 0] - M @ X[:, c]) <= 1.001e-8 * np.linalg.norm(wl.B[:, 0])
        assert np.linalg.norm(wl.C[:, 0] - M.T @ Y[:, c]) <= 1.001e-8 * np.linalg.norm(wl.C[:, 0])
        H = wl.C[:, 0] @ X2[:, c]
        dH = -(Y2[:, c] @ (E @ X2[:, c]))
        move = abs(wl.C[:, 0] @ X[:, c] - H) / abs(H)
        dmove = abs(-(Y[:, c] @ (E @ X[:, c])) - dH) / abs(dH)
        K = s * Er - Ar
        xr = np.linalg.solve(K, Br[:, 0].astype(complex))
        Hr = Cr[:, 0] @ xr
        dHr = -(Cr[:, 0] @ np.linalg.solve(K, Er @ xr))
        assert abs(Hr - H) <= max(1e-7, 20 * move) * abs(H), (c, Hr, H, move)
        assert abs(dHr - dH) <= max(1e-7, 20 * dmove) * abs(dH), (c, dHr, dH, dmove)


def test_batch_full_size_sampled_systems(h):
    sysl = W.uneven_laplace2d_batch()
    mor.mor_set_batch(h, [w.A for w in sysl], [w.B[:, 0] for w in sysl], [w.C[:, 0] for w in sysl])
    nsys, off = mor.mor_batch_info(h)
    assert nsys == 256 and off[-1] == sum(w.n for w in sysl)
    shifts = list(np.logspace(0, 4, 8).astype(np.complex128))
    mor.mor_build_precond(h, shifts[0], 0, mor.MOR_MIXED)
    for z in shifts[1:]:
        mor.mor_update_precond(h, z, 0)
    X, st, code = mor.mor_batch_solve(h, shifts, 0, mor.mor_default_opts())
    assert code == mor.MOR_OK
    rng = np.random.default_rng(5)
    sizes = np.array([w.n for w in sysl])
    picks = {int(np.argmin(sizes)), int(np.argmax(sizes))} | set(rng.choice(nsys, 3, replace=False).tolist())
    for i in sorted(picks):
        w = sysl[i]
        xs = X[off[i]:off[i + 1]]
        for c, s in enumerate(shifts):
            M = oop.A_sigma(w.A, w.E, s)
            b = w.B[:, 0]
            assert np.linalg.norm(b - M @ xs[:, c]) <= 1.001e-8 * np.linalg.norm(b), (i, c)
            assert st[i][c]["status"] == mor.MOR_OK
        xd = spla.spsolve(sp.csc_matrix(oop.A_sigma(w.A, w.E, shifts[0])), w.B[:, 0])
        assert np.linalg.norm(xs[:, 0] - xd) <= 1e-6 * np.linalg.norm(xd)
