"""GPU parity of the two SpMV kernels at every batch width k = 1..16, through
the C ABI, against the oracle, elementwise.

Every width selects its own row layout and lane shape (one thread per row
for narrow rows, otherwise one 16-byte vector per lane with idle lanes past
the row's end), so each (scalar type, k) pair instantiates a different
kernel shape: FP64 and FP32 (real shifts, MOR_REAL_VECTORS), complex128 and
complex64 (complex shifts).  CSR, SELL-32 and the diagonal layout, primal
and transposed.

Bounds (each output is a sum of at most row-nnz + 1 products):
  * operator:  |y - y_ref| <= 30 u (|sE| |E| + |sA| |A|) |x|;
  * chain of L factors F_L ... F_1 applied to x, with the factor values read
    back from the GPU (so that only the SpMV is under test; the factor
    values themselves are checked by the SPAI parity tests):
    |y - y_ref| <= 30 u L (|F_L| ... |F_1| |x|),
with u = 2^-53 (FP64) or 2^-24 (FP32; x rounded to FP32 first).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_2003_12759_gb300 as mor
import workloads as W
from oracle import operator as oop, spai as ospai

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24
KS = list(range(1, 17))


@pytest.fixture(scope="module")
def h():
    mor.load_library()
    hh = mor.mor_create(0)
    yield hh
    mor.mor_destroy(hh)


@pytest.fixture(scope="module")
def wl():
    # 13^3 convection-diffusion, E diagonal: n = 2197 rows (ragged against 32-row
    # slices and every rows-per-block), nonsymmetric (own transposed operator)
    return W.convdiff3d_siso(N=13)


def _shifts(k, real):
    if real:
        return np.array([3.0 + 7.0 * c for c in range(k)], dtype=complex)
    return np.array([2.0 + 5.0 * c + (0.5 + 0.25 * c) * 1j for c in range(k)], dtype=complex)


def _x(n, k, real, precision, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, k)) + (0 if real else 1j * rng.standard_normal((n, k)))
    X = np.asarray(X, dtype=complex)
    if precision == mor.MOR_MIXED:
        X = X.astype(np.complex64).astype(np.complex128)
    return X


@pytest.mark.parametrize("fmt", [mor.MOR_FMT_CSR, mor.MOR_FMT_SELL, mor.MOR_FMT_DIA])
@pytest.mark.parametrize("precision", [mor.MOR_FP64, mor.MOR_MIXED])
@pytest.mark.parametrize("real", [True, False])
@pytest.mark.parametrize("transpose", [0, 1])
def test_operator_every_width(h, wl, fmt, precision, real, transpose):
    mor.mor_set_system(h, wl.A, wl.B, wl.C, E_diag=wl.E, fmt=fmt)
    n = wl.n
    Ea = sp.diags(np.abs(wl.E))
    Aa = abs(wl.A).T if transpose else abs(wl.A)
    u = U64 if precision == mor.MOR_FP64 else U32
    for k in KS:
        sig = _shifts(k, real)
        X = _x(n, k, real, precision, 100 + k)
        Y = mor.mor_apply_operator(h, sig, X, transpose=transpose, precision=precision, real=real)
        if real:
            assert np.all(Y.imag == 0), k
        for c in range(k):
            ref = oop.A_sigma(wl.A, wl.E, sig[c], transpose=bool(transpose)) @ X[:, c]
            bnd = abs(sig[c]) * (Ea @ np.abs(X[:, c])) + Aa @ np.abs(X[:, c])
            err = np.abs(Y[:, c] - ref)
            assert np.all(err <= 30 * u * bnd + 1e-300), (k, c, float(np.max(err / (bnd + 1e-300))))


@pytest.mark.parametrize("fmt", [mor.MOR_FMT_CSR, mor.MOR_FMT_SELL, mor.MOR_FMT_DIA])
@pytest.mark.parametrize("precision", [mor.MOR_FP64, mor.MOR_MIXED])
@pytest.mark.parametrize("real", [True, False])
def test_chain_apply_every_width(h, wl, fmt, precision, real):
    mor.mor_set_system(h, wl.A, wl.B, wl.C, E_diag=wl.E, fmt=fmt)
    n = wl.n
    s = [5.0, 9.0, 30.0] if real else [5.0 + 1.0j, 9.0 + 2.0j, 30.0 + 1.0j]
    mor.mor_build_precond(h, s[0], 0, precision)
    mor.mor_update_precond(h, s[1], 0)
    mor.mor_update_precond(h, s[2], 0)
    rowptr, col = mor.mor_get_pattern(h, 0)
    F = []
    for i in range(3):
        vals, _, _ = mor.mor_get_factor(h, 0, i)
        F.append(sp.csr_matrix((vals.real if real else vals, col, rowptr), shape=(n, n)))
    u = U64 if precision == mor.MOR_FP64 else U32
    for k in KS:
        # column c uses the prefix ending at shift c % 3 (P_1, Q_2 P_1, Q_3 Q_2 P_1)
        sig = np.array([s[c % 3] for c in range(k)], dtype=complex)
        X = _x(n, k, real, precision, 200 + k)
        Y = mor.mor_apply_precond(h, sig, X, real=real)
        for c in range(k):
            L = c % 3 + 1
            ref = ospai.chain_apply(F[:L], X[:, c])
            bnd = np.abs(X[:, c])
            for f in F[:L]:
                bnd = abs(f) @ bnd
            err = np.abs(Y[:, c] - ref)
            assert np.all(err <= 30 * u * L * bnd + 1e-300), (k, c, float(np.max(err / (bnd + 1e-300))))


def _irregular_rows_system(n=2000, seed=31):
    """Tridiagonal rows plus 100 rows of 40 extra entries (rows 600..699): rows
    of 3 entries (no whole gather chunk, only a remainder) next to rows of up
    to 43 (many chunks and every remainder length), in one launch."""
    rng = np.random.default_rng(seed)
    T = sp.diags([np.ones(n - 1), np.zeros(n), np.ones(n - 1)], [-1, 0, 1], format="lil")
    for i in range(600, 700):
        for j in rng.choice(n, 40, replace=False):
            if abs(int(j) - i) > 1:
                T[i, int(j)] = 0.1 * rng.standard_normal()
    R = sp.csr_matrix(T)
    dg = np.asarray(abs(R).sum(axis=1)).ravel() + rng.uniform(1.0, 2.0, n)
    A = sp.csr_matrix(-(R + sp.diags(dg)))
    A.sort_indices()
    return A, rng.standard_normal((n, 1)), rng.standard_normal((n, 1))


@pytest.mark.parametrize("precision", [mor.MOR_FP64, mor.MOR_MIXED])
@pytest.mark.parametrize("real", [True, False])
def test_chain_apply_irregular_rows(h, precision, real):
    """The CSR factor SpMV over rows of very different lengths, every width,
    against the oracle's chain apply with the GPU's factor values."""
    A, B, C = _irregular_rows_system()
    n = A.shape[0]
    mor.mor_set_system(h, A, B, C, fmt=mor.MOR_FMT_CSR)
    s = [2.0, 6.0] if real else [2.0 + 1.0j, 6.0 + 0.5j]
    mor.mor_build_precond(h, s[0], 0, precision)
    mor.mor_update_precond(h, s[1], 0)
    rowptr, col = mor.mor_get_pattern(h, 0)
    assert np.diff(rowptr).max() >= 40
    F = []
    for i in range(2):
        vals, _, _ = mor.mor_get_factor(h, 0, i)
        F.append(sp.csr_matrix((vals.real if real else vals, col, rowptr), shape=(n, n)))
    u = U64 if precision == mor.MOR_FP64 else U32
    for k in KS:
        sig = np.array([s[c % 2] for c in range(k)], dtype=complex)
        X = _x(n, k, real, precision, 300 + k)
        Y = mor.mor_apply_precond(h, sig, X, real=real)
        for c in range(k):
            L = c % 2 + 1
            ref = ospai.chain_apply(F[:L], X[:, c])
            bnd = np.abs(X[:, c])
            for f in F[:L]:
                bnd = abs(f) @ bnd
            err = np.abs(Y[:, c] - ref)
            assert np.all(err <= 30 * u * L * bnd + 1e-300), (k, c, float(np.max(err / (bnd + 1e-300))))


@pytest.mark.parametrize("precision", [mor.MOR_FP64, mor.MOR_MIXED])
def test_solve_diagonal_layout_equals_csr(h, wl, precision):
    """The same shifted solves with the operator and the chain stored in the
    diagonal layout and in CSR: the layouts sum a row's entries in the same
    (column) order, the diagonal layout adding exact zeros for its padding, so
    the solves take the same iterations and agree to rounding."""
    s = [4.0 + 1.0j, 9.0 + 2.0j, 30.0]
    rng = np.random.default_rng(5)
    R = rng.standard_normal((wl.n, 3)) + 0j
    out = {}
    for fmt in (mor.MOR_FMT_CSR, mor.MOR_FMT_DIA):
        mor.mor_set_system(h, wl.A, wl.B, wl.C, E_diag=wl.E, fmt=fmt)
        assert mor.mor_get_info(h)["format"] == fmt
        mor.mor_build_precond(h, s[0], 0, precision)
        mor.mor_update_precond(h, s[1], 0)
        mor.mor_update_precond(h, s[2], 0)
        X, st, code = mor.mor_solve_shifts(h, s, 0, mor.mor_default_opts(precision=precision), R=R)
        assert code == mor.MOR_OK
        out[fmt] = (X, [x["iters"] for x in st])
    (Xc, ic), (Xd, idg) = out[mor.MOR_FMT_CSR], out[mor.MOR_FMT_DIA]
    assert ic == idg
    np.testing.assert_allclose(Xd, Xc, rtol=0, atol=1e-12 * np.abs(Xc).max())


def test_diagonal_layout_refuses_irregular_rows(h):
    """A pattern with hundreds of distinct diagonals is refused with MOR_EINVAL;
    the automatic choice then stays among CSR and SELL-32."""
    A, B, C = _irregular_rows_system()
    with pytest.raises(mor.MorError, match="diagonals"):
        mor.mor_set_system(h, A, B, C, fmt=mor.MOR_FMT_DIA)
    mor.mor_set_system(h, A, B, C, fmt=mor.MOR_FMT_AUTO)
    assert mor.mor_get_info(h)["format"] in (mor.MOR_FMT_CSR, mor.MOR_FMT_SELL)


@pytest.mark.parametrize("precision", [mor.MOR_FP64, mor.MOR_MIXED])
@pytest.mark.parametrize("real", [True, False])
def test_five_diagonal_layout_every_width(h, precision, real):
    """A 2D five-point pattern (41 x 41 grid: 5 diagonals, offsets 0, +-1, +-41)
    in the diagonal layout: the operator and a two-factor chain at every width,
    elementwise against the oracle (the kernels specialised to 5 diagonals and
    their edge rows, within +-41 rows of either end)."""
    wl = W.laplace2d_siso(N=41)
    A = sp.csr_matrix(wl.A)
    n = A.shape[0]
    mor.mor_set_system(h, A, wl.B, wl.C, fmt=mor.MOR_FMT_DIA)
    assert mor.mor_get_info(h)["format"] == mor.MOR_FMT_DIA
    u = U64 if precision == mor.MOR_FP64 else U32
    Aa = abs(A)
    for k in KS:
        sig = _shifts(k, real)
        X = _x(n, k, real, precision, 400 + k)
        Y = mor.mor_apply_operator(h, sig, X, precision=precision, real=real)
        for c in range(k):
            ref = oop.A_sigma(A, None, sig[c]) @ X[:, c]
            bnd = abs(sig[c]) * np.abs(X[:, c]) + Aa @ np.abs(X[:, c])
            assert np.all(np.abs(Y[:, c] - ref) <= 30 * u * bnd + 1e-300), (k, c)
    s = [3.0, 8.0] if real else [3.0 + 1.0j, 8.0 + 0.5j]
    mor.mor_build_precond(h, s[0], 0, precision)
    mor.mor_update_precond(h, s[1], 0)
    rowptr, col = mor.mor_get_pattern(h, 0)
    F = []
    for i in range(2):
        vals, _, _ = mor.mor_get_factor(h, 0, i)
        F.append(sp.csr_matrix((vals.real if real else vals, col, rowptr), shape=(n, n)))
    for k in KS:
        sig = np.array([s[c % 2] for c in range(k)], dtype=complex)
        X = _x(n, k, real, precision, 500 + k)
        Y = mor.mor_apply_precond(h, sig, X, real=real)
        for c in range(k):
            L = c % 2 + 1
            ref = ospai.chain_apply(F[:L], X[:, c])
            bnd = np.abs(X[:, c])
            for f in F[:L]:
                bnd = abs(f) @ bnd
            assert np.all(np.abs(Y[:, c] - ref) <= 30 * u * L * bnd + 1e-300), (k, c)
