"""GPU parity of the individual kernels of the path, through the C ABI,
against the CPU oracle on the same seeded inputs.

Tolerances (derived from the arithmetic):
  * operator SpMV: each output is a sum of at most (row nnz + 1) products;
    |y_gpu - y_oracle| <= 30 u (|sE| |E| + |sA| |A|) |x| elementwise, with
    u = 2^-53 (FP64) or 2^-24 (FP32, inputs rounded to FP32 first);
  * SPAI / reuse columns: each column is a small full-rank least-squares
    problem solved by Householder QR; FP64 columns agree to 1e-9 relative
    (condition numbers of the blocks are below 1e3), FP32 to 1e-4;
  * dense FP64 kernels (Gram-Schmidt, projection, poles, transfer function):
    1e-10 relative unless noted.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_2003_12759_gb300 as mor
import workloads as W
from oracle import operator as oop, spai as ospai, irka as oirka

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def h():
    mor.load_library()
    hh = mor.mor_create(0)
    yield hh
    mor.mor_destroy(hh)


def _E_abs(wl):
    n = wl.n
    if wl.E is None:
        return sp.identity(n, format="csr")
    if isinstance(wl.E, np.ndarray):
        return sp.diags(np.abs(wl.E))
    return abs(wl.E)


SYSTEMS = {
    # ragged sizes: not multiples of 32 or 256, several thread blocks
    "laplace2d_n1369": lambda: W.laplace2d_siso(N=37),
    "convdiff3d_n2197": lambda: W.convdiff3d_siso(N=13),
    "rand_csrE_n700": lambda: W.random_sparse_system(700, 0.01, seed=3, e_kind="csr"),
    "rand_diagE_n33": lambda: W.random_sparse_system(33, 0.2, seed=4, e_kind="diag"),
}


def _set(h, wl, fmt=mor.MOR_FMT_AUTO):
    if wl.E is None:
        mor.mor_set_system(h, wl.A, wl.B, wl.C, fmt=fmt)
    elif isinstance(wl.E, np.ndarray):
        mor.mor_set_system(h, wl.A, wl.B, wl.C, E_diag=wl.E, fmt=fmt)
    else:
        mor.mor_set_system(h, wl.A, wl.B, wl.C, E=wl.E, fmt=fmt)


def _dia_ok(name):
    """Stencil patterns have few diagonals; the random ones are refused by the diagonal layout."""
    return not name.startswith("rand")


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("fmt", [mor.MOR_FMT_CSR, mor.MOR_FMT_SELL, mor.MOR_FMT_DIA])
@pytest.mark.parametrize("transpose", [0, 1])
@pytest.mark.parametrize("precision", [mor.MOR_FP64, mor.MOR_MIXED])
def test_operator_spmv(h, name, fmt, transpose, precision):
    wl = SYSTEMS[name]()
    if fmt == mor.MOR_FMT_DIA and not _dia_ok(name):
        with pytest.raises(mor.MorError, match="diagonals"):
            _set(h, wl, fmt)
        return
    _set(h, wl, fmt)
    assert mor.mor_get_info(h)["format"] == fmt
    rng = np.random.default_rng(10)
    for k in (1, 3, 16):
        sig = np.array([2.0 + 0.5j * c if c % 2 else 10.0 * (c + 1) for c in range(k)], dtype=complex)
        X = rng.standard_normal((wl.n, k)) + 1j * rng.standard_normal((wl.n, k))
        if precision == mor.MOR_MIXED:
            X = X.astype(np.complex64).astype(np.complex128)
        Y = mor.mor_apply_operator(h, sig, X, transpose=transpose, precision=precision)
        Ea, Aa = _E_abs(wl), abs(wl.A)
        if transpose:
            Ea, Aa = Ea.T, Aa.T
        u = U64 if precision == mor.MOR_FP64 else U32
        for c in range(k):
            ref = oop.A_sigma(wl.A, wl.E, sig[c], transpose=bool(transpose)) @ X[:, c]
            bnd = (abs(sig[c]) * (Ea @ np.abs(X[:, c])) + Aa @ np.abs(X[:, c]))
            assert np.all(np.abs(Y[:, c] - ref) <= 30 * u * bnd + 1e-300), (name, k, c)


def test_operator_second_order(h):
    """(s^2 + alpha s) M + (1 + beta s) K applied on the fly (27-point K)."""
    wl = W.stencil27_second_order(nx=9, ny=8, nz=7)
    mor.mor_set_system_2nd(h, wl.K, wl.M_diag, wl.alpha, wl.beta, wl.F, wl.C)
    sig = np.array([0.3 + 0.2j, 2.0])
    rng = np.random.default_rng(1)
    X = rng.standard_normal((wl.n, 2)) + 1j * rng.standard_normal((wl.n, 2))
    Y = mor.mor_apply_operator(h, sig, X, precision=mor.MOR_FP64)
    for c in range(2):
        ref = oop.A_sigma_2nd(wl.K, wl.M_diag, wl.alpha, wl.beta, sig[c]) @ X[:, c]
        np.testing.assert_allclose(Y[:, c], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def _oracle_factor_csr(h, wl, M_new, M_old, transpose):
    """Oracle factor on the library's pattern, returned in the library's CSR order."""
    S = ospai.spai_pattern(wl.A, wl.E, transpose=bool(transpose))
    X = ospai.spai(M_new, S) if M_old is None else ospai.reuse_factor(M_old, M_new, S)
    rowptr, col = mor.mor_get_pattern(h, transpose)
    # the library's pattern is the oracle's S (pattern(A) + pattern(E) + diagonal), entry for entry
    assert np.array_equal(S.indptr, rowptr) and np.array_equal(S.indices, col)
    dense_rows = np.repeat(np.arange(wl.n), np.diff(rowptr))
    return np.asarray(X[dense_rows, col]).ravel(), rowptr, col


@pytest.mark.parametrize("name,fmt", [("laplace2d_n1369", mor.MOR_FMT_SELL), ("convdiff3d_n2197", mor.MOR_FMT_SELL),
                                      ("rand_csrE_n700", mor.MOR_FMT_SELL), ("convdiff3d_n2197", mor.MOR_FMT_DIA)])
@pytest.mark.parametrize("transpose", [0, 1])
@pytest.mark.parametrize("precision", [mor.MOR_FP64, mor.MOR_MIXED])
def test_spai_build_and_update(h, name, fmt, transpose, precision):
    """Factors written into the storage layout (SELL-32: padded slices; DIA:
    diagonals) and read back in CSR order, against the oracle."""
    wl = SYSTEMS[name]()
    _set(h, wl, fmt)
    s1, s2 = 12.0 + 3.0j, 20.0 - 1.0j
    mor.mor_build_precond(h, s1, transpose, precision)
    mor.mor_update_precond(h, s2, transpose)
    L, prec = mor.mor_chain_info(h, transpose)
    assert L == 2 and prec == precision
    tol = 1e-9 if precision == mor.MOR_FP64 else 2e-4
    M1 = oop.A_sigma(wl.A, wl.E, s1, transpose=bool(transpose))
    M2 = oop.A_sigma(wl.A, wl.E, s2, transpose=bool(transpose))
    for idx, (Mn, Mo) in enumerate([(M1, None), (M2, M1)]):
        vals, sf, st = mor.mor_get_factor(h, transpose, idx)
        ref, rowptr, col = _oracle_factor_csr(h, wl, Mn, Mo, transpose)
        assert st == (s1 if idx == 0 else s2)
        # compare column by column (each column is one least-squares problem)
        Pg = sp.csr_matrix((vals, col, rowptr), shape=(wl.n, wl.n)).tocsc()
        Po = sp.csr_matrix((ref, col, rowptr), shape=(wl.n, wl.n)).tocsc()
        for j in range(0, wl.n, max(1, wl.n // 200)):
            a = Pg[:, j].toarray().ravel()
            b = Po[:, j].toarray().ravel()
            assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b), (idx, j)


def test_spai_real_shift_equal_shift_identity(h):
    """Reuse with sigma_new = sigma_old gives Q = I on the GPU too."""
    wl = SYSTEMS["convdiff3d_n2197"]()
    _set(h, wl)
    mor.mor_build_precond(h, 7.0, 0, mor.MOR_FP64)
    mor.mor_update_precond(h, 7.0, 0)
    vals, _, _ = mor.mor_get_factor(h, 0, 1)
    rowptr, col = mor.mor_get_pattern(h, 0)
    Q = sp.csr_matrix((vals, col, rowptr), shape=(wl.n, wl.n)).toarray()
    np.testing.assert_allclose(Q, np.eye(wl.n), atol=1e-12)


@pytest.mark.parametrize("precision", [mor.MOR_FP64, mor.MOR_MIXED])
def test_chain_apply_prefixes(h, precision):
    """mor_apply_precond applies, for each shift, the chain prefix that ends at
    the factor built for it: P_1 for s1, Q_2 P_1 for s2, Q_3 Q_2 P_1 for s3."""
    wl = SYSTEMS["convdiff3d_n2197"]()
    _set(h, wl)
    s = [5.0, 9.0 + 2.0j, 30.0 + 1.0j]
    mor.mor_build_precond(h, s[0], 0, precision)
    mor.mor_update_precond(h, s[1], 0)
    mor.mor_update_precond(h, s[2], 0)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((wl.n, 3)) + 1j * rng.standard_normal((wl.n, 3))
    Y = mor.mor_apply_precond(h, s, X)
    S = ospai.spai_pattern(wl.A, wl.E)
    Ms = [oop.A_sigma(wl.A, wl.E, x) for x in s]
    F = [ospai.spai(Ms[0], S), ospai.reuse_factor(Ms[0], Ms[1], S), ospai.reuse_factor(Ms[1], Ms[2], S)]
    tol = 1e-9 if precision == mor.MOR_FP64 else 1e-4
    for c in range(3):
        ref = ospai.chain_apply(F[: c + 1], X[:, c])
        assert np.linalg.norm(Y[:, c] - ref) <= tol * np.linalg.norm(ref)


def test_orthonormalize_cgs2(h):
    wl = SYSTEMS["laplace2d_n1369"]()
    _set(h, wl)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((wl.n, 10))
    X[:, 7] = X[:, 6] + 1e-6 * rng.standard_normal(wl.n)
    V = mor.mor_orthonormalize(h, X)
    assert np.linalg.norm(V.T @ V - np.eye(10)) <= 1e-13
    assert np.linalg.norm(X - V @ (V.T @ X)) <= 1e-10 * np.linalg.norm(X)
    Vo, _ = oirka.cgs2(X)
    np.testing.assert_allclose(V, Vo, atol=1e-9)


def test_orthonormalize_dependent_column_is_reported(h):
    wl = SYSTEMS["rand_diagE_n33"]()
    _set(h, wl)
    X = np.ones((wl.n, 3))
    with pytest.raises(mor.MorError) as e:
        mor.mor_orthonormalize(h, X)
    assert e.value.code == mor.MOR_ESINGULAR


@pytest.mark.parametrize("name", ["convdiff3d_n2197", "rand_csrE_n700"])
def test_project_matches_oracle(h, name):
    wl = SYSTEMS[name]()
    _set(h, wl)
    rng = np.random.default_rng(5)
    V, _ = oirka.cgs2(rng.standard_normal((wl.n, 6)))
    Wb, _ = oirka.cgs2(rng.standard_normal((wl.n, 6)))
    rom = mor.mor_project(h, V, Wb)
    Ar, Er, Br, Cr = rom.arrays()
    ro = oirka.project(wl.A, wl.E, wl.B, wl.C, V, Wb)
    for g, o in zip((Ar, Er, Br, Cr), ro):
        np.testing.assert_allclose(g, o, rtol=1e-10, atol=1e-10 * np.abs(o).max())


@pytest.mark.parametrize("r", [1, 2, 6, 10, 16, 33])
def test_reduced_poles_vs_lapack(h, r):
    wl = SYSTEMS["rand_diagE_n33"]()
    _set(h, wl)
    rng = np.random.default_rng(r)
    Ar = rng.standard_normal((r, r)) - 3 * np.eye(r)
    Er = rng.standard_normal((r, r)) + 4 * np.eye(r)
    rom = mor.reduced_from_arrays(Ar, Er, np.ones((r, 1)), np.ones((r, 1)))
    lam, shifts = mor.mor_reduced_poles(h, rom)
    ref = oirka.reduced_poles(Ar, Er)
    scale = np.abs(ref).max()
    for x in ref:
        assert np.min(np.abs(lam - x)) <= 1e-10 * scale
    np.testing.assert_allclose(shifts, oirka.mirror_shifts(ref), rtol=1e-9, atol=1e-10 * scale)


def test_eval_tf_vs_oracle(h):
    wl = SYSTEMS["rand_diagE_n33"]()
    _set(h, wl)
    rng = np.random.default_rng(2)
    r, m, q = 12, 3, 2
    Ar = rng.standard_normal((r, r)) - 4 * np.eye(r)
    Er = np.eye(r) + 0.1 * rng.standard_normal((r, r))
    Br = rng.standard_normal((r, m))
    Cr = rng.standard_normal((r, q))
    rom = mor.reduced_from_arrays(Ar, Er, Br, Cr)
    w = np.logspace(0, 5, 1000)
    Hg = mor.mor_eval_tf(h, rom, w)
    Ho = oop.transfer_function_reduced(Ar, Er, Br, Cr, 1j * w)
    np.testing.assert_allclose(Hg, Ho, rtol=1e-11, atol=1e-13 * np.abs(Ho).max())


def test_invalid_inputs_are_rejected(h):
    A = sp.csr_matrix(np.array([[2.0, 1.0], [0.0, 3.0]]))
    B = np.ones((2, 1))
    bad = (2, np.array([0, 2, 1], np.int32), np.array([0, 1, 1], np.int32), np.ones(3))     # rowptr decreases
    with pytest.raises(mor.MorError) as e:
        mor.mor_set_system(h, bad, B, B)
    assert e.value.code == mor.MOR_EINVAL
    bad2 = (2, np.array([0, 2, 3], np.int32), np.array([1, 0, 1], np.int32), np.ones(3))    # unsorted row
    with pytest.raises(mor.MorError):
        mor.mor_set_system(h, bad2, B, B)
    bad3 = (2, np.array([0, 1, 2], np.int32), np.array([0, 5], np.int32), np.ones(2))      # out of range
    with pytest.raises(mor.MorError):
        mor.mor_set_system(h, bad3, B, B)
    mor.mor_set_system(h, A, B, B)
    with pytest.raises(mor.MorError) as e:
        mor.mor_update_precond(h, 1.0, 0)
    assert e.value.code == mor.MOR_ESTATE
