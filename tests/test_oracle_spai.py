"""Pins of the oracle's SPAI columns, reuse factors and chain (Sec. III,
Eq. gen-precond-par, Table II, Appendix B) against brute force and closed
forms."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import operator as op
from oracle import spai


def _sys(n=40, seed=7, e_kind="diag"):
    return W.random_sparse_system(n, 0.08, seed=seed, e_kind=e_kind)


def test_shadow_sets_bruteforce():
    """I_j = union over k in J_j of the rows of column k (python sets)."""
    wl = _sys(25, seed=1, e_kind="csr")
    S = spai.spai_pattern(wl.A, wl.E)
    Jp, Ji, Ip, Ii = spai.pattern_sets(S)
    Sd = S.toarray() != 0
    for j in range(25):
        J = set(np.nonzero(Sd[:, j])[0])
        I = set()
        for k in J:
            I |= set(np.nonzero(Sd[:, k])[0])
        assert list(Ji[Jp[j]:Jp[j + 1]]) == sorted(J)
        assert list(Ii[Ip[j]:Ip[j + 1]]) == sorted(I)


@pytest.mark.parametrize("sigma", [2.0, 1.0 + 3.0j])
@pytest.mark.parametrize("e_kind", ["identity", "diag", "csr"])
def test_spai_columns_match_full_row_lstsq(sigma, e_kind):
    """Each SPAI column equals numpy.linalg.lstsq of e_j against ALL n rows of
    M(:, J_j): the shadow restriction drops no information."""
    wl = _sys(40, seed=11, e_kind=e_kind)
    M = op.A_sigma(wl.A, wl.E, sigma)
    S = spai.spai_pattern(wl.A, wl.E)
    P = spai.spai(M, S).toarray()
    Md = M.toarray()
    Sd = S.toarray() != 0
    for j in range(40):
        J = np.nonzero(Sd[:, j])[0]
        e = np.zeros(40, dtype=Md.dtype)
        e[j] = 1
        ref = np.linalg.lstsq(Md[:, J], e, rcond=None)[0]
        np.testing.assert_allclose(P[J, j], ref, rtol=1e-10, atol=1e-13)
        off = np.setdiff1d(np.arange(40), J)
        assert np.all(P[off, j] == 0)
        # normal equations on all rows
        G = Md[:, J]
        np.testing.assert_allclose(G.conj().T @ (G @ P[J, j] - e), 0, atol=1e-12)


def test_spai_full_pattern_is_inverse():
    """Full pattern on a small dense matrix: P = A^{-1} (||A P - I|| ~ eps)."""
    rng = np.random.default_rng(3)
    n = 9
    Ad = rng.standard_normal((n, n)) + 5 * np.eye(n)
    A = sp.csr_matrix(Ad)
    S = sp.csr_matrix(np.ones((n, n)))
    for sigma in [0.5, 1.0 + 2.0j]:
        M = op.A_sigma(A, None, sigma)
        P = spai.spai(M, S).toarray()
        assert np.linalg.norm(M.toarray() @ P - np.eye(n)) < 1e-12


def test_spai_diagonal_matrix_exact():
    """A diagonal matrix with any pattern containing the diagonal: P = A^{-1}."""
    n = 15
    d = np.linspace(1, 3, n)
    A = sp.diags(-d, format="csr")
    S = sp.csr_matrix(sp.diags([np.ones(n - 1), np.ones(n), np.ones(n - 1)], [-1, 0, 1]))
    M = op.A_sigma(A, None, 2.0 + 1.0j)
    P = spai.spai(M, S).toarray()
    np.testing.assert_allclose(P, np.diag(1.0 / (2.0 + 1.0j + d)), atol=1e-15)


def test_reuse_equal_shifts_gives_identity():
    """sigma_new = sigma_old  =>  Q = I (Table II with A_{i-1} = A_i)."""
    wl = _sys(40, seed=5)
    S = spai.spai_pattern(wl.A, wl.E)
    M = op.A_sigma(wl.A, wl.E, 3.0 - 1.0j)
    Q = spai.reuse_factor(M, M, S).toarray()
    np.testing.assert_allclose(Q, np.eye(40), atol=1e-12)


def test_reuse_full_pattern_closed_form():
    """Full pattern: Q_i = A_i^{-1} A_{i-1} = (I + (s_i - s_{i-1}) A_{i-1}^{-1} E)^{-1}
    (Appendix B) and A_{i-1} P_{i-1} = A_i Q_i P_{i-1} (Sec. III.B)."""
    rng = np.random.default_rng(8)
    n = 8
    Ad = -(rng.standard_normal((n, n)) + 6 * np.eye(n))
    Ed = np.diag(rng.uniform(0.5, 1.5, n))
    A, E = sp.csr_matrix(Ad), sp.csr_matrix(Ed)
    S = sp.csr_matrix(np.ones((n, n)))
    s0, s1 = 1.0 + 0.5j, 2.5 + 1.0j
    M0, M1 = op.A_sigma(A, E, s0).toarray(), op.A_sigma(A, E, s1).toarray()
    Q = spai.reuse_factor(sp.csr_matrix(M0), sp.csr_matrix(M1), S).toarray()
    closed = np.linalg.inv(np.eye(n) + (s1 - s0) * np.linalg.solve(M0, Ed))
    np.testing.assert_allclose(Q, closed, atol=1e-12)
    P0 = spai.spai(sp.csr_matrix(M0), sp.csr_matrix(np.ones((n, n)) * (np.abs(Ad) > 0.5))).toarray()
    np.testing.assert_allclose(M1 @ Q @ P0, M0 @ P0, atol=1e-11)


def test_reuse_columns_match_full_row_lstsq():
    """Q columns with the static pattern: lstsq of A_{i-1}(:, j) against all
    rows of A_i(:, J_j)."""
    wl = _sys(35, seed=21, e_kind="csr")
    S = spai.spai_pattern(wl.A, wl.E)
    M0 = op.A_sigma(wl.A, wl.E, 1.0 + 1.0j)
    M1 = op.A_sigma(wl.A, wl.E, 1.4 + 0.7j)
    Q = spai.reuse_factor(M0, M1, S).toarray()
    M0d, M1d = M0.toarray(), M1.toarray()
    Sd = S.toarray() != 0
    for j in range(35):
        J = np.nonzero(Sd[:, j])[0]
        ref = np.linalg.lstsq(M1d[:, J], M0d[:, j], rcond=None)[0]
        np.testing.assert_allclose(Q[J, j], ref, rtol=1e-10, atol=1e-13)


def test_chain_apply_order():
    """chain [F1, F2, F3] applies F1 first: P x = F3 F2 F1 x."""
    rng = np.random.default_rng(2)
    Fs = [sp.csr_matrix(rng.standard_normal((6, 6))) for _ in range(3)]
    x = rng.standard_normal(6)
    ref = Fs[2].toarray() @ (Fs[1].toarray() @ (Fs[0].toarray() @ x))
    np.testing.assert_allclose(spai.chain_apply(Fs, x), ref, rtol=1e-13)


def test_frobenius_ratio_of_shift_change():
    """||A_{i-1} - A_i||_F = |s_i - s_{i-1}| ||E||_F for first-order systems."""
    wl = _sys(30, seed=4, e_kind="diag")
    M0 = op.A_sigma(wl.A, wl.E, 1.0)
    M1 = op.A_sigma(wl.A, wl.E, 1.0 + 2.0j)
    _, hor = spai.frobenius_ratios(M0, M1)
    num = abs(2.0j) * np.linalg.norm(wl.E)
    assert abs(hor - num / sp.linalg.norm(M0)) < 1e-12
