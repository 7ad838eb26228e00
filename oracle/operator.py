"""Shifted operator and transfer functions (oracle; test infrastructure only).

First-order systems  E x' = A x + B u,  y = C^T x  (Sec. II, the first-order
form of Algorithms 2 and 3 with the descriptor matrix written E).  Every
shifted solve of the method is with the matrix  A(sigma) = sigma E - A
(Algorithm 3 line 4 writes it sigma_i D - K); the transposed solves use
A(sigma)^T (Algorithm 2 line 5, Algorithm 3 line 10).

Second-order systems  M x'' + D x' + K x = F u  (Eq. linear-non-para, Sec. II)
give the matrix  s^2 M + s D + K  (Algorithm 1 line 4).

Everything is FP64 / complex128 and built explicitly with scipy.sparse;
nothing here is optimised.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def E_matrix(E, n: int) -> sp.csr_matrix:
    """The descriptor matrix as a sparse matrix: None -> I, 1-D -> diag."""
    if E is None:
        return sp.identity(n, format="csr", dtype=np.float64)
    if isinstance(E, np.ndarray) and E.ndim == 1:
        return sp.diags(E.astype(np.float64), 0, shape=(n, n), format="csr")
    return sp.csr_matrix(E, dtype=np.float64)


def A_sigma(A, E, sigma, transpose: bool = False) -> sp.csr_matrix:
    """sigma E - A (or its plain transpose), formed explicitly.

    Real sigma gives a float64 matrix, complex sigma a complex128 matrix.
    Parity: pinned by the closed-form eigenpairs of the Laplacian and by
    interior row sums (tests/test_oracle_operator.py)."""
    n = A.shape[0]
    Em = E_matrix(E, n)
    s = complex(sigma)
    if s.imag == 0.0:
        M = s.real * Em - A
    else:
        M = s * Em.astype(np.complex128) - A.astype(np.complex128)
    M = sp.csr_matrix(M)
    if transpose:
        M = sp.csr_matrix(M.T)
    M.sort_indices()
    return M


def A_sigma_2nd(K, M_diag, alpha, beta, sigma) -> sp.csr_matrix:
    """sigma^2 M + sigma D + K with Rayleigh damping D = alpha M + beta K
    (Eq. linear-non-para and Algorithm 1 line 4).  Parity: pinned by the
    expansion test against the three separate terms."""
    s = complex(sigma)
    n = K.shape[0]
    Mm = sp.diags(M_diag, 0, shape=(n, n), format="csr")
    D = alpha * Mm + beta * K
    if s.imag == 0.0:
        s = s.real
        out = s * s * Mm + s * D + K
    else:
        out = (s * s) * Mm.astype(np.complex128) + s * D.astype(np.complex128) + K.astype(np.complex128)
    out = sp.csr_matrix(out)
    out.sort_indices()
    return out


def transfer_function(A, E, B, C, s_values) -> np.ndarray:
    """H(s) = C^T (s E - A)^{-1} B for each s (q x m per point), by sparse
    LU (scipy splu).  Used as the exact reference on small systems."""
    out = []
    for s in np.atleast_1d(s_values):
        M = sp.csc_matrix(A_sigma(A, E, s).astype(np.complex128))
        lu = spla.splu(M)
        X = lu.solve(B.astype(np.complex128))
        out.append(C.T.astype(np.complex128) @ X)
    return np.asarray(out)


def transfer_function_reduced(Ar, Er, Br, Cr, s_values) -> np.ndarray:
    """H_r(s) = C_r^T (s E_r - A_r)^{-1} B_r for each s (dense LU)."""
    out = []
    for s in np.atleast_1d(s_values):
        X = np.linalg.solve(s * Er - Ar, Br.astype(np.complex128))
        out.append(Cr.T @ X)
    return np.asarray(out)
