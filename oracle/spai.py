"""SPAI preconditioner, its reuse update, and the factor chain (oracle).

Test infrastructure only; shares no code with the CUDA library.

Sec. III.A, Eq. (gen-precond) / (gen-precond-par): the right preconditioner P
minimises ||I - A P||_F^2, which splits into n independent column problems
    min_{p_j} || e_j - A p_j ||_2 ,   j = 1..n.
Sec. III.B, Table II (second approach): given P_{i-1} for A_{i-1}, the
preconditioner for A_i is P_i = Q_i P_{i-1}, where Q_i minimises
||A_{i-1} - A_i Q_i||_F, again column by column with right-hand side the
j-th column of A_{i-1}.  P_i is never formed: it is applied as the chain of
sparse mat-vecs Q_i (Q_{i-1} ( ... (P_1 x))) (Sec. III.C, Algorithm 4).

Sparsity pattern (the paper uses MSPAI's adaptive pattern, which is not
reproduced): every P and Q column j is restricted to J_j = the pattern of
column j of S, where S = pattern(A) + pattern(E) + diagonal, i.e. the pattern
of sigma E - A for generic sigma.  The least-squares problem of column j only
involves the rows I_j where the columns M(:, J_j) have non-zeros (the
"shadow" of J_j); rows outside I_j add a constant to the objective and do not
change the minimiser.  Structurally I_j is the pattern of column j of S*S.
"""
from __future__ import annotations

from collections import defaultdict

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def spai_pattern(A, E=None, transpose: bool = False) -> sp.csr_matrix:
    """0/1 pattern S of sigma E - A for generic sigma, diagonal included.
    ``transpose`` gives the pattern of the transposed operator."""
    n = A.shape[0]
    S = abs(sp.csr_matrix(A, dtype=np.float64))
    if E is not None:
        if isinstance(E, np.ndarray) and E.ndim == 1:
            pass  # a diagonal is already in the pattern
        else:
            S = S + abs(sp.csr_matrix(E, dtype=np.float64))
    S = S + sp.identity(n, format="csr")
    S = sp.csr_matrix(S)
    S.data[:] = 1.0
    if transpose:
        S = sp.csr_matrix(S.T)
    S.sum_duplicates()
    S.sort_indices()
    S.data[:] = 1.0
    return S


def pattern_sets(S: sp.csr_matrix):
    """For every column j: J_j (rows of column j of S, sorted) and I_j (the
    union of the patterns of the columns k in J_j, sorted).

    Returns (Jptr, Jidx, Iptr, Iidx) in compressed form."""
    Sc = sp.csc_matrix(S)
    Sc.sort_indices()
    # I_j = { i : exists k in J_j with S_ik != 0 } = pattern of column j of S*S
    S2 = sp.csc_matrix(abs(Sc) @ abs(Sc))
    S2.sort_indices()
    return (Sc.indptr.astype(np.int64), Sc.indices.astype(np.int64),
            S2.indptr.astype(np.int64), S2.indices.astype(np.int64))


def _lookup(M: sp.csr_matrix, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """Dense gather M[rows, cols] (broadcast arrays) from a canonical CSR
    matrix: 0 where M has no entry."""
    n = M.shape[1]
    M = sp.csr_matrix(M)
    M.sort_indices()
    r_of = np.repeat(np.arange(M.shape[0], dtype=np.int64), np.diff(M.indptr))
    keys = r_of * n + M.indices.astype(np.int64)        # sorted (canonical CSR)
    q = rows.astype(np.int64) * n + cols.astype(np.int64)
    pos = np.searchsorted(keys, q)
    pos_c = np.minimum(pos, len(keys) - 1)
    hit = (pos < len(keys)) & (keys[pos_c] == q)
    out = np.zeros(q.shape, dtype=M.dtype)
    out[hit] = M.data[pos_c[hit]]
    return out


def column_least_squares(M, R, S: sp.csr_matrix, columns=None) -> sp.csr_matrix:
    """The matrix X with pattern S whose column j solves
        min_x || R(:, j) - M(:, J_j) x ||_2 ,   x supported on J_j.

    R = I gives the SPAI columns of Eq. (gen-precond-par); R = A_{i-1} gives
    the reuse factor Q_i of Table II (second approach).  Each column is an
    independent dense least-squares problem on the rows I_j, solved by
    Householder QR (numpy.linalg.qr, LAPACK geqrf) and a triangular solve;
    columns with the same (|I_j|, |J_j|) are stacked into one batched call,
    which does not couple them.  ``columns`` restricts the work to a subset
    (the other columns of X are left zero).

    Parity: pinned against per-column numpy.linalg.lstsq on all n rows, the
    normal equations, P = A^{-1} with a full pattern, Q = I for equal shifts
    and Q = A_i^{-1} A_{i-1} with a full pattern (tests/test_oracle_spai.py).
    """
    M = sp.csr_matrix(M)
    R = sp.csr_matrix(R)
    dtype = np.result_type(M.dtype, R.dtype, np.float64)
    Jptr, Jidx, Iptr, Iidx = pattern_sets(S)
    n = S.shape[0]
    cols = np.arange(n) if columns is None else np.asarray(columns, dtype=np.int64)
    groups = defaultdict(list)
    for j in cols:
        groups[(int(Iptr[j + 1] - Iptr[j]), int(Jptr[j + 1] - Jptr[j]))].append(int(j))
    # X stored by columns on S's pattern (CSC of S)
    Sc = sp.csc_matrix(S)
    Sc.sort_indices()
    xval = np.zeros(Sc.nnz, dtype=dtype)
    for (nI, nJ), js in groups.items():
        js = np.asarray(js, dtype=np.int64)
        Irows = np.stack([Iidx[Iptr[j]:Iptr[j + 1]] for j in js])          # b x nI
        Jcols = np.stack([Jidx[Jptr[j]:Jptr[j + 1]] for j in js])          # b x nJ
        G = _lookup(M, Irows[:, :, None], Jcols[:, None, :]).astype(dtype)  # b x nI x nJ
        rhs = _lookup(R, Irows, np.broadcast_to(js[:, None], Irows.shape)).astype(dtype)
        Qf, Rf = np.linalg.qr(G, mode="reduced")
        y = np.einsum("bij,bi->bj", Qf.conj(), rhs)
        x = np.linalg.solve(Rf, y[:, :, None])[:, :, 0]
        for t, j in enumerate(js):
            xval[Sc.indptr[j]:Sc.indptr[j + 1]] = x[t]
    X = sp.csc_matrix((xval, Sc.indices.copy(), Sc.indptr.copy()), shape=(n, n))
    X = sp.csr_matrix(X)
    X.sort_indices()
    return X


def spai(M, S: sp.csr_matrix) -> sp.csr_matrix:
    """SPAI of M on pattern S: min ||I - M P||_F^2 split into columns
    (Sec. III.A, Eq. gen-precond-par)."""
    n = M.shape[0]
    return column_least_squares(M, sp.identity(n, format="csr"), S)


def reuse_factor(M_old, M_new, S: sp.csr_matrix) -> sp.csr_matrix:
    """Q minimising ||M_old - M_new Q||_F on pattern S (Table II, second
    approach; horizontal and vertical reuse of Sec. III.C)."""
    return column_least_squares(M_new, M_old, S)


def chain_apply(factors, x):
    """P x with P = F_L ... F_2 F_1 (factors[0] = F_1 is applied first):
    the preconditioner is never formed (Sec. III.B; Algorithm 4 applies
    Q_i ... Q_2 P_1 as successive mat-vecs)."""
    z = x
    for F in factors:
        z = F @ z
    return z


def frobenius_ratios(M_prev, M_new):
    """The two diagnostics of Tables III/VII: ||I - M_new||_F / ||I||_F and
    ||M_prev - M_new||_F / ||M_prev||_F (None when there is no M_prev)."""
    n = M_new.shape[0]
    I = sp.identity(n, format="csr")
    std = spla.norm(I - M_new) / np.sqrt(n)
    if M_prev is None:
        return std, None
    return std, spla.norm(M_prev - M_new) / spla.norm(M_prev)
