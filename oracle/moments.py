"""Multi-moment matching with repeated solves at fixed shifts (oracle; test
infrastructure only).  Shares no code with the CUDA library.

The higher moments of QB-IHOMM (Sec. II) are blocks of the form
[(sigma D - K)^{-1} D]^j (sigma D - K)^{-1} F, i.e. for the first-order
system E x' = A x + B u, y = C^T x (descriptor E in the role of D, A in the
role of K) the sequence
    X_0 = (sigma E - A)^{-1} B,   X_j = (sigma E - A)^{-1} E X_{j-1},
J solves with one matrix per shift, all with the same preconditioner.  The
transposed sequence Y_j with (sigma E - A)^{-T}, E^T and C gives the left
blocks.  Projection: V = orth of [Re X_j, Im X_j] (one-sided, W = V) or in
addition W = orth of [Re Y_j, Im Y_j] (two-sided), and the reduced pencil
(W^T A V, W^T E V), W^T B, V^T C.

Because X_j = (-1)^j / j! d^j/ds^j (sE - A)^{-1} B at s = sigma, the
one-sided ROM interpolates H and its first J - 1 derivatives at every shift,
the two-sided one its first 2J - 1 (rational Krylov moment matching); the
tests pin both against derivatives of the full transfer function.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from .operator import A_sigma, E_matrix
from .irka import cgs2
from .spai import spai, spai_pattern, chain_apply
from .krylov import bicgstab


def moment_blocks(A, E, R, sigma, J: int, transpose: bool = False, solver: str = "dense",
                  tol: float = 1e-8, precond: bool = True):
    """[X_0, ..., X_{J-1}] with X_0 = M^{-1} R and X_j = M^{-1} E' X_{j-1},
    M = sigma E - A (or its transpose, with E' = E^T).  solver 'dense' (LU)
    or 'bicgstab' with one SPAI of M reused for every block (the matrix does
    not change between the moments)."""
    if J < 1:
        raise ValueError("J must be >= 1")
    n = A.shape[0]
    M = A_sigma(A, E, sigma, transpose=transpose)
    Em = E_matrix(E, n)
    if transpose:
        Em = Em.T.tocsr()
    dtype = np.result_type(M.dtype, R.dtype, np.float64)
    if solver == "dense":
        Md = M.toarray()

        def solve(Rb):
            return np.linalg.solve(Md, Rb.astype(dtype))
    else:
        P = spai(M, spai_pattern(A, E, transpose=transpose)) if precond else None

        def solve(Rb):
            X = np.zeros((n, Rb.shape[1]), dtype=dtype)
            for c in range(Rb.shape[1]):
                x, _, _, _ = bicgstab(lambda v: M @ v, (lambda v: chain_apply([P], v)) if P is not None else None,
                                      Rb[:, c].astype(dtype), tol=tol)
                X[:, c] = x
            return X
    out = [solve(R)]
    for _ in range(1, J):
        out.append(solve(Em @ out[-1]))
    return out


def _real_span(blocks, shifts):
    cols = []
    for X, s in zip(blocks, shifts):
        cols.append(X.real)
        if complex(s).imag != 0.0:
            cols.append(X.imag)
    return cgs2(np.concatenate(cols, axis=1))[0]


def multi_moment_rom(A, E, B, C, shifts, J: int, two_sided: bool = True, solver: str = "dense",
                     tol: float = 1e-8):
    """Reduced pencil (A_r, E_r, B_r, C_r) from J moment blocks at every
    shift (one member of each conjugate pair suffices: Re and Im span both)."""
    n = A.shape[0]
    Em = E_matrix(E, n)
    vb, vs, wb, ws = [], [], [], []
    for s in shifts:
        for X in moment_blocks(A, E, B, s, J, solver=solver, tol=tol):
            vb.append(X)
            vs.append(s)
        if two_sided:
            for Y in moment_blocks(A, E, C, s, J, transpose=True, solver=solver, tol=tol):
                wb.append(Y)
                ws.append(s)
    V = _real_span(vb, vs)
    W = _real_span(wb, ws) if two_sided else V
    if W.shape[1] != V.shape[1]:
        raise ValueError("left and right bases differ in size")
    return W.T @ (A @ V), W.T @ (Em @ V), W.T @ B, V.T @ C
