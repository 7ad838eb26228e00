"""Second-order model reduction with reused SPAI preconditioners (oracle;
test infrastructure only).  Shares no code with the CUDA library.

Systems  M x'' + D x' + K x = F u,  y = C^T x,  D = alpha M + beta K
(Eq. linear-non-para), M diagonal.  One AIRGA iteration (Algorithm 1):
  lines 3-5  X^(0)(s_i) = (s_i^2 M + s_i D + K)^{-1} F at the expansion points
             (one solve per column of F, right-preconditioned, with the reuse
             schedule of Algorithm 4 on s^2 M + s D + K);
  lines 7-12 the inner moment loop, here run for a fixed number J of moments
             per point (``moments``; J = 1 skips it): V_j = X^(j-1) / ||X^(j-1)||_F
             and X^(j)(s_i) = -(s_i^2 M + s_i D + K)^{-1} M V_j, solved with the
             same matrix and the same (reused) preconditioner as X^(0)(s_i);
  Galerkin   V = orth([Re X^(j)(s_i), Im X^(j)(s_i)]) by CGS2 (the Frobenius
             normalisations do not change the span), M_r = V^T M V,
             K_r = V^T K V, D_r = alpha M_r + beta K_r, F_r = V^T F, C_r = V^T C
             (Sec. II);
  line 11    "all expansion points are updated": the rule is not stated.
The inner loop's own stopping test (an H2 change, Sec. IV) and an adaptive r
are not taken: J is an input.
Reading taken for line 11: the new points are the mirror images
sigma = |Re lambda| - i Im lambda of the eigenvalues lambda of the reduced
quadratic eigenproblem (lambda^2 M_r + lambda D_r + K_r) x = 0 of smallest
modulus, as many as there were points, closed under conjugation: taken in
order of increasing |lambda| (ties by Re, then Im), a conjugate pair only
when two places are left; if one place is left and no real eigenvalue comes
before the candidates run out, that place gets the real point |lambda| of the
first pair that did not fit.  Only the point with Im >= 0 of a conjugate
pair is solved; it contributes 2 m J real basis columns, a real point m J,
so r = m J (number of points).
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .operator import A_sigma_2nd
from .spai import spai, reuse_factor, spai_pattern, chain_apply
from .krylov import bicgstab, gmres
from .irka import cgs2, sort_shifts, solve_shifts_of, pair_conjugates, ReuseSchedule, IrkaResult


class ReuseSchedule2(ReuseSchedule):
    """Algorithm 4's schedule on s^2 M + s D + K (pattern of K plus the
    diagonal); the matrix is symmetric, so one chain serves every solve."""

    def __init__(self, K, M_diag, alpha, beta, mode: str = "reuse", max_chain: Optional[int] = None):
        self.K, self.Md, self.alpha, self.beta = K, M_diag, alpha, beta
        self.transpose = False
        self.mode = mode
        self.max_chain = max_chain
        self.S = spai_pattern(K, None)
        self.vertical = []
        self.sigma1_prev = None
        self.builds = []

    def _Asig(self, s):
        return A_sigma_2nd(self.K, self.Md, self.alpha, self.beta, s)


def transfer_function_2nd(K, M_diag, alpha, beta, F, C, s_values) -> np.ndarray:
    """H(s) = C^T (s^2 M + s D + K)^{-1} F (dense LU; small systems)."""
    out = []
    for s in np.atleast_1d(s_values):
        A = A_sigma_2nd(K, M_diag, alpha, beta, s).toarray().astype(np.complex128)
        out.append(C.T @ np.linalg.solve(A, F.astype(np.complex128)))
    return np.asarray(out)


def transfer_function_2nd_reduced(Mr, Dr, Kr, Fr, Cr, s_values) -> np.ndarray:
    """H_r(s) = C_r^T (s^2 M_r + s D_r + K_r)^{-1} F_r."""
    out = []
    for s in np.atleast_1d(s_values):
        out.append(Cr.T @ np.linalg.solve(s * s * Mr + s * Dr + Kr, Fr.astype(np.complex128)))
    return np.asarray(out)


def qep_eigenvalues(Mr, Dr, Kr) -> np.ndarray:
    """The 2r eigenvalues of lambda^2 M_r + lambda D_r + K_r by the first
    companion linearisation [[0, I], [-K_r, -D_r]] z = lambda [[I, 0], [0, M_r]] z,
    z = [x; lambda x], solved by LAPACK (scipy.linalg.eig)."""
    r = Mr.shape[0]
    I = np.eye(r)
    Z = np.zeros((r, r))
    A2 = np.block([[Z, I], [-Kr, -Dr]])
    E2 = np.block([[I, Z], [Z, Mr]])
    return np.asarray(sla.eig(A2, E2, right=False), dtype=np.complex128)


def select_points(lam: np.ndarray, count: int) -> np.ndarray:
    """The reading of Algorithm 1 line 11 (module docstring): `count` new
    points from the eigenvalues `lam`, smallest modulus first, conjugate-closed."""
    lam = pair_conjugates(lam)
    cands = []                                  # (modulus, re, im, size)
    for z in lam:
        if z.imag == 0.0:
            cands.append((abs(z), z.real, 0.0, 1))
        elif z.imag > 0.0:
            cands.append((abs(z), z.real, z.imag, 2))
    cands.sort(key=lambda c: (c[0], c[1], c[2]))
    pts = []
    left = count
    skipped = None
    for mod, re, im, size in cands:
        if left == 0:
            break
        if size <= left:
            lamz = complex(re, im)
            sig = abs(lamz.real) - 1j * lamz.imag
            pts.append(sig)
            if size == 2:
                pts.append(np.conj(sig))
            left -= size
        elif skipped is None:
            skipped = mod
    if left > 0:
        if skipped is None:
            raise ValueError("not enough eigenvalues for the expansion points")
        pts.append(complex(skipped, 0.0))
    return sort_shifts(np.array(pts, dtype=np.complex128))


def real_block_basis(blocks, points) -> np.ndarray:
    """Re X and (for a complex point) Im X of each solved block, side by side."""
    cols = []
    for X, s in zip(blocks, points):
        cols.append(X.real)
        if s.imag != 0.0:
            cols.append(X.imag)
    return np.concatenate(cols, axis=1)


def airga_step(K, M_diag, alpha, beta, F, C, points, sched: ReuseSchedule2, z: int, solver: str = "bicgstab",
               tol: float = 1e-8, maxit: int = 20000, moments: int = 1):
    """One iteration (module docstring) with ``moments`` = J blocks per
    solved point.  Returns (new points, (M_r, D_r, K_r, F_r, C_r), iteration
    counts, true relative residuals, solved points)."""
    if moments < 1:
        raise ValueError("moments must be >= 1")
    s_solve = solve_shifts_of(points)
    chains = sched.chains(z, s_solve)
    if solver == "dense":
        def krylov(apply_A, apply_P, b, tol=None, maxit=None, M=None):
            x = np.linalg.solve(M.toarray(), b)
            return x, 0, np.linalg.norm(b - M @ x) / np.linalg.norm(b), 0
    else:
        base = bicgstab if solver == "bicgstab" else gmres

        def krylov(apply_A, apply_P, b, tol=tol, maxit=maxit, M=None):
            return base(apply_A, apply_P, b, tol=tol, maxit=maxit)
    blocks, bpts, its, rr = [], [], [], []
    for s, ch in zip(s_solve, chains):
        M = A_sigma_2nd(K, M_diag, alpha, beta, s)

        def block_solve(R):
            X = np.zeros((K.shape[0], R.shape[1]), dtype=np.complex128)
            for j in range(R.shape[1]):
                rhs = R[:, j] if np.iscomplexobj(R) and M.dtype.kind == "c" else np.real(R[:, j])
                x, it, rel, _ = krylov(lambda v, M=M: M @ v, (lambda v, f=ch: chain_apply(f, v)) if ch else None,
                                       rhs.astype(M.dtype), M=M)
                X[:, j] = x
                its.append(it)
                rr.append(rel)
            return X

        X = block_solve(F)                                   # X^(0)(s)
        blocks.append(X)
        bpts.append(s)
        for _ in range(1, moments):
            Vj = X / np.linalg.norm(X, "fro")                # V_j = X^(j-1) / ||X^(j-1)||_F
            X = block_solve(-(M_diag[:, None] * Vj))         # X^(j) = -A(s)^{-1} M V_j
            blocks.append(X)
            bpts.append(s)
    V, _ = cgs2(real_block_basis(blocks, bpts))
    Mr = V.T @ (M_diag[:, None] * V)
    Kr = V.T @ (K @ V)
    Dr = alpha * Mr + beta * Kr
    rom = (Mr, Dr, Kr, V.T @ F, V.T @ C)
    new = select_points(qep_eigenvalues(Mr, Dr, Kr), len(points))
    return new, rom, its, rr, s_solve


def airga(K, M_diag, alpha, beta, F, C, points, iters: int, mode: str = "reuse", solver: str = "bicgstab",
          tol: float = 1e-8, maxit: int = 20000, max_chain: Optional[int] = None, moments: int = 1):
    """``iters`` iterations from the initial expansion points, ``moments``
    blocks per point.  The result's (Ar, Er, Br, Cr) slots hold (K_r, M_r,
    F_r, C_r); D_r = alpha M_r + beta K_r."""
    sched = ReuseSchedule2(K, M_diag, alpha, beta, mode=mode, max_chain=max_chain)
    p = sort_shifts(points)
    res = IrkaResult([p], None, None, None, None)
    solved = []
    for z in range(1, iters + 1):
        p, rom, its, rr, s_solve = airga_step(K, M_diag, alpha, beta, F, C, p, sched, z, solver=solver, tol=tol,
                                              maxit=maxit, moments=moments)
        res.shifts_history.append(p)
        res.Ar, res.Er, res.Br, res.Cr = rom[2], rom[0], rom[3], rom[4]
        res.iters.append(its)
        res.relres.append(rr)
        solved.append((s_solve, rom))
    res.builds = sched.builds
    return res, solved
