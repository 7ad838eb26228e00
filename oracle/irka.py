"""IRKA with reused SPAI preconditioners (oracle; test infrastructure only).

Shares no code with the CUDA library.

The iteration is BIRKA (Algorithm 2) with all bilinear terms N_j = 0, which
is IRKA for E x' = A x + B u, y = C^T x:
  line 3   eigen-decompose the reduced pencil; the new shifts are the mirror
           images of the reduced poles, sigma_i = -lambda_i;
  line 4   v_i = (sigma_i E - A)^{-1} B b_i   (SISO: b_i = 1);
  line 5   w_i = (sigma_i E - A)^{-T} C c_i   (plain transpose);
  line 6   V = orth(V), W = orth(W)  (two-pass classical Gram-Schmidt);
  line 7   reduced system from the pencil (W^T A V, W^T E V), W^T B, V^T C.
The Petrov-Galerkin form (W^T V)^{-1} W^T A V of Sec. II describes the same
transfer function H_r; this oracle uses the pencil form.

Every solve is right-preconditioned; the preconditioners follow the reuse
schedule of Algorithm 4 (second approach of Table II) with IRKA's iteration z
in the role of the AIRGA iteration and the sorted shifts in the role of the
expansion points:
  z = 1, i = 1 :  P_1^(1) = SPAI(A_1^(1))                  (full build)
  z > 1, i = 1 :  Q_1^(z) from min ||A_1^(z-1) - A_1^(z) Q||_F   (vertical)
  i > 1        :  Q_i^(z) from min ||A_{i-1}^(z) - A_i^(z) Q||_F (horizontal)
and the preconditioner of (z, i) is Q_i^(z) ... Q_2^(z) Q_1^(z) ... Q_1^(2)
P_1^(1), applied factor by factor.  The transposed solves get their own
chain built the same way on A(sigma)^T ("similarly", Appendix A).  When A and
E are symmetric, A(sigma)^T = A(sigma) and the primal chain is reused.

Readings (the paper is silent): shifts are kept sorted by (Re, |Im|, -Im) so
that conjugate pairs are adjacent, positive imaginary part first; only the
member with Im >= 0 of each pair is solved (the other solution is its
conjugate) and it contributes the two real basis columns Re v, Im v; a reduced
pole with Re lambda > 0 is reflected, sigma = |Re lambda| - i Im lambda
(equal to -lambda for stable poles).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .operator import A_sigma, E_matrix, transfer_function_reduced
from .spai import spai, reuse_factor, spai_pattern, chain_apply, frobenius_ratios
from .krylov import bicgstab, gmres, STATUS_OK


# ----------------------------------------------------------------------------
# orthogonalisation, projection, reduced poles
# ----------------------------------------------------------------------------
def cgs2(X: np.ndarray):
    """Two-pass classical Gram-Schmidt, column by column: for column j,
    twice h = V^T v, v <- v - V h, then v / ||v||.  Returns (V, R) with
    X = V R.  Parity: pinned by orthogonality, span and X = V R."""
    n, k = X.shape
    V = np.zeros((n, k), dtype=X.dtype)
    R = np.zeros((k, k), dtype=X.dtype)
    for j in range(k):
        v = X[:, j].copy()
        for _ in range(2):
            h = V[:, :j].conj().T @ v
            v = v - V[:, :j] @ h
            R[:j, j] += h
        nv = np.linalg.norm(v)
        R[j, j] = nv
        V[:, j] = v / nv
    return V, R


def project(A, E, B, C, V, W):
    """Reduced pencil and vectors: E_r = W^T E V, A_r = W^T A V,
    B_r = W^T B, C_r = V^T C (Algorithm 2 line 7 in pencil form)."""
    n = A.shape[0]
    Em = E_matrix(E, n)
    return (W.T @ (A @ V), W.T @ (Em @ V), W.T @ B, V.T @ C)


def reduced_poles(Ar, Er) -> np.ndarray:
    """Generalized eigenvalues of (A_r, E_r) by LAPACK (scipy.linalg.eig)."""
    lam = sla.eig(Ar, Er, right=False)
    return np.asarray(lam, dtype=np.complex128)


def sort_shifts(s: np.ndarray) -> np.ndarray:
    """Sort by (Re, |Im|, -Im): conjugate pairs adjacent, +Im first."""
    s = np.asarray(s, dtype=np.complex128)
    order = np.lexsort((-s.imag, np.abs(s.imag), s.real))
    return s[order]


def pair_conjugates(lam: np.ndarray) -> np.ndarray:
    """Make the non-real members of a real pencil's spectrum exact conjugate
    pairs: each value with Im > 0 is matched to the nearest conj of a value
    with Im < 0 and both become (mean Re) +- i (mean |Im|).  LAPACK returns
    pairs whose real parts can differ in the last bit, which would otherwise
    let the sort split a pair."""
    lam = np.asarray(lam, dtype=np.complex128).copy()
    pos = [i for i in range(len(lam)) if lam[i].imag > 0]
    neg = [i for i in range(len(lam)) if lam[i].imag < 0]
    if len(pos) != len(neg):
        raise ValueError("spectrum of a real pencil is not closed under conjugation")
    free = list(neg)
    for i in pos:
        k = min(free, key=lambda t: abs(lam[t] - np.conj(lam[i])))
        free.remove(k)
        re = 0.5 * (lam[i].real + lam[k].real)
        im = 0.5 * (lam[i].imag - lam[k].imag)
        lam[i] = complex(re, im)
        lam[k] = complex(re, -im)
    return lam


def mirror_shifts(lam: np.ndarray) -> np.ndarray:
    """sigma_i = -lambda_i for stable poles, |Re| - i Im in general."""
    lam = pair_conjugates(lam)
    return sort_shifts(np.abs(lam.real) - 1j * lam.imag)


def solve_shifts_of(shifts: np.ndarray) -> np.ndarray:
    """The shifts that are actually solved: one per conjugate pair (Im >= 0)."""
    s = sort_shifts(shifts)
    return s[s.imag >= 0.0]


def real_basis(cols: List[np.ndarray], shifts: np.ndarray) -> np.ndarray:
    """Real basis columns from the solutions at the solved shifts: a real
    shift gives Re v, a complex one gives Re v and Im v."""
    out = []
    for v, s in zip(cols, shifts):
        out.append(v.real)
        if s.imag != 0.0:
            out.append(v.imag)
    return np.stack(out, axis=1)


# ----------------------------------------------------------------------------
# the reuse schedule (Algorithm 4)
# ----------------------------------------------------------------------------
class ReuseSchedule:
    """Keeps the vertical chain [P_1^(1), Q_1^(2), ..., Q_1^(z)] of one
    operator (primal or transposed) and returns, for the shifts of the
    current iteration, the factor chain of every shift.

    mode: 'reuse' (Algorithm 4: the second approach of Table II, P_i = Q_i
    P_{i-1}), 'first' (the first approach of Table II along the shifts of an
    iteration: P_i = Q_i P_1 with Q_i from min ||A_1 - A_i Q||_F, so every
    chain is the vertical chain plus one factor), 'auto' (Algorithm 4 with
    the reuse decision read from the Frobenius ratios the paper tabulates,
    see ``reuse_ok``), 'fresh' (a new SPAI per shift, the paper's "SPAI
    case"), or 'none' (unpreconditioned).  ``max_chain`` (default: no limit,
    as in the paper) rebuilds P_1 from scratch when the vertical chain would
    grow beyond it."""

    def __init__(self, A, E, transpose: bool, mode: str = "reuse",
                 max_chain: Optional[int] = None):
        self.A, self.E, self.transpose = A, E, transpose
        self.mode = mode
        self.max_chain = max_chain
        self.S = spai_pattern(A, E, transpose=transpose)
        self.vertical = []
        self.sigma1_prev = None
        self.builds = []     # (z, i, kind) records, kind in {'spai','vertical','horizontal'}

    def _Asig(self, s):
        return A_sigma(self.A, self.E, s, transpose=self.transpose)

    def reuse_ok(self, s_old, s_new) -> bool:
        """Reading of the paper's reuse criterion (Sec. IV, the discussion
        of its Frobenius-ratio table): reuse pays when ||I - A_new||_F /
        ||I||_F is large and ||A_old - A_new||_F / ||A_old||_F is small; the
        paper fixes no thresholds, so 'small' is read as below 1 and below
        the first ratio.  Otherwise a fresh SPAI is built for the new shift."""
        std, change = frobenius_ratios(self._Asig(s_old), self._Asig(s_new))
        return change < min(1.0, std)

    def chains(self, z: int, solve_shifts: np.ndarray):
        if self.mode == "none":
            return [[] for _ in solve_shifts]
        if self.mode == "fresh":
            out = []
            for i, s in enumerate(solve_shifts):
                out.append([spai(self._Asig(s), self.S)])
                self.builds.append((z, i + 1, "spai"))
            return out
        s1 = solve_shifts[0]
        rebuild = (not self.vertical) or (self.max_chain is not None and len(self.vertical) + 1 > self.max_chain)
        if not rebuild and self.mode == "auto":
            rebuild = not self.reuse_ok(self.sigma1_prev, s1)
        if rebuild:
            self.vertical = [spai(self._Asig(s1), self.S)]
            self.builds.append((z, 1, "spai"))
        else:
            self.vertical.append(reuse_factor(self._Asig(self.sigma1_prev), self._Asig(s1), self.S))
            self.builds.append((z, 1, "vertical"))
        self.sigma1_prev = s1
        out = [list(self.vertical)]
        for i in range(1, len(solve_shifts)):
            if self.mode == "first":
                Q = reuse_factor(self._Asig(s1), self._Asig(solve_shifts[i]), self.S)
                self.builds.append((z, i + 1, "first"))
                out.append(list(self.vertical) + [Q])
            elif self.mode == "auto" and not self.reuse_ok(solve_shifts[i - 1], solve_shifts[i]):
                self.builds.append((z, i + 1, "spai"))
                out.append([spai(self._Asig(solve_shifts[i]), self.S)])
            else:
                Q = reuse_factor(self._Asig(solve_shifts[i - 1]), self._Asig(solve_shifts[i]), self.S)
                self.builds.append((z, i + 1, "horizontal"))
                out.append(out[-1] + [Q])
        return out


# ----------------------------------------------------------------------------
# IRKA
# ----------------------------------------------------------------------------
@dataclass
class IrkaResult:
    shifts_history: List[np.ndarray]
    Ar: np.ndarray
    Er: np.ndarray
    Br: np.ndarray
    Cr: np.ndarray
    iters: List[List[int]] = field(default_factory=list)      # per iteration, per solve
    relres: List[List[float]] = field(default_factory=list)
    hermite: List[dict] = field(default_factory=list)
    builds: list = field(default_factory=list)


def _is_symmetric(A, E) -> bool:
    if (A != A.T).nnz != 0:
        return False
    if E is None or (isinstance(E, np.ndarray) and E.ndim == 1):
        return True
    return (E != E.T).nnz == 0


def irka_step(A, E, B, C, shifts, sched_V: ReuseSchedule, sched_W: Optional[ReuseSchedule],
              z: int, solver: str = "bicgstab", tol: float = 1e-8, maxit: int = 20000,
              hermite: bool = False):
    """One IRKA iteration (Algorithm 2 lines 3-7 with N_j = 0, SISO) with the
    reuse schedule of Algorithm 4.  Returns (new shifts, (Ar, Er, Br, Cr),
    iteration counts, true relative residuals, hermite data)."""
    s_solve = solve_shifts_of(shifts)
    chains_V = sched_V.chains(z, s_solve)
    chains_W = chains_V if sched_W is None else sched_W.chains(z, s_solve)
    vs, ws, its, rr = [], [], [], []
    if solver == "dense":
        krylov = _dense_krylov
    else:
        krylov = bicgstab if solver == "bicgstab" else gmres
    for s, cv, cw in zip(s_solve, chains_V, chains_W):
        M = A_sigma(A, E, s)
        MT = sp.csr_matrix(M.T)
        b = B[:, 0].astype(M.dtype)
        c = C[:, 0].astype(M.dtype)
        v, itv, rv, stv = krylov(lambda x: M @ x, (lambda x, f=cv: chain_apply(f, x)) if cv else None,
                                 b, tol=tol, maxit=maxit)
        w, itw, rw, stw = krylov(lambda x: MT @ x, (lambda x, f=cw: chain_apply(f, x)) if cw else None,
                                 c, tol=tol, maxit=maxit)
        vs.append(v)
        ws.append(w)
        its += [itv, itw]
        rr += [rv, rw]
    V, _ = cgs2(real_basis(vs, s_solve))
    W, _ = cgs2(real_basis(ws, s_solve))
    Ar, Er, Br, Cr = project(A, E, B, C, V, W)
    herm = None
    if hermite:
        Em = E_matrix(E, A.shape[0])
        herm = {"sigma": s_solve,
                "H": np.array([C[:, 0] @ v for v in vs]),
                "dH": np.array([-(w @ (Em @ v)) for v, w in zip(vs, ws)]),
                "Hr": np.array([transfer_function_reduced(Ar, Er, Br, Cr, s)[0, 0, 0] for s in s_solve]),
                "dHr": np.array([_dHr(Ar, Er, Br, Cr, s) for s in s_solve])}
    new = mirror_shifts(reduced_poles(Ar, Er))
    return new, (Ar, Er, Br, Cr), its, rr, herm


# ----------------------------------------------------------------------------
# tangential (MIMO) IRKA: the directions of Algorithm 2 line 3
# ----------------------------------------------------------------------------
def tangential_directions(Ar, Er, Br, Cr):
    """Reduced poles and tangential directions, Algorithm 2 line 3 with
    N_j = 0, read on the pencil: K = E_r^{-1} A_r = R Lambda R^{-1}
    (eigenvectors R by LAPACK), F = E_r^{-1} B_r, C = C_r^T.  The pole
    lambda_i = Lambda_ii carries the right direction b_i = column i of
    F^T R^{-T}, i.e. row i of R^{-1} F, and the left direction c_i = column i
    of C R.  Returns (lam (r,), btil (r, m), ctil (r, q)), row i belonging to
    lambda_i."""
    K = np.linalg.solve(Er, Ar)
    F = np.linalg.solve(Er, Br)
    lam, R = sla.eig(K)
    btil = np.linalg.solve(R, F.astype(np.complex128))
    ctil = (Cr.T.astype(np.complex128) @ R).T
    return np.asarray(lam, dtype=np.complex128), btil, ctil


def mirror_with_directions(lam, btil, ctil):
    """New shifts sigma_i = |Re lambda_i| - i Im lambda_i (as mirror_shifts)
    with each pole's directions, sorted by (Re, |Im|, -Im); the -Im member of
    a conjugate pair gets the conjugate directions of the +Im member."""
    lam = pair_conjugates(lam)
    sig = np.abs(lam.real) - 1j * lam.imag
    order = np.lexsort((-sig.imag, np.abs(sig.imag), sig.real))
    sig, bt, ct = sig[order], np.array(btil[order]), np.array(ctil[order])
    i = 0
    while i < len(sig):
        if sig[i].imag > 0:
            bt[i + 1] = np.conj(bt[i])
            ct[i + 1] = np.conj(ct[i])
            i += 2
        else:
            i += 1
    return sig, bt, ct


def irka_step_tangential(A, E, B, C, shifts, btil, ctil, sched_V: ReuseSchedule,
                         sched_W: Optional[ReuseSchedule], z: int, solver: str = "bicgstab",
                         tol: float = 1e-8, maxit: int = 20000):
    """One tangential IRKA iteration for a MIMO system (Algorithm 2 lines 3-7
    with N_j = 0): at each solved shift sigma_i with directions b_i, c_i,
    v_i = A(sigma_i)^{-1} B b_i and w_i = A(sigma_i)^{-T} C c_i (lines 4-5),
    V, W by CGS2 of the real bases (line 6), the reduced pencil (line 7), and
    the new shifts and directions from its eigenvectors (line 3 of the next
    iteration).  btil (r x m) and ctil (r x q) hold the directions row by row
    in the order of `shifts`.  Returns (new shifts, new btil, new ctil,
    (Ar, Er, Br, Cr), iteration counts, true relative residuals, solved data)."""
    shifts = np.asarray(shifts, dtype=np.complex128)
    order = np.lexsort((-shifts.imag, np.abs(shifts.imag), shifts.real))
    keep = shifts[order].imag >= 0.0
    s_solve = shifts[order][keep]
    b_solve = np.asarray(btil)[order][keep]
    c_solve = np.asarray(ctil)[order][keep]
    chains_V = sched_V.chains(z, s_solve)
    chains_W = chains_V if sched_W is None else sched_W.chains(z, s_solve)
    if solver == "dense":
        krylov = _dense_krylov
    else:
        krylov = bicgstab if solver == "bicgstab" else gmres
    vs, ws, its, rr = [], [], [], []
    for s, bi, ci, cv, cw in zip(s_solve, b_solve, c_solve, chains_V, chains_W):
        M = A_sigma(A, E, s)
        MT = sp.csr_matrix(M.T)
        dt = np.result_type(M.dtype, bi.dtype, ci.dtype)
        b = (B @ bi).astype(dt)
        c = (C @ ci).astype(dt)
        v, itv, rv, _ = krylov(lambda x, M=M: M @ x, (lambda x, f=cv: chain_apply(f, x)) if cv else None,
                               b, tol=tol, maxit=maxit)
        w, itw, rw, _ = krylov(lambda x, MT=MT: MT @ x, (lambda x, f=cw: chain_apply(f, x)) if cw else None,
                               c, tol=tol, maxit=maxit)
        vs.append(v)
        ws.append(w)
        its += [itv, itw]
        rr += [rv, rw]
    V, _ = cgs2(real_basis(vs, s_solve))
    W, _ = cgs2(real_basis(ws, s_solve))
    rom = project(A, E, B, C, V, W)
    lam, bt, ct = tangential_directions(*rom)
    new, bnew, cnew = mirror_with_directions(lam, bt, ct)
    solved = {"sigma": s_solve, "b": b_solve, "c": c_solve}
    return new, bnew, cnew, rom, its, rr, solved


def _dense_krylov(apply_A, apply_P, b, tol=None, maxit=None):
    """Exact solve for pins: assemble the operator column by column and use
    dense LU (small n only).  The preconditioner is ignored."""
    n = b.shape[0]
    I = np.eye(n, dtype=b.dtype)
    Md = np.stack([apply_A(I[:, j]) for j in range(n)], axis=1)
    x = np.linalg.solve(Md, b)
    return x, 0, np.linalg.norm(b - Md @ x) / np.linalg.norm(b), STATUS_OK


def _dHr(Ar, Er, Br, Cr, s):
    """H_r'(s) = -C_r^T (s E_r - A_r)^{-1} E_r (s E_r - A_r)^{-1} B_r."""
    K = s * Er - Ar
    x = np.linalg.solve(K, Br[:, 0].astype(np.complex128))
    y = np.linalg.solve(K, Er @ x)
    return -(Cr[:, 0] @ y)


def irka(A, E, B, C, shifts, iters: int, mode: str = "reuse", solver: str = "bicgstab",
         tol: float = 1e-8, maxit: int = 20000, max_chain: Optional[int] = None,
         hermite: bool = False) -> IrkaResult:
    """``iters`` IRKA iterations from the initial ``shifts`` (SISO)."""
    sym = _is_symmetric(A, E)
    sV = ReuseSchedule(A, E, transpose=False, mode=mode, max_chain=max_chain)
    sW = None if sym else ReuseSchedule(A, E, transpose=True, mode=mode, max_chain=max_chain)
    s = sort_shifts(shifts)
    res = IrkaResult([s], None, None, None, None)
    for z in range(1, iters + 1):
        s, rom, its, rr, herm = irka_step(A, E, B, C, s, sV, sW, z, solver=solver, tol=tol,
                                          maxit=maxit, hermite=hermite)
        res.shifts_history.append(s)
        res.Ar, res.Er, res.Br, res.Cr = rom
        res.iters.append(its)
        res.relres.append(rr)
        if herm is not None:
            res.hermite.append(herm)
    res.builds = sV.builds + ([] if sW is None else sW.builds)
    return res


def irka_tangential(A, E, B, C, shifts, btil, ctil, iters: int, mode: str = "reuse",
                    solver: str = "bicgstab", tol: float = 1e-8, maxit: int = 20000,
                    max_chain: Optional[int] = None):
    """``iters`` tangential IRKA iterations (MIMO) from the initial shifts and
    directions.  Returns (IrkaResult, list of per-iteration solved data: the
    shifts solved and the directions used)."""
    sym = _is_symmetric(A, E)
    sV = ReuseSchedule(A, E, transpose=False, mode=mode, max_chain=max_chain)
    sW = None if sym else ReuseSchedule(A, E, transpose=True, mode=mode, max_chain=max_chain)
    s, bt, ct = np.asarray(shifts, dtype=np.complex128), np.asarray(btil), np.asarray(ctil)
    res = IrkaResult([sort_shifts(s)], None, None, None, None)
    used = []
    for z in range(1, iters + 1):
        s, bt, ct, rom, its, rr, solved = irka_step_tangential(A, E, B, C, s, bt, ct, sV, sW, z, solver=solver,
                                                               tol=tol, maxit=maxit)
        res.shifts_history.append(s)
        res.Ar, res.Er, res.Br, res.Cr = rom
        res.iters.append(its)
        res.relres.append(rr)
        used.append(solved)
    res.builds = sV.builds + ([] if sW is None else sW.builds)
    res.btil, res.ctil = bt, ct
    return res, used
