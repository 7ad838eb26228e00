"""Right-preconditioned Krylov solvers and a dense direct solve (oracle).

Test infrastructure only; shares no code with the CUDA library.

Sec. III.A: the preconditioned system is A P y = b with x = P y (right
preconditioning), so the residual the iteration tracks is the true residual
of the unpreconditioned system.  Sec. IV uses GMRES (tolerance 1e-6); this
library's default solver is BiCGSTAB (van der Vorst 1992) with the relative
residual target 1e-8.  Both start from x_0 = 0.

Readings fixed here (the paper does not state them):
  * inner products are Hermitian (x^H y) for complex shifts;
  * convergence is tested on the recursively updated residual after each
    full BiCGSTAB iteration, ||r|| <= tol ||b||; on exit the true residual
    b - A x is recomputed, and if it still exceeds tol ||b|| the iteration
    restarts from the current x (r = r_hat = b - A x);
  * a zero rho, r_hat^H v or t^H t is a breakdown and also triggers a
    restart; after 3 restarts the status is BREAKDOWN;
  * GMRES(m): Arnoldi with modified Gram-Schmidt and Givens rotations,
    restart length m = 50.
"""
from __future__ import annotations

import numpy as np

STATUS_OK = 0
STATUS_NOCONV = 4
STATUS_BREAKDOWN = 5


def _vdot(a, b):
    return np.vdot(a, b)  # conjugates the first argument


def bicgstab(apply_A, apply_P, b, tol=1e-8, maxit=10000, max_restarts=3):
    """Right-preconditioned BiCGSTAB for A x = b (A P y = b, x = P y).

    ``apply_P`` may be None (no preconditioner).  Returns
    (x, iterations, true relative residual, status).

    Parity: pinned against dense LU solutions and independently recomputed
    residuals (tests/test_oracle_krylov.py)."""
    if apply_P is None:
        apply_P = lambda v: v  # noqa: E731
    dtype = np.result_type(b.dtype, np.float64)
    b = b.astype(dtype)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    if bnorm == 0.0:
        return x, 0, 0.0, STATUS_OK
    r = b.copy()
    it = 0
    restarts = 0
    while True:
        rhat = r.copy()
        rho_old = alpha = omega = 1.0
        v = np.zeros_like(b)
        p = np.zeros_like(b)
        broke = False
        converged = False
        while it < maxit:
            rho = _vdot(rhat, r)
            if rho == 0.0:
                broke = True
                break
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
            phat = apply_P(p)
            v = apply_A(phat)
            rv = _vdot(rhat, v)
            if rv == 0.0:
                broke = True
                break
            alpha = rho / rv
            s = r - alpha * v
            shat = apply_P(s)
            t = apply_A(shat)
            tt = _vdot(t, t).real
            if tt == 0.0:
                broke = True
                break
            omega = _vdot(t, s) / tt
            x = x + alpha * phat + omega * shat
            r = s - omega * t
            rho_old = rho
            it += 1
            if np.linalg.norm(r) <= tol * bnorm:
                converged = True
                break
        rt = b - apply_A(x)
        relres = np.linalg.norm(rt) / bnorm
        if relres <= tol:
            return x, it, relres, STATUS_OK
        if it >= maxit:
            return x, it, relres, STATUS_NOCONV
        if broke or converged:
            restarts += 1
            if restarts > max_restarts:
                return x, it, relres, STATUS_BREAKDOWN if broke else STATUS_NOCONV
            r = rt
            continue


def gmres(apply_A, apply_P, b, tol=1e-8, m=50, maxit=10000):
    """Restarted right-preconditioned GMRES(m) (Saad 2003, Sec. 9.3.2):
    Arnoldi on A P with modified Gram-Schmidt, least-squares by Givens
    rotations, x = x_0 + P V_k y_k at each restart.  Returns
    (x, iterations, true relative residual, status).

    Parity: pinned against dense LU (tests/test_oracle_krylov.py)."""
    if apply_P is None:
        apply_P = lambda v: v  # noqa: E731
    dtype = np.result_type(b.dtype, np.float64)
    b = b.astype(dtype)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    if bnorm == 0.0:
        return x, 0, 0.0, STATUS_OK
    it = 0
    n = b.shape[0]
    while it < maxit:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            break
        V = np.zeros((n, m + 1), dtype=dtype)
        H = np.zeros((m + 1, m), dtype=dtype)
        cs = np.zeros(m, dtype=dtype)
        sn = np.zeros(m, dtype=dtype)
        g = np.zeros(m + 1, dtype=dtype)
        g[0] = beta
        V[:, 0] = r / beta
        k = 0
        for j in range(m):
            w = apply_A(apply_P(V[:, j]))
            for i in range(j + 1):                 # modified Gram-Schmidt
                H[i, j] = _vdot(V[:, i], w)
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[:, j + 1] = w / H[j + 1, j]
            for i in range(j):                     # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, c = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            if den == 0.0:
                cs[j], sn[j] = 1.0, 0.0
            else:
                if a == 0.0:
                    cs[j], sn[j] = 0.0, 1.0
                else:
                    cs[j] = abs(a) / den
                    sn[j] = (a / abs(a)) * np.conj(c) / den
            H[j, j] = cs[j] * a + sn[j] * c
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            it += 1
            if abs(g[j + 1]) <= tol * bnorm or it >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + apply_P(V[:, :k] @ y)
    rt = b - apply_A(x)
    relres = np.linalg.norm(rt) / bnorm
    return x, it, relres, (STATUS_OK if relres <= tol else STATUS_NOCONV)


def block_gmres(apply_A, apply_P, B, tol=1e-8, m=50, maxit=10000):
    """Restarted right-preconditioned block GMRES(m) for A X = B with p
    right-hand sides (Saad 2003, Sec. 6.12: block Arnoldi and block GMRES;
    right preconditioning as in Sec. 9.3.2): one block Krylov space
    span{R_0, (AP) R_0, ..., (AP)^{j-1} R_0} serves all p columns.  Block
    Arnoldi by block modified Gram-Schmidt (two passes) and a QR of each new
    block; the block least-squares problem min ||E_1 R_0' - Hbar_j Y||_F
    (R_0 = V_1 R_0') is solved by numpy's lstsq, and the iteration stops when
    every column's residual in it is below tol ||b_c||.  At a restart
    X = X_0 + P [V_1 ... V_j] Y.  Returns (X, block iterations, true relative
    residual per column, status).

    Parity: pinned against dense LU, against gmres for p = 1, by the block
    space containing every column's own Krylov space (no more block
    iterations than the slowest column's GMRES) and by termination within
    ceil(n / p) block steps (tests/test_oracle_krylov.py)."""
    if apply_P is None:
        apply_P = lambda v: v  # noqa: E731
    B = np.atleast_2d(B.T).T if B.ndim == 1 else B
    dtype = np.result_type(B.dtype, np.float64)
    B = B.astype(dtype)
    n, p = B.shape
    bn = np.linalg.norm(B, axis=0)
    X = np.zeros_like(B)
    it = 0
    while it < maxit:
        R = B - apply_A(X)
        if np.all(np.linalg.norm(R, axis=0) <= tol * bn):
            break
        Q, R0 = np.linalg.qr(R)
        V = [Q]
        Hbar = np.zeros(((m + 1) * p, m * p), dtype=dtype)
        G = np.zeros(((m + 1) * p, p), dtype=dtype)
        G[:p] = R0
        Y = None
        k = 0
        for j in range(m):
            W = apply_A(apply_P(V[j]))
            for _ in range(2):                             # block MGS, two passes
                for i in range(j + 1):
                    Hij = V[i].conj().T @ W
                    Hbar[i * p:(i + 1) * p, j * p:(j + 1) * p] += Hij
                    W = W - V[i] @ Hij
            Qj, Rj = np.linalg.qr(W)
            Hbar[(j + 1) * p:(j + 2) * p, j * p:(j + 1) * p] = Rj
            V.append(Qj)
            k = j + 1
            it += 1
            Hk = Hbar[:(k + 1) * p, :k * p]
            Y = np.linalg.lstsq(Hk, G[:(k + 1) * p], rcond=None)[0]
            res = np.linalg.norm(G[:(k + 1) * p] - Hk @ Y, axis=0)
            if np.all(res <= tol * bn) or it >= maxit:
                break
        X = X + apply_P(np.hstack(V[:k]) @ Y)
    rel = np.linalg.norm(B - apply_A(X), axis=0) / np.where(bn > 0, bn, 1.0)
    return X, it, rel, (STATUS_OK if np.all(rel <= tol) else STATUS_NOCONV)


def dense_solve(M_sparse, b):
    """Exact reference: dense LU with partial pivoting (numpy.linalg.solve)."""
    Md = M_sparse.toarray()
    return np.linalg.solve(Md, b.astype(np.result_type(Md.dtype, b.dtype)))
