"""Pins of the multi-moment oracle (repeated solves with one matrix and one
preconditioner per shift, the higher moments of QB-IHOMM in first-order
form): the ROM interpolates the transfer function and its derivatives at
every shift, as many as rational Krylov moment matching gives (J - 1
one-sided, 2J - 1 two-sided), checked against derivatives of the full H
computed by their closed form H^(k)(s) = (-1)^k k! C^T [(sE - A)^{-1} E]^k
(sE - A)^{-1} B; one moment fewer leaves the last derivative unmatched."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import moments, operator as op


def _derivs(A, E, B, C, s, K):
    """H(s), H'(s), ..., H^(K)(s) (dense)."""
    n = A.shape[0]
    Ad = A.toarray() if hasattr(A, "toarray") else A
    Em = op.E_matrix(E, n)
    Ed = Em.toarray() if hasattr(Em, "toarray") else Em
    M = s * Ed - Ad
    X = np.linalg.solve(M, B.astype(complex))
    out = [C.T @ X]
    for k in range(1, K + 1):
        X = np.linalg.solve(M, Ed @ X)
        out.append(((-1) ** k) * math.factorial(k) * (C.T @ X))
    return out


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(a)


def _check(wl, shifts, J, unmatched_floor):
    for two_sided, nmatch in ((False, J), (True, 2 * J)):
        Ar, Er, Br, Cr = moments.multi_moment_rom(wl.A, wl.E, wl.B, wl.C, shifts, J, two_sided=two_sided)
        worst_unmatched = 0.0
        for s in list(shifts) + [np.conj(shifts[0])]:
            full = _derivs(wl.A, wl.E, wl.B, wl.C, s, nmatch)
            red = _derivs(Ar, Er, Br, Cr, s, nmatch)
            for k in range(nmatch):
                assert _rel(full[k], red[k]) <= 1e-12, (two_sided, s, k)
            worst_unmatched = max(worst_unmatched, _rel(full[nmatch], red[nmatch]))
        # the next derivative is not matched, so the bar above can fail
        assert worst_unmatched > unmatched_floor, (two_sided, nmatch, worst_unmatched)


@pytest.mark.parametrize("J", [1, 2, 3])
def test_derivative_matching_convection_diffusion(J):
    """n = 343, E diagonal, SISO: matched derivatives agree to <= 3e-15
    (bar 1e-12); the first unmatched one differs by >= 2e-11 (floor 2e-12)."""
    _check(W.convdiff3d_siso(N=7), np.array([20.0 + 5.0j, 200.0]), J, 2e-12)


@pytest.mark.parametrize("e_kind", ["identity", "csr"])
@pytest.mark.parametrize("J", [1, 2])
def test_derivative_matching_mimo_e_kinds(e_kind, J):
    """n = 300, m = q = 2, identity and general sparse E (these strongly
    diagonal systems have smooth transfer functions: the first unmatched
    derivative differs by >= 5e-8, floor 1e-9)."""
    wl = W.random_sparse_system(300, 0.02, seed=21, e_kind=e_kind, m=2, q=2)
    _check(wl, np.array([1.0 + 0.5j, 4.0]), J, 1e-9)


def test_moment_blocks_iterative_match_dense():
    """BiCGSTAB with one SPAI reused for every moment block of a shift
    reproduces the dense blocks (relative to each block) to 1e-6."""
    wl = W.convdiff3d_siso(N=8)
    for s in (20.0 + 5.0j, 60.0):
        d = moments.moment_blocks(wl.A, wl.E, wl.B, s, 3, solver="dense")
        i = moments.moment_blocks(wl.A, wl.E, wl.B, s, 3, solver="bicgstab", tol=1e-10)
        for a, b in zip(d, i):
            assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)
        dT = moments.moment_blocks(wl.A, wl.E, wl.C, s, 2, transpose=True, solver="dense")
        iT = moments.moment_blocks(wl.A, wl.E, wl.C, s, 2, transpose=True, solver="bicgstab", tol=1e-10)
        for a, b in zip(dT, iT):
            assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)
