"""GPU parity of the moment blocks with one matrix and one preconditioner per
shift (mor_moment_blocks; the higher moments of QB-IHOMM in first-order
form) against the oracle, through the C ABI:

  * every block X_j(s_i) = A(s_i)^{-1} E X_{j-1}(s_i) against the oracle's
    dense-LU blocks, relative to the block, at 1e-6 (the same bar as the
    oracle's own iterative-vs-dense pin; 1e-8 true relative residuals, and
    the conditioning of these small shifted systems is below 1e2), for the
    primal (B) and transposed (C) sequences, identity, diagonal and general
    sparse E, FP64 and mixed precision, fresh SPAI per shift and the chain;
  * the ROM projected on the real spans of the GPU's blocks (GPU
    Gram-Schmidt and projection) interpolates H and its first J - 1
    derivatives at every shift (one-sided) or 2J - 1 (two-sided), against
    the closed-form derivatives (-1)^k k! C^T [(sE - A)^{-1} E]^k (sE -
    A)^{-1} B of the full system, at 1e-6.
"""
import math

import numpy as np
import pytest

import paper_2003_12759_gb300 as mor
import workloads as W
from oracle import moments as omom, operator as oop

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    mor.load_library()
    hh = mor.mor_create(0)
    yield hh
    mor.mor_destroy(hh)


def _set(h, wl):
    if wl.E is None:
        mor.mor_set_system(h, wl.A, wl.B, wl.C)
    elif isinstance(wl.E, np.ndarray):
        mor.mor_set_system(h, wl.A, wl.B, wl.C, E_diag=wl.E)
    else:
        mor.mor_set_system(h, wl.A, wl.B, wl.C, E=wl.E)


SYSTEMS = {
    "convdiff_diagE": lambda: W.convdiff3d_siso(N=8),
    "rand_identityE_mimo": lambda: W.random_sparse_system(300, 0.02, seed=21, e_kind="identity", m=2, q=2),
    "rand_csrE_mimo": lambda: W.random_sparse_system(300, 0.02, seed=21, e_kind="csr", m=2, q=2),
}
SHIFTS = {
    "convdiff_diagE": np.array([20.0 + 5.0j, 200.0]),
    "rand_identityE_mimo": np.array([1.0 + 0.5j, 4.0]),
    "rand_csrE_mimo": np.array([1.0 + 0.5j, 4.0]),
}


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("precision,precond", [(mor.MOR_FP64, 1), (mor.MOR_MIXED, 1), (mor.MOR_MIXED, 0)])
def test_moment_blocks_match_dense_oracle(h, name, precision, precond):
    wl = SYSTEMS[name]()
    _set(h, wl)
    shifts = SHIFTS[name]
    J = 3
    opts = mor.mor_default_opts(precision=precision, precond=precond)
    for transpose, R in ((0, wl.B), (1, wl.C)):
        blocks, stats, code = mor.mor_moment_blocks(h, shifts, J, transpose=transpose, opts=opts)
        assert code == mor.MOR_OK
        assert all(x["relres"] <= 1.001e-8 for x in stats)
        for i, s in enumerate(shifts):
            ref = omom.moment_blocks(wl.A, wl.E, R, s, J, transpose=bool(transpose), solver="dense")
            for j in range(J):
                a, b = ref[j], blocks[i][j]
                assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a), (name, transpose, i, j)


def _derivs(A, E, B, C, s, K):
    n = A.shape[0]
    Ad = A.toarray() if hasattr(A, "toarray") else A
    Em = oop.E_matrix(E, n)
    Ed = Em.toarray() if hasattr(Em, "toarray") else Em
    M = s * Ed - Ad
    X = np.linalg.solve(M, B.astype(complex))
    out = [C.T @ X]
    for k in range(1, K + 1):
        X = np.linalg.solve(M, Ed @ X)
        out.append(((-1) ** k) * math.factorial(k) * (C.T @ X))
    return out


def _real_span(blocks, shifts):
    cols = []
    for bl, s in zip(blocks, shifts):
        for X in bl:
            cols.append(X.real)
            if s.imag != 0:
                cols.append(X.imag)
    return np.concatenate(cols, axis=1)


@pytest.mark.parametrize("name", ["convdiff_diagE", "rand_csrE_mimo"])
@pytest.mark.parametrize("J", [1, 2])
def test_moment_rom_matches_derivatives(h, name, J):
    wl = SYSTEMS[name]()
    _set(h, wl)
    shifts = SHIFTS[name]
    opts = mor.mor_default_opts(precision=mor.MOR_MIXED, precond=0)
    Xb, _, _ = mor.mor_moment_blocks(h, shifts, J, transpose=0, opts=opts)
    Yb, _, _ = mor.mor_moment_blocks(h, shifts, J, transpose=1, opts=opts)
    V = mor.mor_orthonormalize(h, _real_span(Xb, shifts))
    W_ = mor.mor_orthonormalize(h, _real_span(Yb, shifts))
    for two_sided, nmatch in ((False, J), (True, 2 * J)):
        rom = mor.mor_project(h, V, W_ if two_sided else V)
        Ar, Er, Br, Cr = rom.arrays()
        for s in list(shifts) + [np.conj(shifts[0])]:
            full = _derivs(wl.A, wl.E, wl.B, wl.C, s, nmatch - 1)
            red = _derivs(Ar, Er, Br, Cr, s, nmatch - 1)
            for k in range(nmatch):
                rel = np.linalg.norm(full[k] - red[k]) / np.linalg.norm(full[k])
                assert rel <= 1e-6, (name, J, two_sided, s, k, rel)


def test_moment_blocks_argument_errors(h):
    wl = W.stencil27_second_order(nx=4, ny=4, nz=4, m=1)
    mor.mor_set_system_2nd(h, wl.K, wl.M_diag, wl.alpha, wl.beta, wl.F, wl.C)
    with pytest.raises(RuntimeError):            # second-order system
        mor.mor_moment_blocks(h, [1.0], 2)
    wl = SYSTEMS["convdiff_diagE"]()
    _set(h, wl)
    with pytest.raises(RuntimeError):            # J = 0
        mor.mor_moment_blocks(h, [1.0], 0)
