"""Seeded generators of the synthetic first- and second-order systems.

Every function draws from ``numpy.random.default_rng(seed)`` in a fixed,
documented order so that the oracle and the CUDA path see byte-identical
inputs.  Matrices are returned as canonical ``scipy.sparse.csr_matrix``
(sorted column indices, no duplicates, explicit diagonal kept).

First-order systems are ``E x' = A x + B u, y = C^T x``; the shifted
operator of the method is ``sigma E - A``.  Second-order systems are
``M x'' + D x' + K x = F u`` with Rayleigh damping ``D = alpha M + beta K``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.sparse as sp


# --------------------------------------------------------------------------
# containers
# --------------------------------------------------------------------------
@dataclass
class Workload:
    """A first-order system ``E x' = A x + B u, y = C^T x`` plus its shifts.

    ``E`` is ``None`` (identity), a 1-D array (diagonal) or a CSR matrix.
    ``B`` is n x m and ``C`` is n x q, both float64, column-major friendly.
    ``shifts`` is the initial shift set (complex128, closed under
    conjugation, conjugate pairs adjacent with the positive imaginary part
    first).
    """

    name: str
    A: sp.csr_matrix
    E: object
    B: np.ndarray
    C: np.ndarray
    shifts: np.ndarray
    r: int
    irka_iters: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.shape[0]


@dataclass
class SecondOrderWorkload:
    """``M x'' + D x' + K x = F u``, ``y = C^T x``, ``D = alpha M + beta K``.

    ``M`` is stored as its diagonal (1-D array).
    """

    name: str
    K: sp.csr_matrix
    M_diag: np.ndarray
    alpha: float
    beta: float
    F: np.ndarray
    C: np.ndarray
    shifts: np.ndarray
    r: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.K.shape[0]


# --------------------------------------------------------------------------
# stencil matrices
# --------------------------------------------------------------------------
def _tridiag(N: int, lo: float, mid: float, hi: float) -> sp.csr_matrix:
    return sp.diags([np.full(N - 1, lo), np.full(N, mid), np.full(N - 1, hi)],
                    [-1, 0, 1], shape=(N, N), format="csr")


def _canon(M) -> sp.csr_matrix:
    M = sp.csr_matrix(M, dtype=np.float64)
    M.sum_duplicates()
    M.sort_indices()
    return M


def laplacian_2d(N: int, scaled: bool = True) -> sp.csr_matrix:
    """5-point ``-Laplacian`` on an N x N interior grid with Dirichlet
    boundary, grid spacing h = 1/(N+1); entries scaled by 1/h^2 when
    ``scaled`` (diagonal 4/h^2, neighbours -1/h^2).  Row index = i + N*j."""
    T = _tridiag(N, -1.0, 2.0, -1.0)
    I = sp.identity(N, format="csr")
    L = sp.kron(I, T) + sp.kron(T, I)
    if scaled:
        h = 1.0 / (N + 1)
        L = L / (h * h)
    return _canon(L)


def convection_diffusion_3d(N: int, peclet: float = 10.0) -> sp.csr_matrix:
    """7-point ``-Delta_h + w . grad_h`` on an N^3 interior grid, h = 1/(N+1),
    unit diffusion, w = (Pe/sqrt 3)(1,1,1) (global Peclet number Pe on the
    unit cube) and first-order upwind differences for the convective term
    (w > 0 so the backward neighbour is upwind).  Row index = i + N j + N^2 k.
    The returned matrix is the *positive* operator L; the system matrix of
    the workload is A = -L."""
    h = 1.0 / (N + 1)
    wd = peclet / math.sqrt(3.0)
    # 1D diffusion  (-1, 2, -1)/h^2  plus 1D upwind convection  w (u_i - u_{i-1})/h
    T = _tridiag(N, -1.0 / h**2 - wd / h, 2.0 / h**2 + wd / h, -1.0 / h**2)
    I = sp.identity(N, format="csr")
    L = sp.kron(sp.kron(I, I), T) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(T, I), I)
    return _canon(L)


def stencil27_3d(nx: int, ny: int, nz: int) -> sp.csr_matrix:
    """27-point SPD stencil, unscaled: centre 26, each of the 26 neighbours -1,
    Dirichlet truncation at the boundary.  Equal to 27 I - T_z (x) T_y (x) T_x
    with T = tridiag(1, 1, 1), whose eigenvalues lie in (-27, 27), so the
    matrix is SPD.  Row index = i + nx j + nx ny k."""
    Tx = _tridiag(nx, 1.0, 1.0, 1.0)
    Ty = _tridiag(ny, 1.0, 1.0, 1.0)
    Tz = _tridiag(nz, 1.0, 1.0, 1.0)
    n = nx * ny * nz
    K = 27.0 * sp.identity(n, format="csr") - sp.kron(sp.kron(Tz, Ty), Tx)
    return _canon(K)


def csr_arrays(M: sp.csr_matrix):
    """(rowptr int32, col int32, val float64) of a canonical CSR matrix."""
    M = _canon(M)
    return (np.ascontiguousarray(M.indptr, dtype=np.int32),
            np.ascontiguousarray(M.indices, dtype=np.int32),
            np.ascontiguousarray(M.data, dtype=np.float64))


def conj_pairs(a: np.ndarray, ratio: float = 0.5) -> np.ndarray:
    """Shifts a_k (1 +- ratio i), each pair adjacent, positive imaginary first."""
    out = []
    for ak in a:
        out.append(complex(ak, ratio * ak))
        out.append(complex(ak, -ratio * ak))
    return np.asarray(out, dtype=np.complex128)


# --------------------------------------------------------------------------
# the five configurations
# --------------------------------------------------------------------------
def laplace2d_siso(N: int = 100, seed: int = 0) -> Workload:
    """Plain FP64 IRKA, SISO: A = -L2 (5-point Laplacian, N x N grid,
    h = 1/(N+1), scaled), E = I, B, C ~ N(0,1) (drawn in that order),
    r = 6, initial real shifts logspace(1, 4, 6), 20 IRKA iterations."""
    A = _canon(-laplacian_2d(N))
    n = A.shape[0]
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, 1))
    C = rng.standard_normal((n, 1))
    shifts = np.logspace(1, 4, 6).astype(np.complex128)
    return Workload("laplace2d_n%d" % n, A, None, B, C, shifts, r=6,
                    irka_iters=20, meta={"grid": (N, N), "seed": seed})


def convdiff3d_siso(N: int = 100, seed: int = 1) -> Workload:
    """Nonsymmetric 3D convection-diffusion (7-point, Peclet 10, upwind) on
    N^3, A = -L, E = diag(U[0.5, 1.5]); draws B, C ~ N(0,1) then E's
    diagonal.  r = 10 complex shifts: 5 conjugate pairs a_k (1 +- 0.5 i),
    a_k = logspace(1, 4, 5)."""
    A = _canon(-convection_diffusion_3d(N))
    n = A.shape[0]
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, 1))
    C = rng.standard_normal((n, 1))
    Ed = rng.uniform(0.5, 1.5, n)
    shifts = conj_pairs(np.logspace(1, 4, 5))
    return Workload("convdiff3d_n%d" % n, A, Ed, B, C, shifts, r=10,
                    meta={"grid": (N, N, N), "seed": seed, "peclet": 10.0})


def uneven_laplace2d_batch(num_systems: int = 256, n_lo: int = 2000, n_hi: int = 60000,
                           seed: int = 2) -> List[Workload]:
    """256 independent systems.  Draw order: all sizes n_s ~ U{n_lo..n_hi},
    then per system B, C ~ N(0,1) and the diagonal U[0,1].  nx = ceil(sqrt
    n_s); A_s = -(L2(nx x nx, h = 1/(nx+1)) + diag(U[0,1])) restricted to its
    leading n_s x n_s block (a principal submatrix of an SPD matrix, hence
    SPD, so A_s is stable); E = I; 8 real shifts logspace(0, 4, 8)."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(n_lo, n_hi + 1, size=num_systems)
    out = []
    for s, ns in enumerate(sizes):
        ns = int(ns)
        nx = int(math.ceil(math.sqrt(ns)))
        L = laplacian_2d(nx)[:ns, :ns]
        B = rng.standard_normal((ns, 1))
        C = rng.standard_normal((ns, 1))
        d = rng.uniform(0.0, 1.0, ns)
        A = _canon(-(L + sp.diags(d)))
        shifts = np.logspace(0, 4, 8).astype(np.complex128)
        out.append(Workload("uneven_batch_sys%03d_n%d" % (s, ns), A, None, B, C,
                            shifts, r=8, meta={"nx": nx, "seed": seed}))
    return out


def stencil27_second_order(nx: int = 110, ny: int = 110, nz: int = 99, seed: int = 3,
                           m: int = 4) -> SecondOrderWorkload:
    """Second-order structural-like system: K = 27-point SPD stencil on
    nx x ny x nz, M = diag(U[1, 2]), D = 1e-3 M + 1e-4 K.  Draw order:
    F, C ~ N(0,1) (n x m each), then M's diagonal.  Shifts: 6 conjugate
    pairs a_k (1 +- 0.5 i), a_k = logspace(-1, 1, 6); r = 12."""
    K = stencil27_3d(nx, ny, nz)
    n = K.shape[0]
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((n, m))
    C = rng.standard_normal((n, m))
    Md = rng.uniform(1.0, 2.0, n)
    shifts = conj_pairs(np.logspace(-1, 1, 6))
    return SecondOrderWorkload("stencil27_second_order_n%d" % n, K, Md, 1e-3, 1e-4, F, C,
                               shifts, r=12, meta={"grid": (nx, ny, nz), "seed": seed})


def convdiff3d_mimo(N: int = 200, seed: int = 4, m: int = 8) -> Workload:
    """MIMO 3D convection-diffusion on N^3 (the operator of convdiff3d_siso, h = 1/(N+1)),
    E = I, B, C ~ N(0,1) n x m (drawn in that order); the timed sweep is 48
    real shifts logspace(0, 4, 48) times the full m-column block; r = 16."""
    A = _canon(-convection_diffusion_3d(N))
    n = A.shape[0]
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, m))
    C = rng.standard_normal((n, m))
    shifts = np.logspace(0, 4, 48).astype(np.complex128)
    return Workload("convdiff3d_mimo_n%d" % n, A, None, B, C, shifts, r=16,
                    meta={"grid": (N, N, N), "seed": seed})


def random_sparse_system(n: int, density: float, seed: int, e_kind: str = "identity",
                         m: int = 1, q: int = 1, nonsym: bool = True) -> Workload:
    """Small random sparse test system: A = -(dominant diagonal + random
    sparse off-diagonal) so sigma E - A is well conditioned for Re sigma >= 0.
    Draw order: off-diagonal pattern/values, diagonal, E, B, C.
    ``e_kind``: 'identity' | 'diag' | 'csr'."""
    rng = np.random.default_rng(seed)
    R = sp.random(n, n, density=density, random_state=rng, format="csr",
                  data_rvs=lambda k: rng.standard_normal(k))
    if not nonsym:
        R = R + R.T
    R = R - sp.diags(R.diagonal())
    rowsum = np.asarray(abs(R).sum(axis=1)).ravel()
    dg = rowsum + rng.uniform(1.0, 2.0, n)
    A = _canon(-(R + sp.diags(dg)))
    if e_kind == "identity":
        E = None
    elif e_kind == "diag":
        E = rng.uniform(0.5, 1.5, n)
    elif e_kind == "csr":
        S = sp.random(n, n, density=density / 2, random_state=rng, format="csr",
                      data_rvs=lambda k: 0.1 * rng.standard_normal(k))
        S = S - sp.diags(S.diagonal())
        srs = np.asarray(abs(S).sum(axis=1)).ravel()
        E = _canon(S + sp.diags(srs + rng.uniform(1.0, 2.0, n)))
    else:
        raise ValueError(e_kind)
    B = rng.standard_normal((n, m))
    C = rng.standard_normal((n, q))
    shifts = np.array([1.0 + 0.5j, 1.0 - 0.5j, 3.0], dtype=np.complex128)
    return Workload("rand_n%d_s%d" % (n, seed), A, E, B, C, shifts, r=3,
                    meta={"seed": seed, "e_kind": e_kind})
