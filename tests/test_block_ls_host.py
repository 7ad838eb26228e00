"""The host side of the GPU block GMRES (csrc/block_ls.h: the incremental
Householder least-squares solve of the block Hessenberg system, the block
Cholesky factor, the triangular inverse, and the rank-revealing block
orthonormalisation by pivoted Cholesky of the Gram matrix) compiled with g++
and checked against LAPACK through NumPy: after every block step of random
complex block Hessenberg systems, the least-squares residual of each
right-hand side and the solution Y equal numpy.linalg.lstsq's; R^H R = G and
R R^{-1} = I; for blocks of known rank, V = W C is orthonormal on the rank
and zero beyond it, and W = V F.  No GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2003_12759_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "block_ls.h"
typedef std::complex<double> cx;
static std::vector<cx> read(int n) {
  std::vector<cx> v(n);
  for (auto& z : v) { double a, b; if (scanf("%lf %lf", &a, &b) != 2) throw 1; z = cx(a, b); }
  return v;
}
int main() {
  int p, m;
  if (scanf("%d %d", &p, &m) != 2) return 1;
  std::vector<cx> R0 = read(p * p);
  BlockLS ls;
  ls.reset(p, m, R0.data());
  for (int j = 0; j < m; ++j) {
    std::vector<cx> hcol = read((j + 2) * p * p);
    ls.add_block(hcol.data());
    for (int b = 0; b < p; ++b) printf("%.17g ", ls.resnorm(b));
    printf("\n");
    std::vector<cx> Y((size_t)(j + 1) * p * p);
    ls.solve(Y.data());
    for (auto z : Y) printf("%.17g %.17g ", z.real(), z.imag());
    printf("\n");
  }
  std::vector<cx> G = read(p * p), R(p * p), Ri(p * p);
  int rank = block_cholesky(p, G.data(), R.data(), 1e-14);
  printf("%d\n", rank);
  block_triu_inverse(p, R.data(), Ri.data());
  for (auto z : R) printf("%.17g %.17g ", z.real(), z.imag());
  printf("\n");
  for (auto z : Ri) printf("%.17g %.17g ", z.real(), z.imag());
  printf("\n");
  // rank-revealing block orthonormalisation of a Gram matrix that follows
  int q;
  if (scanf("%d", &q) != 1) return 0;
  std::vector<cx> G2 = read(q * q), Cf(q * q), Ff(q * q);
  double tol;
  if (scanf("%lf", &tol) != 1) return 1;
  int r = block_orth_factor(q, G2.data(), tol, Cf.data(), Ff.data());
  printf("%d\n", r);
  for (auto z : Cf) printf("%.17g %.17g ", z.real(), z.imag());
  printf("\n");
  for (auto z : Ff) printf("%.17g %.17g ", z.real(), z.imag());
  printf("\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("block_ls")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def _fmt(a):
    a = np.asarray(a, dtype=complex).ravel(order="F")
    return " ".join("%.17g %.17g" % (z.real, z.imag) for z in a)


@pytest.mark.parametrize("p,m,seed", [(1, 6, 0), (3, 5, 1), (4, 7, 2), (8, 3, 3)])
def test_block_least_squares_matches_lstsq(harness, p, m, seed):
    rng = np.random.default_rng(seed)
    cr = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)   # noqa: E731
    R0 = np.triu(cr(p, p))
    Hbar = np.zeros(((m + 1) * p, m * p), dtype=complex)
    for j in range(m):
        Hbar[: (j + 1) * p, j * p:(j + 1) * p] = cr((j + 1) * p, p)
        Hbar[(j + 1) * p:(j + 2) * p, j * p:(j + 1) * p] = np.triu(cr(p, p))
    G = cr(p, p)
    G = G.conj().T @ G + 0.1 * np.eye(p)
    inp = "%d %d\n%s\n" % (p, m, _fmt(R0))
    for j in range(m):
        inp += _fmt(Hbar[: (j + 2) * p, j * p:(j + 1) * p]) + "\n"
    inp += _fmt(G) + "\n"
    out = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    E1R0 = np.zeros(((m + 1) * p, p), dtype=complex)
    E1R0[:p] = R0
    for k in range(1, m + 1):
        res = np.array([float(x) for x in out[2 * (k - 1)].split()])
        vals = np.array([float(x) for x in out[2 * (k - 1) + 1].split()])
        Y = (vals[0::2] + 1j * vals[1::2]).reshape((k * p, p), order="F")
        Hk = Hbar[: (k + 1) * p, : k * p]
        rhs = E1R0[: (k + 1) * p]
        Yref = np.linalg.lstsq(Hk, rhs, rcond=None)[0]
        rref = np.linalg.norm(rhs - Hk @ Yref, axis=0)
        np.testing.assert_allclose(res, rref, rtol=1e-9, atol=1e-12 * np.linalg.norm(R0))
        np.testing.assert_allclose(Y, Yref, rtol=1e-8, atol=1e-10 * np.abs(Yref).max())
    rank = int(out[2 * m])
    assert rank == p
    v = np.array([float(x) for x in out[2 * m + 1].split()])
    R = (v[0::2] + 1j * v[1::2]).reshape((p, p), order="F")
    v = np.array([float(x) for x in out[2 * m + 2].split()])
    Ri = (v[0::2] + 1j * v[1::2]).reshape((p, p), order="F")
    assert np.allclose(np.tril(R, -1), 0)
    np.testing.assert_allclose(R.conj().T @ R, G, rtol=1e-12, atol=1e-12 * np.abs(G).max())
    np.testing.assert_allclose(R @ Ri, np.eye(p), atol=1e-10)


def test_block_cholesky_reports_rank_deficiency(harness):
    """A Gram matrix of dependent columns stops the factor at its rank."""
    p = 3
    rng = np.random.default_rng(7)
    X = rng.standard_normal((20, 2)) + 1j * rng.standard_normal((20, 2))
    X = np.column_stack([X, X[:, 0] + 2 * X[:, 1]])       # third column dependent
    G = X.conj().T @ X
    inp = "%d %d\n%s\n%s\n%s\n" % (p, 1, _fmt(np.eye(p)), _fmt(np.vstack([np.eye(p), np.eye(p)])), _fmt(G))
    out = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    assert int(out[2]) == 2


def _run_orth(harness, W, tol):
    p = W.shape[1]
    G = W.conj().T @ W
    inp = "%d %d\n%s\n%s\n%s\n%d\n%s\n%.17g\n" % (1, 1, _fmt(np.eye(1)), _fmt(np.ones((2, 1))), _fmt(np.eye(1)),
                                                   p, _fmt(G), tol)
    out = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    r = int(out[5])
    v = np.array([float(x) for x in out[6].split()])
    Cm = (v[0::2] + 1j * v[1::2]).reshape((p, p), order="F")
    v = np.array([float(x) for x in out[7].split()])
    Fm = (v[0::2] + 1j * v[1::2]).reshape((p, p), order="F")
    return r, Cm, Fm


@pytest.mark.parametrize("p,rank,seed", [(4, 4, 0), (6, 4, 1), (8, 5, 2), (3, 1, 3)])
def test_block_orth_factor_rank_revealing(harness, p, rank, seed):
    """V = W C has r orthonormal columns and p - r zero ones, W = V F, and r
    is the numerical rank of W (dependent columns are deflated; the pivot
    tolerance 1e-12 of the largest Gram diagonal sits above the rounding of
    the Gram matrix, ~1e-16)."""
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((40, rank)) + 1j * rng.standard_normal((40, rank))
    W = B @ (rng.standard_normal((rank, p)) + 1j * rng.standard_normal((rank, p)))
    r, Cm, Fm = _run_orth(harness, W, 1e-12)
    assert r == rank
    V = W @ Cm
    np.testing.assert_allclose(V[:, :r].conj().T @ V[:, :r], np.eye(r), atol=1e-10)
    assert np.abs(V[:, r:]).max(initial=0.0) == 0.0
    np.testing.assert_allclose(V @ Fm, W, atol=1e-9 * np.abs(W).max())
    assert np.abs(Fm[r:]).max(initial=0.0) == 0.0
