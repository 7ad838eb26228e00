"""The small dense FP64 routines the GPU runs with one thread per problem
(csrc/small_eig.cuh: reduced poles by Hessenberg + Francis double-shift QR;
csrc/small_tangent.cuh: tangential directions by inverse iteration) are
plain host/device C++: compiled here for the host with g++ and checked
against LAPACK (scipy) and the oracle's directions.  No GPU needed."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import irka

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2003_12759_gb300", "csrc")

HARNESS = r"""
#define __host__
#define __device__
#include <cstdio>
#include <vector>
#include "small_eig.cuh"
#include "small_tangent.cuh"
int main() {
  int r, m, q;
  if (scanf("%d %d %d", &r, &m, &q) != 3) return 1;
  std::vector<double> A(r * r), E(r * r), B(r * m), C(r * q), M(r * r), LU(r * r), F(r * m);
  for (auto* v : {&A, &E, &B, &C}) for (double& x : *v) if (scanf("%lf", &x) != 1) return 1;
  std::vector<double> wr(r), wi(r), sr(r), si(r);
  std::vector<int> piv(r);
  int st = small_eig(r, A.data(), E.data(), M.data(), LU.data(), piv.data(), wr.data(), wi.data());
  if (st == 0) mirror_sort(r, wr.data(), wi.data(), sr.data(), si.data());
  printf("%d\n", st);
  for (int i = 0; i < r; ++i) printf("%.17g %.17g %.17g %.17g\n", wr[i], wi[i], sr[i], si[i]);
  if (tangent_prepare(r, m, A.data(), E.data(), B.data(), M.data(), F.data(), LU.data(), piv.data())) return 2;
  std::vector<tz> K(r * r), x(r), y(r), bt(m), ct(q);
  for (int i = 0; i < r; ++i) {
    tangent_dirs(r, m, q, M.data(), F.data(), C.data(), tz_c(wr[i], wi[i]), K.data(), piv.data(), x.data(), y.data(),
                 bt.data(), ct.data());
    for (int j = 0; j < m; ++j) printf("%.17g %.17g ", bt[j].re, bt[j].im);
    for (int j = 0; j < q; ++j) printf("%.17g %.17g ", ct[j].re, ct[j].im);
    printf("\n");
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("small_dense")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def _run(exe, Ar, Er, Br, Cr):
    r, m, q = Ar.shape[0], Br.shape[1], Cr.shape[1]
    data = "%d %d %d\n" % (r, m, q) + " ".join("%.17g" % v for M in (Ar, Er, Br, Cr) for v in M.ravel(order="F"))
    out = subprocess.run([exe], input=data, capture_output=True, text=True, check=True).stdout.split("\n")
    assert int(out[0]) == 0
    ev = np.array([[float(t) for t in out[1 + i].split()] for i in range(r)])
    lam = ev[:, 0] + 1j * ev[:, 1]
    sig = ev[:, 2] + 1j * ev[:, 3]
    dirs = np.array([[float(t) for t in out[1 + r + i].split()] for i in range(r)])
    z = dirs[:, 0::2] + 1j * dirs[:, 1::2]
    return lam, sig, z[:, :m], z[:, m:]


def _pencil(rng, r, m, q, stable=True):
    X = rng.standard_normal((r, r))
    D = -rng.uniform(0.5, 20.0, r) if stable else rng.standard_normal(r) * 5
    Er = np.eye(r) + 0.2 * rng.standard_normal((r, r))
    Ar = Er @ X @ np.diag(D) @ np.linalg.inv(X) + 0.3 * rng.standard_normal((r, r))   # complex pairs too
    return Ar, Er, rng.standard_normal((r, m)), rng.standard_normal((r, q))


@pytest.mark.parametrize("seed,r", [(1, 4), (2, 7), (3, 12), (4, 16), (5, 31)])
def test_poles_and_mirrored_shifts_match_lapack(harness, seed, r):
    rng = np.random.default_rng(seed)
    Ar, Er, Br, Cr = _pencil(rng, r, 2, 3, stable=(seed % 2 == 1))
    lam, sig, _, _ = _run(harness, Ar, Er, Br, Cr)
    ref = irka.reduced_poles(Ar, Er)
    scale = np.max(np.abs(ref))
    # same multiset of eigenvalues
    for z in ref:
        assert np.min(np.abs(lam - z)) <= 1e-10 * scale
    np.testing.assert_allclose(sig, irka.mirror_shifts(ref), rtol=0, atol=1e-10 * scale)


@pytest.mark.parametrize("seed,r,m,q", [(6, 5, 3, 2), (7, 9, 1, 1), (8, 14, 4, 4), (9, 20, 8, 8)])
def test_tangential_directions_match_oracle(harness, seed, r, m, q):
    """The residues c_i b_i^T (independent of the eigenvector scale) of each
    pole agree with the oracle's LAPACK eigenvectors, and they rebuild H_r."""
    rng = np.random.default_rng(seed)
    Ar, Er, Br, Cr = _pencil(rng, r, m, q)
    lam, _, bt, ct = _run(harness, Ar, Er, Br, Cr)
    lo, bo, co = irka.tangential_directions(Ar, Er, Br, Cr)
    for i in range(r):
        j = int(np.argmin(np.abs(lo - lam[i])))
        Ri = np.outer(ct[i], bt[i])
        Ro = np.outer(co[j], bo[j])
        assert np.linalg.norm(Ri - Ro) <= 1e-7 * np.linalg.norm(Ro), i
    s = 0.3 + 1.7j
    Hr = Cr.T @ np.linalg.solve(s * Er - Ar, Br)
    Hres = sum(np.outer(ct[i], bt[i]) / (s - lam[i]) for i in range(r))
    np.testing.assert_allclose(Hres, Hr, rtol=1e-7, atol=1e-9 * np.linalg.norm(Hr))


QEP_HARNESS = r"""
#define __host__
#define __device__
#include <cstdio>
#include <vector>
#include "small_qep.cuh"
int main() {
  int r, count;
  double alpha, beta;
  if (scanf("%d %d %lf %lf", &r, &count, &alpha, &beta) != 4) return 1;
  std::vector<double> M(r * r), K(r * r);
  for (double& x : M) if (scanf("%lf", &x) != 1) return 1;
  for (double& x : K) if (scanf("%lf", &x) != 1) return 1;
  const int n2 = 2 * r;
  std::vector<double> A2(n2 * n2), E2(n2 * n2), W1(n2 * n2), W2(n2 * n2), wr(n2), wi(n2), pr(count), pi(count), w(3 * n2);
  std::vector<int> piv(n2);
  qep_pencil(r, M.data(), K.data(), alpha, beta, A2.data(), E2.data());
  int st = small_eig(n2, A2.data(), E2.data(), W1.data(), W2.data(), piv.data(), wr.data(), wi.data());
  printf("%d\n", st);
  for (int i = 0; i < n2; ++i) printf("%.17g %.17g\n", wr[i], wi[i]);
  int s2 = qep_select(n2, wr.data(), wi.data(), count, pr.data(), pi.data(), w.data());
  printf("%d\n", s2);
  for (int i = 0; i < count; ++i) printf("%.17g %.17g\n", pr[i], pi[i]);
  return 0;
}
"""


@pytest.fixture(scope="module")
def qep_harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("small_qep")
    src = d / "q.cpp"
    src.write_text(QEP_HARNESS)
    exe = d / "q"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


@pytest.mark.parametrize("seed,r,count", [(1, 3, 3), (2, 6, 3), (3, 12, 3), (4, 12, 4), (5, 20, 5)])
def test_qep_poles_and_point_update_match_oracle(qep_harness, seed, r, count):
    from oracle import airga
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((r, r))
    Mr = X @ X.T + r * np.eye(r)
    Y = rng.standard_normal((r, r))
    Kr = Y @ Y.T + 0.1 * np.eye(r)
    alpha, beta = 1e-3 * (1 + seed), 1e-4 * seed
    data = "%d %d %.17g %.17g\n" % (r, count, alpha, beta) + " ".join(
        "%.17g" % v for A in (Mr, Kr) for v in A.ravel(order="F"))
    out = subprocess.run([qep_harness], input=data, capture_output=True, text=True, check=True).stdout.split("\n")
    assert int(out[0]) == 0
    lam = np.array([complex(*map(float, out[1 + i].split())) for i in range(2 * r)])
    ref = airga.qep_eigenvalues(Mr, alpha * Mr + beta * Kr, Kr)
    for z in ref:
        assert np.min(np.abs(lam - z)) <= 1e-9 * abs(z)
    assert int(out[1 + 2 * r]) == 0
    pts = np.array([complex(*map(float, out[2 + 2 * r + i].split())) for i in range(count)])
    np.testing.assert_allclose(pts, airga.select_points(ref, count), rtol=1e-9)
