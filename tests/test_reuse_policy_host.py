"""The reuse-or-rebuild decision of the library's schedule
(csrc/reuse_policy.h: the paper's Frobenius ratios in closed form from a few
scalar products of the stored matrices) is plain host C++: compiled here
with g++ and checked against the oracle, which forms every shifted matrix
and takes its norms directly (oracle.spai.frobenius_ratios and the schedule's
reuse_ok).  First order with identity, diagonal and general sparse E, and
second order with Rayleigh damping.  No GPU needed."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import irka, airga, spai as ospai, operator as op

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2003_12759_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "reuse_policy.h"
static bool read_csr(long n, std::vector<int32_t>& rp, std::vector<int32_t>& col, std::vector<double>& val) {
  long nnz;
  if (scanf("%ld", &nnz) != 1) return false;
  rp.resize(n + 1); col.resize(nnz); val.resize(nnz);
  for (auto& x : rp) if (scanf("%d", &x) != 1) return false;
  for (auto& x : col) if (scanf("%d", &x) != 1) return false;
  for (auto& x : val) if (scanf("%lf", &x) != 1) return false;
  return true;
}
int main() {
  int order, pkind, npairs;
  long n;
  double alpha, beta;
  if (scanf("%d %lf %lf %ld %d", &order, &alpha, &beta, &n, &pkind) != 5) return 1;
  std::vector<int32_t> qrp, qcol, prp, pcol;
  std::vector<double> qval, pval, pdiag;
  if (!read_csr(n, qrp, qcol, qval)) return 1;
  if (pkind == 1) { pdiag.resize(n); for (auto& x : pdiag) if (scanf("%lf", &x) != 1) return 1; }
  if (pkind == 2 && !read_csr(n, prp, pcol, pval)) return 1;
  FrobScalars f = frob_scalars(order, alpha, beta, n, pkind == 1 ? pdiag.data() : nullptr,
                               pkind == 2 ? prp.data() : nullptr, pkind == 2 ? pcol.data() : nullptr,
                               pkind == 2 ? pval.data() : nullptr, qrp.data(), qcol.data(), qval.data());
  if (scanf("%d", &npairs) != 1) return 1;
  for (int i = 0; i < npairs; ++i) {
    frob_z a, b;
    if (scanf("%lf %lf %lf %lf", &a.re, &a.im, &b.re, &b.im) != 4) return 1;
    printf("%.17g %.17g %d\n", frob_ratio_identity(f, b), frob_ratio_change(f, a, b), frob_reuse_ok(f, a, b) ? 1 : 0);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("reuse_policy")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def _csr_text(M):
    M = sp.csr_matrix(M)
    M.sort_indices()
    return "%d\n%s\n%s\n%s\n" % (M.nnz, " ".join(map(str, M.indptr)), " ".join(map(str, M.indices)),
                                  " ".join("%.17g" % v for v in M.data))


def _run(exe, order, alpha, beta, Q, P, pairs):
    n = Q.shape[0]
    if P is None:
        pk, ptxt = 0, ""
    elif isinstance(P, np.ndarray) and P.ndim == 1:
        pk, ptxt = 1, " ".join("%.17g" % v for v in P) + "\n"
    else:
        pk, ptxt = 2, _csr_text(P)
    data = "%d %.17g %.17g %d %d\n" % (order, alpha, beta, n, pk) + _csr_text(Q) + ptxt
    data += "%d\n" % len(pairs) + "".join("%.17g %.17g %.17g %.17g\n" % (a.real, a.imag, b.real, b.imag)
                                           for a, b in pairs)
    out = subprocess.run([exe], input=data, capture_output=True, text=True, check=True).stdout.split("\n")
    return [(float(t[0]), float(t[1]), int(t[2])) for t in (l.split() for l in out if l.strip())]


PAIRS = [(1.0 + 0.5j, 1.0 - 0.5j), (3.0, 3.3), (10.0 + 2.0j, 11.0 + 2.5j), (2.0, 50.0), (0.5 + 4.0j, 0.6 + 4.1j),
         (7.0, 7.0)]


@pytest.mark.parametrize("e_kind", ["identity", "diag", "csr"])
def test_first_order_ratios_and_decisions_match_oracle(harness, e_kind):
    wl = W.random_sparse_system(40, 0.1, seed=12, e_kind=e_kind)
    got = _run(harness, 1, 0.0, 0.0, wl.A, wl.E, PAIRS)
    sched = irka.ReuseSchedule(wl.A, wl.E, transpose=False, mode="auto")
    for (a, b), (gi, gc, gd) in zip(PAIRS, got):
        std, change = ospai.frobenius_ratios(op.A_sigma(wl.A, wl.E, a), op.A_sigma(wl.A, wl.E, b))
        assert abs(gi - std) <= 1e-12 * std
        assert abs(gc - change) <= 1e-10 * max(change, 1e-300) + 1e-15
        assert gd == int(sched.reuse_ok(a, b))
    # transposition changes none of the quantities
    schedT = irka.ReuseSchedule(wl.A, wl.E, transpose=True, mode="auto")
    assert [int(schedT.reuse_ok(a, b)) for a, b in PAIRS] == [g[2] for g in got]
    assert [g[2] for g in got][-1] == 1            # equal shifts: change 0, reused
    assert [g[2] for g in got][3] == 0             # 2 -> 50: change ratio above 1, rebuilt


def test_second_order_ratios_and_decisions_match_oracle(harness):
    wl = W.stencil27_second_order(nx=4, ny=3, nz=3, m=1)
    pairs = [(0.2 + 0.1j, 0.25 + 0.1j), (1.0, 1.2), (0.3 + 2.0j, 0.3 + 2.2j), (0.1, 30.0)]
    got = _run(harness, 2, wl.alpha, wl.beta, wl.K, wl.M_diag, pairs)
    sched = airga.ReuseSchedule2(wl.K, wl.M_diag, wl.alpha, wl.beta, mode="auto")
    for (a, b), (gi, gc, gd) in zip(pairs, got):
        Ma = op.A_sigma_2nd(wl.K, wl.M_diag, wl.alpha, wl.beta, a)
        Mb = op.A_sigma_2nd(wl.K, wl.M_diag, wl.alpha, wl.beta, b)
        std, change = ospai.frobenius_ratios(Ma, Mb)
        assert abs(gi - std) <= 1e-12 * std
        assert abs(gc - change) <= 1e-10 * change
        assert gd == int(sched.reuse_ok(a, b))
    assert sorted(set(g[2] for g in got)) == [0, 1]    # both decisions occur
