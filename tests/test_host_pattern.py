"""The host-side sparsity construction of the library (csrc/host_pattern.h:
the static pattern S = pattern(A) + pattern(E) + diagonal with aligned
values, its transpose, the SPAI shadow sets I_j, the SELL-32 layout and the
diagonal layout) is
plain C++: compiled here with g++ and checked against the oracle's pattern
and shadow sets (oracle.spai.spai_pattern / pattern_sets, which take I_j as
the pattern of column j of S S) and against scipy's transpose.  No GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import spai as ospai

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2003_12759_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include "host_pattern.h"
using namespace mor_host;
static bool rd(long n, HostCSR& M) {
  long nnz;
  if (scanf("%ld", &nnz) != 1) return false;
  M.n = n; M.rowptr.resize(n + 1); M.col.resize(nnz); M.val.resize(nnz);
  for (auto& x : M.rowptr) if (scanf("%d", &x) != 1) return false;
  for (auto& x : M.col) if (scanf("%d", &x) != 1) return false;
  for (auto& x : M.val) if (scanf("%lf", &x) != 1) return false;
  return true;
}
template <class T> static void pr(const std::vector<T>& v, const char* fmt) {
  printf("%zu", v.size());
  for (const T& x : v) printf(fmt, x);
  printf("\n");
}
int main() {
  long n; int ek;
  HostCSR A, E;
  if (scanf("%ld", &n) != 1 || !rd(n, A) || scanf("%d", &ek) != 1) return 1;
  if (ek && !rd(n, E)) return 1;
  HostCSR S, T;
  std::vector<double> sa, se;
  merge_pattern(A, ek ? &E : nullptr, S, sa, se);
  std::vector<int64_t> t2p;
  transpose_pattern(S, T, t2p);
  pr(S.rowptr, " %d"); pr(S.col, " %d"); pr(sa, " %.17g"); pr(se, " %.17g");
  pr(T.rowptr, " %d"); pr(T.col, " %d"); pr(t2p, " %lld");
  for (const HostCSR* c : {&T, &S}) {
    std::vector<int64_t> iptr; std::vector<int32_t> iidx; int nI, nJ;
    shadow_sets(*c, iptr, iidx, nI, nJ);
    pr(iptr, " %lld"); pr(iidx, " %d"); printf("%d %d\n", nI, nJ);
  }
  std::vector<int64_t> sptr, lay; std::vector<int32_t> scol;
  sell_layout(S, sptr, scol, lay);
  pr(sptr, " %lld"); pr(scol, " %d"); pr(lay, " %lld");
  for (int md : {32, 3}) {
    std::vector<int32_t> offs; std::vector<int64_t> dlay;
    const bool ok = dia_layout(S, md, 1.25, offs, dlay);
    printf("%d\n", ok ? 1 : 0);
    pr(offs, " %d"); pr(dlay, " %lld");
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("host_pattern")
    (d / "h.cpp").write_text(HARNESS)
    exe = d / "h"
    subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-I", CSRC, str(d / "h.cpp"), "-o", str(exe)], check=True)
    return str(exe)


def _csr_text(M):
    M = sp.csr_matrix(M)
    M.sort_indices()
    return "%d\n%s\n%s\n%s\n" % (M.nnz, " ".join(map(str, M.indptr)), " ".join(map(str, M.indices)),
                                  " ".join("%.17g" % v for v in M.data))


def _run(exe, A, E):
    n = A.shape[0]
    data = "%d\n" % n + _csr_text(A) + ("1\n" + _csr_text(E) if E is not None else "0\n")
    lines = subprocess.run([exe], input=data, capture_output=True, text=True, check=True).stdout.split("\n")

    def arr(i, typ):
        t = lines[i].split()
        assert int(t[0]) == len(t) - 1
        return np.array([typ(x) for x in t[1:]])
    out = {"Srp": arr(0, int), "Scol": arr(1, int), "sa": arr(2, float), "se": arr(3, float),
           "Trp": arr(4, int), "Tcol": arr(5, int), "t2p": arr(6, int),
           "IprimT": arr(7, int), "IidxT": arr(8, int), "nIJ_T": tuple(map(int, lines[9].split())),
           "IprimS": arr(10, int), "IidxS": arr(11, int), "nIJ_S": tuple(map(int, lines[12].split())),
           "sptr": arr(13, int), "scol": arr(14, int), "lay": arr(15, int),
           "dia_ok": int(lines[16]), "doffs": arr(17, int), "dlay": arr(18, int),
           "dia3_ok": int(lines[19]), "doffs3": arr(20, int), "dlay3": arr(21, int)}
    return out


CASES = {
    "rand_diagE": lambda: W.random_sparse_system(257, 0.02, seed=3, e_kind="diag"),
    "rand_csrE": lambda: W.random_sparse_system(130, 0.04, seed=5, e_kind="csr"),
    "convdiff_n343": lambda: W.convdiff3d_siso(N=7),
}


@pytest.mark.parametrize("name", list(CASES))
def test_pattern_transpose_shadows_and_sell_match_oracle(harness, name):
    wl = CASES[name]()
    A = sp.csr_matrix(wl.A)
    Ecsr = wl.E if (wl.E is not None and not (isinstance(wl.E, np.ndarray) and wl.E.ndim == 1)) else None
    got = _run(harness, A, Ecsr)
    n = A.shape[0]
    # S against the oracle's static pattern; A's and E's values aligned to it
    S = ospai.spai_pattern(wl.A, wl.E)
    assert np.array_equal(got["Srp"], S.indptr) and np.array_equal(got["Scol"], S.indices)
    Sm = sp.csr_matrix((np.ones(len(got["Scol"])), got["Scol"], got["Srp"]), shape=(n, n))
    rows = np.repeat(np.arange(n), np.diff(got["Srp"]))
    assert np.array_equal(got["sa"], np.asarray(A[rows, got["Scol"]]).ravel())
    if Ecsr is not None:
        assert np.array_equal(got["se"], np.asarray(sp.csr_matrix(Ecsr)[rows, got["Scol"]]).ravel())
    # transpose and the position map
    St = sp.csr_matrix(Sm.T)
    St.sort_indices()
    assert np.array_equal(got["Trp"], St.indptr) and np.array_equal(got["Tcol"], St.indices)
    trows = np.repeat(np.arange(n), np.diff(got["Trp"]))
    assert np.array_equal(rows[got["t2p"]], got["Tcol"]) and np.array_equal(got["Scol"][got["t2p"]], trows)
    # shadow sets of the primal operator (columns of S = rows of S^T) and of the transposed one
    for key, Sref in (("T", S), ("S", sp.csr_matrix(S.T))):
        Jptr, Jidx, Iptr, Iidx = ospai.pattern_sets(Sref)
        assert np.array_equal(got["Iprim" + key], Iptr) and np.array_equal(got["Iidx" + key], Iidx)
        nI, nJ = got["nIJ_" + key]
        assert nI == np.max(np.diff(Iptr)) and nJ == np.max(np.diff(Jptr))
    # SELL-32: every CSR entry at its layout position, slices as wide as their longest row,
    # padding indices valid
    sptr, scol, lay = got["sptr"], got["scol"], got["lay"]
    assert len(sptr) == (n + 31) // 32 + 1
    lens = np.diff(got["Srp"])
    for s in range(len(sptr) - 1):
        assert sptr[s + 1] - sptr[s] == 32 * lens[s * 32:(s + 1) * 32].max()
    assert np.array_equal(scol[lay], got["Scol"])
    assert scol.min() >= 0 and scol.max() < n
    assert len(np.unique(lay)) == len(lay)
    # diagonal layout: eligible only with at most 32 diagonals and at most 25% padding; then the
    # offsets are the distinct c - r ascending and entry (r, c) sits at d n + r
    rows_all = np.repeat(np.arange(n), lens)
    offs = np.unique(got["Scol"] - rows_all)
    eligible = len(offs) <= 32 and len(offs) * n <= 1.25 * len(rows_all)
    assert got["dia_ok"] == int(eligible), (name, len(offs))
    assert eligible == name.startswith("convdiff")           # 7 diagonals; the random ones have hundreds
    if eligible:
        assert np.array_equal(got["doffs"], offs)
        d = np.searchsorted(offs, got["Scol"] - rows_all)
        assert np.array_equal(got["dlay"], d * n + rows_all)
    else:
        assert len(got["doffs"]) == 0 and len(got["dlay"]) == 0
    assert got["dia3_ok"] == 0 and len(got["doffs3"]) == 0      # more than 3 diagonals


DIA_HARNESS = r"""
#include <cstdio>
#include "host_pattern.h"
using namespace mor_host;
int main() {
  long n, nnz; int maxd; double fill;
  if (scanf("%ld %ld %d %lf", &n, &nnz, &maxd, &fill) != 4) return 1;
  HostCSR S; S.n = n; S.rowptr.resize(n + 1); S.col.resize(nnz);
  for (auto& x : S.rowptr) if (scanf("%d", &x) != 1) return 1;
  for (auto& x : S.col) if (scanf("%d", &x) != 1) return 1;
  std::vector<int32_t> offs; std::vector<int64_t> lay;
  const bool ok = dia_layout(S, maxd, fill, offs, lay);
  printf("%d %zu %zu\n", ok ? 1 : 0, offs.size(), lay.size());
  return 0;
}
"""


@pytest.fixture(scope="module")
def dia_harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("dia_layout")
    (d / "h.cpp").write_text(DIA_HARNESS)
    exe = d / "h"
    subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-I", CSRC, str(d / "h.cpp"), "-o", str(exe)], check=True)
    return str(exe)


def _banded(n, offsets):
    """Pattern with the given diagonals, every in-range position present."""
    rows, cols = [], []
    for o in offsets:
        for r in range(max(0, -o), min(n, n - o)):
            rows.append(r)
            cols.append(r + o)
    M = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    M.sort_indices()
    return M


def _dia_run(exe, M, maxd=32, fill=1.25):
    n = M.shape[0]
    inp = "%d %d %d %.17g\n%s\n%s\n" % (n, M.nnz, maxd, fill, " ".join(map(str, M.indptr)),
                                        " ".join(map(str, M.indices)))
    ok, no, nl = map(int, subprocess.run([exe], input=inp, capture_output=True, text=True,
                                         check=True).stdout.split())
    return ok, no, nl


def test_dia_layout_limits(dia_harness):
    """The diagonal layout takes at most max_diag diagonals and at most max_fill
    stored entries per nonzero: 32 diagonals pass and 33 do not; the padding
    bound is checked on both sides of 1.25."""
    n = 400
    M32 = _banded(n, list(range(-16, 16)))           # 32 diagonals
    ok, no, nl = _dia_run(dia_harness, M32)
    assert (ok, no, nl) == (1, 32, M32.nnz)
    M33 = _banded(n, list(range(-16, 17)))
    assert _dia_run(dia_harness, M33)[0] == 0
    # two far diagonals: stored entries 3 n against nnz = 3 n - 2 o
    o = 60
    M3 = _banded(n, [-o, 0, o])
    fill = 3 * n / M3.nnz
    assert _dia_run(dia_harness, M3, fill=fill * 1.001)[0] == 1
    assert _dia_run(dia_harness, M3, fill=fill * 0.999)[0] == 0
