"""The row layout rule of the lock-step blocks (csrc/mor_internal.h:
row_stride pads k shift columns to a stride ld whose row is a whole number
of 16-byte vectors, lane_shape spreads a row over a power-of-two number of
lanes) compiled with g++ and checked for every scalar type and every k the
library batches (1..16): ld >= k, ld fits the 16-column limit, padded rows
are whole 16-byte vectors, the lanes of a row stay inside one warp and cover
the row exactly (or one column per lane).  No GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2003_12759_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r"""
#include <cstdio>
#include "mor_internal.h"
int main() {
  for (int st = 0; st < 4; ++st)
    for (int k = 1; k <= MOR_KMAX; ++k) {
      const int ld = row_stride(st, k);
      int tpr = 0, cpt = 0;
      lane_shape(st, ld, &tpr, &cpt);
      printf("%d %d %d %d %d %d\n", st, (int)st_size(st), k, ld, tpr, cpt);
    }
  return 0;
}
"""


def test_row_stride_and_lane_shape():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("no C++ compiler or CUDA headers")
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "h.cpp")
        open(src, "w").write(HARNESS)
        exe = os.path.join(d, "h")
        subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", CUDA_INC,
                        src, "-o", exe], check=True)
        rows = [tuple(map(int, l.split())) for l in subprocess.run([exe], capture_output=True, text=True,
                                                                  check=True).stdout.split("\n") if l.strip()]
    assert len(rows) == 4 * 16
    for st, es, k, ld, tpr, cpt in rows:
        assert k <= ld <= 16, (st, k, ld)
        assert ld == k or (ld * es) % 16 == 0, (st, k, ld)          # padded rows: whole 16-byte vectors
        assert tpr >= 1 and (tpr & (tpr - 1)) == 0 and tpr <= 32, (st, ld, tpr)
        assert tpr * cpt == ld or (cpt == 1 and tpr >= ld), (st, ld, tpr, cpt)
        assert cpt * es <= 16 or tpr == 1, (st, ld, tpr, cpt)       # one vector per lane unless one lane per row
