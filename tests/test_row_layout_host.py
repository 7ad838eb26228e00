"""The row layout rule of the lock-step blocks (csrc/mor_internal.h:
row_stride pads k shift columns to the next whole 16-byte vector, lane_shape
gives each lane one 16-byte vector and a row a power-of-two number of lanes,
the last ones idle) compiled with g++ and checked for every scalar type and
every k the library batches (1..16): ld >= k, ld fits the 16-column limit,
rows of 16 bytes or more are whole 16-byte vectors with less than one vector
of padding, narrow rows are one thread per row, the lanes of a row stay
inside one warp and cover it, and every (type, lanes, columns per lane)
shape is instantiated in csrc/shape_dispatch.cuh.  No GPU."""
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
  // the FP64 refinement of a solve reuses the inner solve's stride:
  // (inner type, its wide type) = (F32, F64), (C32, C64)
  const int wide[4] = {ST_F64, ST_F64, ST_C64, ST_C64};
  for (int st = 0; st < 4; ++st)
    for (int k = 1; k <= MOR_KMAX; ++k) {
      const int ld = row_stride(st, k);
      int tpr = 0, cpt = 0;
      lane_shape(wide[st], ld, &tpr, &cpt);
      printf("W %d %d %d %d %d %d\n", wide[st], (int)st_size(wide[st]), k, ld, tpr, cpt);
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
        lines = [l for l in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
                 if l.strip()]
    rows = [tuple(map(int, l.split())) for l in lines if not l.startswith("W")]
    cross = [tuple(map(int, l.split()[1:])) for l in lines if l.startswith("W")]
    assert len(rows) == 4 * 16 and len(cross) == 4 * 16
    import re
    names = {"float": 0, "double": 1, "cfloat": 2, "cdouble": 3}
    disp = open(os.path.join(CSRC, "shape_dispatch.cuh")).read()
    shapes = {(int({"ST_F32": 0, "ST_F64": 1, "ST_C32": 2, "ST_C64": 3}[a]), int(c), int(d))
              for a, b, c, d in re.findall(r"MOR_SHAPE_CASE\((ST_\w+), (\w+), (\d+), (\d+)\)", disp)}
    assert shapes, "no shapes parsed"
    for st, es, k, ld, tpr, cpt in rows:
        assert k <= ld <= 16, (st, k, ld)
        if k * es < 16:                                             # narrow rows: one thread per row
            assert (ld, tpr, cpt) == (k, 1, k), (st, k, ld, tpr, cpt)
        else:
            assert (ld * es) % 16 == 0 and (ld - k) * es < 16, (st, k, ld)   # whole vectors, < 1 vector padding
            assert cpt * es == 16, (st, ld, cpt)                    # one 16-byte vector per lane
            assert tpr & (tpr - 1) == 0 and tpr * cpt >= ld > (tpr // 2) * cpt, (st, ld, tpr, cpt)
        assert tpr <= 32, (st, ld, tpr)
        assert (st, tpr, cpt) in shapes, ("shape not instantiated", st, tpr, cpt)
    for st, es, k, ld, tpr, cpt in cross:
        # a stride of another type: 16-byte lanes only on whole 16-byte rows, else scalar rows
        if cpt * es == 16:
            assert (ld * es) % 16 == 0 and tpr * cpt >= ld, (st, k, ld, tpr, cpt)
        else:
            assert tpr == 1 and cpt == ld, (st, k, ld, tpr, cpt)
        assert (st, tpr, cpt) in shapes, ("shape not instantiated", st, tpr, cpt)
