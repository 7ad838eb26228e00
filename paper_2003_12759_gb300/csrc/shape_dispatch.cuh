// Compile-time instantiation of the (scalar type, lanes per row, columns per
// lane) shapes the solve uses; see row_stride / lane_shape in mor_internal.h.
#pragma once
#include "mor_internal.h"
#include "mor_types.cuh"

#define MOR_SHAPE_CASE(ST, S, T, C) \
  if (st == ST && tpr == T && cpt == C) return f.template operator()<S, T, C>();

// Calls f.template operator()<S, TPR, CPT>() for the shape of (st, ld).
template <class F>
int dispatch_shape(int st, int ld, F&& f) {
  int tpr = 1, cpt = 1;
  lane_shape(st, ld, &tpr, &cpt);
  MOR_SHAPE_CASE(ST_F32, float, 1, 1) MOR_SHAPE_CASE(ST_F32, float, 1, 2) MOR_SHAPE_CASE(ST_F32, float, 1, 3)
  MOR_SHAPE_CASE(ST_F32, float, 1, 4) MOR_SHAPE_CASE(ST_F32, float, 2, 4) MOR_SHAPE_CASE(ST_F32, float, 4, 4)
  MOR_SHAPE_CASE(ST_F64, double, 1, 1) MOR_SHAPE_CASE(ST_F64, double, 1, 2) MOR_SHAPE_CASE(ST_F64, double, 2, 2)
  MOR_SHAPE_CASE(ST_F64, double, 4, 2) MOR_SHAPE_CASE(ST_F64, double, 8, 2) MOR_SHAPE_CASE(ST_F64, double, 1, 3)
  MOR_SHAPE_CASE(ST_C32, cfloat, 1, 1) MOR_SHAPE_CASE(ST_C32, cfloat, 1, 2) MOR_SHAPE_CASE(ST_C32, cfloat, 2, 2)
  MOR_SHAPE_CASE(ST_C32, cfloat, 4, 2) MOR_SHAPE_CASE(ST_C32, cfloat, 8, 2)
  MOR_SHAPE_CASE(ST_C64, cdouble, 1, 1) MOR_SHAPE_CASE(ST_C64, cdouble, 2, 1) MOR_SHAPE_CASE(ST_C64, cdouble, 4, 1)
  MOR_SHAPE_CASE(ST_C64, cdouble, 8, 1) MOR_SHAPE_CASE(ST_C64, cdouble, 16, 1)
  return (int)cudaErrorInvalidValue;
}
