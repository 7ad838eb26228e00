// Factor SpMV in the diagonal layout, specialised to patterns of ND
// diagonals (5: 2D five-point stencils, 7: 3D seven-point stencils) with
// FP32 / complex64 vectors, the inner solves' types, for rows of two or more
// lanes.  Measured on the 100^3 chain (complex64, L2 flushed; us per launch,
// this kernel against the generic diagonal-layout one): k = 3: 26.2 / 34.3,
// k = 6: 37.9 / 44.1, k = 7: 45.1 / 56.3; ncu at k = 6 counts 36% fewer
// instructions.
//
// Same product as factor_spmv_kernel<..., DIA = true> (a factor of the chain
// Q_L ... Q_2 P_1 of Sec. III.B applied to k columns; row r sums, in the order
// of the diagonals, f(d n + r) x(r + o_d)), with the per-diagonal constants
// passed by value as kernel parameters: the offsets o_d, the offsets times the
// row stride, and the start of each diagonal's values.  The parameters sit in
// the constant bank and, the diagonal loop being unrolled at compile time,
// enter the address arithmetic without loads.  Interior rows (every r + o_d
// inside 0 .. n - 1) gather at x(r) + o_d ld without a clamp; the few edge rows
// go one diagonal at a time with the column clamped into range (those
// positions are padding, value 0).
#include "mor_internal.h"
#include "krylov_state.cuh"
#include "shape_dispatch.cuh"

#include <type_traits>

#ifndef MOR_DIA_ND
#define MOR_DIA_ND 1
#endif

namespace {

template <int ND> struct DiaConst {
  long long offld[ND];     // o_d times the row stride ld (elements)
  int off[ND];             // o_d, ascending
  const void* fd[ND];      // values of diagonal d (f + d n)
};

template <typename S> __device__ __forceinline__ S zero_() { return S(0); }

template <typename S, typename V, typename W, int CPT>
__device__ __forceinline__ void mac(Pack<S, CPT>& acc, const W fv, const Pack<S, CPT>& xv) {
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    if constexpr (is_cplx<V>::value) fma_s(acc.v[j], fv, xv.v[j]);
    else fma_r(acc.v[j], fv, xv.v[j]);
  }
}

// diagonals per chunk (values and gathers of a chunk in flight together) and
// blocks per SM the registers are held to.  Measured (k = 3 / 6 / 7 / 8, us
// per launch, L2 flushed): chunk 4 at 8 blocks (32 registers) 29.2 / 38.5 /
// 46.6 / 43.6; chunk 8 at 6 (40) 27.2 / 36.4 / 50.6 / 49.8; at 5 (48) 27.2 /
// 39.4 / 51.8 / 50.7; at 4 (56) 25.1 / 37.4 / 45.6 / 42.5; chunk 2 at 8
// 28.2 / 38.4 / 46.6 / 46.6 -- within a few percent of one another.
#ifndef MOR_DIA_ND_CHUNK
#define MOR_DIA_ND_CHUNK 4
#endif
#ifndef MOR_DIA_ND_MINB
#define MOR_DIA_ND_MINB 8
#endif

template <typename S, typename V, int TPR, int CPT, int ND>
__global__ void __launch_bounds__(256, MOR_DIA_ND_MINB) factor_dia_nd_kernel(SegView sg, DiaConst<ND> dc, int n,
                                                               const int* __restrict__ apply, int ld,
                                                               const S* __restrict__ x, S* __restrict__ y,
                                                               const int* done, const KState* __restrict__ kst) {
  typedef typename real_of<S>::type RS;
  typedef typename std::conditional<is_cplx<V>::value, cplx<RS>, RS>::type W;
  if (done && *done) return;
  // three or five lanes per row: the threads past the last whole row group of
  // the block have no row
  if constexpr ((TPR & (TPR - 1)) != 0) {
    if ((int)threadIdx.x >= (256 / TPR) * TPR) return;
  }
  const int sub = threadIdx.x % TPR;
  const int c0 = sub * CPT;
  if (c0 >= ld) return;
  unsigned mask = 0;
#pragma unroll
  for (int j = 0; j < CPT; ++j) mask |= (apply[c0 + j] != 0 ? 1u : 0u) << j;
  int64_t rb64, re64;
  {
    const int seg = seg_of_chunk(sg, blockIdx.x);
    if (kst) {
      // inside a Krylov iteration: lanes whose columns of this segment have all stopped skip
      const KState* ks = kst + (size_t)seg * ld + c0;
      bool any = false;
#pragma unroll
      for (int j = 0; j < CPT; ++j) any |= (ks[j].active != 0);
      if (!any) return;
    }
    chunk_rows(sg, seg, blockIdx.x, rb64, re64);
  }
  const int rpb = blockDim.x / TPR;
  const int re = (int)re64;
  for (int r = (int)rb64 + (int)threadIdx.x / TPR; r < re; r += rpb) {
    Pack<S, CPT> acc;
#pragma unroll
    for (int j = 0; j < CPT; ++j) acc.v[j] = zero_<S>();
    if (mask) {
      if (r + dc.off[0] >= 0 && r + dc.off[ND - 1] < n) {
        const S* xr = x + (int64_t)r * ld + c0;
        // chunks of CH diagonals: values and gathers of a chunk in flight together
        constexpr int CH = MOR_DIA_ND_CHUNK;
#pragma unroll
        for (int d0 = 0; d0 < ND; d0 += CH) {
          W fv[CH];
          Pack<S, CPT> xv[CH];
#pragma unroll
          for (int u = 0; u < CH; ++u)
            if (d0 + u < ND) {
              fv[u] = cvt_<W, V>::f(((const V* __restrict__)dc.fd[d0 + u])[r]);
              xv[u] = ldp<S, CPT>(xr + dc.offld[d0 + u]);
            }
#pragma unroll
          for (int u = 0; u < CH; ++u)
            if (d0 + u < ND) mac<S, V, W, CPT>(acc, fv[u], xv[u]);
        }
      } else {
        for (int d = 0; d < ND; ++d) {
          const int c = r + dc.off[d];
          const int cc = c < 0 ? 0 : (c >= n ? n - 1 : c);
          const W fv = cvt_<W, V>::f(((const V* __restrict__)dc.fd[d])[r]);
          mac<S, V, W, CPT>(acc, fv, ldp<S, CPT>(x + (int64_t)cc * ld + c0));
        }
      }
    }
    const int64_t q = (int64_t)r * ld + c0;
    if (mask != (1u << CPT) - 1u) {
      const Pack<S, CPT> xo = ldp<S, CPT>(x + q);
#pragma unroll
      for (int j = 0; j < CPT; ++j)
        if (!((mask >> j) & 1u)) acc.v[j] = xo.v[j];
    }
    stp<S, CPT>(y + q, acc);
  }
}

template <typename S, typename V, int TPR, int CPT, int ND>
int launch_nd(const SegView& sg, const PatView& pv, const void* fvals, const int* apply, int ld, const void* x,
              void* y, const int* done, const void* kstate, cudaStream_t s) {
  DiaConst<ND> dc;
  for (int d = 0; d < ND; ++d) {
    dc.off[d] = pv.h_doff[d];
    dc.offld[d] = (long long)pv.h_doff[d] * ld;
    dc.fd[d] = (const V*)fvals + (size_t)d * pv.n;
  }
  const SegView g = fit_grid(sg, (const void*)factor_dia_nd_kernel<S, V, TPR, CPT, ND>, TPR);
  factor_dia_nd_kernel<S, V, TPR, CPT, ND><<<g.nblocks, 256, 0, s>>>(g, dc, pv.n, apply, ld, (const S*)x, (S*)y, done,
                                                                     (const KState*)kstate);
  return 0;
}

// One thread per row (k = 1, 2 complex64): the generic diagonal-layout kernel
// measured as fast or faster (k = 1: 16.9 against 18.0 us), so those shapes
// are left to it.
template <typename S, int TPR, int CPT>
int launch_shape(int fst, const SegView& sg, const PatView& pv, const void* fvals, const int* apply, int ld,
                 const void* x, void* y, const int* done, const void* kstate, cudaStream_t s) {
  if constexpr (CPT * sizeof(S) > 16 || TPR == 1) {
    return -1;
  } else {
    auto by_nd = [&]<typename V>() -> int {
      if (pv.ndiag == 7) return launch_nd<S, V, TPR, CPT, 7>(sg, pv, fvals, apply, ld, x, y, done, kstate, s);
      if (pv.ndiag == 5) return launch_nd<S, V, TPR, CPT, 5>(sg, pv, fvals, apply, ld, x, y, done, kstate, s);
      return -1;
    };
    if constexpr (is_cplx<S>::value) {
      if (fst == ST_C32) return by_nd.template operator()<cfloat>();
      if (fst == ST_F32) return by_nd.template operator()<float>();
      return -1;
    } else {
      if (fst == ST_F32) return by_nd.template operator()<float>();
      return -1;
    }
  }
}

}  // namespace

int launch_factor_dia_nd(int st, int fst, const SegView& sg, const PatView& pv, const void* fvals, const int* apply,
                         int ld, const void* x, void* y, const int* done, const void* kstate, cudaStream_t s) {
#if !MOR_DIA_ND
  return -1;
#else
  if (pv.fmt != FMT_DIA || !pv.h_doff || (pv.ndiag != 5 && pv.ndiag != 7)) return -1;
  if (st != ST_C32 && st != ST_F32) return -1;
  if (ld < 1 || ld > MOR_LDMAX) return -1;
  // rows of exactly three (five) 16-byte vectors: three (five) lanes per row,
  // no idle lane (the power-of-two mapping would give four or eight)
  if ((int)st_size(st) * ld == 48) {
    if (st == ST_C32) return launch_shape<cfloat, 3, 2>(fst, sg, pv, fvals, apply, ld, x, y, done, kstate, s);
    return launch_shape<float, 3, 4>(fst, sg, pv, fvals, apply, ld, x, y, done, kstate, s);
  }
  if ((int)st_size(st) * ld == 80) {
    if (st == ST_C32) return launch_shape<cfloat, 5, 2>(fst, sg, pv, fvals, apply, ld, x, y, done, kstate, s);
    return launch_shape<float, 5, 4>(fst, sg, pv, fvals, apply, ld, x, y, done, kstate, s);
  }
  return dispatch_shape(st, ld, [&]<typename S, int TPR, int CPT>() -> int {
    if constexpr (std::is_same<S, cfloat>::value || std::is_same<S, float>::value)
      return launch_shape<S, TPR, CPT>(fst, sg, pv, fvals, apply, ld, x, y, done, kstate, s);
    else
      return -1;
  });
#endif
}
