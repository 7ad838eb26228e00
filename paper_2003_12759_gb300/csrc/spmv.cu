// Shifted-operator SpMV and preconditioner-factor SpMV.
//
// Operator (Sec. II; Algorithm 3 line 4 writes it sigma_i D - K):
//     Y(:, c) = sE_c * (E X(:, c)) + sA_c * (A X(:, c))       [+ Bv(:, c)]
// with per-column complex coefficients: first-order systems use
// (sE, sA) = (sigma_c, -1), i.e. sigma_c E - A; second-order systems
// (Rayleigh damping, Algorithm 1 line 4) use (s^2 + alpha s, 1 + beta s) on
// (M, K).  The shifted matrix is never formed: one pass over the pattern
// reads the A values (and E values when E is a general sparse matrix) once
// for all k columns of the batch, which is the point of batching the shifts.
//
// Factor SpMV: Y(:, c) = F X(:, c) for the columns the factor applies to,
// Y(:, c) = X(:, c) otherwise (the chain prefix of a shift, Sec. III.B: the
// preconditioner Q_i ... Q_2 P_1 is applied as successive mat-vecs).
//
// Vectors are n x k, row-major with row stride k (the k values of one row are
// contiguous), so every gathered x[col] serves all k columns from one
// sector.  Patterns are CSR or SELL-32 (slices of 32 rows stored
// column-major, so a warp's index/value loads are fully coalesced).
#include "mor_internal.h"
#include "krylov_state.cuh"

#include "shape_dispatch.cuh"

#include <type_traits>

namespace {

template <typename S> struct CoefS { S sE[MOR_LDMAX]; S sA[MOR_LDMAX]; };

// Tuning of the two SpMV kernels, measured on the 7-point 100^3 pattern with
// complex64 shift columns (CUDA events, L2 flushed before every launch).
// Both kernels are latency-bound on the chain row pointer -> index -> gather,
// so resident warps matter more than gathers in flight per thread: the
// register allocation is held to a full SM of 256-thread blocks (32
// registers) for lane slices of at most 16 bytes, and a row's nonzeros are
// gathered in whole chunks (all gathers of a chunk in flight) plus a
// one-by-one remainder.  A sweep of chunk depth x blocks per SM with the
// last chunk predicated past the row's end instead of the remainder (factor /
// operator SpMV, k = 7): 4 x 8 blocks 64 / 102 us, 8 x 8: 65 / 100, 8 x 6:
// 75 / 113, 8 x 5: 76 / 109, 8 x 4: 77 / 104, 8 x 3: 94 / 132 -- at 32
// registers the compiler keeps only a few gathers in flight whatever the
// chunk, and fewer resident warps cost more than deeper chunks gain; the
// whole chunks with a one-by-one remainder measured 60 / 99 us (k = 7) and
// 58 us (factor, k = 6) against 65 and 64 us predicated.  FP64
// data keeps fewer blocks (6 in the factor kernel for two real columns, 5 in
// the operator kernel), where 32 registers would spill.  Wider lane slices
// take no bound and chunk 1.
#ifndef MOR_FACTOR_GCH
#define MOR_FACTOR_GCH 4
#endif
#ifndef MOR_OP_GCH
#define MOR_OP_GCH 2
#endif
template <typename S, int CPT> constexpr bool narrow_slice() { return CPT * sizeof(S) <= 16; }
template <typename S, int CPT> constexpr int factor_chunk() { return narrow_slice<S, CPT>() ? MOR_FACTOR_GCH : 1; }
template <typename S, int CPT> constexpr int op_chunk() { return narrow_slice<S, CPT>() ? MOR_OP_GCH : 1; }
#ifndef MOR_FACTOR_MINB
#define MOR_FACTOR_MINB 8
#endif
template <typename S, int CPT> constexpr int min_blocks() {
  return narrow_slice<S, CPT>() ? ((sizeof(S) == 8 && !is_cplx<S>::value && CPT > 1 && MOR_FACTOR_MINB > 6)
                                       ? 6 : MOR_FACTOR_MINB) : 1;
}
#ifndef MOR_OP_MINB
#define MOR_OP_MINB 8
#endif
template <typename S, int CPT> constexpr int op_min_blocks() {
  return narrow_slice<S, CPT>() ? (sizeof(typename real_of<S>::type) == 8 ? 5 : MOR_OP_MINB) : 1;
}
// the operator SpMV in the diagonal layout: no index loads, so a row's loads
// are independent and deeper chunks cost only registers
#ifndef MOR_OP_DIA_GCH
#define MOR_OP_DIA_GCH 4
#endif
#ifndef MOR_OP_DIA_MINB
#define MOR_OP_DIA_MINB 8
#endif
template <typename S, int CPT, bool DIA> constexpr int op_blocks() {
  return (DIA && narrow_slice<S, CPT>() && sizeof(typename real_of<S>::type) == 4) ? MOR_OP_DIA_MINB
                                                                                  : op_min_blocks<S, CPT>();
}
template <typename S, int CPT, bool DIA> constexpr int op_gch() {
  return (DIA && narrow_slice<S, CPT>()) ? MOR_OP_DIA_GCH : op_chunk<S, CPT>();
}

template <typename S> __device__ __forceinline__ S zero_() { return S(0); }

// L2 eviction priorities for the SpMVs of a preconditioner chain: every factor
// of the chain (and the operator) shares one pattern, so the row pointers and
// column indices are loaded with evict_last (kept across the chain's
// launches), the factor values, read once per chain, with evict_first; the
// output vector, the next factor's input, is written with the default policy.
// Measured on the 100^3 sweep (complex64, L2 flushed before each launch):
// factor SpMV k = 1: 30.2 -> 26.3 us, k = 6: 65.1 -> 60.0 us, k = 7: 65.6 ->
// 63.4 us; the IRKA step time moved within run-to-run noise (294 vs 296 ms).
// MOR_L2_HINTS = 0 uses plain loads.
#ifndef MOR_L2_HINTS
#define MOR_L2_HINTS 1
#endif
struct L2Pol { uint64_t last, first; };
__device__ __forceinline__ L2Pol l2_policies() {
  L2Pol p{0, 0};
#if MOR_L2_HINTS
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p.last));
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p.first));
#endif
  return p;
}
__device__ __forceinline__ int ldh(const int* a, uint64_t pol) {
#if MOR_L2_HINTS
  int v;
  asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
  return v;
#else
  (void)pol;
  return __ldg(a);
#endif
}
__device__ __forceinline__ float ldh(const float* a, uint64_t pol) {
#if MOR_L2_HINTS
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
  return v;
#else
  (void)pol;
  return __ldg(a);
#endif
}
__device__ __forceinline__ double ldh(const double* a, uint64_t pol) {
#if MOR_L2_HINTS
  double v;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
  return v;
#else
  (void)pol;
  return __ldg(a);
#endif
}
__device__ __forceinline__ cfloat ldh(const cfloat* a, uint64_t pol) {
#if MOR_L2_HINTS
  float x, y;
  asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(x), "=f"(y) : "l"(a), "l"(pol));
  return cfloat(x, y);
#else
  (void)pol;
  return *a;
#endif
}
__device__ __forceinline__ cdouble ldh(const cdouble* a, uint64_t pol) {
#if MOR_L2_HINTS
  double x, y;
  asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(x), "=d"(y) : "l"(a), "l"(pol));
  return cdouble(x, y);
#else
  (void)pol;
  return *a;
#endif
}


// Per-diagonal constants of the operator SpMV in the diagonal layout for a
// pattern of ND diagonals (ND = 0: read at run time), passed by value (the
// constant bank): offsets, offsets times the row stride, and the start of
// each diagonal's A (and E) values.
template <int ND> struct OpDiaC {
  long long offld[ND];
  int off[ND];
  const void* ad[ND];
  const void* ed[ND];
};
template <> struct OpDiaC<0> { int unused; };

// R diagonals d .. d + R - 1 of an operator row r in the diagonal layout
// (column clamped into range: out-of-range columns are padding of value 0).
template <int R, bool ECSR, typename S, typename RV, int CPT>
__device__ __forceinline__ void op_dia_gather(S (&accA)[CPT], S (&accE)[CPT], const int* __restrict__ doff,
                                              const RV* __restrict__ a, const RV* __restrict__ e, int d, int r, int n,
                                              int ld, int c0, const S* __restrict__ x) {
  int cc[R];
  RV av[R], ev[R];
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int c = r + __ldg(doff + d + u);
    cc[u] = c < 0 ? 0 : (c >= n ? n - 1 : c);
    av[u] = __ldg(a + (d + u) * n + r);
    if constexpr (ECSR) ev[u] = __ldg(e + (d + u) * n + r);
    else ev[u] = RV(0);
  }
  Pack<S, CPT> xv[R];
#pragma unroll
  for (int u = 0; u < R; ++u) xv[u] = ldp<S, CPT>(x + (int64_t)cc[u] * ld + c0);
#pragma unroll
  for (int u = 0; u < R; ++u)
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      fma_r(accA[j], av[u], xv[u].v[j]);
      if constexpr (ECSR) fma_r(accE[j], ev[u], xv[u].v[j]);
    }
}

// Y(:, c) = sE_c (E X(:, c)) + sA_c (A X(:, c)) [+ B(:, c)], with an optional
// fused per-column reduction.  TPR lanes per row, lane `sub` owns the CPT
// columns sub * CPT ... sub * CPT + CPT - 1 of the n x ld blocks.  The
// coefficients are read from shared memory where they are used and row
// indices are 32-bit, to hold the register bound of op_min_blocks.
template <typename S, int TPR, int CPT, bool ECSR, bool DIA, int ND>
__global__ void __launch_bounds__(256, (op_blocks<S, CPT, DIA>())) op_spmv_kernel(SegView sg, PatView pv, OpVals ov,
                                                                                CoefS<S> cf, int ld,
                                                                                const S* __restrict__ x, S* __restrict__ y,
                                                                                const S* __restrict__ bv, RedArgs red,
                                                                                OpDiaC<ND> dc) {
  typedef typename real_of<S>::type R;
  if (red.done && *red.done) return;
  __shared__ S csE[MOR_LDMAX], csA[MOR_LDMAX];
  if (threadIdx.x < ld) { csE[threadIdx.x] = cf.sE[threadIdx.x]; csA[threadIdx.x] = cf.sA[threadIdx.x]; }
  __syncthreads();
  const R* __restrict__ a = (const R*)ov.a;
  const R* __restrict__ e = (const R*)ov.e;
  const R* __restrict__ ed = (const R*)ov.ediag;
  const S* __restrict__ w = (const S*)red.w;
  const int sub = threadIdx.x % TPR;
  const int c0 = sub * CPT;
  const int seg = seg_of_chunk(sg, blockIdx.x);
  // inside a Krylov iteration, a lane whose columns of this segment have all stopped
  // (converged, or every column of a finished system of a batch) has no work: its
  // rows of y are read only by stopped columns, and its reduction terms stay zero
  bool act = c0 < ld;
  if (act && red.state && red.fin >= FIN_ALPHA) {
    const KState* ks = (const KState*)red.state + (size_t)seg * ld + c0;
    bool any = false;
#pragma unroll
    for (int j = 0; j < CPT; ++j) any |= (ks[j].active != 0);
    act = any;
  }
  S v0[CPT], v1[CPT];
#pragma unroll
  for (int j = 0; j < CPT; ++j) { v0[j] = zero_<S>(); v1[j] = zero_<S>(); }
  const int rpb = blockDim.x / TPR;
  int64_t rb64, re64;
  chunk_rows(sg, seg, blockIdx.x, rb64, re64);
  const int re = (int)re64;
  const bool sell = pv.fmt == FMT_SELL;
  const L2Pol pol = l2_policies();
  const int ekind = ECSR ? EK_CSR : ov.ekind;   // E a general sparse matrix: compile-time branch
  constexpr int GCH = op_gch<S, CPT, DIA>();
  static_assert(GCH <= 4, "the remainder below takes at most 3 diagonals");
  if (act) {
    for (int r = (int)rb64 + (int)threadIdx.x / TPR; r < re; r += rpb) {
      S accA[CPT], accE[CPT];
#pragma unroll
      for (int j = 0; j < CPT; ++j) { accA[j] = zero_<S>(); accE[j] = zero_<S>(); }
      if constexpr (DIA && ND > 0) {
        if (r + dc.off[0] >= 0 && r + dc.off[ND - 1] < pv.n) {
          // interior row: every column r + o_d in range, no clamp
          const S* xr = x + (int64_t)r * ld + c0;
#pragma unroll
          for (int d0 = 0; d0 < ND; d0 += 4) {
            R av[4], ev[4];
            Pack<S, CPT> xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (d0 + u < ND) {
                av[u] = ((const R* __restrict__)dc.ad[d0 + u])[r];
                if constexpr (ECSR) ev[u] = ((const R* __restrict__)dc.ed[d0 + u])[r];
                xv[u] = ldp<S, CPT>(xr + dc.offld[d0 + u]);
              }
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (d0 + u < ND) {
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                  fma_r(accA[j], av[u], xv[u].v[j]);
                  if constexpr (ECSR) fma_r(accE[j], ev[u], xv[u].v[j]);
                }
              }
          }
        } else {
          for (int d = 0; d < ND; ++d) op_dia_gather<1, ECSR, S, R, CPT>(accA, accE, pv.doff, a, e, d, r, pv.n, ld, c0, x);
        }
      } else if constexpr (DIA) {
        int d = 0;
        for (; d + GCH <= pv.ndiag; d += GCH)
          op_dia_gather<GCH, ECSR, S, R, CPT>(accA, accE, pv.doff, a, e, d, r, pv.n, ld, c0, x);
        if constexpr (GCH > 1) {
          const int rem = pv.ndiag - d;     // 0 .. GCH - 1
          if constexpr (GCH > 3) {
            if (rem == 3) op_dia_gather<3, ECSR, S, R, CPT>(accA, accE, pv.doff, a, e, d, r, pv.n, ld, c0, x);
          }
          if constexpr (GCH > 2) {
            if (rem == 2) op_dia_gather<2, ECSR, S, R, CPT>(accA, accE, pv.doff, a, e, d, r, pv.n, ld, c0, x);
          }
          if (rem == 1) op_dia_gather<1, ECSR, S, R, CPT>(accA, accE, pv.doff, a, e, d, r, pv.n, ld, c0, x);
        }
      } else {
        int p0, p1, step;
        if (sell) {
          const int64_t base = pv.sptr[r >> 5];
          const int wd = (int)((pv.sptr[(r >> 5) + 1] - base) >> 5);
          p0 = (int)base + (r & 31);
          p1 = p0 + 32 * wd;
          step = 32;
        } else {
          p0 = ldh(pv.rowptr + r, pol.last);
          p1 = ldh(pv.rowptr + r + 1, pol.last);
          step = 1;
        }
        int pc = p0;
        for (; pc + (GCH - 1) * step < p1; pc += GCH * step) {
          int cc[GCH];
          R av[GCH], ev[GCH];
#pragma unroll
          for (int u = 0; u < GCH; ++u) {
            cc[u] = ldh(pv.col + pc + u * step, pol.last);
            av[u] = __ldg(a + pc + u * step);
            if constexpr (ECSR) ev[u] = __ldg(e + pc + u * step);
            else ev[u] = R(0);
          }
          Pack<S, CPT> xv[GCH];
#pragma unroll
          for (int u = 0; u < GCH; ++u) xv[u] = ldp<S, CPT>(x + (int64_t)cc[u] * ld + c0);
#pragma unroll
          for (int u = 0; u < GCH; ++u)
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
              fma_r(accA[j], av[u], xv[u].v[j]);
              if constexpr (ECSR) fma_r(accE[j], ev[u], xv[u].v[j]);
            }
        }
        for (; pc < p1; pc += step) {
          const int cc = ldh(pv.col + pc, pol.last);
          const R av = __ldg(a + pc);
          const Pack<S, CPT> xv = ldp<S, CPT>(x + (int64_t)cc * ld + c0);
          if constexpr (ECSR) {
            const R ev = __ldg(e + pc);
#pragma unroll
            for (int j = 0; j < CPT; ++j) { fma_r(accA[j], av, xv.v[j]); fma_r(accE[j], ev, xv.v[j]); }
          } else {
#pragma unroll
            for (int j = 0; j < CPT; ++j) fma_r(accA[j], av, xv.v[j]);
          }
        }
      }
      const int64_t q = (int64_t)r * ld + c0;
      if constexpr (!ECSR) {
        const Pack<S, CPT> xr = ldp<S, CPT>(x + q);
        const R d = (ekind == EK_DIAG) ? __ldg(ed + r) : R(1);
#pragma unroll
        for (int j = 0; j < CPT; ++j) accE[j] = scale_(d, xr.v[j]);
      }
      Pack<S, CPT> yv;
#pragma unroll
      for (int j = 0; j < CPT; ++j) yv.v[j] = csE[c0 + j] * accE[j] + csA[c0 + j] * accA[j];
      if (bv) {
        const Pack<S, CPT> bb = ldp<S, CPT>(bv + q);
#pragma unroll
        for (int j = 0; j < CPT; ++j) yv.v[j] += bb.v[j];
      }
      stp<S, CPT>(y + q, yv);
      if (red.mode == RED_DOT_W) {
        const Pack<S, CPT> wv = ldp<S, CPT>(w + q);
#pragma unroll
        for (int j = 0; j < CPT; ++j) fma_s(v0[j], conj_(wv.v[j]), yv.v[j]);
      } else if (red.mode == RED_DOT_TT) {
        const Pack<S, CPT> wv = ldp<S, CPT>(w + q);
#pragma unroll
        for (int j = 0; j < CPT; ++j) { fma_s(v0[j], conj_(yv.v[j]), wv.v[j]); v1[j] += S(abs2_(yv.v[j])); }
      } else if (red.mode == RED_NORM) {
#pragma unroll
        for (int j = 0; j < CPT; ++j) v0[j] += S(abs2_(yv.v[j]));
      }
    }
  }
  if (red.mode != RED_NONE)
    col_reduce_finalize<S, TPR, CPT>(v0, v1, ld, sg, seg, blockIdx.x, (double*)red.part, red.fin, (KState*)red.state,
                                     (cdouble*)red.out, (int*)red.done);
}

// R entries of a factor row starting at position pc (stride step): indices
// and values first, then all R gathers in flight, then the products in
// storage order.
template <int R, typename S, typename V, typename W, int CPT>
__device__ __forceinline__ void factor_gather(Pack<S, CPT>& acc, const int* __restrict__ col,
                                              const V* __restrict__ f, int pc, int step, int ld, int c0,
                                              const S* __restrict__ x, const L2Pol& pol) {
  int cc[R];
  W fv[R];
#pragma unroll
  for (int u = 0; u < R; ++u) {
    cc[u] = ldh(col + pc + u * step, pol.last);
    fv[u] = cvt_<W, V>::f(ldh(f + pc + u * step, pol.first));
  }
  Pack<S, CPT> xv[R];
#pragma unroll
  for (int u = 0; u < R; ++u) xv[u] = ldp<S, CPT>(x + (int64_t)cc[u] * ld + c0);
#pragma unroll
  for (int u = 0; u < R; ++u)
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      if constexpr (is_cplx<V>::value) fma_s(acc.v[j], fv[u], xv[u].v[j]);
      else fma_r(acc.v[j], fv[u], xv[u].v[j]);
    }
}

// R diagonals d .. d + R - 1 of row r in the diagonal layout: value at
// (d + u) n + r, column r + doff[d + u].  A column outside 0 .. n - 1 is
// padding (value 0): the index is clamped into range so that every load is
// in bounds and unconditional.
template <int R, typename S, typename V, typename W, int CPT>
__device__ __forceinline__ void factor_dia_gather(Pack<S, CPT>& acc, const int* __restrict__ doff,
                                                  const V* __restrict__ f, int d, int r, int n, int ld, int c0,
                                                  const S* __restrict__ x, const L2Pol& pol) {
  int cc[R];
  W fv[R];
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int c = r + __ldg(doff + d + u);
    cc[u] = c < 0 ? 0 : (c >= n ? n - 1 : c);
    fv[u] = cvt_<W, V>::f(ldh(f + (d + u) * n + r, pol.first));
  }
  Pack<S, CPT> xv[R];
#pragma unroll
  for (int u = 0; u < R; ++u) xv[u] = ldp<S, CPT>(x + (int64_t)cc[u] * ld + c0);
#pragma unroll
  for (int u = 0; u < R; ++u)
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      if constexpr (is_cplx<V>::value) fma_s(acc.v[j], fv[u], xv[u].v[j]);
      else fma_r(acc.v[j], fv[u], xv[u].v[j]);
    }
}

// Y(:, c) = F X(:, c) where the factor applies to column c, else Y(:, c) = X(:, c).
// With Krylov states (kst), lanes whose columns of the block's segment have all
// stopped leave their rows of Y as they were.
// Kept lean (32-bit row indices, a column bit mask, the copy-through value
// loaded only at the end) so that the register bound of min_blocks holds
// without spills.
template <typename S, typename V, int TPR, int CPT, bool DIA>
__global__ void __launch_bounds__(256, min_blocks<S, CPT>()) factor_spmv_kernel(SegView sg, PatView pv, const V* __restrict__ f,
                                                          const int* __restrict__ apply, int ld,
                                                          const S* __restrict__ x, S* __restrict__ y,
                                                          const int* done, const KState* __restrict__ kst) {
  if (done && *done) return;
  // three lanes per row (rows of three 16-byte vectors): the threads past the
  // last whole row group of the block have no row
  if constexpr ((TPR & (TPR - 1)) != 0) {
    if ((int)threadIdx.x >= (256 / TPR) * TPR) return;
  }
  typedef typename real_of<S>::type RS;
  typedef typename std::conditional<is_cplx<V>::value, cplx<RS>, RS>::type W;
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
  const bool sell = pv.fmt == FMT_SELL;
  const L2Pol pol = l2_policies();
  for (int r = (int)rb64 + (int)threadIdx.x / TPR; r < re; r += rpb) {
    Pack<S, CPT> acc;
#pragma unroll
    for (int j = 0; j < CPT; ++j) acc.v[j] = zero_<S>();
    // whole chunks of GCH entries, then the remainder (fewer than GCH) as one
    // more chunk, so that a row of c GCH + t entries waits on c + 1 rounds of
    // gathers; the sum runs in storage order (columns ascending) either way.
    // FP32 factor values under FP64 vectors are widened on load (W).
    constexpr int GCH = factor_chunk<S, CPT>();
    static_assert(GCH <= 4, "the remainder below takes at most 3 entries");
    if constexpr (DIA) {
      if (mask) {
      const int nd = pv.ndiag, n = pv.n;
      int d = 0;
      for (; d + GCH <= nd; d += GCH) factor_dia_gather<GCH, S, V, W, CPT>(acc, pv.doff, f, d, r, n, ld, c0, x, pol);
      if constexpr (GCH > 1) {
        const int rem = nd - d;
        if constexpr (GCH > 3) {
          if (rem == 3) factor_dia_gather<3, S, V, W, CPT>(acc, pv.doff, f, d, r, n, ld, c0, x, pol);
        }
        if constexpr (GCH > 2) {
          if (rem == 2) factor_dia_gather<2, S, V, W, CPT>(acc, pv.doff, f, d, r, n, ld, c0, x, pol);
        }
        if (rem == 1) factor_dia_gather<1, S, V, W, CPT>(acc, pv.doff, f, d, r, n, ld, c0, x, pol);
      }
      }
    } else if (mask) {
      int p0, p1, step;
      if (sell) {
        const int64_t base = pv.sptr[r >> 5];
        const int w = (int)((pv.sptr[(r >> 5) + 1] - base) >> 5);
        // SELL positions exceed 32 bits only for > 2^31 stored entries, which the set-up rejects
        p0 = (int)base + (r & 31);
        p1 = p0 + 32 * w;
        step = 32;
      } else {
        p0 = ldh(pv.rowptr + r, pol.last);
        p1 = ldh(pv.rowptr + r + 1, pol.last);
        step = 1;
      }
      int pc = p0;
      for (; pc + (GCH - 1) * step < p1; pc += GCH * step)
        factor_gather<GCH, S, V, W, CPT>(acc, pv.col, f, pc, step, ld, c0, x, pol);
      if constexpr (GCH > 1) {
        const int rem = (p1 - pc) / step;     // 0 .. 3
        if constexpr (GCH > 3) {
          if (rem == 3) factor_gather<3, S, V, W, CPT>(acc, pv.col, f, pc, step, ld, c0, x, pol);
        }
        if constexpr (GCH > 2) {
          if (rem == 2) factor_gather<2, S, V, W, CPT>(acc, pv.col, f, pc, step, ld, c0, x, pol);
        }
        if (rem == 1) factor_gather<1, S, V, W, CPT>(acc, pv.col, f, pc, step, ld, c0, x, pol);
      }
    }
    const int64_t q = (int64_t)r * ld + c0;
    if (mask != (1u << CPT) - 1u) {
      const Pack<S, CPT> xo = ldp<S, CPT>(x + q);
#pragma unroll
      for (int j = 0; j < CPT; ++j) if (!((mask >> j) & 1u)) acc.v[j] = xo.v[j];
    }
    stp<S, CPT>(y + q, acc);
  }
}

}  // namespace

int launch_op_spmv(int st, const SegView& sg, const PatView& pv, const OpVals& ov, const Coef* coefs, int ld,
                   const void* x, void* y, const void* b, const RedArgs* red, cudaStream_t s, int kreal) {
  if (ld < 1 || ld > MOR_LDMAX) return (int)cudaErrorInvalidValue;
  RedArgs ra;
  if (red) ra = *red;
  else { ra.mode = RED_NONE; ra.w = nullptr; ra.part = nullptr; ra.counter = nullptr; ra.fin = 0;
         ra.state = nullptr; ra.out = nullptr; ra.done = nullptr; }
  int e = dispatch_shape(st, ld, [&]<typename S, int TPR, int CPT>() -> int {
    CoefS<S> cf;
    for (int c = 0; c < MOR_LDMAX; ++c) {
      const Coef q = (c < ld) ? coefs[c] : Coef{0, 0, 0, 0};
      if constexpr (is_cplx<S>::value) {
        typedef typename real_of<S>::type R;
        cf.sE[c] = S((R)q.sEr, (R)q.sEi);
        cf.sA[c] = S((R)q.sAr, (R)q.sAi);
      } else {
        cf.sE[c] = (S)q.sEr;
        cf.sA[c] = (S)q.sAr;
      }
    }
    auto run = [&]<bool ECSR, bool DIA, int ND>() {
      OpDiaC<ND> dc{};
      if constexpr (ND > 0) {
        typedef typename real_of<S>::type R;
        for (int d = 0; d < ND; ++d) {
          dc.off[d] = pv.h_doff[d];
          dc.offld[d] = (long long)pv.h_doff[d] * ld;
          dc.ad[d] = (const R*)ov.a + (size_t)d * pv.n;
          dc.ed[d] = ECSR ? (const void*)((const R*)ov.e + (size_t)d * pv.n) : nullptr;
        }
      }
      const SegView g = fit_grid(sg, (const void*)op_spmv_kernel<S, TPR, CPT, ECSR, DIA, ND>, TPR);
      op_spmv_kernel<S, TPR, CPT, ECSR, DIA, ND><<<g.nblocks, 256, 0, s>>>(g, pv, ov, cf, ld, (const S*)x, (S*)y,
                                                                           (const S*)b, ra, dc);
    };
    // the diagonal layout with 5 or 7 diagonals and FP32 / complex64 vectors:
    // the per-diagonal constants by value (OpDiaC)
    auto go = [&]<bool ECSR, bool DIA>() {
      if constexpr (DIA && sizeof(typename real_of<S>::type) == 4 && narrow_slice<S, CPT>()) {
        if (pv.h_doff && pv.ndiag == 7) return run.template operator()<ECSR, true, 7>();
        if (pv.h_doff && pv.ndiag == 5) return run.template operator()<ECSR, true, 5>();
      }
      run.template operator()<ECSR, DIA, 0>();
    };
    const bool dia = pv.fmt == FMT_DIA;
    if (ov.ekind == EK_CSR) {
      if (dia) go.template operator()<true, true>();
      else go.template operator()<true, false>();
    } else {
      if (dia) go.template operator()<false, true>();
      else go.template operator()<false, false>();
    }
    return 0;
  });
  if (e) return e;
  mor_count_launches(1);
  mor_tally(0, st, kreal < 0 ? ld : kreal);
  return (int)cudaGetLastError();
}

// one factor SpMV launch with the lane shape (TPR, CPT) on vectors of type S;
// the factor values are of type fst (FP32 factors may serve FP64 vectors)
template <typename S, int TPR, int CPT>
static int launch_factor_shape(int fst, const SegView& sg, const PatView& pv, const void* fvals, const int* apply,
                               int ld, const void* x, void* y, const int* done, const void* kstate, cudaStream_t s) {
  typedef typename real_of<S>::type R;
  const bool fc = st_is_cplx(fst), f32 = st_is_f32(fst);
  auto go = [&]<typename V>() {
    auto run = [&]<bool DIA>() {
      const SegView g = fit_grid(sg, (const void*)factor_spmv_kernel<S, V, TPR, CPT, DIA>, TPR);
      factor_spmv_kernel<S, V, TPR, CPT, DIA><<<g.nblocks, 256, 0, s>>>(g, pv, (const V*)fvals, apply, ld,
                                                                        (const S*)x, (S*)y, done,
                                                                        (const KState*)kstate);
    };
    if (pv.fmt == FMT_DIA) run.template operator()<true>();
    else run.template operator()<false>();
  };
  if (sizeof(R) == 4 && !f32) return (int)cudaErrorInvalidValue;     // FP64 factors under FP32 vectors
  if constexpr (is_cplx<S>::value) {
    if (fc) {
      if (f32 && sizeof(R) == 8) go.template operator()<cfloat>();
      else go.template operator()<S>();
    } else {
      if (f32 && sizeof(R) == 8) go.template operator()<float>();
      else go.template operator()<R>();
    }
  } else {
    if (fc) return (int)cudaErrorInvalidValue;
    if (f32 && sizeof(R) == 8) go.template operator()<float>();
    else go.template operator()<S>();
  }
  return 0;
}

// Rows of exactly three 16-byte vectors (complex64 k = 5, 6; FP32 k = 9 .. 12;
// ...) get three lanes instead of four with one idle: 85 rows per block pass
// instead of 64.  Measured on the 100^3 chain (complex64, L2 flushed): k = 5
// 56.8 -> 53.8 us, k = 6 56.8 -> 51.7 us.
#ifndef MOR_FACTOR_TPR3
#define MOR_FACTOR_TPR3 1
#endif

int launch_factor_spmv(int st, int fst, const SegView& sg, const PatView& pv, const void* fvals, const int* apply,
                       int ld, const void* x, void* y, const int* done, const void* kstate, cudaStream_t s,
                       int kreal) {
  if (ld < 1 || ld > MOR_LDMAX) return (int)cudaErrorInvalidValue;
  int e = launch_factor_dia_nd(st, fst, sg, pv, fvals, apply, ld, x, y, done, kstate, s);
  if (e == 0) {
    mor_count_launches(1);
    mor_tally(1, st, kreal < 0 ? ld : kreal);
    return (int)cudaGetLastError();
  }
#if MOR_FACTOR_TPR3
  // rows of exactly three 16-byte vectors: three lanes per row (no idle fourth lane)
  if ((int)st_size(st) * ld == 48) {
    switch (st) {
      case ST_F32: e = launch_factor_shape<float, 3, 4>(fst, sg, pv, fvals, apply, ld, x, y, done, kstate, s); break;
      case ST_F64: e = launch_factor_shape<double, 3, 2>(fst, sg, pv, fvals, apply, ld, x, y, done, kstate, s); break;
      case ST_C32: e = launch_factor_shape<cfloat, 3, 2>(fst, sg, pv, fvals, apply, ld, x, y, done, kstate, s); break;
      default: e = launch_factor_shape<cdouble, 3, 1>(fst, sg, pv, fvals, apply, ld, x, y, done, kstate, s); break;
    }
  } else
#endif
  e = dispatch_shape(st, ld, [&]<typename S, int TPR, int CPT>() -> int {
    return launch_factor_shape<S, TPR, CPT>(fst, sg, pv, fvals, apply, ld, x, y, done, kstate, s);
  });
  if (e) return e;
  mor_count_launches(1);
  mor_tally(1, st, kreal < 0 ? ld : kreal);
  return (int)cudaGetLastError();
}
