// Per-column BiCGSTAB state, the scalar "finalize" stages that the last
// block of a fused reduction runs, and the block/grid reduction used by every
// kernel that reduces per shift column.  The recurrence is right-
// preconditioned BiCGSTAB (Sec. III.A: A P y = b, x = P y) started from
// x_0 = 0 with Hermitian inner products; the scalars are kept in FP64 complex
// whatever the vector precision.
//
// Thread mapping shared by the kernels of the solve: a row of the n x ld
// row-major block is handled by TPR consecutive lanes, lane `sub` owning the
// CPT consecutive columns sub * CPT ... (a 16-byte vector when CPT * size =
// 16); each block walks one contiguous range of rows, so that neighbouring
// rows of a stencil reuse the gathered vector entries from L1.
#pragma once
#include "mor_types.cuh"
#include "mor_internal.h"
#include <string.h>

#define MOR_LDMAX_DEV 16

enum {
  FIN_NONE = 0,
  FIN_INIT = 1,    // sums: (r_hat, r), ||r||^2        -> rho, active
  FIN_ALPHA = 2,   // sums: (r_hat, v)                  -> alpha = rho / (r_hat, v)
  FIN_OMEGA = 3,   // sums: (t, s), (t, t)              -> omega = (t, s) / (t, t)
  FIN_RHO = 4      // sums: (r_hat, r), ||r||^2         -> convergence, beta
};

enum { KST_OK = 0, KST_NOCONV = 4, KST_BREAKDOWN = 5, KST_STAGNATED = 6 };

// stag > 0: a column whose best residual has not dropped by 0.1% for
// max(stag, iterations it took to reach that best) iterations stops with
// KST_STAGNATED (an FP32 inner solve that has reached its working accuracy;
// the FP64 refinement restarts it from the true residual).  The window grows
// with the solve, so that the long plateaus of BiCGSTAB on hard shifts (a few
// hundred iterations after a few hundred of progress) do not stop it.
struct KState {
  cdouble rho, rho_old, alpha, omega, beta;
  double rnorm2, target2, best2;
  int active, iters, maxit, status, best_it, stag;
};

// sums[c*2 + q] for column c, reduction q
__device__ inline int krylov_finalize(int stage, int k, const cdouble* sums, KState* st) {
  int any = 0;
  for (int c = 0; c < k; ++c) {
    KState& S = st[c];
    if (stage == FIN_INIT) {
      S.rho = sums[2 * c];
      S.rho_old = cdouble(1.0);
      S.alpha = cdouble(1.0);
      S.omega = cdouble(1.0);
      S.beta = cdouble(0.0);
      S.rnorm2 = sums[2 * c + 1].re;
      S.best2 = S.rnorm2;
      S.best_it = 0;
      S.iters = 0;
      S.status = KST_OK;
      S.active = (S.rnorm2 > S.target2 && S.maxit > 0) ? 1 : 0;
      if (S.rnorm2 > S.target2 && S.maxit <= 0) S.status = KST_NOCONV;
      if (S.active && S.rho.re == 0.0 && S.rho.im == 0.0) { S.active = 0; S.status = KST_BREAKDOWN; }
    } else if (!S.active) {
      // frozen column
    } else if (stage == FIN_ALPHA) {
      cdouble rv = sums[2 * c];
      if (rv.re == 0.0 && rv.im == 0.0) { S.active = 0; S.status = KST_BREAKDOWN; S.alpha = cdouble(0.0); S.omega = cdouble(0.0); }
      else S.alpha = cdiv(S.rho, rv);
    } else if (stage == FIN_OMEGA) {
      cdouble ts = sums[2 * c];
      double tt = sums[2 * c + 1].re;
      if (tt == 0.0) { S.active = 0; S.status = KST_BREAKDOWN; S.alpha = cdouble(0.0); S.omega = cdouble(0.0); }
      else S.omega = cdouble(ts.re / tt, ts.im / tt);
    } else if (stage == FIN_RHO) {
      S.iters += 1;
      S.rnorm2 = sums[2 * c + 1].re;
      if (S.rnorm2 < 0.999 * S.best2) { S.best2 = S.rnorm2; S.best_it = S.iters; }
      if (S.rnorm2 <= S.target2) { S.active = 0; S.status = KST_OK; }
      else if (S.iters >= S.maxit) { S.active = 0; S.status = KST_NOCONV; }
      else if (S.stag > 0 && S.iters - S.best_it >= max(S.stag, S.best_it)) { S.active = 0; S.status = KST_STAGNATED; }
      else if (!(S.rnorm2 == S.rnorm2)) { S.active = 0; S.status = KST_BREAKDOWN; }   // NaN
      else {
        S.rho_old = S.rho;
        S.rho = sums[2 * c];
        if (S.rho.re == 0.0 && S.rho.im == 0.0) { S.active = 0; S.status = KST_BREAKDOWN; }
        else S.beta = cdiv(S.rho, S.rho_old) * cdiv(S.alpha, S.omega);
      }
    }
    any |= S.active;
  }
  return any;
}

__device__ inline int krylov_any_active(int k, const KState* st) {
  int any = 0;
  for (int c = 0; c < k; ++c) any |= st[c].active;
  return any;
}

// ---------------------------------------------------------------------------
// Vector access to the CPT consecutive columns a lane owns: one 16-byte load
// or store when CPT * sizeof(S) == 16, scalar accesses otherwise.
template <typename S, int CPT> struct Pack { S v[CPT]; };

template <typename S, int CPT>
__device__ __forceinline__ Pack<S, CPT> ldp(const S* p) {
  Pack<S, CPT> o;
  if constexpr (CPT * sizeof(S) == 16) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    memcpy(&o, &t, 16);
  } else {
#pragma unroll
    for (int j = 0; j < CPT; ++j) o.v[j] = p[j];
  }
  return o;
}
template <typename S, int CPT>
__device__ __forceinline__ void stp(S* p, const Pack<S, CPT>& o) {
  if constexpr (CPT * sizeof(S) == 16) {
    float4 t;
    memcpy(&t, &o, 16);
    *reinterpret_cast<float4*>(p) = t;
  } else {
#pragma unroll
    for (int j = 0; j < CPT; ++j) p[j] = o.v[j];
  }
}

// Segment of chunk b and the chunk's row range [r0, r1).  Kernels are
// persistent: a resident wave of blocks walks the chunks b = blockIdx.x,
// blockIdx.x + gridDim.x, ... of the segment table.
__device__ __forceinline__ int seg_of_chunk(const SegView& sg, int b) {
  if (sg.nseg == 1) return 0;
  int lo = 0, hi = sg.nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sg.blk0[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ void chunk_rows(const SegView& sg, int s, int b, int64_t& r0, int64_t& r1) {
  if (sg.nseg == 1) {
    r0 = (int64_t)b * sg.rows_per_block;
    r1 = r0 + sg.rows_per_block < sg.nrows ? r0 + sg.rows_per_block : sg.nrows;
    return;
  }
  r0 = sg.row0[s] + (int64_t)(b - sg.blk0[s]) * sg.rows_per_block;
  const int64_t e = r0 + sg.rows_per_block;
  r1 = e < sg.row0[s + 1] ? e : sg.row0[s + 1];
}

// The block that finishes a segment's last chunk: sum the segment's chunk
// partials in a fixed order and run the finalize stage.  Kept out of line: it
// runs once per segment and launch, so its register needs must not raise the
// allocation (and lower the residency) of the streaming kernels that call it.
static __device__ __noinline__ void seg_finalize(int ld, const SegView& sg, int seg, int b0s, int b1s, double* part, int fin,
                                          KState* state, cdouble* out, int* done) {
  __shared__ __align__(16) double sums_raw[2 * MOR_LDMAX_DEV * 2];
  cdouble* sums = reinterpret_cast<cdouble*>(sums_raw);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int nv = 2 * ld;
  __threadfence();
  // warp w sums values w, w + nwarps, ... over the segment's chunks
  const volatile double* vp = part;
  for (int i = wid; i < nv; i += nwarps) {
    double re = 0.0, im = 0.0;
    for (int blk = b0s + lane; blk < b1s; blk += 32) {
      re += vp[((size_t)blk * nv + i) * 2 + 0];
      im += vp[((size_t)blk * nv + i) * 2 + 1];
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) sums[i] = cdouble(re, im);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (fin != FIN_NONE) {
      KState* st = state + (size_t)seg * ld;
      const int was = (fin == FIN_INIT) ? 0 : krylov_any_active(ld, st);
      const int now = krylov_finalize(fin, ld, sums, st);
      if (fin == FIN_INIT) {
        if (now) atomicAdd(sg.live, 1);
      } else if (was && !now) {
        if (atomicSub(sg.live, 1) == 1 && done) *done = 1;
      }
    } else if (out) {
      for (int i = 0; i < nv; ++i) out[(size_t)seg * nv + i] = sums[i];
    }
    sg.counters[seg] = 0u;   // ready for the next launch (stream order makes this safe)
  }
}

// ---------------------------------------------------------------------------
// Reduce two per-column values (v0[j], v1[j]) of the CPT columns lane `sub`
// owns (columns sub * CPT + j; sub = lane % TPR) over the block for chunk
// `chunk`, write the chunk's FP64 partials part[(chunk * 2 ld + 2c + q) * 2 +
// {re, im}], and let the block that finishes the last chunk of segment `seg`
// (ticket counters[seg]) sum the segment's partials in a fixed order and run
// the finalize stage on that segment's states (or write the sums to
// out[seg * 2 ld ...]).  The finalize keeps sg.live (segments with an active
// column) and `done` (no segment active) current.  Every thread of the block
// must call it, once per chunk.
template <typename S, int TPR, int CPT>
__device__ inline void col_reduce_finalize(const S (&v0)[CPT], const S (&v1)[CPT], int ld, const SegView& sg, int seg,
                                           int chunk, double* part, int fin, KState* state, cdouble* out, int* done) {
  typedef typename real_of<S>::type R;
  __shared__ double sh[8][2 * MOR_LDMAX_DEV][2];
  __shared__ bool am_last;
  __syncthreads();   // the shared buffers are reused chunk after chunk
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int nv = 2 * ld;
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    R a0 = (R)real_(v0[j]), b0 = (R)imag_(v0[j]), a1 = (R)real_(v1[j]), b1 = (R)imag_(v1[j]);
#pragma unroll
    for (int o = 16; o >= TPR; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      b0 += __shfl_xor_sync(0xffffffffu, b0, o);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
      b1 += __shfl_xor_sync(0xffffffffu, b1, o);
    }
    const int c = lane * CPT + j;
    if (lane < TPR && c < ld) {
      sh[wid][2 * c][0] = (double)a0;
      sh[wid][2 * c][1] = (double)b0;
      sh[wid][2 * c + 1][0] = (double)a1;
      sh[wid][2 * c + 1][1] = (double)b1;
    }
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double re = 0.0, im = 0.0;
    for (int w = 0; w < nwarps; ++w) { re += sh[w][threadIdx.x][0]; im += sh[w][threadIdx.x][1]; }
    part[((size_t)chunk * nv + threadIdx.x) * 2 + 0] = re;
    part[((size_t)chunk * nv + threadIdx.x) * 2 + 1] = im;
  }
  __threadfence();
  __syncthreads();
  const int b0s = sg.nseg == 1 ? 0 : sg.blk0[seg];
  const int b1s = sg.nseg == 1 ? sg.nblocks : sg.blk0[seg + 1];
  if (threadIdx.x == 0) am_last = (atomicAdd(sg.counters + seg, 1u) == (unsigned)(b1s - b0s - 1));
  __syncthreads();
  if (!am_last) return;
  seg_finalize(ld, sg, seg, b0s, b1s, part, fin, state, out, done);
}
