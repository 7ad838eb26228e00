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
#include <string.h>

#define MOR_LDMAX_DEV 16

enum {
  FIN_NONE = 0,
  FIN_INIT = 1,    // sums: (r_hat, r), ||r||^2        -> rho, active
  FIN_ALPHA = 2,   // sums: (r_hat, v)                  -> alpha = rho / (r_hat, v)
  FIN_OMEGA = 3,   // sums: (t, s), (t, t)              -> omega = (t, s) / (t, t)
  FIN_RHO = 4      // sums: (r_hat, r), ||r||^2         -> convergence, beta
};

enum { KST_OK = 0, KST_NOCONV = 4, KST_BREAKDOWN = 5 };

struct KState {
  cdouble rho, rho_old, alpha, omega, beta;
  double rnorm2, target2;
  int active, iters, maxit, status;
};

// sums[c*2 + q] for column c, reduction q
__device__ inline void krylov_finalize(int stage, int k, const cdouble* sums, KState* st, int* done) {
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
      if (S.rnorm2 <= S.target2) { S.active = 0; S.status = KST_OK; }
      else if (S.iters >= S.maxit) { S.active = 0; S.status = KST_NOCONV; }
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
  if (done) *done = any ? 0 : 1;
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

// Contiguous row range of this block: [r0, r1), processed rpb rows at a time.
__device__ __forceinline__ void block_rows(int64_t n, int rpb, int64_t& r0, int64_t& r1) {
  int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  chunk = (chunk + rpb - 1) / rpb * rpb;
  r0 = (int64_t)blockIdx.x * chunk;
  r1 = r0 + chunk < n ? r0 + chunk : n;
}

// ---------------------------------------------------------------------------
// Reduce two per-column values (v0[j], v1[j]) of the CPT columns lane `sub`
// owns (columns sub * CPT + j; sub = lane % TPR) over the block, write the
// per-block FP64 partials part[(block * 2 ld + 2c + q) * 2 + {re, im}], and
// let the last block (atomic ticket) sum the partials of all blocks in a fixed
// order and run the finalize stage (or write the sums to `out`).  Every thread
// of the block must call it.
template <typename S, int TPR, int CPT>
__device__ inline void col_reduce_finalize(const S (&v0)[CPT], const S (&v1)[CPT], int ld, double* part,
                                           unsigned* counter, int fin, KState* state, cdouble* out, int* done) {
  typedef typename real_of<S>::type R;
  __shared__ double sh[8][2 * MOR_LDMAX_DEV][2];
  __shared__ bool am_last;
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
    part[((size_t)blockIdx.x * nv + threadIdx.x) * 2 + 0] = re;
    part[((size_t)blockIdx.x * nv + threadIdx.x) * 2 + 1] = im;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  // last block: warp w sums values w, w + nwarps, ... over all blocks (lanes stride the blocks)
  __shared__ cdouble sums[2 * MOR_LDMAX_DEV];
  const volatile double* vp = part;
  for (int i = wid; i < nv; i += nwarps) {
    double re = 0.0, im = 0.0;
    for (int blk = lane; blk < (int)gridDim.x; blk += 32) {
      re += vp[((size_t)blk * nv + i) * 2 + 0];
      im += vp[((size_t)blk * nv + i) * 2 + 1];
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) sums[i] = cdouble(re, im);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (fin != FIN_NONE) krylov_finalize(fin, ld, sums, state, done);
    else if (out) for (int i = 0; i < nv; ++i) out[i] = sums[i];
    *counter = 0u;   // ready for the next launch (stream order makes this safe)
  }
}
