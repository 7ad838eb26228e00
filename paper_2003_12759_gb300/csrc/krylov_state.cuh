// Per-column BiCGSTAB state and the scalar "finalize" stages that the last
// block of a fused reduction runs.  The recurrence is right-preconditioned
// BiCGSTAB (Sec. III.A: A P y = b, x = P y) started from x_0 = 0 with
// Hermitian inner products; the scalars are kept in FP64 complex whatever
// the vector precision.
#pragma once
#include "mor_types.cuh"

enum {
  FIN_NONE = 0,
  FIN_INIT = 1,    // sums: (r_hat, r), ||r||^2        -> rho, active
  FIN_ALPHA = 2,   // sums: (r_hat, v)                  -> alpha = rho / (r_hat, v)
  FIN_OMEGA = 3,   // sums: (t, s), (t, t)              -> omega = (t, s) / (t, t)
  FIN_RHO = 4      // sums: (r_hat, r), ||r||^2         -> convergence, beta
};

enum { KST_RUNNING = 0, KST_OK = 0, KST_NOCONV = 4, KST_BREAKDOWN = 5 };

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
  if (stage == FIN_INIT || stage == FIN_RHO || stage == FIN_ALPHA || stage == FIN_OMEGA) {
    if (done) *done = any ? 0 : 1;
  }
}

// ---------------------------------------------------------------------------
// Block reduction of NV per-thread scalars (NV <= 2*MOR_KMAX) of type S into
// FP64 per-block partials, then the last block (by atomic ticket) reduces the
// partials in a fixed order and runs the finalize stage or writes the sums.
// part layout: part[(block * nv + i) * 2 + {re, im}] (doubles).
template <typename S, int NV>
__device__ inline void block_reduce_finalize(const S (&vals)[NV], int nv, double* part,
                                             unsigned* counter, int fin, KState* state,
                                             cdouble* out, int* done, int k) {
  typedef typename real_of<S>::type R;
  __shared__ double sh_re[8][NV];
  __shared__ double sh_im[8][NV];
  __shared__ bool am_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    if (i < nv) {
      R re = warp_sum((R)real_(vals[i]));
      R im = is_cplx<S>::value ? warp_sum((R)imag_(vals[i])) : R(0);
      if (lane == 0) { sh_re[wid][i] = (double)re; sh_im[wid][i] = (double)im; }
    }
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double re = 0.0, im = 0.0;
    for (int w = 0; w < nwarps; ++w) { re += sh_re[w][threadIdx.x]; im += sh_im[w][threadIdx.x]; }
    part[((size_t)blockIdx.x * nv + threadIdx.x) * 2 + 0] = re;
    part[((size_t)blockIdx.x * nv + threadIdx.x) * 2 + 1] = im;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned ticket = atomicAdd(counter, 1u);
    am_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  // last block: thread t sums blocks t, t + blockDim, ... for all nv values
  double acc_re[NV], acc_im[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) { acc_re[i] = 0.0; acc_im[i] = 0.0; }
  const volatile double* vp = part;
  for (int blk = threadIdx.x; blk < (int)gridDim.x; blk += blockDim.x) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      if (i < nv) {
        acc_re[i] += vp[((size_t)blk * nv + i) * 2 + 0];
        acc_im[i] += vp[((size_t)blk * nv + i) * 2 + 1];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    if (i < nv) {
      double re = warp_sum(acc_re[i]);
      double im = warp_sum(acc_im[i]);
      if (lane == 0) { sh_re[wid][i] = re; sh_im[wid][i] = im; }
    }
  }
  __syncthreads();
  __shared__ cdouble sums[NV];
  if (threadIdx.x < nv) {
    double re = 0.0, im = 0.0;
    for (int w = 0; w < nwarps; ++w) { re += sh_re[w][threadIdx.x]; im += sh_im[w][threadIdx.x]; }
    sums[threadIdx.x] = cdouble(re, im);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (fin != FIN_NONE) krylov_finalize(fin, k, sums, state, done);
    else if (out) for (int i = 0; i < nv; ++i) out[i] = sums[i];
    *counter = 0u;   // ready for the next launch (stream order makes this safe)
  }
}
