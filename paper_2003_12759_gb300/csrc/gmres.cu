// Restarted right-preconditioned GMRES(m) for k shift columns in lock step
// (the Krylov method of the paper's experiments, Sec. IV; GMRES with right
// preconditioning as in Saad 2003, Sec. 9.3.2): Arnoldi on A(sigma) P, the
// least-squares problem by Givens rotations, x += P V_k y_k at every restart.
//
// GPU form of one Arnoldi step j (all columns of the batch at once):
//   z  = P v_j                           chain of factor SpMVs
//   w  = A(sigma) z                      operator SpMV
//   h  = V_{0..j}^H w;  w -= V h         CGS, fused multi-dot / multi-axpy
//   h' = V_{0..j}^H w;  w -= V h', ||w|| CGS re-orthogonalisation (CGS2);
//                                        the last block applies the Givens
//                                        rotations in FP64 (gm_finalize)
//   v_{j+1} = w / ||w||                  scale
// CGS2 reads each basis vector four times per step, no more than modified
// Gram-Schmidt's j dot/axpy pairs, but in four fused passes instead of 2 j
// dependent ones; both orthogonalise to working accuracy.
// Per-column scalars (rotations, g, H, y) are FP64 complex in device memory;
// columns whose residual estimate met the target stop iterating (their
// basis vectors are zeroed), and every Arnoldi kernel returns at once when no
// column iterates, so a whole cycle is replayed from one captured graph.
#include "mor_internal.h"
#include "krylov_state.cuh"

#include "shape_dispatch.cuh"

namespace {

struct GState {
  int active;        // iterating in the current cycle
  int conv;          // residual estimate met the target
  int k;             // Arnoldi steps of the current cycle
  int iters, maxit, status;
  int enabled;       // column takes part in this inner solve
  int pad;
  double target2;    // squared target on the inner residual norm
  double inv_next;   // 1 / ||w|| of the last step, 0 once the column stopped
  double cs[GM_MMAX];
  cdouble sn[GM_MMAX];
  cdouble g[GM_MMAX + 1];
};

template <typename S> __device__ __forceinline__ S cd_to(cdouble z);
template <> __device__ __forceinline__ float cd_to<float>(cdouble z) { return (float)z.re; }
template <> __device__ __forceinline__ double cd_to<double>(cdouble z) { return z.re; }
template <> __device__ __forceinline__ cfloat cd_to<cfloat>(cdouble z) { return cfloat((float)z.re, (float)z.im); }
template <> __device__ __forceinline__ cdouble cd_to<cdouble>(cdouble z) { return z; }

template <typename S> __device__ __forceinline__ cdouble to_cd(S v) { return cdouble((double)real_(v), (double)imag_(v)); }

// basis vectors accumulated per register pass of the multi-dot kernel
template <typename S, int CPT> constexpr int dot_block() {
  constexpr int b = (int)(CPT * sizeof(S));
  return b <= 16 ? 8 : (b <= 32 ? 4 : (b <= 64 ? 2 : 1));
}

// Sum v[j] (the lane's columns sub * CPT + j) over the block; afterwards
// thread c < ld holds the block sum of column c.  All threads must call it.
template <typename S, int TPR, int CPT>
__device__ __forceinline__ cdouble block_col_sum(const S (&v)[CPT], int ld) {
  typedef typename real_of<S>::type R;
  __shared__ double sh[8][MOR_LDMAX_DEV][2];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    R a = (R)real_(v[j]), b = (R)imag_(v[j]);
#pragma unroll
    for (int o = 16; o >= TPR; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int c = lane * CPT + j;
    if (lane < TPR && c < ld) { sh[wid][c][0] = (double)a; sh[wid][c][1] = (double)b; }
  }
  __syncthreads();
  cdouble out(0.0, 0.0);
  if ((int)threadIdx.x < ld)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { out.re += sh[w][threadIdx.x][0]; out.im += sh[w][threadIdx.x][1]; }
  return out;
}

// Ticket on *counter: true in the block that finished last (all partials visible).
__device__ __forceinline__ bool last_block(unsigned* counter) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

#define GM_LANE_SETUP                                   \
  const int sub = threadIdx.x % TPR;                   \
  const int c0 = sub * CPT;                            \
  const int rpb = blockDim.x / TPR;                    \
  int64_t rb, re;                                      \
  chunk_rows(sg, 0, blockIdx.x, rb, re);

// out[i * ld + c] = (V_i(:, c), w(:, c)) for i < nv (Hermitian inner products)
template <typename S, int TPR, int CPT>
__global__ void __launch_bounds__(256) gm_dot_kernel(SegView sg, int ld, const S* __restrict__ V, int64_t vstride,
                                                     int nv, const S* __restrict__ w, double* part, unsigned* counter,
                                                     cdouble* out, const int* done) {
  if (*done) return;
  GM_LANE_SETUP
  constexpr int IB = dot_block<S, CPT>();
  for (int i0 = 0; i0 < nv; i0 += IB) {
    S acc[IB][CPT];
#pragma unroll
    for (int b = 0; b < IB; ++b)
#pragma unroll
      for (int j = 0; j < CPT; ++j) acc[b][j] = S(0);
    if (c0 < ld) {
      for (int64_t r = rb + threadIdx.x / TPR; r < re; r += rpb) {
        const int64_t q = r * ld + c0;
        const Pack<S, CPT> wv = ldp<S, CPT>(w + q);
#pragma unroll
        for (int b = 0; b < IB; ++b) {
          if (i0 + b < nv) {
            const Pack<S, CPT> vv = ldp<S, CPT>(V + (int64_t)(i0 + b) * vstride + q);
#pragma unroll
            for (int j = 0; j < CPT; ++j) fma_s(acc[b][j], conj_(vv.v[j]), wv.v[j]);
          }
        }
      }
    }
#pragma unroll
    for (int b = 0; b < IB; ++b) {
      if (i0 + b >= nv) break;
      const cdouble s = block_col_sum<S, TPR, CPT>(acc[b], ld);
      if ((int)threadIdx.x < ld) {
        double* p = part + (((size_t)blockIdx.x * nv + i0 + b) * ld + threadIdx.x) * 2;
        p[0] = s.re;
        p[1] = s.im;
      }
    }
  }
  if (!last_block(counter)) return;
  const volatile double* vp = part;
  for (int t = threadIdx.x; t < nv * ld; t += blockDim.x) {
    double re2 = 0.0, im2 = 0.0;
    for (int blk = 0; blk < (int)gridDim.x; ++blk) {
      re2 += vp[((size_t)blk * nv * ld + t) * 2 + 0];
      im2 += vp[((size_t)blk * nv * ld + t) * 2 + 1];
    }
    out[t] = cdouble(re2, im2);
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
}

// Givens step of column c after the two CGS passes (h = h1 + h2, ||w||^2 = nrm2).
__device__ __noinline__ void gm_finalize(int ld, int m, const cdouble* h1, const cdouble* h2, const double* nrm2,
                                         GState* st, cdouble* H, int* done) {
  const int c = threadIdx.x;
  if (c < ld) {
    GState& S = st[c];
    if (S.active) {
      const int j = S.k;
      const int M1 = m + 1;
      cdouble* Hc = H + (size_t)c * M1 * m + (size_t)j * M1;
      const double hn = sqrt(nrm2[c]);
      // previous rotations, carried down the column
      cdouble hp = h1[c] + h2[c];
      for (int i = 0; i < j; ++i) {
        const cdouble hi1 = h1[(i + 1) * ld + c] + h2[(i + 1) * ld + c];
        const cdouble t = S.cs[i] * hp + S.sn[i] * hi1;
        hp = S.cs[i] * hi1 - conj_(S.sn[i]) * hp;
        Hc[i] = t;
      }
      // new rotation annihilating ||w|| below the diagonal
      const double aa = sqrt(abs2_(hp));
      const double den = sqrt(aa * aa + hn * hn);
      double csj;
      cdouble snj;
      if (den == 0.0) { csj = 1.0; snj = cdouble(0.0, 0.0); }
      else if (aa == 0.0) { csj = 0.0; snj = cdouble(1.0, 0.0); }
      else { csj = aa / den; snj = cdouble(hp.re / aa * hn / den, hp.im / aa * hn / den); }
      Hc[j] = csj * hp + snj * cdouble(hn, 0.0);
      S.cs[j] = csj;
      S.sn[j] = snj;
      const cdouble gj = S.g[j];
      S.g[j + 1] = -(conj_(snj) * gj);
      S.g[j] = csj * gj;
      S.k = j + 1;
      S.iters += 1;
      const bool finite = (hn == hn) && (S.g[j + 1].re == S.g[j + 1].re);
      const bool conv = finite && (abs2_(S.g[j + 1]) <= S.target2 || hn == 0.0);
      S.inv_next = (finite && hn > 0.0) ? 1.0 / hn : 0.0;
      if (!finite) { S.active = 0; S.status = KST_BREAKDOWN; }
      else if (conv) { S.active = 0; S.conv = 1; }
      else if (S.iters >= S.maxit || S.k >= m) { S.active = 0; }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int any = 0;
    for (int q = 0; q < ld; ++q) any |= st[q].active;
    if (!any) *done = 1;
  }
}

// w = w - sum_i coef_i V_i (mode 0) or w = sum_i coef_i V_i (mode 1), i < nv.
// fin != 0: also ||w||^2 per column, then the Givens step in the last block.
template <typename S, int TPR, int CPT>
__global__ void __launch_bounds__(256) gm_axpy_kernel(SegView sg, int ld, const S* __restrict__ V, int64_t vstride,
                                                      int nv, const cdouble* coef, S* __restrict__ w, int mode, int fin,
                                                      double* part, unsigned* counter, GState* st, cdouble* H, int m,
                                                      const cdouble* h1, const cdouble* h2, int* done) {
  if (done && *done) return;
  __shared__ __align__(16) unsigned char cbuf[(GM_MMAX + 1) * MOR_LDMAX_DEV * sizeof(S)];
  S* cs = reinterpret_cast<S*>(cbuf);
  for (int t = threadIdx.x; t < nv * ld; t += blockDim.x) cs[t] = cd_to<S>(coef[t]);
  __syncthreads();
  GM_LANE_SETUP
  S nacc[CPT];
#pragma unroll
  for (int j = 0; j < CPT; ++j) nacc[j] = S(0);
  if (c0 < ld) {
    for (int64_t r = rb + threadIdx.x / TPR; r < re; r += rpb) {
      const int64_t q = r * ld + c0;
      Pack<S, CPT> acc;
      if (mode == 0) acc = ldp<S, CPT>(w + q);
      else {
#pragma unroll
        for (int j = 0; j < CPT; ++j) acc.v[j] = S(0);
      }
      for (int i = 0; i < nv; ++i) {
        const Pack<S, CPT> vv = ldp<S, CPT>(V + (int64_t)i * vstride + q);
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          if (mode == 0) acc.v[j] -= cs[i * ld + c0 + j] * vv.v[j];
          else fma_s(acc.v[j], cs[i * ld + c0 + j], vv.v[j]);
        }
      }
      stp<S, CPT>(w + q, acc);
      if (fin) {
#pragma unroll
        for (int j = 0; j < CPT; ++j) nacc[j] += S(abs2_(acc.v[j]));
      }
    }
  }
  if (!fin) return;
  const cdouble s = block_col_sum<S, TPR, CPT>(nacc, ld);
  if ((int)threadIdx.x < ld) part[(size_t)blockIdx.x * ld + threadIdx.x] = s.re;
  if (!last_block(counter)) return;
  __shared__ double nrm2[MOR_LDMAX_DEV];
  const volatile double* vp = part;
  if ((int)threadIdx.x < ld) {
    double a = 0.0;
    for (int blk = 0; blk < (int)gridDim.x; ++blk) a += vp[(size_t)blk * ld + threadIdx.x];
    nrm2[threadIdx.x] = a;
  }
  __syncthreads();
  gm_finalize(ld, m, h1, h2, nrm2, st, H, done);
  if (threadIdx.x == 0) *counter = 0u;
}

// v = w / ||w|| for iterating columns (scale from the state), 0 for the others
template <typename S, int TPR, int CPT>
__global__ void __launch_bounds__(256) gm_scale_kernel(SegView sg, int ld, const S* __restrict__ w, S* __restrict__ v,
                                                       const GState* st, int use_active, const int* done) {
  if (done && *done) return;
  GM_LANE_SETUP
  if (c0 >= ld) return;
  typedef typename real_of<S>::type R;
  R sc[CPT];
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    const GState& G = st[c0 + j];
    sc[j] = (R)((use_active ? G.active : 1) ? G.inv_next : 0.0);
  }
  for (int64_t r = rb + threadIdx.x / TPR; r < re; r += rpb) {
    const int64_t q = r * ld + c0;
    Pack<S, CPT> a = ldp<S, CPT>(w + q);
#pragma unroll
    for (int j = 0; j < CPT; ++j) a.v[j] = (sc[j] == R(0)) ? S(0) : scale_(sc[j], a.v[j]);
    stp<S, CPT>(v + q, a);
  }
}

template <typename S, int TPR, int CPT>
__global__ void __launch_bounds__(256) gm_add_kernel(SegView sg, int ld, S* __restrict__ x, const S* __restrict__ z) {
  GM_LANE_SETUP
  if (c0 >= ld) return;
  for (int64_t r = rb + threadIdx.x / TPR; r < re; r += rpb) {
    const int64_t q = r * ld + c0;
    Pack<S, CPT> a = ldp<S, CPT>(x + q);
    const Pack<S, CPT> b = ldp<S, CPT>(z + q);
#pragma unroll
    for (int j = 0; j < CPT; ++j) a.v[j] += b.v[j];
    stp<S, CPT>(x + q, a);
  }
}

// Start of a cycle, one thread per column: beta = ||r||, g = beta e_1, the
// scale 1 / beta for v_0, and which columns iterate.  first != 0 also loads
// the column's target and iteration budget.
__global__ void gm_begin_kernel(int ld, const cdouble* sums, GState* st, const double* target, const int* maxit,
                                const int* enabled, int first, int* done_cycle, int* done_all) {
  const int c = threadIdx.x;
  if (c < ld) {
    GState& S = st[c];
    if (first) {
      S.iters = 0;
      S.maxit = maxit[c];
      S.target2 = target[c] * target[c];
      S.status = KST_OK;
      S.enabled = enabled[c];
    }
    const double b2 = sums[2 * c].re;
    const double beta = sqrt(b2);
    S.k = 0;
    for (int i = 0; i <= GM_MMAX; ++i) S.g[i] = cdouble(0.0, 0.0);
    S.g[0] = cdouble(beta, 0.0);
    S.conv = (b2 <= S.target2) ? 1 : 0;
    const bool finite = (b2 == b2);
    if (!finite) S.status = KST_BREAKDOWN;
    S.active = (S.enabled && finite && !S.conv && S.iters < S.maxit && S.status == KST_OK) ? 1 : 0;
    if (S.enabled && !S.conv && S.iters >= S.maxit && S.status == KST_OK) S.status = KST_NOCONV;
    S.inv_next = (S.active && beta > 0.0) ? 1.0 / beta : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int any = 0;
    for (int q = 0; q < ld; ++q) any |= st[q].active;
    *done_cycle = any ? 0 : 1;
    *done_all = any ? 0 : 1;
  }
}

// y = R^{-1} g per column (R the rotated k x k Hessenberg block), written as
// the coefficients ycoef[i * ld + c] (0 beyond k) of x += P V y; the
// columns that took steps resume iterating in the next cycle.
__global__ void gm_solve_y_kernel(int ld, int m, GState* st, const cdouble* H, cdouble* ycoef) {
  const int c = threadIdx.x;
  if (c >= ld) return;
  GState& S = st[c];
  const int k = S.k;
  const int M1 = m + 1;
  const cdouble* Hc = H + (size_t)c * M1 * m;
  for (int i = m - 1; i >= 0; --i) {
    if (i >= k) { ycoef[i * ld + c] = cdouble(0.0, 0.0); continue; }
    cdouble s = S.g[i];
    for (int l = i + 1; l < k; ++l) s = s - Hc[(size_t)l * M1 + i] * ycoef[l * ld + c];
    const cdouble d = Hc[(size_t)i * M1 + i];
    ycoef[i * ld + c] = (d.re == 0.0 && d.im == 0.0) ? cdouble(0.0, 0.0) : cdiv(s, d);
  }
}

}  // namespace

size_t gmres_state_bytes() { return sizeof(GState); }
int gmres_state_iters(const void* s) { return ((const GState*)s)->iters; }
int gmres_state_status(const void* s) { return ((const GState*)s)->status; }
int gmres_state_conv(const void* s) { return ((const GState*)s)->conv; }

int gmres_launch_dot(int st, const SegView& sg, int ld, const void* V, int64_t vstride, int nv, const void* w,
                     double* part, unsigned* counter, void* out, const int* done, cudaStream_t s) {
  if (sg.nseg != 1 || nv < 1 || nv > GM_MMAX + 1) return (int)cudaErrorInvalidValue;
  int e = dispatch_shape(st, ld, [&]<typename S, int TPR, int CPT>() -> int {
    const SegView g = fit_grid(sg, (const void*)gm_dot_kernel<S, TPR, CPT>, TPR);
    gm_dot_kernel<S, TPR, CPT><<<g.nblocks, 256, 0, s>>>(g, ld, (const S*)V, vstride, nv, (const S*)w, part, counter,
                                                        (cdouble*)out, done);
    return 0;
  });
  if (e) return e;
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int gmres_launch_axpy(int st, const SegView& sg, int ld, const void* V, int64_t vstride, int nv, const void* coef,
                      void* w, int mode, int fin, double* part, unsigned* counter, void* state, void* H, int m,
                      const void* h1, const void* h2, int* done, cudaStream_t s) {
  if (sg.nseg != 1 || nv < 1 || nv > GM_MMAX + 1) return (int)cudaErrorInvalidValue;
  int e = dispatch_shape(st, ld, [&]<typename S, int TPR, int CPT>() -> int {
    const SegView g = fit_grid(sg, (const void*)gm_axpy_kernel<S, TPR, CPT>, TPR);
    gm_axpy_kernel<S, TPR, CPT><<<g.nblocks, 256, 0, s>>>(g, ld, (const S*)V, vstride, nv, (const cdouble*)coef, (S*)w,
                                                         mode, fin, part, counter, (GState*)state, (cdouble*)H, m,
                                                         (const cdouble*)h1, (const cdouble*)h2, done);
    return 0;
  });
  if (e) return e;
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int gmres_launch_scale(int st, const SegView& sg, int ld, const void* w, void* v, const void* state, int use_active,
                       const int* done, cudaStream_t s) {
  int e = dispatch_shape(st, ld, [&]<typename S, int TPR, int CPT>() -> int {
    const SegView g = fit_grid(sg, (const void*)gm_scale_kernel<S, TPR, CPT>, TPR);
    gm_scale_kernel<S, TPR, CPT><<<g.nblocks, 256, 0, s>>>(g, ld, (const S*)w, (S*)v, (const GState*)state, use_active,
                                                          done);
    return 0;
  });
  if (e) return e;
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int gmres_launch_add(int st, const SegView& sg, int ld, void* x, const void* z, cudaStream_t s) {
  int e = dispatch_shape(st, ld, [&]<typename S, int TPR, int CPT>() -> int {
    const SegView g = fit_grid(sg, (const void*)gm_add_kernel<S, TPR, CPT>, TPR);
    gm_add_kernel<S, TPR, CPT><<<g.nblocks, 256, 0, s>>>(g, ld, (S*)x, (const S*)z);
    return 0;
  });
  if (e) return e;
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int gmres_launch_begin(int ld, const void* sums, void* state, const double* target, const int* maxit,
                       const int* enabled, int first, int* done_cycle, int* done_all, cudaStream_t s) {
  gm_begin_kernel<<<1, 32, 0, s>>>(ld, (const cdouble*)sums, (GState*)state, target, maxit, enabled, first, done_cycle,
                                   done_all);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int gmres_launch_solve_y(int ld, int m, void* state, const void* H, void* ycoef, cudaStream_t s) {
  gm_solve_y_kernel<<<1, 32, 0, s>>>(ld, m, (GState*)state, (const cdouble*)H, (cdouble*)ycoef);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}
