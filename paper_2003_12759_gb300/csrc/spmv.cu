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

namespace {

template <typename S, int KB> struct CoefS { S sE[KB]; S sA[KB]; };

template <typename S> __device__ __forceinline__ S zero_() { return S(0); }

// [p0, p1) and step of row r in the stored layout
__device__ __forceinline__ void row_range(const PatView& pv, int r, int64_t& p0, int64_t& p1, int& step) {
  if (pv.fmt == FMT_SELL) {
    const int64_t base = pv.sptr[r >> 5];
    const int64_t w = (pv.sptr[(r >> 5) + 1] - base) >> 5;
    p0 = base + (r & 31);
    p1 = p0 + 32 * w;
    step = 32;
  } else {
    p0 = pv.rowptr[r];
    p1 = pv.rowptr[r + 1];
    step = 1;
  }
}

// Y(:, c) = sE_c (E X(:, c)) + sA_c (A X(:, c)) [+ B(:, c)], with an optional
// fused per-column reduction.  KB lanes per row, lane `sub` owns column sub.
template <typename S, int KB>
__global__ void __launch_bounds__(256) op_spmv_kernel(PatView pv, OpVals ov, CoefS<S, KB> cf, int k,
                                                      const S* __restrict__ x, S* __restrict__ y,
                                                      const S* __restrict__ bv, RedArgs red) {
  typedef typename real_of<S>::type R;
  if (red.done && *red.done) return;
  __shared__ S csE[KB], csA[KB];
  if (threadIdx.x < KB) { csE[threadIdx.x] = cf.sE[threadIdx.x]; csA[threadIdx.x] = cf.sA[threadIdx.x]; }
  __syncthreads();
  const R* __restrict__ a = (const R*)ov.a;
  const R* __restrict__ e = (const R*)ov.e;
  const R* __restrict__ ed = (const R*)ov.ediag;
  const S* __restrict__ w = (const S*)red.w;
  const int sub = threadIdx.x & (KB - 1);
  const bool act = sub < k;
  const S sE = csE[sub], sA = csA[sub];
  S v0 = zero_<S>(), v1 = zero_<S>();
  const int rpb = blockDim.x / KB;
  for (int r = blockIdx.x * rpb + threadIdx.x / KB; r < pv.n; r += gridDim.x * rpb) {
    if (!act) continue;
    int64_t p0, p1;
    int step;
    row_range(pv, r, p0, p1, step);
    S accA = zero_<S>(), accE = zero_<S>();
    if (ov.ekind == EK_CSR) {
      for (int64_t p = p0; p < p1; p += step) {
        const int cc = __ldg(pv.col + p);
        const S xv = x[(int64_t)cc * k + sub];
        fma_r(accA, __ldg(a + p), xv);
        fma_r(accE, __ldg(e + p), xv);
      }
    } else {
#pragma unroll 4
      for (int64_t p = p0; p < p1; p += step) {
        const int cc = __ldg(pv.col + p);
        fma_r(accA, __ldg(a + p), x[(int64_t)cc * k + sub]);
      }
      const S xr = x[(int64_t)r * k + sub];
      accE = (ov.ekind == EK_DIAG) ? scale_(__ldg(ed + r), xr) : xr;
    }
    S yv = sE * accE + sA * accA;
    const int64_t q = (int64_t)r * k + sub;
    if (bv) yv += bv[q];
    y[q] = yv;
    if (red.mode == RED_DOT_W) {
      fma_s(v0, conj_(w[q]), yv);
    } else if (red.mode == RED_DOT_TT) {
      fma_s(v0, conj_(yv), w[q]);
      v1 += S(abs2_(yv));
    } else if (red.mode == RED_NORM) {
      v0 += S(abs2_(yv));
    }
  }
  if (red.mode != RED_NONE)
    col_reduce_finalize<S, KB>(v0, v1, k, (double*)red.part, red.counter, red.fin, (KState*)red.state,
                               (cdouble*)red.out, (int*)red.done);
}

// Y(:, c) = F X(:, c) where the factor applies to column c, else Y(:, c) = X(:, c).
template <typename S, typename V, int KB>
__global__ void __launch_bounds__(256) factor_spmv_kernel(PatView pv, const V* __restrict__ f,
                                                          const int* __restrict__ apply, int k,
                                                          const S* __restrict__ x, S* __restrict__ y,
                                                          const int* done) {
  if (done && *done) return;
  const int sub = threadIdx.x & (KB - 1);
  if (sub >= k) return;
  const int ap = apply[sub];
  const int rpb = blockDim.x / KB;
  for (int r = blockIdx.x * rpb + threadIdx.x / KB; r < pv.n; r += gridDim.x * rpb) {
    const int64_t q = (int64_t)r * k + sub;
    if (!ap) { y[q] = x[q]; continue; }
    int64_t p0, p1;
    int step;
    row_range(pv, r, p0, p1, step);
    S acc = zero_<S>();
#pragma unroll 4
    for (int64_t p = p0; p < p1; p += step) {
      const int cc = __ldg(pv.col + p);
      const V fv = f[p];
      if constexpr (is_cplx<V>::value) fma_s(acc, fv, x[(int64_t)cc * k + sub]);
      else fma_r(acc, fv, x[(int64_t)cc * k + sub]);
    }
    y[q] = acc;
  }
}

template <typename S, int KB>
int op_dispatch(const PatView& pv, const OpVals& ov, const Coef* coefs, int k, const void* x, void* y,
                const void* b, const RedArgs* red, int grid_cap, cudaStream_t s) {
  CoefS<S, KB> cf;
  for (int c = 0; c < KB; ++c) {
    const Coef q = (c < k) ? coefs[c] : Coef{0, 0, 0, 0};
    if constexpr (is_cplx<S>::value) {
      typedef typename real_of<S>::type R;
      cf.sE[c] = S((R)q.sEr, (R)q.sEi);
      cf.sA[c] = S((R)q.sAr, (R)q.sAi);
    } else {
      cf.sE[c] = (S)q.sEr;
      cf.sA[c] = (S)q.sAr;
    }
  }
  RedArgs ra;
  if (red) ra = *red;
  else { ra.mode = RED_NONE; ra.w = nullptr; ra.part = nullptr; ra.counter = nullptr; ra.fin = 0;
         ra.state = nullptr; ra.out = nullptr; ra.done = nullptr; }
  const int threads = 256;
  int64_t blocks = ((int64_t)pv.n * KB + threads - 1) / threads;
  if (grid_cap > 0 && blocks > grid_cap) blocks = grid_cap;
  if (blocks < 1) blocks = 1;
  op_spmv_kernel<S, KB><<<(unsigned)blocks, threads, 0, s>>>(pv, ov, cf, k, (const S*)x, (S*)y,
                                                             (const S*)b, ra);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

template <typename S, typename V, int KB>
int factor_dispatch(const PatView& pv, const void* f, const int* apply, int k, const void* x, void* y,
                    const int* done, cudaStream_t s) {
  const int threads = 256;
  int64_t blocks = ((int64_t)pv.n * KB + threads - 1) / threads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  factor_spmv_kernel<S, V, KB><<<(unsigned)blocks, threads, 0, s>>>(pv, (const V*)f, apply, k,
                                                                    (const S*)x, (S*)y, done);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

#define KB_SWITCH(kb, CALL)                 \
  switch (kb) {                             \
    case 1: { constexpr int KBv = 1; return CALL; } \
    case 2: { constexpr int KBv = 2; return CALL; } \
    case 4: { constexpr int KBv = 4; return CALL; } \
    case 8: { constexpr int KBv = 8; return CALL; } \
    case 16: { constexpr int KBv = 16; return CALL; } \
    default: return (int)cudaErrorInvalidValue; \
  }

}  // namespace

int launch_op_spmv(int st, int kb, const PatView& pv, const OpVals& ov, const Coef* coefs, int k,
                   const void* x, void* y, const void* b, const RedArgs* red, int grid_cap,
                   cudaStream_t s) {
  switch (st) {
    case ST_F32: KB_SWITCH(kb, (op_dispatch<float, KBv>(pv, ov, coefs, k, x, y, b, red, grid_cap, s)));
    case ST_F64: KB_SWITCH(kb, (op_dispatch<double, KBv>(pv, ov, coefs, k, x, y, b, red, grid_cap, s)));
    case ST_C32: KB_SWITCH(kb, (op_dispatch<cfloat, KBv>(pv, ov, coefs, k, x, y, b, red, grid_cap, s)));
    case ST_C64: KB_SWITCH(kb, (op_dispatch<cdouble, KBv>(pv, ov, coefs, k, x, y, b, red, grid_cap, s)));
  }
  return (int)cudaErrorInvalidValue;
}

int launch_factor_spmv(int st, bool fcplx, int kb, const PatView& pv, const void* fvals,
                       const int* apply, int k, const void* x, void* y, const int* done,
                       cudaStream_t s) {
  switch (st) {
    case ST_F32: KB_SWITCH(kb, (factor_dispatch<float, float, KBv>(pv, fvals, apply, k, x, y, done, s)));
    case ST_F64: KB_SWITCH(kb, (factor_dispatch<double, double, KBv>(pv, fvals, apply, k, x, y, done, s)));
    case ST_C32:
      if (fcplx) KB_SWITCH(kb, (factor_dispatch<cfloat, cfloat, KBv>(pv, fvals, apply, k, x, y, done, s)))
      else KB_SWITCH(kb, (factor_dispatch<cfloat, float, KBv>(pv, fvals, apply, k, x, y, done, s)));
    case ST_C64:
      if (fcplx) KB_SWITCH(kb, (factor_dispatch<cdouble, cdouble, KBv>(pv, fvals, apply, k, x, y, done, s)))
      else KB_SWITCH(kb, (factor_dispatch<cdouble, double, KBv>(pv, fvals, apply, k, x, y, done, s)));
  }
  return (int)cudaErrorInvalidValue;
}
