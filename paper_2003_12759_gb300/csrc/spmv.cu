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

template <typename S> __device__ __forceinline__ S mk_coef(double re, double im);
template <> __device__ __forceinline__ float mk_coef<float>(double re, double) { return (float)re; }
template <> __device__ __forceinline__ double mk_coef<double>(double re, double) { return re; }
template <> __device__ __forceinline__ cfloat mk_coef<cfloat>(double re, double im) { return cfloat((float)re, (float)im); }
template <> __device__ __forceinline__ cdouble mk_coef<cdouble>(double re, double im) { return cdouble(re, im); }

template <typename S> __device__ __forceinline__ S zero_() { return S(0); }

// one row of the operator: accumulate A x and E x for all k columns
template <typename S, int KB>
__device__ __forceinline__ void op_row(const PatView& pv, int ekind, const typename real_of<S>::type* __restrict__ a,
                                       const typename real_of<S>::type* __restrict__ e,
                                       const typename real_of<S>::type* __restrict__ ed, int k,
                                       const S* __restrict__ x, int r, S (&accA)[KB], S (&accE)[KB]) {
  typedef typename real_of<S>::type R;
#pragma unroll
  for (int c = 0; c < KB; ++c) { accA[c] = zero_<S>(); accE[c] = zero_<S>(); }
  int64_t p0, p1, step;
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
  for (int64_t p = p0; p < p1; p += step) {
    const int cc = __ldg(pv.col + p);
    const R av = __ldg(a + p);
    const S* xr = x + (int64_t)cc * k;
    if (ekind == EK_CSR) {
      const R ev = __ldg(e + p);
#pragma unroll
      for (int c = 0; c < KB; ++c)
        if (c < k) { S xv = xr[c]; fma_r(accA[c], av, xv); fma_r(accE[c], ev, xv); }
    } else {
#pragma unroll
      for (int c = 0; c < KB; ++c)
        if (c < k) fma_r(accA[c], av, xr[c]);
    }
  }
  if (ekind == EK_DIAG) {
    const R d = __ldg(ed + r);
#pragma unroll
    for (int c = 0; c < KB; ++c)
      if (c < k) accE[c] = scale_(d, x[(int64_t)r * k + c]);
  } else if (ekind == EK_IDENTITY) {
#pragma unroll
    for (int c = 0; c < KB; ++c)
      if (c < k) accE[c] = x[(int64_t)r * k + c];
  }
}

template <typename S, int KB>
__global__ void __launch_bounds__(256) op_spmv_kernel(PatView pv, OpVals ov, CoefS<S, KB> cf, int k,
                                                      const S* __restrict__ x, S* __restrict__ y,
                                                      const S* __restrict__ bv, RedArgs red) {
  typedef typename real_of<S>::type R;
  if (red.done && *red.done) return;
  const R* a = (const R*)ov.a;
  const R* e = (const R*)ov.e;
  const R* ed = (const R*)ov.ediag;
  const S* w = (const S*)red.w;
  S vals[2 * KB];
#pragma unroll
  for (int i = 0; i < 2 * KB; ++i) vals[i] = zero_<S>();
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < pv.n; r += gridDim.x * blockDim.x) {
    S accA[KB], accE[KB];
    op_row<S, KB>(pv, ov.ekind, a, e, ed, k, x, r, accA, accE);
#pragma unroll
    for (int c = 0; c < KB; ++c) {
      if (c < k) {
        S yv = cf.sE[c] * accE[c] + cf.sA[c] * accA[c];
        if (bv) yv += bv[(int64_t)r * k + c];
        y[(int64_t)r * k + c] = yv;
        if (red.mode == RED_DOT_W) {
          fma_s(vals[2 * c], conj_(w[(int64_t)r * k + c]), yv);
        } else if (red.mode == RED_DOT_TT) {
          fma_s(vals[2 * c], conj_(yv), w[(int64_t)r * k + c]);
          vals[2 * c + 1] += S(abs2_(yv));
        } else if (red.mode == RED_NORM) {
          vals[2 * c] += S(abs2_(yv));
        }
      }
    }
  }
  if (red.mode != RED_NONE)
    block_reduce_finalize<S, 2 * KB>(vals, 2 * k, (double*)red.part, red.counter, red.fin,
                                     (KState*)red.state, (cdouble*)red.out, (int*)red.done, k);
}

template <typename S, typename V, int KB>
__global__ void __launch_bounds__(256) factor_spmv_kernel(PatView pv, const V* __restrict__ f,
                                                          const int* __restrict__ apply, int k,
                                                          const S* __restrict__ x, S* __restrict__ y,
                                                          const int* done) {
  if (done && *done) return;
  int ap[KB];
#pragma unroll
  for (int c = 0; c < KB; ++c) ap[c] = (c < k) ? apply[c] : 0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < pv.n; r += gridDim.x * blockDim.x) {
    S acc[KB];
#pragma unroll
    for (int c = 0; c < KB; ++c) acc[c] = zero_<S>();
    int64_t p0, p1, step;
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
    for (int64_t p = p0; p < p1; p += step) {
      const int cc = __ldg(pv.col + p);
      const V fv = f[p];
      const S* xr = x + (int64_t)cc * k;
#pragma unroll
      for (int c = 0; c < KB; ++c)
        if (c < k) {
          if constexpr (is_cplx<V>::value) fma_s(acc[c], fv, xr[c]);
          else fma_r(acc[c], fv, xr[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < KB; ++c)
      if (c < k) y[(int64_t)r * k + c] = ap[c] ? acc[c] : x[(int64_t)r * k + c];
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
  int64_t blocks = ((int64_t)pv.n + threads - 1) / threads;
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
  int64_t blocks = ((int64_t)pv.n + threads - 1) / threads;
  if (blocks > 152 * 16) blocks = 152 * 16;
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
