// Vector kernels of the right-preconditioned BiCGSTAB iteration with fused
// reductions, the FP64 iterative-refinement kernels, and layout conversions.
//
// One BiCGSTAB iteration for k columns in lock step (Sec. III.A; van der
// Vorst's BiCGSTAB applied to A P y = b, x = P y):
//   p  = r + beta (p - omega v)           update_p
//   ph = P p                               chain of factor SpMVs
//   v  = A(sigma) ph,  (r_hat, v)          operator SpMV + FIN_ALPHA
//   s  = r - alpha v                       update_s
//   sh = P s                               chain
//   t  = A(sigma) sh,  (t, s), (t, t)      operator SpMV + FIN_OMEGA
//   x += alpha ph + omega sh,  r = s - omega t,  (r_hat, r), ||r||^2
//                                          update_xr + FIN_RHO
// Scalars live in device memory (KState); columns that converged or broke
// down are frozen; every kernel returns at once when the whole batch is done,
// so a captured graph of several iterations can be replayed blindly.
#include "mor_internal.h"
#include "krylov_state.cuh"

namespace {

template <typename S> __device__ __forceinline__ S from_cd(cdouble z);
template <> __device__ __forceinline__ float from_cd<float>(cdouble z) { return (float)z.re; }
template <> __device__ __forceinline__ double from_cd<double>(cdouble z) { return z.re; }
template <> __device__ __forceinline__ cfloat from_cd<cfloat>(cdouble z) { return cfloat((float)z.re, (float)z.im); }
template <> __device__ __forceinline__ cdouble from_cd<cdouble>(cdouble z) { return z; }

inline int grid_for(int64_t n, int cap) {
  int64_t b = (n + 255) / 256;    // n = number of threads wanted
  if (cap > 0 && b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

template <typename S, int KB>
__global__ void __launch_bounds__(256) update_p_kernel(int n, int k, const S* __restrict__ r, S* __restrict__ p,
                                                       const S* __restrict__ v, const KState* st, const int* done) {
  if (*done) return;
  const int sub = threadIdx.x & (KB - 1);
  if (sub >= k || !st[sub].active) return;
  const S beta = from_cd<S>(st[sub].beta), omega = from_cd<S>(st[sub].omega);
  const int rpb = blockDim.x / KB;
  for (int64_t i = blockIdx.x * (int64_t)rpb + threadIdx.x / KB; i < n; i += (int64_t)gridDim.x * rpb) {
    const int64_t q = i * k + sub;
    p[q] = r[q] + beta * (p[q] - omega * v[q]);
  }
}

template <typename S, int KB>
__global__ void __launch_bounds__(256) update_s_kernel(int n, int k, const S* __restrict__ r, const S* __restrict__ v,
                                                       S* __restrict__ sv, const KState* st, const int* done) {
  if (*done) return;
  const int sub = threadIdx.x & (KB - 1);
  if (sub >= k) return;
  const int act = st[sub].active;
  const S alpha = from_cd<S>(st[sub].alpha);
  const int rpb = blockDim.x / KB;
  for (int64_t i = blockIdx.x * (int64_t)rpb + threadIdx.x / KB; i < n; i += (int64_t)gridDim.x * rpb) {
    const int64_t q = i * k + sub;
    sv[q] = act ? r[q] - alpha * v[q] : r[q];
  }
}

template <typename S, int KB>
__global__ void __launch_bounds__(256) update_xr_kernel(int n, int k, S* __restrict__ x, S* __restrict__ r,
                                                        const S* __restrict__ ph, const S* __restrict__ sh,
                                                        const S* __restrict__ sv, const S* __restrict__ t,
                                                        const S* __restrict__ rhat, double* part, unsigned* counter,
                                                        KState* st, int* done) {
  if (*done) return;
  const int sub = threadIdx.x & (KB - 1);
  const bool act = sub < k && st[sub].active;
  const S alpha = act ? from_cd<S>(st[sub].alpha) : S(0);
  const S omega = act ? from_cd<S>(st[sub].omega) : S(0);
  S v0 = S(0), v1 = S(0);
  const int rpb = blockDim.x / KB;
  if (act) {
    for (int64_t i = blockIdx.x * (int64_t)rpb + threadIdx.x / KB; i < n; i += (int64_t)gridDim.x * rpb) {
      const int64_t q = i * k + sub;
      x[q] = x[q] + alpha * ph[q] + omega * sh[q];
      const S rn = sv[q] - omega * t[q];
      r[q] = rn;
      fma_s(v0, conj_(rhat[q]), rn);
      v1 += S(abs2_(rn));
    }
  }
  col_reduce_finalize<S, KB>(v0, v1, k, part, counter, FIN_RHO, st, nullptr, done);
}

// x = 0, r = r_hat = rhs, p = v = 0, then (r_hat, r), ||r||^2 -> FIN_INIT
template <typename S, int KB>
__global__ void __launch_bounds__(256) init_kernel(int n, int k, const S* __restrict__ rhs, S* __restrict__ x,
                                                   S* __restrict__ r, S* __restrict__ rhat, S* __restrict__ p,
                                                   S* __restrict__ v, double* part, unsigned* counter, KState* st,
                                                   int* done) {
  const int sub = threadIdx.x & (KB - 1);
  S v0 = S(0), v1 = S(0);
  const int rpb = blockDim.x / KB;
  if (sub < k) {
    for (int64_t i = blockIdx.x * (int64_t)rpb + threadIdx.x / KB; i < n; i += (int64_t)gridDim.x * rpb) {
      const int64_t q = i * k + sub;
      const S b = rhs[q];
      x[q] = S(0);
      r[q] = b;
      rhat[q] = b;
      p[q] = S(0);
      v[q] = S(0);
      fma_s(v0, conj_(b), b);
      v1 += S(abs2_(b));
    }
  }
  col_reduce_finalize<S, KB>(v0, v1, k, part, counter, FIN_INIT, st, nullptr, done);
}

__global__ void set_targets_kernel(int k, KState* st, const double* target, const int* maxit) {
  int c = threadIdx.x;
  if (c < k) { st[c].target2 = target[c] * target[c]; st[c].maxit = maxit[c]; }
}

// rhs_in = cast(r64 / ||r64||) for active columns, 0 otherwise
template <typename Sin, typename S64, int KB>
__global__ void scale_cast_kernel(int n, int k, const S64* __restrict__ r64, const double* nrm2,
                                  const int* active, Sin* __restrict__ out) {
  const int sub = threadIdx.x & (KB - 1);
  if (sub >= k) return;
  const int act = active[sub];
  const double inv = (act && nrm2[sub] > 0.0) ? 1.0 / sqrt(nrm2[sub]) : 0.0;
  const int rpb = blockDim.x / KB;
  for (int64_t i = blockIdx.x * (int64_t)rpb + threadIdx.x / KB; i < n; i += (int64_t)gridDim.x * rpb) {
    const int64_t q = i * k + sub;
    out[q] = act ? cvt<Sin>(inv * r64[q]) : Sin(0);
  }
}

template <typename Sin, typename S64, int KB>
__global__ void refine_update_kernel(int n, int k, S64* __restrict__ x64, const Sin* __restrict__ d,
                                     const double* nrm2, const int* active) {
  const int sub = threadIdx.x & (KB - 1);
  if (sub >= k || !active[sub]) return;
  const double sc = sqrt(nrm2[sub]);
  const int rpb = blockDim.x / KB;
  for (int64_t i = blockIdx.x * (int64_t)rpb + threadIdx.x / KB; i < n; i += (int64_t)gridDim.x * rpb) {
    const int64_t q = i * k + sub;
    x64[q] = x64[q] + sc * cvt<S64>(d[q]);
  }
}

// column-major complex128 (n x k) -> row-major S
template <typename S>
__global__ void c128_col_to_row_kernel(int n, int k, const cdouble* __restrict__ src, S* __restrict__ dst) {
  int64_t total = (int64_t)n * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t / k, c = t % k;
    dst[t] = cvt<S>(src[c * n + i]);
  }
}
template <typename S>
__global__ void row_to_c128_col_kernel(int n, int k, const S* __restrict__ src, cdouble* __restrict__ dst) {
  int64_t total = (int64_t)n * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t % n, c = t / n;
    dst[t] = cvt<cdouble>(src[i * k + c]);
  }
}
template <typename S>
__global__ void real_col_to_row_kernel(int n, int k, const double* __restrict__ src, int ld, S* __restrict__ dst) {
  int64_t total = (int64_t)n * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t / k, c = t % k;
    dst[t] = cvt<S>(src[c * (int64_t)ld + i]);
  }
}
template <typename D, typename S>
__global__ void copy_cast_kernel(int64_t count, const S* __restrict__ src, D* __restrict__ dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = cvt<D>(src[t]);
}

#define KB_SWITCH(kb, CALL)                 \
  switch (kb) {                             \
    case 1: { constexpr int KBv = 1; CALL; break; } \
    case 2: { constexpr int KBv = 2; CALL; break; } \
    case 4: { constexpr int KBv = 4; CALL; break; } \
    case 8: { constexpr int KBv = 8; CALL; break; } \
    case 16: { constexpr int KBv = 16; CALL; break; } \
    default: return (int)cudaErrorInvalidValue; \
  }

#define ST_SWITCH(st, CALL)                                   \
  switch (st) {                                               \
    case ST_F32: { typedef float S; CALL; break; }            \
    case ST_F64: { typedef double S; CALL; break; }           \
    case ST_C32: { typedef cfloat S; CALL; break; }           \
    case ST_C64: { typedef cdouble S; CALL; break; }          \
    default: return (int)cudaErrorInvalidValue;               \
  }

}  // namespace

size_t krylov_state_bytes(int) { return sizeof(KState); }

int krylov_launch_update_p(int st, int kb, int n, int k, const void* r, void* p, const void* v,
                           const void* state, const int* done, cudaStream_t s) {
  const int g = grid_for((int64_t)n * kb, 152 * 32);
  ST_SWITCH(st, KB_SWITCH(kb, (update_p_kernel<S, KBv><<<g, 256, 0, s>>>(n, k, (const S*)r, (S*)p, (const S*)v,
                                                                        (const KState*)state, done))));
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int krylov_launch_update_s(int st, int kb, int n, int k, const void* r, const void* v, void* sv,
                           const void* state, const int* done, cudaStream_t s) {
  const int g = grid_for((int64_t)n * kb, 152 * 32);
  ST_SWITCH(st, KB_SWITCH(kb, (update_s_kernel<S, KBv><<<g, 256, 0, s>>>(n, k, (const S*)r, (const S*)v, (S*)sv,
                                                                        (const KState*)state, done))));
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int krylov_launch_update_xr(int st, int kb, int n, int k, void* x, void* r, const void* phat,
                            const void* shat, const void* sv, const void* t, const void* rhat,
                            void* part, unsigned* counter, void* state, int* done, int grid_cap,
                            cudaStream_t s) {
  const int g = grid_for((int64_t)n * kb, grid_cap);
  ST_SWITCH(st, KB_SWITCH(kb, (update_xr_kernel<S, KBv><<<g, 256, 0, s>>>(
                                  n, k, (S*)x, (S*)r, (const S*)phat, (const S*)shat, (const S*)sv,
                                  (const S*)t, (const S*)rhat, (double*)part, counter, (KState*)state, done))));
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int krylov_launch_init(int st, int kb, int n, int k, const void* rhs, void* x, void* r, void* rhat,
                       void* p, void* v, void* part, unsigned* counter, void* state,
                       const double* target, const int* maxit, int* done, int grid_cap,
                       cudaStream_t s) {
  set_targets_kernel<<<1, 32, 0, s>>>(k, (KState*)state, target, maxit);
  mor_count_launches(1);
  const int g = grid_for((int64_t)n * kb, grid_cap);
  ST_SWITCH(st, KB_SWITCH(kb, (init_kernel<S, KBv><<<g, 256, 0, s>>>(n, k, (const S*)rhs, (S*)x, (S*)r, (S*)rhat,
                                                                    (S*)p, (S*)v, (double*)part, counter,
                                                                    (KState*)state, done))));
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int krylov_read_state(int, const void* state_dev, int k, int* iters, int* status, cudaStream_t s) {
  KState h[MOR_KMAX];
  cudaError_t e = cudaMemcpyAsync(h, state_dev, sizeof(KState) * k, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return (int)e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return (int)e;
  for (int c = 0; c < k; ++c) { iters[c] = h[c].iters; status[c] = h[c].status; }
  return 0;
}

int refine_launch_scale_cast(int st_in, int kb, int n, int k, const void* r64, const double* nrm2,
                             const int* active, void* rhs_in, cudaStream_t s) {
  const int g = grid_for((int64_t)n * kb, 152 * 32);
  switch (st_in) {
    case ST_F32: KB_SWITCH(kb, (scale_cast_kernel<float, double, KBv><<<g, 256, 0, s>>>(n, k, (const double*)r64, nrm2, active, (float*)rhs_in))); break;
    case ST_F64: KB_SWITCH(kb, (scale_cast_kernel<double, double, KBv><<<g, 256, 0, s>>>(n, k, (const double*)r64, nrm2, active, (double*)rhs_in))); break;
    case ST_C32: KB_SWITCH(kb, (scale_cast_kernel<cfloat, cdouble, KBv><<<g, 256, 0, s>>>(n, k, (const cdouble*)r64, nrm2, active, (cfloat*)rhs_in))); break;
    case ST_C64: KB_SWITCH(kb, (scale_cast_kernel<cdouble, cdouble, KBv><<<g, 256, 0, s>>>(n, k, (const cdouble*)r64, nrm2, active, (cdouble*)rhs_in))); break;
    default: return (int)cudaErrorInvalidValue;
  }
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int refine_launch_update(int st_in, int kb, int n, int k, void* x64, const void* d,
                         const double* nrm2, const int* active, cudaStream_t s) {
  const int g = grid_for((int64_t)n * kb, 152 * 32);
  switch (st_in) {
    case ST_F32: KB_SWITCH(kb, (refine_update_kernel<float, double, KBv><<<g, 256, 0, s>>>(n, k, (double*)x64, (const float*)d, nrm2, active))); break;
    case ST_F64: KB_SWITCH(kb, (refine_update_kernel<double, double, KBv><<<g, 256, 0, s>>>(n, k, (double*)x64, (const double*)d, nrm2, active))); break;
    case ST_C32: KB_SWITCH(kb, (refine_update_kernel<cfloat, cdouble, KBv><<<g, 256, 0, s>>>(n, k, (cdouble*)x64, (const cfloat*)d, nrm2, active))); break;
    case ST_C64: KB_SWITCH(kb, (refine_update_kernel<cdouble, cdouble, KBv><<<g, 256, 0, s>>>(n, k, (cdouble*)x64, (const cdouble*)d, nrm2, active))); break;
    default: return (int)cudaErrorInvalidValue;
  }
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int conv_launch_colmajor_c128_to_rowmajor(int st, int n, int k, const void* src, void* dst, cudaStream_t s) {
  const int g = grid_for((int64_t)n * k, 152 * 8);
  ST_SWITCH(st, (c128_col_to_row_kernel<S><<<g, 256, 0, s>>>(n, k, (const cdouble*)src, (S*)dst)));
  mor_count_launches(1);
  return (int)cudaGetLastError();
}
int conv_launch_rowmajor_to_colmajor_c128(int st, int n, int k, const void* src, void* dst, cudaStream_t s) {
  const int g = grid_for((int64_t)n * k, 152 * 8);
  ST_SWITCH(st, (row_to_c128_col_kernel<S><<<g, 256, 0, s>>>(n, k, (const S*)src, (cdouble*)dst)));
  mor_count_launches(1);
  return (int)cudaGetLastError();
}
int conv_launch_real_col_to_rowmajor(int st, int n, int k, const double* src, int ld, void* dst, cudaStream_t s) {
  const int g = grid_for((int64_t)n * k, 152 * 8);
  ST_SWITCH(st, (real_col_to_row_kernel<S><<<g, 256, 0, s>>>(n, k, src, ld, (S*)dst)));
  mor_count_launches(1);
  return (int)cudaGetLastError();
}
int conv_launch_copy_cast(int st_dst, int st_src, int64_t count, const void* src, void* dst, cudaStream_t s) {
  const int g = grid_for(count, 152 * 8);
  if (st_src == ST_F64 && st_dst == ST_F32) copy_cast_kernel<float, double><<<g, 256, 0, s>>>(count, (const double*)src, (float*)dst);
  else if (st_src == ST_C64 && st_dst == ST_C32) copy_cast_kernel<cfloat, cdouble><<<g, 256, 0, s>>>(count, (const cdouble*)src, (cfloat*)dst);
  else if (st_src == ST_F32 && st_dst == ST_C64) copy_cast_kernel<cdouble, float><<<g, 256, 0, s>>>(count, (const float*)src, (cdouble*)dst);
  else if (st_src == ST_C32 && st_dst == ST_C64) copy_cast_kernel<cdouble, cfloat><<<g, 256, 0, s>>>(count, (const cfloat*)src, (cdouble*)dst);
  else if (st_src == ST_F64 && st_dst == ST_C64) copy_cast_kernel<cdouble, double><<<g, 256, 0, s>>>(count, (const double*)src, (cdouble*)dst);
  else if (st_src == ST_C64 && st_dst == ST_C64) copy_cast_kernel<cdouble, cdouble><<<g, 256, 0, s>>>(count, (const cdouble*)src, (cdouble*)dst);
  else if (st_src == ST_F64 && st_dst == ST_C32) copy_cast_kernel<cfloat, double><<<g, 256, 0, s>>>(count, (const double*)src, (cfloat*)dst);
  else if (st_src == ST_F32 && st_dst == ST_C32) copy_cast_kernel<cfloat, float><<<g, 256, 0, s>>>(count, (const float*)src, (cfloat*)dst);
  else if (st_src == ST_F64 && st_dst == ST_F64) copy_cast_kernel<double, double><<<g, 256, 0, s>>>(count, (const double*)src, (double*)dst);
  else if (st_src == ST_F32 && st_dst == ST_F32) copy_cast_kernel<float, float><<<g, 256, 0, s>>>(count, (const float*)src, (float*)dst);
  else return (int)cudaErrorInvalidValue;
  mor_count_launches(1);
  return (int)cudaGetLastError();
}
