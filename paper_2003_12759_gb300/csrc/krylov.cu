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

#include "shape_dispatch.cuh"

#include <algorithm>
#include <mutex>
#include <unordered_map>

namespace {

template <typename S> __device__ __forceinline__ S from_cd(cdouble z);
template <> __device__ __forceinline__ float from_cd<float>(cdouble z) { return (float)z.re; }
template <> __device__ __forceinline__ double from_cd<double>(cdouble z) { return z.re; }
template <> __device__ __forceinline__ cfloat from_cd<cfloat>(cdouble z) { return cfloat((float)z.re, (float)z.im); }
template <> __device__ __forceinline__ cdouble from_cd<cdouble>(cdouble z) { return z; }

inline int grid_for(int64_t threads, int cap) {
  int64_t b = (threads + 255) / 256;
  if (cap > 0 && b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// lane geometry shared by the elementwise kernels: segment, rows, owned columns
#define MOR_LANE_SETUP                                  \
  const int sub = threadIdx.x % TPR;                   \
  const int c0 = sub * CPT;                            \
  const int rpb = blockDim.x / TPR;                    \
  const int seg = seg_of_chunk(sg, blockIdx.x);                    \
  int64_t rb, re;                                      \
  chunk_rows(sg, seg, blockIdx.x, rb, re);

template <typename S, int TPR, int CPT>
__global__ void __launch_bounds__(256) update_p_kernel(SegView sg, int ld, const S* __restrict__ r, S* __restrict__ p,
                                                       const S* __restrict__ v, const KState* st, const int* done) {
  if (*done) return;
  MOR_LANE_SETUP
  if (c0 >= ld) return;
  st += (size_t)seg * ld;
  S beta[CPT], omega[CPT];
  int act[CPT];
  bool any = false;
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    act[j] = st[c0 + j].active;
    beta[j] = from_cd<S>(st[c0 + j].beta);
    omega[j] = from_cd<S>(st[c0 + j].omega);
    any |= (act[j] != 0);
  }
  if (!any) return;
  for (int64_t i = rb + threadIdx.x / TPR; i < re; i += rpb) {
    const int64_t q = i * ld + c0;
    const Pack<S, CPT> rv = ldp<S, CPT>(r + q), vv = ldp<S, CPT>(v + q);
    Pack<S, CPT> pv = ldp<S, CPT>(p + q);
#pragma unroll
    for (int j = 0; j < CPT; ++j)
      if (act[j]) pv.v[j] = rv.v[j] + beta[j] * (pv.v[j] - omega[j] * vv.v[j]);
    stp<S, CPT>(p + q, pv);
  }
}

template <typename S, int TPR, int CPT>
__global__ void __launch_bounds__(256) update_s_kernel(SegView sg, int ld, const S* __restrict__ r, const S* __restrict__ v,
                                                       S* __restrict__ sv, const KState* st, const int* done) {
  if (*done) return;
  MOR_LANE_SETUP
  if (c0 >= ld) return;
  st += (size_t)seg * ld;
  S alpha[CPT];
  int act[CPT];
#pragma unroll
  for (int j = 0; j < CPT; ++j) { act[j] = st[c0 + j].active; alpha[j] = from_cd<S>(st[c0 + j].alpha); }
  for (int64_t i = rb + threadIdx.x / TPR; i < re; i += rpb) {
    const int64_t q = i * ld + c0;
    const Pack<S, CPT> rv = ldp<S, CPT>(r + q), vv = ldp<S, CPT>(v + q);
    Pack<S, CPT> o;
#pragma unroll
    for (int j = 0; j < CPT; ++j) o.v[j] = act[j] ? rv.v[j] - alpha[j] * vv.v[j] : rv.v[j];
    stp<S, CPT>(sv + q, o);
  }
}

template <typename S, int TPR, int CPT>
__global__ void __launch_bounds__(256) update_xr_kernel(SegView sg, int ld, S* __restrict__ x, S* __restrict__ r,
                                                        const S* __restrict__ ph, const S* __restrict__ sh,
                                                        const S* __restrict__ sv, const S* __restrict__ t,
                                                        const S* __restrict__ rhat, double* part, KState* st,
                                                        int* done) {
  if (*done) return;
  MOR_LANE_SETUP
  const bool lane_on = c0 < ld;
  const KState* sts = st + (size_t)seg * ld;
  S alpha[CPT], omega[CPT], v0[CPT], v1[CPT];
  int act[CPT];
  bool any = false, all = true;
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    act[j] = lane_on ? sts[c0 + j].active : 0;
    alpha[j] = act[j] ? from_cd<S>(sts[c0 + j].alpha) : S(0);
    omega[j] = act[j] ? from_cd<S>(sts[c0 + j].omega) : S(0);
    v0[j] = S(0);
    v1[j] = S(0);
    any |= (act[j] != 0);
    all &= (act[j] != 0);
  }
  if (any) {
    for (int64_t i = rb + threadIdx.x / TPR; i < re; i += rpb) {
      const int64_t q = i * ld + c0;
      Pack<S, CPT> xv = ldp<S, CPT>(x + q);
      const Pack<S, CPT> pv = ldp<S, CPT>(ph + q), shv = ldp<S, CPT>(sh + q), svv = ldp<S, CPT>(sv + q),
                         tv = ldp<S, CPT>(t + q), rh = ldp<S, CPT>(rhat + q);
      // r is read only to carry stopped columns through: a lane whose columns
      // are all active overwrites every one of them
      Pack<S, CPT> rn;
      if (!all) rn = ldp<S, CPT>(r + q);
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        if (act[j]) {
          xv.v[j] = xv.v[j] + alpha[j] * pv.v[j] + omega[j] * shv.v[j];
          rn.v[j] = svv.v[j] - omega[j] * tv.v[j];
          fma_s(v0[j], conj_(rh.v[j]), rn.v[j]);
          v1[j] += S(abs2_(rn.v[j]));
        }
      }
      stp<S, CPT>(x + q, xv);
      stp<S, CPT>(r + q, rn);
    }
  }
  col_reduce_finalize<S, TPR, CPT>(v0, v1, ld, sg, seg, blockIdx.x, part, FIN_RHO, st, nullptr, done);
}

// x = 0, r = r_hat = rhs, p = v = 0, then (r_hat, r), ||r||^2 -> FIN_INIT
template <typename S, int TPR, int CPT>
__global__ void __launch_bounds__(256) init_kernel(SegView sg, int ld, const S* __restrict__ rhs, S* __restrict__ x,
                                                   S* __restrict__ r, S* __restrict__ rhat, S* __restrict__ p,
                                                   S* __restrict__ v, double* part, KState* st, int* done) {
  MOR_LANE_SETUP
  S v0[CPT], v1[CPT];
#pragma unroll
  for (int j = 0; j < CPT; ++j) { v0[j] = S(0); v1[j] = S(0); }
  if (c0 < ld) {
    Pack<S, CPT> z;
#pragma unroll
    for (int j = 0; j < CPT; ++j) z.v[j] = S(0);
    for (int64_t i = rb + threadIdx.x / TPR; i < re; i += rpb) {
      const int64_t q = i * ld + c0;
      const Pack<S, CPT> b = ldp<S, CPT>(rhs + q);
      stp<S, CPT>(x + q, z);
      stp<S, CPT>(r + q, b);
      stp<S, CPT>(rhat + q, b);
      stp<S, CPT>(p + q, z);
      stp<S, CPT>(v + q, z);
#pragma unroll
      for (int j = 0; j < CPT; ++j) { fma_s(v0[j], conj_(b.v[j]), b.v[j]); v1[j] += S(abs2_(b.v[j])); }
    }
  }
  col_reduce_finalize<S, TPR, CPT>(v0, v1, ld, sg, seg, blockIdx.x, part, FIN_INIT, st, nullptr, done);
}

__global__ void set_targets_kernel(int count, KState* st, const double* target, const int* maxit, int stag) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < count; c += gridDim.x * blockDim.x) {
    st[c].target2 = target[c] * target[c];
    st[c].maxit = maxit[c];
    st[c].stag = stag;
  }
}
__global__ void set_done_kernel(const int* live, int* done) { *done = (*live == 0) ? 1 : 0; }

template <typename S> struct wide_of { typedef S type; };
template <> struct wide_of<float> { typedef double type; };
template <> struct wide_of<cfloat> { typedef cdouble type; };

// rhs_in = cast(r64 / ||r64||) for active columns, 0 otherwise
template <typename S, int TPR, int CPT>
__global__ void scale_cast_kernel(SegView sg, int ld, const typename wide_of<S>::type* __restrict__ r64,
                                  const double* nrm2, const int* active, S* __restrict__ out) {
  typedef typename wide_of<S>::type W;
  MOR_LANE_SETUP
  if (c0 >= ld) return;
  active += (size_t)seg * ld;
  nrm2 += (size_t)seg * ld;
  double inv[CPT];
  int act[CPT];
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    act[j] = active[c0 + j];
    inv[j] = (act[j] && nrm2[c0 + j] > 0.0) ? 1.0 / sqrt(nrm2[c0 + j]) : 0.0;
  }
  for (int64_t i = rb + threadIdx.x / TPR; i < re; i += rpb) {
    const int64_t q = i * ld + c0;
    Pack<S, CPT> o;
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      const W w = r64[q + j];
      o.v[j] = act[j] ? cvt<S>(inv[j] * w) : S(0);
    }
    stp<S, CPT>(out + q, o);
  }
}

template <typename S, int TPR, int CPT>
__global__ void refine_update_kernel(SegView sg, int ld, typename wide_of<S>::type* __restrict__ x64,
                                     const S* __restrict__ d, const double* nrm2, const int* active) {
  typedef typename wide_of<S>::type W;
  MOR_LANE_SETUP
  if (c0 >= ld) return;
  active += (size_t)seg * ld;
  nrm2 += (size_t)seg * ld;
  double sc[CPT];
  int act[CPT];
#pragma unroll
  for (int j = 0; j < CPT; ++j) { act[j] = active[c0 + j]; sc[j] = sqrt(nrm2[c0 + j]); }
  for (int64_t i = rb + threadIdx.x / TPR; i < re; i += rpb) {
    const int64_t q = i * ld + c0;
    const Pack<S, CPT> dv = ldp<S, CPT>(d + q);
#pragma unroll
    for (int j = 0; j < CPT; ++j)
      if (act[j]) x64[q + j] = x64[q + j] + sc[j] * cvt<W>(dv.v[j]);
  }
}

// column-major complex128 (n x k) -> row-major S with stride ld (columns k..ld-1 untouched)
template <typename S>
__global__ void c128_col_to_row_kernel(int n, int k, int ld, const cdouble* __restrict__ src, S* __restrict__ dst) {
  int64_t total = (int64_t)n * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t / k, c = t % k;
    dst[i * ld + c] = cvt<S>(src[c * n + i]);
  }
}
template <typename S>
__global__ void row_to_c128_col_kernel(int n, int k, int ld, const S* __restrict__ src, cdouble* __restrict__ dst) {
  int64_t total = (int64_t)n * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t % n, c = t / n;
    dst[t] = cvt<cdouble>(src[i * ld + c]);
  }
}
template <typename S>
__global__ void real_col_to_row_kernel(int n, int k, int ld, const double* __restrict__ src, int64_t lds,
                                       S* __restrict__ dst) {
  int64_t total = (int64_t)n * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t / k, c = t % k;
    dst[i * ld + c] = cvt<S>(src[c * lds + i]);
  }
}
template <typename D, typename S>
__global__ void copy_cast_kernel(int64_t count, const S* __restrict__ src, D* __restrict__ dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = cvt<D>(src[t]);
}

// dst(i, c) = c < ncols ? src(i, map[c]) : 0 for c < ld_dst (column compaction)
template <typename T>
__global__ void gather_cols_kernel(int64_t n, int ld_src, int ld_dst, int ncols, const int* __restrict__ map,
                                   const T* __restrict__ src, T* __restrict__ dst) {
  const int64_t total = n * ld_dst;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ld_dst;
    const int c = (int)(t - i * ld_dst);
    T v;
    memset(&v, 0, sizeof(T));
    if (c < ncols) v = src[i * ld_src + map[c]];
    dst[t] = v;
  }
}
// dst(i, dmap[c]) = src(i, smap[c]) for c < ncols
template <typename T>
__global__ void scatter_cols_kernel(int64_t n, int ld_src, int ld_dst, int ncols, const int* __restrict__ smap,
                                    const int* __restrict__ dmap, const T* __restrict__ src, T* __restrict__ dst) {
  const int64_t total = n * ncols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ncols;
    const int c = (int)(t - i * ncols);
    dst[i * ld_dst + dmap[c]] = src[i * ld_src + smap[c]];
  }
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

int mor_device_sms() {
  static std::mutex mu;
  static std::unordered_map<int, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  cache[dev] = sms;
  return sms;
}

SegView fit_grid(const SegView& sg, const void* kern, int tpr) {
  if (sg.nseg != 1) return sg;
  static std::mutex mu;
  static std::unordered_map<const void*, int> occ_cache;
  int occ = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = occ_cache.find(kern);
    if (it != occ_cache.end()) occ = it->second;
  }
  if (occ <= 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0) != cudaSuccess || occ < 1) occ = 1;
    std::lock_guard<std::mutex> lk(mu);
    occ_cache[kern] = occ;
  }
  // one resident wave (measured faster than 2 or 4 waves of smaller blocks);
  // 256-thread blocks give occ <= 8, so grids stay within sms * 8 blocks,
  // the size every per-block partial buffer is allocated for
  if (occ > 8) occ = 8;
  const int64_t pass = 256 / tpr;
  const int64_t passes = (sg.nrows + pass - 1) / pass;
  int64_t grid = std::min<int64_t>((int64_t)sg.sms * occ, std::max<int64_t>(passes, 1));
  const int64_t ppb = (passes + grid - 1) / grid;   // passes per block
  SegView g = sg;
  g.rows_per_block = std::max<int64_t>(ppb, 1) * pass;
  g.nblocks = (int)std::max<int64_t>((sg.nrows + g.rows_per_block - 1) / g.rows_per_block, 1);
  return g;
}

int krylov_launch_update_p(int st, const SegView& sg, int ld, const void* r, void* p, const void* v, const void* state,
                           const int* done, cudaStream_t s) {
  int e = dispatch_shape(st, ld, [&]<typename S, int TPR, int CPT>() -> int {
    const SegView g = fit_grid(sg, (const void*)update_p_kernel<S, TPR, CPT>, TPR); update_p_kernel<S, TPR, CPT><<<g.nblocks, 256, 0, s>>>(g, ld, (const S*)r, (S*)p, (const S*)v,
                                                            (const KState*)state, done);
    return 0;
  });
  if (e) return e;
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int krylov_launch_update_s(int st, const SegView& sg, int ld, const void* r, const void* v, void* sv, const void* state,
                           const int* done, cudaStream_t s) {
  int e = dispatch_shape(st, ld, [&]<typename S, int TPR, int CPT>() -> int {
    const SegView g = fit_grid(sg, (const void*)update_s_kernel<S, TPR, CPT>, TPR); update_s_kernel<S, TPR, CPT><<<g.nblocks, 256, 0, s>>>(g, ld, (const S*)r, (const S*)v, (S*)sv,
                                                            (const KState*)state, done);
    return 0;
  });
  if (e) return e;
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int krylov_launch_update_xr(int st, const SegView& sg, int ld, void* x, void* r, const void* phat, const void* shat,
                            const void* sv, const void* t, const void* rhat, void* part, void* state, int* done,
                            cudaStream_t s) {
  int e = dispatch_shape(st, ld, [&]<typename S, int TPR, int CPT>() -> int {
    const SegView g = fit_grid(sg, (const void*)update_xr_kernel<S, TPR, CPT>, TPR); update_xr_kernel<S, TPR, CPT><<<g.nblocks, 256, 0, s>>>(g, ld, (S*)x, (S*)r, (const S*)phat, (const S*)shat,
                                                             (const S*)sv, (const S*)t, (const S*)rhat, (double*)part,
                                                             (KState*)state, done);
    return 0;
  });
  if (e) return e;
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int krylov_launch_init(int st, const SegView& sg, int ld, const void* rhs, void* x, void* r, void* rhat, void* p,
                       void* v, void* part, void* state, const double* target, const int* maxit, int stag, int* done,
                       cudaStream_t s) {
  const int count = sg.nseg * ld;
  set_targets_kernel<<<(count + 255) / 256, 256, 0, s>>>(count, (KState*)state, target, maxit, stag);
  mor_count_launches(1);
  cudaError_t ce = cudaMemsetAsync(sg.live, 0, sizeof(int), s);
  if (ce != cudaSuccess) return (int)ce;
  int e = dispatch_shape(st, ld, [&]<typename S, int TPR, int CPT>() -> int {
    const SegView g = fit_grid(sg, (const void*)init_kernel<S, TPR, CPT>, TPR); init_kernel<S, TPR, CPT><<<g.nblocks, 256, 0, s>>>(g, ld, (const S*)rhs, (S*)x, (S*)r, (S*)rhat, (S*)p, (S*)v,
                                                        (double*)part, (KState*)state, done);
    return 0;
  });
  if (e) return e;
  mor_count_launches(1);
  set_done_kernel<<<1, 1, 0, s>>>(sg.live, done);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int krylov_read_state(int, const void* state_dev, int k, int* iters, int* status, cudaStream_t s) {
  if (k > MOR_LDMAX) return (int)cudaErrorInvalidValue;
  KState h[MOR_LDMAX];
  cudaError_t e = cudaMemcpyAsync(h, state_dev, sizeof(KState) * k, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return (int)e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return (int)e;
  for (int c = 0; c < k; ++c) { iters[c] = h[c].iters; status[c] = h[c].status; }
  return 0;
}

int refine_launch_scale_cast(int st_in, const SegView& sg, int ld, const void* r64, const double* nrm2, const int* active,
                             void* rhs_in, cudaStream_t s) {
  int e = dispatch_shape(st_in, ld, [&]<typename S, int TPR, int CPT>() -> int {
    typedef typename wide_of<S>::type W;
    const SegView g = fit_grid(sg, (const void*)scale_cast_kernel<S, TPR, CPT>, TPR); scale_cast_kernel<S, TPR, CPT><<<g.nblocks, 256, 0, s>>>(g, ld, (const W*)r64, nrm2, active, (S*)rhs_in);
    return 0;
  });
  if (e) return e;
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int refine_launch_update(int st_in, const SegView& sg, int ld, void* x64, const void* d, const double* nrm2,
                         const int* active, cudaStream_t s) {
  int e = dispatch_shape(st_in, ld, [&]<typename S, int TPR, int CPT>() -> int {
    typedef typename wide_of<S>::type W;
    const SegView g = fit_grid(sg, (const void*)refine_update_kernel<S, TPR, CPT>, TPR); refine_update_kernel<S, TPR, CPT><<<g.nblocks, 256, 0, s>>>(g, ld, (W*)x64, (const S*)d, nrm2, active);
    return 0;
  });
  if (e) return e;
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int conv_launch_colmajor_c128_to_rowmajor(int st, int n, int k, int ld, const void* src, void* dst, cudaStream_t s) {
  const int g = grid_for((int64_t)n * k, mor_device_sms() * 8);
  ST_SWITCH(st, (c128_col_to_row_kernel<S><<<g, 256, 0, s>>>(n, k, ld, (const cdouble*)src, (S*)dst)));
  mor_count_launches(1);
  return (int)cudaGetLastError();
}
int conv_launch_rowmajor_to_colmajor_c128(int st, int n, int k, int ld, const void* src, void* dst, cudaStream_t s) {
  const int g = grid_for((int64_t)n * k, mor_device_sms() * 8);
  ST_SWITCH(st, (row_to_c128_col_kernel<S><<<g, 256, 0, s>>>(n, k, ld, (const S*)src, (cdouble*)dst)));
  mor_count_launches(1);
  return (int)cudaGetLastError();
}
int conv_launch_real_col_to_rowmajor(int st, int n, int k, int ld, const double* src, int64_t lds, void* dst,
                                     cudaStream_t s) {
  const int g = grid_for((int64_t)n * k, mor_device_sms() * 8);
  ST_SWITCH(st, (real_col_to_row_kernel<S><<<g, 256, 0, s>>>(n, k, ld, src, lds, (S*)dst)));
  mor_count_launches(1);
  return (int)cudaGetLastError();
}
int conv_launch_copy_cast(int st_dst, int st_src, int64_t count, const void* src, void* dst, cudaStream_t s) {
  const int g = grid_for(count, mor_device_sms() * 8);
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

int conv_launch_gather_cols(int st, int64_t n, int ld_src, int ld_dst, int ncols, const int* map, const void* src,
                            void* dst, cudaStream_t s) {
  const int g = grid_for(n * ld_dst, mor_device_sms() * 8);
  const size_t es = st_size(st);
  if (es == 4) gather_cols_kernel<uint32_t><<<g, 256, 0, s>>>(n, ld_src, ld_dst, ncols, map, (const uint32_t*)src, (uint32_t*)dst);
  else if (es == 8) gather_cols_kernel<uint2><<<g, 256, 0, s>>>(n, ld_src, ld_dst, ncols, map, (const uint2*)src, (uint2*)dst);
  else gather_cols_kernel<uint4><<<g, 256, 0, s>>>(n, ld_src, ld_dst, ncols, map, (const uint4*)src, (uint4*)dst);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int conv_launch_scatter_cols(int st, int64_t n, int ld_src, int ld_dst, int ncols, const int* smap, const int* dmap,
                             const void* src, void* dst, cudaStream_t s) {
  const int g = grid_for(n * ncols, mor_device_sms() * 8);
  const size_t es = st_size(st);
  if (es == 4) scatter_cols_kernel<uint32_t><<<g, 256, 0, s>>>(n, ld_src, ld_dst, ncols, smap, dmap, (const uint32_t*)src, (uint32_t*)dst);
  else if (es == 8) scatter_cols_kernel<uint2><<<g, 256, 0, s>>>(n, ld_src, ld_dst, ncols, smap, dmap, (const uint2*)src, (uint2*)dst);
  else scatter_cols_kernel<uint4><<<g, 256, 0, s>>>(n, ld_src, ld_dst, ncols, smap, dmap, (const uint4*)src, (uint4*)dst);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int krylov_write_state(const void* host_states, void* state_dev, int k, cudaStream_t s) {
  return (int)cudaMemcpyAsync(state_dev, host_states, sizeof(KState) * k, cudaMemcpyHostToDevice, s);
}
int krylov_read_states(void* host_states, const void* state_dev, int k, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(host_states, state_dev, sizeof(KState) * k, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaStreamSynchronize(s);
}
int krylov_state_active(const void* host_state) { return ((const KState*)host_state)->active; }
int krylov_state_iters(const void* host_state) { return ((const KState*)host_state)->iters; }
int krylov_state_status(const void* host_state) { return ((const KState*)host_state)->status; }
int krylov_status_stagnated(int status) { return status == KST_STAGNATED; }
void krylov_state_make_dummy(void* host_state) {
  KState* k = (KState*)host_state;
  memset(k, 0, sizeof(KState));
  k->target2 = 1.0;
}
