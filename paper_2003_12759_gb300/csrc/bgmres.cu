// Kernels of restarted block GMRES(m) (Saad 2003, Sec. 6.12) for the p right-
// hand sides of one shift: the p columns of an n x ld row-major block share
// one block Krylov space of A(sigma) P.  The basis [V_0 .. V_j] is kept
// stacked, row-major n x ldv (row r holds V_0[r, 0..p), V_1[r, 0..p), ...),
// so that one pass over the rows serves every block of the basis:
//   bg_dot     H = V^H W       (K = (j+1) p basis columns against the p
//                               columns of W; per-block partials, fixed-order
//                               reduction by the last block)
//   bg_update  W = W - V C     (block classical Gram-Schmidt update), or
//              Y = V C         (Y = W R^{-1} of CholQR, x += P V y at a restart)
//   bg_copy    copy p columns between a contiguous block and the stack.
// The block least-squares problem and the small Cholesky factors run on the
// host in FP64 (csrc/block_ls.h).
#include "mor_internal.h"
#include "krylov_state.cuh"

#include <algorithm>
#include <cuda_pipeline.h>

namespace {

template <typename S> __device__ __forceinline__ cdouble to_cd(S v) { return cdouble((double)real_(v), (double)imag_(v)); }
template <typename S> __device__ __forceinline__ S from_cd(cdouble z);
template <> __device__ __forceinline__ float from_cd<float>(cdouble z) { return (float)z.re; }
template <> __device__ __forceinline__ double from_cd<double>(cdouble z) { return z.re; }
template <> __device__ __forceinline__ cfloat from_cd<cfloat>(cdouble z) { return cfloat((float)z.re, (float)z.im); }
template <> __device__ __forceinline__ cdouble from_cd<cdouble>(cdouble z) { return z; }

constexpr int BG_PMAX = 8;       // right-hand sides per block

// out[kk * P + b] = sum_r conj(V[r, kk]) W[r, b], kk < K, b < P.  The block's
// threads form G = 256 / KT row groups of KT threads (KT = K rounded up to a
// multiple of 32, at most 256); thread (g, t) owns the basis columns kk = t +
// KT u (u < U) and all P columns of W.  The block walks its contiguous row
// range in tiles of BG_TILE rows: the tile's rows of W are staged in shared
// memory (every thread reads all of them), and group g takes the tile rows
// g, g + G, ..., whose V loads are independent (unrolled, all in flight).
// The groups' sums meet in shared memory; bg_reduce sums the blocks'
// partials in a fixed order.
constexpr int BG_RPT = 16;          // tile rows per thread of the dot kernel
template <typename S, int U>
__global__ void __launch_bounds__(256) bg_dot_kernel(int64_t n, int K, int P, const S* __restrict__ V, int64_t ldv,
                                                     const S* __restrict__ W, int64_t ldw, double* part) {
  __shared__ double red[128 * BG_PMAX][2];
  __shared__ S ws[BG_RPT * 8][BG_PMAX];
  const int KT = K >= 256 ? 256 : ((K + 31) / 32) * 32;
  const int G = 256 / KT;
  const int g = threadIdx.x / KT, t = threadIdx.x % KT;
  const int TR = BG_RPT * G;                     // tile rows: 16 per thread
  S acc[U][BG_PMAX];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int b = 0; b < BG_PMAX; ++b) acc[u][b] = S(0);
  const int64_t rpb = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rpb;
  const int64_t r1 = r0 + rpb < n ? r0 + rpb : n;
  for (int64_t tr = r0; tr < r1; tr += TR) {
    const int rows = (int)(r1 - tr < TR ? r1 - tr : TR);
    __syncthreads();
    for (int i = threadIdx.x; i < TR * BG_PMAX; i += blockDim.x) {
      const int rr = i / BG_PMAX, b = i % BG_PMAX;
      ws[rr][b] = (rr < rows && b < P) ? W[(tr + rr) * ldw + b] : S(0);
    }
    __syncthreads();
    if (g < G) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int kk = t + KT * u;
        if (kk < K) {
          // all 16 loads of the thread's rows in flight, then the products
          S vr[BG_RPT];
#pragma unroll
          for (int i = 0; i < BG_RPT; ++i) {
            const int rr = g + i * G;
            vr[i] = rr < rows ? conj_(V[(tr + rr) * ldv + kk]) : S(0);
          }
#pragma unroll
          for (int i = 0; i < BG_RPT; ++i) {
            const int rr = g + i * G;
#pragma unroll
            for (int b = 0; b < BG_PMAX; ++b) fma_s(acc[u][b], vr[i], ws[rr < TR ? rr : 0][b]);
          }
        }
      }
    }
  }
  const int nout = K * P;
  if (G > 1) {
    // K <= 128 here: sum the G groups' accumulators in a fixed order
    for (int gg = 0; gg < G; ++gg) {
      if (g == gg && t < K) {
#pragma unroll
        for (int b = 0; b < BG_PMAX; ++b) {
          if (b >= P) break;
          const double re = (double)real_(acc[0][b]), im = (double)imag_(acc[0][b]);
          if (gg == 0) { red[t * P + b][0] = re; red[t * P + b][1] = im; }
          else { red[t * P + b][0] += re; red[t * P + b][1] += im; }
        }
      }
      __syncthreads();
    }
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
      double* q = part + ((size_t)blockIdx.x * nout + o) * 2;
      q[0] = red[o][0];
      q[1] = red[o][1];
    }
  } else if (g == 0) {
    // one row group (K > 128): threads past KT (when KT < 256) hold nothing
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int kk = t + KT * u;
      if (kk < K) {
#pragma unroll
        for (int b = 0; b < BG_PMAX; ++b) {
          if (b >= P) break;
          double* q = part + ((size_t)blockIdx.x * nout + (size_t)kk * P + b) * 2;
          q[0] = (double)real_(acc[u][b]);
          q[1] = (double)imag_(acc[u][b]);
        }
      }
    }
  }
}

// out[o] = sum over the dot kernel's blocks of their partials: one warp per
// output, lane l summing blocks l, l + 32, ..., then a fixed-order warp sum
__global__ void bg_reduce_kernel(int nout, int nblk, const double* __restrict__ part, cdouble* __restrict__ out) {
  const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (o >= nout) return;
  double re = 0.0, im = 0.0;
  for (int blk = lane; blk < nblk; blk += 32) {
    re += part[((size_t)blk * nout + o) * 2 + 0];
    im += part[((size_t)blk * nout + o) * 2 + 1];
  }
  re = warp_sum(re);
  im = warp_sum(im);
  if (lane == 0) out[o] = cdouble(re, im);
}

// mode 0: Y[r, b] = W[r, b] - sum_kk V[r, kk] C[kk * P + b]
// mode 1: Y[r, b] =          sum_kk V[r, kk] C[kk * P + b]
// The block walks tiles of T <= 32 rows: the tile's rows of V (T x K) are
// loaded into shared memory with coalesced loads, then thread (row rr, column
// b) of the 32 x 8 layout sums over kk from shared memory (four independent
// partial sums, combined in a fixed order).  Shared memory: C (K x P), then
// the V tile (T x K).
template <typename S>
__global__ void __launch_bounds__(256) bg_update_kernel(int64_t n, int K, int P, int T, const S* __restrict__ V,
                                                        int64_t ldv, const cdouble* __restrict__ C, const S* W,
                                                        int64_t ldw, int mode, S* Y, int64_t ldy) {
  extern __shared__ __align__(16) unsigned char bg_smem[];
  S* cs = reinterpret_cast<S*>(bg_smem);
  S* vs = cs + (size_t)K * P;
  for (int t = threadIdx.x; t < K * P; t += blockDim.x) cs[t] = from_cd<S>(C[t]);
  const int b = threadIdx.x & 7;
  const int rl = threadIdx.x >> 3;
  const int64_t ntiles = (n + T - 1) / T;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * T;
    const int rows = (int)(n - r0 < T ? n - r0 : T);
    __syncthreads();
    // asynchronous copies: every element of the tile in flight at once
    for (int i = threadIdx.x; i < rows * K; i += blockDim.x) {
      const int rr = i / K, kk = i % K;
      __pipeline_memcpy_async(vs + i, V + (r0 + rr) * ldv + kk, sizeof(S));
    }
    __pipeline_commit();
    __pipeline_wait_prior(0);
    __syncthreads();
    if (rl < rows && b < P) {
      const S* vr = vs + (size_t)rl * K;
      S a0 = S(0), a1 = S(0), a2 = S(0), a3 = S(0);
      int kk = 0;
      for (; kk + 3 < K; kk += 4) {
        fma_s(a0, vr[kk], cs[kk * P + b]);
        fma_s(a1, vr[kk + 1], cs[(kk + 1) * P + b]);
        fma_s(a2, vr[kk + 2], cs[(kk + 2) * P + b]);
        fma_s(a3, vr[kk + 3], cs[(kk + 3) * P + b]);
      }
      for (; kk < K; ++kk) fma_s(a0, vr[kk], cs[kk * P + b]);
      const S sum = (a0 + a1) + (a2 + a3);
      const int64_t r = r0 + rl;
      Y[r * ldy + b] = mode == 0 ? W[r * ldw + b] - sum : sum;
    }
  }
}

// dst[r * ldd + off + b] = src[r * lds + b], b < P
template <typename S>
__global__ void bg_copy_kernel(int64_t n, int P, const S* __restrict__ src, int64_t lds, S* __restrict__ dst,
                               int64_t ldd, int64_t off) {
  const int64_t tot = n * P;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / P;
    const int b = (int)(t % P);
    dst[r * ldd + off + b] = src[r * lds + b];
  }
}

#define BG_ST_SWITCH(st, ...)                                 \
  switch (st) {                                               \
    case ST_F32: { typedef float S; __VA_ARGS__; break; }     \
    case ST_F64: { typedef double S; __VA_ARGS__; break; }    \
    case ST_C32: { typedef cfloat S; __VA_ARGS__; break; }    \
    case ST_C64: { typedef cdouble S; __VA_ARGS__; break; }   \
    default: return (int)cudaErrorInvalidValue;               \
  }

}  // namespace

int bgmres_max_cols() { return BG_PMAX; }

int bgmres_dot_grid() { return 2 * mor_device_sms(); }

size_t bgmres_part_doubles(int K, int P) { return (size_t)2 * K * P * (size_t)bgmres_dot_grid(); }

int bgmres_launch_dot(int st, int64_t n, int K, int P, const void* V, int64_t ldv, const void* W, int64_t ldw,
                      double* part, unsigned* counter, void* out, cudaStream_t s) {
  (void)counter;
  if (K < 1 || K > 1024 || P < 1 || P > BG_PMAX) return (int)cudaErrorInvalidValue;
  const int grid = bgmres_dot_grid();
  const int U = (K + 255) / 256;
  BG_ST_SWITCH(st, {
    if (U == 1) bg_dot_kernel<S, 1><<<grid, 256, 0, s>>>(n, K, P, (const S*)V, ldv, (const S*)W, ldw, part);
    else if (U == 2) bg_dot_kernel<S, 2><<<grid, 256, 0, s>>>(n, K, P, (const S*)V, ldv, (const S*)W, ldw, part);
    else bg_dot_kernel<S, 4><<<grid, 256, 0, s>>>(n, K, P, (const S*)V, ldv, (const S*)W, ldw, part);
  });
  const int nout = K * P;
  bg_reduce_kernel<<<(nout + 7) / 8, 256, 0, s>>>(nout, grid, part, (cdouble*)out);
  mor_count_launches(2);
  return (int)cudaGetLastError();
}

int bgmres_launch_update(int st, int64_t n, int K, int P, const void* V, int64_t ldv, const void* C, const void* W,
                         int64_t ldw, int mode, void* Y, int64_t ldy, cudaStream_t s) {
  if (K < 1 || P < 1 || P > BG_PMAX) return (int)cudaErrorInvalidValue;
  const size_t es = st_size(st);
  const size_t cbytes = es * (size_t)K * P;
  // rows per tile: the V tile and C within 96 KB of shared memory, at most 32
  int T = (int)std::min<size_t>(32, ((size_t)96 * 1024 > cbytes ? ((size_t)96 * 1024 - cbytes) : 0) / (es * K));
  if (T < 1) return (int)cudaErrorInvalidValue;
  const size_t sm = cbytes + es * (size_t)T * K;
  const int grid = (int)std::min<int64_t>((n + T - 1) / T, (int64_t)mor_device_sms() * 4);
  BG_ST_SWITCH(st, {
    cudaError_t e = cudaFuncSetAttribute(bg_update_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    bg_update_kernel<S><<<grid, 256, sm, s>>>(n, K, P, T, (const S*)V, ldv, (const cdouble*)C, (const S*)W, ldw,
                                              mode, (S*)Y, ldy);
  });
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int bgmres_launch_copy(int st, int64_t n, int P, const void* src, int64_t lds, void* dst, int64_t ldd, int64_t off,
                       cudaStream_t s) {
  const int grid = (int)std::min<int64_t>((n * P + 255) / 256, (int64_t)mor_device_sms() * 8);
  BG_ST_SWITCH(st, (bg_copy_kernel<S><<<grid, 256, 0, s>>>(n, P, (const S*)src, lds, (S*)dst, ldd, off)));
  mor_count_launches(1);
  return (int)cudaGetLastError();
}
