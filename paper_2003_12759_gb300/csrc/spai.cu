// Batched column least squares for the SPAI preconditioner and its reuse
// factor (Sec. III.A Eq. gen-precond-par; Table II second approach):
//
//   build  (update = 0):  p_j = argmin || e_j - A(s_new) p ||_2
//   reuse  (update = 1):  q_j = argmin || A(s_old) e_j - A(s_new) q ||_2
//
// with p_j, q_j supported on J_j (the pattern of column j).  Only the rows
// I_j reached by the columns J_j enter the problem (the others add a
// constant), so each column is a dense |I_j| x |J_j| least-squares problem.
//
// GB300 mapping: one group of LPC lanes per column (LPC = 4 ... 32 so that a
// lane owns at most four rows; 32 / LPC columns per warp).  A group gathers
// the block G = A(s_new)(I_j, J_j) straight from the stored sparse columns
// (the shifted matrix is never formed: each entry is sE e + sA a), stages it
// in shared memory column-major, factors it by Householder QR with
// group-shuffle reductions, applies Q^H to the right-hand side and
// back-substitutes.  The solution is scattered straight into the factor's
// value array in the operator's storage layout.  A warp per column, with 25
// rows on 32 lanes and five-step reductions, spent 5.2k warp instructions
// per column of the 7-point stencil and kept the FP64 pipe half busy forming
// the entries in FP64; FP32 / complex64 factors now gather from FP32 copies.
#include "mor_internal.h"
#include "mor_types.cuh"

#include <algorithm>

namespace {

__device__ __forceinline__ float div_s(float a, float b) { return a / b; }
__device__ __forceinline__ double div_s(double a, double b) { return a / b; }
template <typename R> __device__ __forceinline__ cplx<R> div_s(cplx<R> a, cplx<R> b) {
  R d = b.re * b.re + b.im * b.im;
  return cplx<R>((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}

// A(s) entry of column `kc` at column-entry q (row = colidx[q]), in the
// precision V of the column data (FP32 for FP32 / complex64 factors: the
// FP64 pipe of this GPU is narrow, and the factor is rounded to FP32 anyway)
template <typename V> struct ColData {
  const V* ca;
  const V* ce;
  const V* ediag;
};
template <typename V>
__device__ __forceinline__ cplx<V> entry(const ColData<V>& d, int ekind, const cplx<V> (&cf)[2], int64_t q, int row,
                                         int kc) {
  V ev = V(0);
  if (ekind == EK_CSR) ev = d.ce[q];
  else if (row == kc) ev = (ekind == EK_DIAG) ? d.ediag[kc] : V(1);
  const V av = d.ca[q];
  return cplx<V>(cf[0].re * ev + cf[1].re * av, cf[0].im * ev + cf[1].im * av);
}

template <typename S, typename V> __device__ __forceinline__ S to_s(cplx<V> z);
template <> __device__ __forceinline__ float to_s<float, float>(cplx<float> z) { return z.re; }
template <> __device__ __forceinline__ cfloat to_s<cfloat, float>(cplx<float> z) { return z; }
template <> __device__ __forceinline__ double to_s<double, double>(cplx<double> z) { return z.re; }
template <> __device__ __forceinline__ cdouble to_s<cdouble, double>(cplx<double> z) { return z; }

__device__ __forceinline__ int find_row(const int* Il, int nI, int row) {
  int lo = 0, hi = nI - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (Il[mid] < row) lo = mid + 1; else hi = mid;
  }
  return lo;   // I_j contains every row of the gathered columns by construction
}

// Shared memory of one column's problem, padded so that the columns of a
// warp's groups start W = LPC * sizeof(S) bytes apart modulo 128: a group's
// access of LPC consecutive elements then shares each 128-byte bank
// wavefront with other groups' accesses without bank conflicts (unpadded,
// 1824-byte columns of the 7-point stencil gave 217M conflicts per 10^6
// columns and an L1 pipe 88% busy).
template <typename S, int LPC>
__host__ __device__ inline size_t col_bytes(int nImax, int nJmax) {
  size_t b = ((size_t)nImax * nJmax + nImax + 2 * nJmax) * sizeof(S) + (size_t)nImax * sizeof(int);
  b = (b + 15) & ~(size_t)15;
  constexpr size_t W = (size_t)LPC * sizeof(S);
  if (W < 128) {
    while (b % 128 != W % 128) b += 16;
  }
  return b;
}

// sum over the LPC lanes of a column group (xor offsets below LPC stay inside the group)
template <int LPC, typename T> __device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = LPC >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <int LPC, typename R> __device__ __forceinline__ cplx<R> group_sum(cplx<R> v) {
#pragma unroll
  for (int o = LPC >> 1; o > 0; o >>= 1) {
    v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
    v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
  }
  return v;
}
__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// One column per group of LPC lanes, 32 / LPC columns per warp: each group
// gathers G = A(s_new)(I_j, J_j) into shared memory (column-major, lane l of
// the group owns rows l, l + LPC, ...), factors it by Householder QR with
// group reductions, applies Q^H to the right-hand side and back-substitutes.
// Loop bounds are the maxima over the warp's groups (a group past its own
// sizes computes nothing), so every shuffle runs with the whole warp.
template <typename S, typename V, int LPC>
__global__ void __launch_bounds__(256) spai_kernel(SpaiArgs a, ColData<V> cd, S* __restrict__ out) {
  typedef typename real_of<S>::type R;
  constexpr int CPW = 32 / LPC;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int grp = lane / LPC, gl = lane % LPC;
  unsigned char* base = smem + ((size_t)wid * CPW + grp) * col_bytes<S, LPC>(a.nImax, a.nJmax);
  S* G = (S*)base;                                   // nJmax columns of nImax rows
  S* rhs = G + (size_t)a.nImax * a.nJmax;
  S* Rd = rhs + a.nImax;                             // diagonal of R
  S* qv = Rd + a.nJmax;                              // solution
  int* Il = (int*)(qv + a.nJmax);
  const int ld = a.nImax;
  const cplx<V> cnew[2] = {cplx<V>((V)a.cnew.sEr, (V)a.cnew.sEi), cplx<V>((V)a.cnew.sAr, (V)a.cnew.sAi)};
  const cplx<V> cold[2] = {cplx<V>((V)a.cold.sEr, (V)a.cold.sEi), cplx<V>((V)a.cold.sAr, (V)a.cold.sAi)};

  for (int j0 = (blockIdx.x * nw + wid) * CPW; j0 < a.n; j0 += gridDim.x * nw * CPW) {
    const int j = j0 + grp;
    const bool valid = j < a.n;
    int64_t i0 = 0;
    int nI = 0, c0 = 0, nJ = 0;
    if (valid) {
      i0 = a.iptr[j];
      nI = (int)(a.iptr[j + 1] - i0);
      c0 = a.colptr[j];
      nJ = a.colptr[j + 1] - c0;
    }
    const int nJw = warp_max(nJ);
    for (int t = gl; t < nI; t += LPC) Il[t] = a.iidx[i0 + t];
    for (int t = gl; t < nJ * ld; t += LPC) G[t] = S(0);
    for (int t = gl; t < nI; t += LPC) rhs[t] = S(0);
    __syncwarp();
    // gather G = A(s_new)(I_j, J_j) column by column
    for (int t = 0; t < nJ; ++t) {
      const int kc = a.colidx[c0 + t];
      const int q0 = a.colptr[kc], q1 = a.colptr[kc + 1];
      for (int q = q0 + gl; q < q1; q += LPC) {
        const int row = a.colidx[q];
        G[t * ld + find_row(Il, nI, row)] = to_s<S, V>(entry(cd, a.ekind, cnew, q, row, kc));
      }
    }
    // right-hand side restricted to I_j
    if (valid) {
      if (!a.update) {
        if (gl == 0) rhs[find_row(Il, nI, j)] = S(1);
      } else {
        for (int q = c0 + gl; q < c0 + nJ; q += LPC) {
          const int row = a.colidx[q];
          rhs[find_row(Il, nI, row)] = to_s<S, V>(entry(cd, a.ekind, cold, q, row, j));
        }
      }
    }
    __syncwarp();
    // Householder QR, lane gl of the group owns rows gl, gl + LPC, ...
    bool singular = false;
    for (int c = 0; c < nJw; ++c) {
      const bool act = c < nJ;
      S* gc = G + c * ld;
      R s2 = R(0);
      if (act)
        for (int rr = gl; rr < nI; rr += LPC) if (rr >= c) s2 += abs2_(gc[rr]);
      s2 = group_sum<LPC>(s2);
      const S x0 = act ? gc[c] : S(0);
      __syncwarp();
      const R alpha = sqrt(s2);
      const bool ok = act && (alpha > R(0));
      if (act && !ok) {
        singular = true;
        if (gl == 0) Rd[c] = S(0);
      }
      const R ax0 = sqrt(abs2_(x0));
      const S ph = (ax0 > R(0)) ? x0 * (R(1) / ax0) : S(1);
      const S v0 = x0 + ph * alpha;
      const R vn2 = s2 - ax0 * ax0 + abs2_(v0);
      const R beta = ok ? R(2) / vn2 : R(0);
      if (ok && gl == (c % LPC)) gc[c] = v0;
      if (ok && gl == 0) Rd[c] = -(ph * alpha);
      __syncwarp();
      for (int c2 = c + 1; c2 < nJw; ++c2) {
        const bool act2 = ok && c2 < nJ;
        S* g2 = G + c2 * ld;
        S w = S(0);
        if (act2)
          for (int rr = gl; rr < nI; rr += LPC) if (rr >= c) fma_s(w, conj_(gc[rr]), g2[rr]);
        w = group_sum<LPC>(w);
        const S bw = w * beta;
        if (act2)
          for (int rr = gl; rr < nI; rr += LPC) if (rr >= c) g2[rr] -= gc[rr] * bw;
      }
      {
        S w = S(0);
        if (ok)
          for (int rr = gl; rr < nI; rr += LPC) if (rr >= c) fma_s(w, conj_(gc[rr]), rhs[rr]);
        w = group_sum<LPC>(w);
        const S bw = w * beta;
        if (ok)
          for (int rr = gl; rr < nI; rr += LPC) if (rr >= c) rhs[rr] -= gc[rr] * bw;
      }
      __syncwarp();
    }
    // back substitution R q = (Q^H rhs)(0:nJ) (lane 0 of the group), then scatter
    if (valid && gl == 0) {
      if (singular) {
        for (int c = 0; c < nJ; ++c) qv[c] = S(0);
        atomicAdd(a.nsingular, 1);
      } else {
        for (int c = nJ - 1; c >= 0; --c) {
          S acc = rhs[c];
          for (int c2 = c + 1; c2 < nJ; ++c2) acc -= G[c2 * ld + c] * qv[c2];
          qv[c] = div_s(acc, Rd[c]);
        }
      }
    }
    __syncwarp();
    for (int t = gl; t < nJ; t += LPC) out[a.outpos[c0 + t]] = qv[t];
    __syncwarp();
  }
}

template <typename S, typename V, int LPC>
int spai_launch(const SpaiArgs& a, const ColData<V>& cd, void* out, cudaStream_t s) {
  constexpr int CPW = 32 / LPC;
  const size_t wb = col_bytes<S, LPC>(a.nImax, a.nJmax) * CPW;     // per warp
  int nw = 8;
  while (nw > 1 && wb * nw > 48 * 1024) nw >>= 1;
  if (wb * nw > 200 * 1024) return (int)cudaErrorInvalidValue;
  const size_t sm = wb * nw;
  cudaError_t e = cudaFuncSetAttribute(spai_kernel<S, V, LPC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return (int)e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, spai_kernel<S, V, LPC>, nw * 32, sm);
  if (e != cudaSuccess || occ < 1) occ = 1;
  const int sms = mor_device_sms();
  const int64_t per_block = (int64_t)nw * CPW;
  int64_t blocks = ((int64_t)a.n + per_block - 1) / per_block;
  blocks = std::min<int64_t>(blocks, (int64_t)sms * occ);
  spai_kernel<S, V, LPC><<<(unsigned)std::max<int64_t>(blocks, 1), nw * 32, sm, s>>>(a, cd, (S*)out);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

// lanes per column: each lane owns at most 4 rows of the |I_j| x |J_j| block
template <typename S, typename V>
int spai_reg_launch(const SpaiArgs& a, const ColData<V>& cd, void* out, cudaStream_t s);
template <typename S> size_t spai_reg_smem(const SpaiArgs& a, int nw);

#ifndef MOR_SPAI_REG
#define MOR_SPAI_REG 1
#endif

template <typename S, typename V>
int spai_dispatch(const SpaiArgs& a, const ColData<V>& cd, void* out, cudaStream_t s) {
#if MOR_SPAI_REG
  // small columns (the 7-point stencil's 25 x 7) on registers, when one
  // warp's staging fits the default 48 KB of shared memory
  if (a.nImax <= 32 && a.nJmax <= 8 && spai_reg_smem<S>(a, 1) <= 48 * 1024)
    return spai_reg_launch<S, V>(a, cd, out, s);
#endif
  if (a.nImax <= 16) return spai_launch<S, V, 4>(a, cd, out, s);
  if (a.nImax <= 32) return spai_launch<S, V, 8>(a, cd, out, s);
  if (a.nImax <= 64) return spai_launch<S, V, 16>(a, cd, out, s);
  return spai_launch<S, V, 32>(a, cd, out, s);
}

// value of lane src (a lane index of the whole warp)
template <typename T> __device__ __forceinline__ T shfl_s(T v, int src) { return __shfl_sync(0xffffffffu, v, src); }
template <typename R> __device__ __forceinline__ cplx<R> shfl_s(cplx<R> v, int src) {
  return cplx<R>(__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src));
}

// The same column least squares for small columns (|I_j| <= 32, |J_j| <= 8:
// the 7-point stencil has 25 x 7) with the block held in registers during
// the factorisation: groups of 8 lanes, lane l of a group owning rows l,
// l + 8, l + 16, l + 24 of all 8 columns.  The gather still stages G through
// shared memory (entries land on rows found by search in I_j); then every
// Householder step, the application of the reflectors to the later columns
// and to the right-hand side, and the back substitution run on registers
// with the loops unrolled, in the order (and with the sums) of spai_kernel.
// The row of the pivot of step c < 8 is row c, held by lane c of the group
// in its first register, which is where the back substitution reads R.
// blocks per SM the register allocation is held to.  Measured on the 100^3
// pattern (10^6 columns, 25 x 7 blocks), build / reuse update in ms, complex64
// and FP32: 1 block (168 registers) 2.43 / 2.31 and 1.50 / 1.43; 4 blocks
// (118) 2.13 / 2.00 and 1.49 / 1.44; 5 blocks (96) 2.01 / 1.91 and 1.29 /
// 1.23.  Complex128 blocks keep their registers (236 a thread; any bound
// spills kilobytes).
#ifndef MOR_SPAI_REG_MINB
#define MOR_SPAI_REG_MINB 5
#endif
template <typename S> constexpr int spai_reg_minb() { return sizeof(S) == 16 ? 1 : MOR_SPAI_REG_MINB; }
template <typename S, typename V>
__global__ void __launch_bounds__(128, spai_reg_minb<S>()) spai_reg_kernel(SpaiArgs a, ColData<V> cd, S* __restrict__ out) {
  typedef typename real_of<S>::type R;
  constexpr int LPC = 8, NR = 4, NJ = 8, CPW = 32 / LPC;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int grp = lane / LPC, gl = lane % LPC, gbase = lane & ~(LPC - 1);
  unsigned char* base = smem + ((size_t)wid * CPW + grp) * col_bytes<S, LPC>(a.nImax, a.nJmax);
  S* G = (S*)base;                                   // nJmax columns of nImax rows
  S* rhs = G + (size_t)a.nImax * a.nJmax;
  int* Il = (int*)(rhs + a.nImax + 2 * a.nJmax);
  const int ld = a.nImax;
  const cplx<V> cnew[2] = {cplx<V>((V)a.cnew.sEr, (V)a.cnew.sEi), cplx<V>((V)a.cnew.sAr, (V)a.cnew.sAi)};
  const cplx<V> cold[2] = {cplx<V>((V)a.cold.sEr, (V)a.cold.sEi), cplx<V>((V)a.cold.sAr, (V)a.cold.sAi)};

  for (int j0 = (blockIdx.x * nw + wid) * CPW; j0 < a.n; j0 += gridDim.x * nw * CPW) {
    const int j = j0 + grp;
    const bool valid = j < a.n;
    int64_t i0 = 0;
    int nI = 0, c0 = 0, nJ = 0;
    if (valid) {
      i0 = a.iptr[j];
      nI = (int)(a.iptr[j + 1] - i0);
      c0 = a.colptr[j];
      nJ = a.colptr[j + 1] - c0;
    }
    for (int t = gl; t < nI; t += LPC) Il[t] = a.iidx[i0 + t];
    for (int t = gl; t < nJ * ld; t += LPC) G[t] = S(0);
    for (int t = gl; t < nI; t += LPC) rhs[t] = S(0);
    __syncwarp();
    for (int t = 0; t < nJ; ++t) {
      const int kc = a.colidx[c0 + t];
      const int q0 = a.colptr[kc], q1 = a.colptr[kc + 1];
      for (int q = q0 + gl; q < q1; q += LPC) {
        const int row = a.colidx[q];
        G[t * ld + find_row(Il, nI, row)] = to_s<S, V>(entry(cd, a.ekind, cnew, q, row, kc));
      }
    }
    if (valid) {
      if (!a.update) {
        if (gl == 0) rhs[find_row(Il, nI, j)] = S(1);
      } else {
        for (int q = c0 + gl; q < c0 + nJ; q += LPC) {
          const int row = a.colidx[q];
          rhs[find_row(Il, nI, row)] = to_s<S, V>(entry(cd, a.ekind, cold, q, row, j));
        }
      }
    }
    __syncwarp();
    // the block and the right-hand side into registers (zero past the sizes)
    S g[NJ][NR], rv[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const int rr = gl + LPC * i;
      const bool in = rr < nI;
      const S rh = rhs[in ? rr : 0];             // indices clamped into the group's block
      rv[i] = in ? rh : S(0);
#pragma unroll
      for (int t = 0; t < NJ; ++t) {
        const bool e = in && t < nJ;
        const S gv = G[e ? t * ld + rr : 0];
        g[t][i] = e ? gv : S(0);
      }
    }
    __syncwarp();
    bool singular = false;
    S rd[NJ];
#pragma unroll
    for (int c = 0; c < NJ; ++c) {
      const bool act = c < nJ;
      // rows >= c: all of a lane's rows but possibly its first (c < 8)
      R s2 = R(0);
#pragma unroll
      for (int i = 0; i < NR; ++i)
        if (i > 0 || gl >= c) s2 += abs2_(g[c][i]);
      s2 = act ? s2 : R(0);
      s2 = group_sum<LPC>(s2);
      S x0 = shfl_s(g[c][0], gbase + c);     // every lane shuffles; inactive groups take zero
      if (!act) x0 = S(0);
      const R alpha = sqrt(s2);
      const bool ok = act && (alpha > R(0));
      if (act && !ok) singular = true;
      const R ax0 = sqrt(abs2_(x0));
      const S ph = (ax0 > R(0)) ? x0 * (R(1) / ax0) : S(1);
      const S v0 = x0 + ph * alpha;
      const R vn2 = s2 - ax0 * ax0 + abs2_(v0);
      const R beta = ok ? R(2) / vn2 : R(0);
      if (ok && gl == c) g[c][0] = v0;
      rd[c] = ok ? -(ph * alpha) : S(0);
      // the later columns c2 > c (a fixed trip count, so that both loops unroll
      // and the block stays in registers)
#pragma unroll
      for (int c2 = 1; c2 < NJ; ++c2) {
        if (c2 <= c) continue;
        const bool act2 = ok && c2 < nJ;
        S w = S(0);
#pragma unroll
        for (int i = 0; i < NR; ++i)
          if (i > 0 || gl >= c) fma_s(w, conj_(g[c][i]), g[c2][i]);
        w = act2 ? w : S(0);
        w = group_sum<LPC>(w);
        const S bw = w * beta;
        if (act2) {
#pragma unroll
          for (int i = 0; i < NR; ++i)
            if (i > 0 || gl >= c) g[c2][i] -= g[c][i] * bw;
        }
      }
      {
        S w = S(0);
#pragma unroll
        for (int i = 0; i < NR; ++i)
          if (i > 0 || gl >= c) fma_s(w, conj_(g[c][i]), rv[i]);
        w = ok ? w : S(0);
        w = group_sum<LPC>(w);
        const S bw = w * beta;
        if (ok) {
#pragma unroll
          for (int i = 0; i < NR; ++i)
            if (i > 0 || gl >= c) rv[i] -= g[c][i] * bw;
        }
      }
    }
    // back substitution R q = (Q^H rhs)(0:nJ): row c of R and of the rotated
    // right-hand side sit in lane c's first registers
    S qv[NJ];
#pragma unroll
    for (int c = NJ - 1; c >= 0; --c) {
      S acc = rv[0];
#pragma unroll
      for (int c2 = c + 1; c2 < NJ; ++c2)
        if (c2 < nJ) acc -= g[c2][0] * qv[c2];
      acc = shfl_s(acc, gbase + c);
      qv[c] = (c < nJ && !singular) ? div_s(acc, rd[c]) : S(0);
    }
    if (valid && singular && gl == 0) atomicAdd(a.nsingular, 1);
    S mine = qv[0];
#pragma unroll
    for (int c = 1; c < NJ; ++c)
      if (gl == c) mine = qv[c];
    if (gl < nJ) out[a.outpos[c0 + gl]] = mine;
    __syncwarp();
  }
}

// shared memory of a block of nw warps of spai_reg_kernel (the gather's staging)
template <typename S> size_t spai_reg_smem(const SpaiArgs& a, int nw) { return col_bytes<S, 8>(a.nImax, a.nJmax) * 4 * nw; }

template <typename S, typename V>
int spai_reg_launch(const SpaiArgs& a, const ColData<V>& cd, void* out, cudaStream_t s) {
  constexpr int CPW = 4;
  int nw = 4;
  while (nw > 1 && spai_reg_smem<S>(a, nw) > 48 * 1024) nw >>= 1;
  const size_t sm = spai_reg_smem<S>(a, nw);
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, spai_reg_kernel<S, V>, nw * 32, sm);
  if (e != cudaSuccess || occ < 1) occ = 1;
  const int sms = mor_device_sms();
  const int64_t per_block = (int64_t)nw * CPW;
  int64_t blocks = ((int64_t)a.n + per_block - 1) / per_block;
  blocks = std::min<int64_t>(blocks, (int64_t)sms * occ);
  spai_reg_kernel<S, V><<<(unsigned)std::max<int64_t>(blocks, 1), nw * 32, sm, s>>>(a, cd, (S*)out);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

}  // namespace

int launch_spai(int st, const SpaiArgs& a, void* out, cudaStream_t s) {
  const ColData<float> c32{a.ca32, a.ce32, a.ediag32};
  const ColData<double> c64{a.ca, a.ce, a.ediag};
  switch (st) {
    case ST_F32: return spai_dispatch<float, float>(a, c32, out, s);
    case ST_F64: return spai_dispatch<double, double>(a, c64, out, s);
    case ST_C32: return spai_dispatch<cfloat, float>(a, c32, out, s);
    case ST_C64: return spai_dispatch<cdouble, double>(a, c64, out, s);
  }
  return (int)cudaErrorInvalidValue;
}
