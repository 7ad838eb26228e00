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
// GB300 mapping: one warp per column.  The warp gathers the block
// G = A(s_new)(I_j, J_j) straight from the stored sparse columns (the shifted
// matrix is never formed: each entry is sE e + sA a), stages it in shared
// memory column-major (lane l owns rows l, l + 32, ...), factors it by
// Householder QR with warp-shuffle reductions, applies Q^H to the right-hand
// side and back-substitutes.  The solution is scattered straight into the
// factor's value array in the operator's storage layout.
#include "mor_internal.h"
#include "mor_types.cuh"

namespace {

template <typename S> __device__ __forceinline__ S from_cd(cdouble z);
template <> __device__ __forceinline__ float from_cd<float>(cdouble z) { return (float)z.re; }
template <> __device__ __forceinline__ double from_cd<double>(cdouble z) { return z.re; }
template <> __device__ __forceinline__ cfloat from_cd<cfloat>(cdouble z) { return cfloat((float)z.re, (float)z.im); }
template <> __device__ __forceinline__ cdouble from_cd<cdouble>(cdouble z) { return z; }

__device__ __forceinline__ float div_s(float a, float b) { return a / b; }
__device__ __forceinline__ double div_s(double a, double b) { return a / b; }
template <typename R> __device__ __forceinline__ cplx<R> div_s(cplx<R> a, cplx<R> b) {
  R d = b.re * b.re + b.im * b.im;
  return cplx<R>((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}

// A(s) entry of column `kc` at column-entry q (row = colidx[q])
__device__ __forceinline__ cdouble entry(const SpaiArgs& a, const Coef& cf, int64_t q, int row, int kc) {
  double ev = 0.0;
  if (a.ekind == EK_CSR) ev = a.ce[q];
  else if (row == kc) ev = (a.ekind == EK_DIAG) ? a.ediag[kc] : 1.0;
  const double av = a.ca[q];
  return cdouble(cf.sEr * ev + cf.sAr * av, cf.sEi * ev + cf.sAi * av);
}

__device__ __forceinline__ int find_row(const int* Il, int nI, int row) {
  int lo = 0, hi = nI - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (Il[mid] < row) lo = mid + 1; else hi = mid;
  }
  return lo;   // I_j contains every row of the gathered columns by construction
}

template <typename S>
__host__ __device__ inline size_t warp_bytes(int nImax, int nJmax) {
  size_t b = ((size_t)nImax * nJmax + nImax + 2 * nJmax) * sizeof(S) + (size_t)nImax * sizeof(int);
  return (b + 15) & ~(size_t)15;
}

template <typename S>
__global__ void __launch_bounds__(256) spai_kernel(SpaiArgs a, S* __restrict__ out) {
  typedef typename real_of<S>::type R;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned char* base = smem + (size_t)wid * warp_bytes<S>(a.nImax, a.nJmax);
  S* G = (S*)base;                                   // nJmax columns of nImax rows
  S* rhs = G + (size_t)a.nImax * a.nJmax;
  S* Rd = rhs + a.nImax;                             // diagonal of R
  S* qv = Rd + a.nJmax;                              // solution
  int* Il = (int*)(qv + a.nJmax);
  const int ld = a.nImax;

  for (int j = blockIdx.x * nw + wid; j < a.n; j += gridDim.x * nw) {
    const int64_t i0 = a.iptr[j];
    const int nI = (int)(a.iptr[j + 1] - i0);
    const int c0 = a.colptr[j];
    const int nJ = a.colptr[j + 1] - c0;
    for (int t = lane; t < nI; t += 32) Il[t] = a.iidx[i0 + t];
    for (int t = lane; t < nJ * ld; t += 32) G[t] = S(0);
    for (int t = lane; t < nI; t += 32) rhs[t] = S(0);
    __syncwarp();
    // gather G = A(s_new)(I_j, J_j) column by column
    for (int t = 0; t < nJ; ++t) {
      const int kc = a.colidx[c0 + t];
      const int q0 = a.colptr[kc], q1 = a.colptr[kc + 1];
      for (int q = q0 + lane; q < q1; q += 32) {
        const int row = a.colidx[q];
        G[t * ld + find_row(Il, nI, row)] = from_cd<S>(entry(a, a.cnew, q, row, kc));
      }
    }
    // right-hand side restricted to I_j
    if (!a.update) {
      if (lane == 0) rhs[find_row(Il, nI, j)] = S(1);
    } else {
      for (int q = c0 + lane; q < c0 + nJ; q += 32) {
        const int row = a.colidx[q];
        rhs[find_row(Il, nI, row)] = from_cd<S>(entry(a, a.cold, q, row, j));
      }
    }
    __syncwarp();
    // Householder QR, lane l owns rows l, l+32, ...
    bool singular = false;
    for (int c = 0; c < nJ; ++c) {
      S* gc = G + c * ld;
      R s2 = R(0);
      for (int rr = lane; rr < nI; rr += 32) if (rr >= c) s2 += abs2_(gc[rr]);
      s2 = warp_sum(s2);
      const S x0 = gc[c];
      __syncwarp();
      const R alpha = sqrt(s2);
      if (!(alpha > R(0))) {
        singular = true;
        if (lane == 0) Rd[c] = S(0);
        __syncwarp();
        continue;
      }
      const R ax0 = sqrt(abs2_(x0));
      const S ph = (ax0 > R(0)) ? x0 * (R(1) / ax0) : S(1);
      const S v0 = x0 + ph * alpha;
      const R vn2 = s2 - ax0 * ax0 + abs2_(v0);
      const R beta = R(2) / vn2;
      if (lane == (c & 31)) gc[c] = v0;
      if (lane == 0) Rd[c] = -(ph * alpha);
      __syncwarp();
      for (int c2 = c + 1; c2 < nJ; ++c2) {
        S* g2 = G + c2 * ld;
        S w = S(0);
        for (int rr = lane; rr < nI; rr += 32) if (rr >= c) fma_s(w, conj_(gc[rr]), g2[rr]);
        w = warp_sum(w);
        const S bw = w * beta;
        for (int rr = lane; rr < nI; rr += 32) if (rr >= c) g2[rr] -= gc[rr] * bw;
      }
      {
        S w = S(0);
        for (int rr = lane; rr < nI; rr += 32) if (rr >= c) fma_s(w, conj_(gc[rr]), rhs[rr]);
        w = warp_sum(w);
        const S bw = w * beta;
        for (int rr = lane; rr < nI; rr += 32) if (rr >= c) rhs[rr] -= gc[rr] * bw;
      }
      __syncwarp();
    }
    // back substitution R q = (Q^H rhs)(0:nJ)  (lane 0), then scatter
    if (lane == 0) {
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
    for (int t = lane; t < nJ; t += 32) out[a.outpos[c0 + t]] = qv[t];
    __syncwarp();
  }
}

template <typename S>
int spai_dispatch(const SpaiArgs& a, void* out, cudaStream_t s) {
  const size_t wb = warp_bytes<S>(a.nImax, a.nJmax);
  int nw = 8;
  while (nw > 1 && wb * nw > 100 * 1024) nw >>= 1;
  if (wb * nw > 200 * 1024) return (int)cudaErrorInvalidValue;
  const size_t sm = wb * nw;
  cudaError_t e = cudaFuncSetAttribute(spai_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return (int)e;
  int64_t blocks = ((int64_t)a.n + nw - 1) / nw;
  if (blocks > 152 * 16) blocks = 152 * 16;
  spai_kernel<S><<<(unsigned)blocks, nw * 32, sm, s>>>(a, (S*)out);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

}  // namespace

int launch_spai(int st, const SpaiArgs& a, void* out, cudaStream_t s) {
  switch (st) {
    case ST_F32: return spai_dispatch<float>(a, out, s);
    case ST_F64: return spai_dispatch<double>(a, out, s);
    case ST_C32: return spai_dispatch<cfloat>(a, out, s);
    case ST_C64: return spai_dispatch<cdouble>(a, out, s);
  }
  return (int)cudaErrorInvalidValue;
}
