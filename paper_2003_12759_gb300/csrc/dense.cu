// FP64 kernels on the tall-skinny projection bases and the reduced system:
//   gram      G = X^T Y for n x a and n x b column-major blocks (one pass
//             over n, tiles staged in shared memory, fixed-order reduction
//             of per-block partials by the last block) -- used for the
//             Gram-Schmidt coefficients (Algorithm 2 line 6) and the
//             Petrov-Galerkin products W^T A V, W^T E V, W^T B, V^T C
//             (Algorithm 2 line 7);
//   gs_update v -= V(:, 0:j) h;   scale  v /= ||v||;
//   eig       reduced poles and mirrored, sorted shifts (Algorithm 2 line 3);
//   tf        H_r(i w) = C_r^T (i w E_r - A_r)^{-1} B_r, one block per w.
#include "mor_internal.h"
#include "mor_types.cuh"
#include "small_eig.cuh"
#include "small_tangent.cuh"
#include "small_qep.cuh"

#include <algorithm>

namespace {

constexpr int GRAM_TR = 32;      // rows per tile
constexpr int GRAM_MAXC = 64;    // max columns of X plus Y

__global__ void __launch_bounds__(256) gram_kernel(int n, int a, int b, const double* __restrict__ X, int64_t ldx,
                                                   const double* __restrict__ Y, int64_t ldy, double* __restrict__ out,
                                                   double* part, unsigned* counter) {
  __shared__ double Xs[GRAM_TR][GRAM_MAXC + 1];
  __shared__ double Ys[GRAM_TR][GRAM_MAXC + 1];
  __shared__ bool am_last;
  const int npairs = a * b;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};        // pairs tid, tid+256, tid+512, tid+768
  const int ntiles = (n + GRAM_TR - 1) / GRAM_TR;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int r0 = tile * GRAM_TR;
    for (int t = threadIdx.x; t < GRAM_TR * a; t += blockDim.x) {
      const int rr = t % GRAM_TR, c = t / GRAM_TR;
      Xs[rr][c] = (r0 + rr < n) ? X[(int64_t)c * ldx + r0 + rr] : 0.0;
    }
    for (int t = threadIdx.x; t < GRAM_TR * b; t += blockDim.x) {
      const int rr = t % GRAM_TR, c = t / GRAM_TR;
      Ys[rr][c] = (r0 + rr < n) ? Y[(int64_t)c * ldy + r0 + rr] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int pr = threadIdx.x + 256 * u;
      if (pr < npairs) {
        const int i = pr % a, j = pr / a;
        double s = acc[u];
#pragma unroll 8
        for (int rr = 0; rr < GRAM_TR; ++rr) s = fma(Xs[rr][i], Ys[rr][j], s);
        acc[u] = s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int pr = threadIdx.x + 256 * u;
    if (pr < npairs) part[(size_t)blockIdx.x * npairs + pr] = acc[u];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  const volatile double* vp = part;
  for (int pr = threadIdx.x; pr < npairs; pr += blockDim.x) {
    double s = 0.0;
    for (int blk = 0; blk < (int)gridDim.x; ++blk) s += vp[(size_t)blk * npairs + pr];
    out[pr] = s;          // out[i + a*j] = X(:,i)^T Y(:,j)
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
}

// Tall-skinny form of gram for b <= 2 (the Gram-Schmidt coefficients and
// norms): out[i + a j] = X(:, i)^T Y(:, j), i < a <= 64.  One pass over the
// rows in registers (eight columns of X per blockIdx.y, the b columns of Y
// read once per row), per-block partials, and a fixed-order sum by the last
// block of each column group (ticket counters[blockIdx.y]).  The tiled gram
// kernel above staged 32-row tiles with two barriers each and ran ~10x
// below the bandwidth of this access pattern.
template <int B>
__global__ void __launch_bounds__(256) gram_skinny_kernel(int64_t n, int a, const double* __restrict__ X, int64_t ldx,
                                                          const double* __restrict__ Y, int64_t ldy,
                                                          double* __restrict__ out, double* part, unsigned* counters) {
  constexpr int CW = 8;
  constexpr int NV = CW * B;
  const int i0 = blockIdx.y * CW;
  double acc[CW][B];
#pragma unroll
  for (int c = 0; c < CW; ++c)
#pragma unroll
    for (int j = 0; j < B; ++j) acc[c][j] = 0.0;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x) {
    double y[B];
#pragma unroll
    for (int j = 0; j < B; ++j) y[j] = Y[row + j * ldy];
#pragma unroll
    for (int c = 0; c < CW; ++c)
      if (i0 + c < a) {
        const double x = X[row + (int64_t)(i0 + c) * ldx];
#pragma unroll
        for (int j = 0; j < B; ++j) acc[c][j] = fma(x, y[j], acc[c][j]);
      }
  }
  __shared__ double sh[8][NV];
  __shared__ bool am_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double t = warp_sum(acc[v / B][v % B]);
    if (lane == 0) sh[wid][v] = t;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w][threadIdx.x];
    part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * NV + threadIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counters + blockIdx.y, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  if (threadIdx.x < NV) {
    const volatile double* vp = part;
    double t = 0.0;
    for (int blk = 0; blk < (int)gridDim.x; ++blk) t += vp[((size_t)blockIdx.y * gridDim.x + blk) * NV + threadIdx.x];
    const int c = threadIdx.x / B, j = threadIdx.x % B;
    if (i0 + c < a) out[(i0 + c) + (size_t)a * j] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) counters[blockIdx.y] = 0u;
}

__global__ void gs_update_kernel(int n, int j, const double* __restrict__ V, int64_t ldv,
                                 const double* __restrict__ h, double* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = v[i];
    for (int c = 0; c < j; ++c) s -= V[(int64_t)c * ldv + i] * h[c];
    v[i] = s;
  }
}

__global__ void scale_kernel(int n, double* __restrict__ v, const double* nrm2) {
  const double inv = 1.0 / sqrt(nrm2[0]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] *= inv;
}

__global__ void diag_mul_kernel(int n, int k, const double* __restrict__ d, const double* __restrict__ X,
                                double* __restrict__ Y) {
  int64_t total = (int64_t)n * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    Y[t] = d[t % n] * X[t];
}

// out: wr[r], wi[r], sr[r], si[r], status  (one thread)
__global__ void eig_kernel(int r, const double* Ar, const double* Er, double* out, double* work, int* iwork) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* wr = out;
  double* wi = out + r;
  double* sr = out + 2 * r;
  double* si = out + 3 * r;
  int st = small_eig(r, Ar, Er, work, work + r * r, iwork, wr, wi);
  if (st == 0) mirror_sort(r, wr, wi, sr, si);
  out[4 * r] = (double)st;
}

// Tangential directions of r poles, one thread per pole (r <= 64): thread 0
// forms M = E_r^{-1} A_r and F = E_r^{-1} B_r, then every thread runs the
// inverse iterations of its pole.  out: r x m right directions, then r x q
// left ones (complex, row i for pole i), then the status (1: E_r singular).
__global__ void tangent_kernel(int r, int m, int q, const double* Ar, const double* Er, const double* Br,
                               const double* Cr, const double* lam, double* out, double* work, int* iwork) {
  double* M = work;
  double* F = M + (size_t)r * r;
  double* LU = F + (size_t)r * m;
  double* per = LU + (size_t)r * r;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = tangent_prepare(r, m, Ar, Er, Br, M, F, LU, iwork);
  __syncthreads();
  const int t = threadIdx.x;
  if (t == 0) out[2 * (size_t)r * (m + q)] = (double)bad;
  if (bad || t >= r) return;
  tz* K = (tz*)(per + (size_t)t * (2 * r * r + 4 * r));
  tz* x = K + (size_t)r * r;
  tz* y = x + r;
  tz* bt = (tz*)out + (size_t)t * m;
  tz* ct = (tz*)(out + 2 * (size_t)r * m) + (size_t)t * q;
  tangent_dirs(r, m, q, M, F, Cr, tz_c(lam[2 * t], lam[2 * t + 1]), K, iwork + r + t * r, x, y, bt, ct);
}

// Second-order point update (one thread): the companion pencil of the
// reduced QEP, its 2r eigenvalues (small_eig) and `count` new points
// (qep_select).  out: 2r eigenvalues (re, im), count points (re, im), status
// (0; 1 singular M_r; 2 QR did not converge; 3 too few eigenvalues).
__global__ void qep_kernel(int r, int count, const double* Kr, const double* Mr, double alpha, double beta,
                           double* out, double* work, int* iwork) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int n2 = 2 * r;
  double* A2 = work;
  double* E2 = A2 + (size_t)n2 * n2;
  double* W1 = E2 + (size_t)n2 * n2;
  double* W2 = W1 + (size_t)n2 * n2;
  double* wr = W2 + (size_t)n2 * n2;
  double* wi = wr + n2;
  double* sel = wi + n2;
  double* pr = sel + 3 * n2;
  double* pi = pr + count;
  qep_pencil(r, Mr, Kr, alpha, beta, A2, E2);
  int st = small_eig(n2, A2, E2, W1, W2, iwork, wr, wi);
  if (st == 0 && qep_select(n2, wr, wi, count, pr, pi, sel) != 0) st = 3;
  for (int i = 0; i < n2; ++i) { out[2 * i] = wr[i]; out[2 * i + 1] = wi[i]; }
  for (int i = 0; i < count; ++i) { out[2 * n2 + 2 * i] = (st == 0) ? pr[i] : 0.0; out[2 * n2 + 2 * i + 1] = (st == 0) ? pi[i] : 0.0; }
  out[2 * n2 + 2 * count] = (double)st;
}

// one block per frequency; (i w E_r - A_r) X = B_r by LU with partial
// pivoting in shared memory, then H = C_r^T X.
// order 1: (i w E_r - A_r); order 2 (A_r = K_r, E_r = M_r): s^2 M_r + s D_r + K_r
// at s = i w, i.e. (K_r - w^2 M_r) + i w (alpha M_r + beta K_r).
__global__ void tf_kernel(int r, int m, int q, const double* __restrict__ Ar, const double* __restrict__ Er,
                          const double* __restrict__ Br, const double* __restrict__ Cr, const double* __restrict__ omega,
                          int nw, cdouble* __restrict__ H, int order, double alpha, double beta) {
  extern __shared__ __align__(16) unsigned char sm[];
  cdouble* K = (cdouble*)sm;                 // r x r, column-major
  cdouble* X = K + r * r;                    // r x m
  __shared__ int pivrow;
  const int w = blockIdx.x;
  if (w >= nw) return;
  const double om = omega[w];
  for (int t = threadIdx.x; t < r * r; t += blockDim.x)
    K[t] = (order == 2) ? cdouble(Ar[t] - om * om * Er[t], om * (alpha * Er[t] + beta * Ar[t])) : cdouble(-Ar[t], om * Er[t]);
  for (int t = threadIdx.x; t < r * m; t += blockDim.x) X[t] = cdouble(Br[t], 0.0);
  __syncthreads();
  for (int kk = 0; kk < r; ++kk) {
    if (threadIdx.x == 0) {
      int p = kk;
      double best = cabs_(K[kk + kk * r]);
      for (int i = kk + 1; i < r; ++i) { double v = cabs_(K[i + kk * r]); if (v > best) { best = v; p = i; } }
      pivrow = p;
    }
    __syncthreads();
    const int p = pivrow;
    if (p != kk) {
      for (int j = threadIdx.x; j < r; j += blockDim.x) { cdouble t = K[kk + j * r]; K[kk + j * r] = K[p + j * r]; K[p + j * r] = t; }
      for (int j = threadIdx.x; j < m; j += blockDim.x) { cdouble t = X[kk + j * r]; X[kk + j * r] = X[p + j * r]; X[p + j * r] = t; }
    }
    __syncthreads();
    const cdouble d = K[kk + kk * r];
    // eliminate rows below kk
    for (int t = threadIdx.x; t < (r - kk - 1); t += blockDim.x) {
      const int i = kk + 1 + t;
      K[i + kk * r] = cdiv(K[i + kk * r], d);
    }
    __syncthreads();
    const int rows = r - kk - 1;
    for (int t = threadIdx.x; t < rows * (r - kk - 1 + m); t += blockDim.x) {
      const int i = kk + 1 + t % rows;
      const int jj = t / rows;
      const cdouble l = K[i + kk * r];
      if (jj < r - kk - 1) {
        const int j = kk + 1 + jj;
        K[i + j * r] -= l * K[kk + j * r];
      } else {
        const int j = jj - (r - kk - 1);
        X[i + j * r] -= l * X[kk + j * r];
      }
    }
    __syncthreads();
  }
  // back substitution, one thread per right-hand side
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    for (int i = r - 1; i >= 0; --i) {
      cdouble s = X[i + j * r];
      for (int c = i + 1; c < r; ++c) s -= K[i + c * r] * X[c + j * r];
      X[i + j * r] = cdiv(s, K[i + i * r]);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < q * m; t += blockDim.x) {
    const int iq = t % q, im = t / q;
    cdouble s(0.0, 0.0);
    for (int i = 0; i < r; ++i) s += Cr[i + (size_t)iq * r] * X[i + im * r];
    H[w + (size_t)nw * (iq + (size_t)q * im)] = s;
  }
}

inline int grid_for(int64_t n, int cap) {
  int64_t b = (n + 255) / 256;
  if (cap > 0 && b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

int dense_launch_gram(int n, int a, int b, const double* X, int64_t ldx, const double* Y, int64_t ldy,
                      double* out, double* part, unsigned* counter, int grid_cap, cudaStream_t s) {
  if (a < 1 || b < 1 || a + b > GRAM_MAXC || a * b > 1024) return (int)cudaErrorInvalidValue;
  if (b <= 2 && a <= 64) {
    // counter[0 .. ceil(a / 8) - 1] are the column groups' tickets
    dim3 g((unsigned)std::max<int64_t>(1, std::min<int64_t>(grid_cap / 2, ((int64_t)n + 255) / 256)), (unsigned)((a + 7) / 8));
    if (b == 1) gram_skinny_kernel<1><<<g, 256, 0, s>>>(n, a, X, ldx, Y, ldy, out, part, counter);
    else gram_skinny_kernel<2><<<g, 256, 0, s>>>(n, a, X, ldx, Y, ldy, out, part, counter);
    mor_count_launches(1);
    return (int)cudaGetLastError();
  }
  int64_t blocks = ((int64_t)n + GRAM_TR - 1) / GRAM_TR;
  if (blocks > grid_cap) blocks = grid_cap;
  if (blocks < 1) blocks = 1;
  gram_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, a, b, X, ldx, Y, ldy, out, part, counter);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int dense_launch_gs_update(int n, int j, const double* V, int64_t ldv, const double* h, double* v, cudaStream_t s) {
  gs_update_kernel<<<grid_for(n, mor_device_sms() * 8), 256, 0, s>>>(n, j, V, ldv, h, v);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int dense_launch_scale(int n, double* v, const double* nrm2, cudaStream_t s) {
  scale_kernel<<<grid_for(n, mor_device_sms() * 8), 256, 0, s>>>(n, v, nrm2);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int dense_launch_diag_mul(int n, int k, const double* d, const double* X, double* Y, cudaStream_t s) {
  diag_mul_kernel<<<grid_for((int64_t)n * k, mor_device_sms() * 8), 256, 0, s>>>(n, k, d, X, Y);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int dense_launch_eig(int r, const double* Ar, const double* Er, double* out, cudaStream_t s) {
  // work: 2 r^2 doubles + r ints, placed after the 4r+1 outputs
  double* work = out + 4 * r + 1;
  int* iwork = (int*)(work + 2 * r * r);
  eig_kernel<<<1, 32, 0, s>>>(r, Ar, Er, out, work, iwork);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

size_t dense_qep_work(int r, int count) { return (size_t)4 * (2 * r) * (2 * r) + (size_t)5 * (2 * r) + 2 * (size_t)count; }

int dense_launch_qep(int r, int count, const double* Kr, const double* Mr, double alpha, double beta, double* out,
                     double* work, int* iwork, cudaStream_t s) {
  qep_kernel<<<1, 32, 0, s>>>(r, count, Kr, Mr, alpha, beta, out, work, iwork);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

size_t dense_tangent_work(int r, int m) { return (size_t)2 * r * r + (size_t)r * m + (size_t)r * (2 * r * r + 4 * r); }

int dense_launch_tangent(int r, int m, int q, const double* Ar, const double* Er, const double* Br, const double* Cr,
                         const double* lam, double* out, double* work, int* iwork, cudaStream_t s) {
  if (r < 1 || r > 64) return (int)cudaErrorInvalidValue;
  tangent_kernel<<<1, 64, 0, s>>>(r, m, q, Ar, Er, Br, Cr, lam, out, work, iwork);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}

int dense_launch_tf(int r, int m, int q, const double* Ar, const double* Er, const double* Br, const double* Cr,
                    const double* omega, int nw, double* H, cudaStream_t s, int order, double alpha, double beta) {
  size_t sm = sizeof(cdouble) * ((size_t)r * r + (size_t)r * m);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(tf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
  }
  tf_kernel<<<nw, 128, sm, s>>>(r, m, q, Ar, Er, Br, Cr, omega, nw, (cdouble*)H, order, alpha, beta);
  mor_count_launches(1);
  return (int)cudaGetLastError();
}
