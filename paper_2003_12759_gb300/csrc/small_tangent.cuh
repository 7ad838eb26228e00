// Tangential directions of IRKA for MIMO systems (Algorithm 2 line 3 with
// N_j = 0, read on the reduced pencil): K = E_r^{-1} A_r = R Lambda R^{-1},
// F = E_r^{-1} B_r, C = C_r^T.  The pole lambda_i carries the right direction
// b_i = row i of R^{-1} F and the left direction c_i = column i of C R.
//
// Per pole lambda (one thread): the right eigenvector x (K x = lambda x) and
// the left one y (y^T K = lambda y^T) by two steps of inverse iteration on
// K - lambda I each (complex LU with partial pivoting, FP64; a pivot that
// vanishes because lambda is an exact eigenvalue is replaced by a tiny
// multiple of ||K||), y scaled so that y^T x = 1 -- then y^T is the row of
// R^{-1} that belongs to the column x of R -- and b = F^T y, c = C_r^T x.
// Only the products c_i b_i^T are independent of the eigenvector scale; the
// scale of b_i and c_i does not change the spans IRKA projects on.
// Plain host/device C++ (no CUDA types), so that it also runs on the host.
#pragma once
#include <math.h>

#define TG_IDX(i, j, ld) ((i) + (size_t)(j) * (ld))

struct tz { double re, im; };
__host__ __device__ inline tz tz_c(double a, double b) { tz z; z.re = a; z.im = b; return z; }
__host__ __device__ inline tz tz_add(tz a, tz b) { return tz_c(a.re + b.re, a.im + b.im); }
__host__ __device__ inline tz tz_sub(tz a, tz b) { return tz_c(a.re - b.re, a.im - b.im); }
__host__ __device__ inline tz tz_mul(tz a, tz b) { return tz_c(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
__host__ __device__ inline double tz_abs(tz a) { return hypot(a.re, a.im); }
// a / b by Smith's scaling (no overflow of |b|^2)
__host__ __device__ inline tz tz_div(tz a, tz b) {
  if (fabs(b.re) >= fabs(b.im)) {
    const double t = b.im / b.re, d = b.re + b.im * t;
    return tz_c((a.re + a.im * t) / d, (a.im - a.re * t) / d);
  }
  const double t = b.re / b.im, d = b.re * t + b.im;
  return tz_c((a.re * t + a.im) / d, (a.im * t - a.re) / d);
}

// M = E_r^{-1} A_r (r x r) and F = E_r^{-1} B_r (r x m), column-major, by LU
// with partial pivoting of E_r (LU: r*r work, piv: r).  Returns 1 if E_r is
// singular, 0 otherwise.
__host__ __device__ inline int tangent_prepare(int r, int m, const double* Ar, const double* Er, const double* Br,
                                               double* M, double* F, double* LU, int* piv) {
  for (int i = 0; i < r * r; ++i) LU[i] = Er[i];
  for (int k = 0; k < r; ++k) {
    int p = k;
    double best = fabs(LU[TG_IDX(k, k, r)]);
    for (int i = k + 1; i < r; ++i)
      if (fabs(LU[TG_IDX(i, k, r)]) > best) { best = fabs(LU[TG_IDX(i, k, r)]); p = i; }
    piv[k] = p;
    if (best == 0.0) return 1;
    if (p != k)
      for (int j = 0; j < r; ++j) {
        const double t = LU[TG_IDX(k, j, r)];
        LU[TG_IDX(k, j, r)] = LU[TG_IDX(p, j, r)];
        LU[TG_IDX(p, j, r)] = t;
      }
    for (int i = k + 1; i < r; ++i) {
      const double l = LU[TG_IDX(i, k, r)] / LU[TG_IDX(k, k, r)];
      LU[TG_IDX(i, k, r)] = l;
      for (int j = k + 1; j < r; ++j) LU[TG_IDX(i, j, r)] -= l * LU[TG_IDX(k, j, r)];
    }
  }
  for (int c = 0; c < r + m; ++c) {
    double* x = (c < r) ? M + (size_t)c * r : F + (size_t)(c - r) * r;
    const double* b = (c < r) ? Ar + (size_t)c * r : Br + (size_t)(c - r) * r;
    for (int i = 0; i < r; ++i) x[i] = b[i];
    for (int k = 0; k < r; ++k) {
      const double t = x[k];
      x[k] = x[piv[k]];
      x[piv[k]] = t;
    }
    for (int i = 1; i < r; ++i)
      for (int k = 0; k < i; ++k) x[i] -= LU[TG_IDX(i, k, r)] * x[k];
    for (int i = r - 1; i >= 0; --i) {
      for (int k = i + 1; k < r; ++k) x[i] -= LU[TG_IDX(i, k, r)] * x[k];
      x[i] /= LU[TG_IDX(i, i, r)];
    }
  }
  return 0;
}

// solve (K - lambda I) z = z in place from its LU (trans = 0) or
// (K - lambda I)^T z = z (trans = 1)
__host__ __device__ inline void tangent_solve(int r, const tz* K, const int* piv, tz* z, int trans) {
  if (!trans) {
    for (int k = 0; k < r; ++k) {
      const tz t = z[k];
      z[k] = z[piv[k]];
      z[piv[k]] = t;
    }
    for (int i = 1; i < r; ++i)
      for (int k = 0; k < i; ++k) z[i] = tz_sub(z[i], tz_mul(K[TG_IDX(i, k, r)], z[k]));
    for (int i = r - 1; i >= 0; --i) {
      for (int k = i + 1; k < r; ++k) z[i] = tz_sub(z[i], tz_mul(K[TG_IDX(i, k, r)], z[k]));
      z[i] = tz_div(z[i], K[TG_IDX(i, i, r)]);
    }
  } else {
    // P K = L U  =>  K^T = U^T L^T P:  U^T u = z, L^T w = u, z = P^T w
    for (int i = 0; i < r; ++i) {
      for (int k = 0; k < i; ++k) z[i] = tz_sub(z[i], tz_mul(K[TG_IDX(k, i, r)], z[k]));
      z[i] = tz_div(z[i], K[TG_IDX(i, i, r)]);
    }
    for (int i = r - 2; i >= 0; --i)
      for (int k = i + 1; k < r; ++k) z[i] = tz_sub(z[i], tz_mul(K[TG_IDX(k, i, r)], z[k]));
    for (int k = r - 1; k >= 0; --k) {
      const tz t = z[k];
      z[k] = z[piv[k]];
      z[piv[k]] = t;
    }
  }
}

__host__ __device__ inline void tangent_normalize(int r, tz* z) {
  double s = 0.0;
  for (int i = 0; i < r; ++i) s += z[i].re * z[i].re + z[i].im * z[i].im;
  s = sqrt(s);
  if (s > 0.0)
    for (int i = 0; i < r; ++i) { z[i].re /= s; z[i].im /= s; }
}

// Directions of the pole lam of M (from tangent_prepare): bt (m), ct (q).
// Work: K (r*r), x, y (r each), piv (r).
__host__ __device__ inline void tangent_dirs(int r, int m, int q, const double* M, const double* F, const double* Cr,
                                             tz lam, tz* K, int* piv, tz* x, tz* y, tz* bt, tz* ct) {
  double nrm = tz_abs(lam);
  for (int i = 0; i < r * r; ++i) nrm = fmax(nrm, fabs(M[i]));
  for (int j = 0; j < r; ++j)
    for (int i = 0; i < r; ++i) K[TG_IDX(i, j, r)] = tz_c(M[TG_IDX(i, j, r)] - (i == j ? lam.re : 0.0), i == j ? -lam.im : 0.0);
  const double tiny = 1e-15 * (nrm > 0.0 ? nrm : 1.0);
  for (int k = 0; k < r; ++k) {
    int p = k;
    double best = tz_abs(K[TG_IDX(k, k, r)]);
    for (int i = k + 1; i < r; ++i)
      if (tz_abs(K[TG_IDX(i, k, r)]) > best) { best = tz_abs(K[TG_IDX(i, k, r)]); p = i; }
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < r; ++j) {
        const tz t = K[TG_IDX(k, j, r)];
        K[TG_IDX(k, j, r)] = K[TG_IDX(p, j, r)];
        K[TG_IDX(p, j, r)] = t;
      }
    if (best < tiny) K[TG_IDX(k, k, r)] = tz_c(tiny, 0.0);
    const tz d = K[TG_IDX(k, k, r)];
    for (int i = k + 1; i < r; ++i) {
      const tz l = tz_div(K[TG_IDX(i, k, r)], d);
      K[TG_IDX(i, k, r)] = l;
      for (int j = k + 1; j < r; ++j) K[TG_IDX(i, j, r)] = tz_sub(K[TG_IDX(i, j, r)], tz_mul(l, K[TG_IDX(k, j, r)]));
    }
  }
  for (int i = 0; i < r; ++i) { x[i] = tz_c(1.0, 0.0); y[i] = tz_c(1.0, 0.0); }
  for (int it = 0; it < 2; ++it) {
    tangent_solve(r, K, piv, x, 0);
    tangent_normalize(r, x);
    tangent_solve(r, K, piv, y, 1);
    tangent_normalize(r, y);
  }
  tz s = tz_c(0.0, 0.0);
  for (int i = 0; i < r; ++i) s = tz_add(s, tz_mul(y[i], x[i]));
  for (int i = 0; i < r; ++i) y[i] = tz_div(y[i], s);
  for (int j = 0; j < m; ++j) {
    tz a = tz_c(0.0, 0.0);
    for (int l = 0; l < r; ++l) a = tz_add(a, tz_c(F[TG_IDX(l, j, r)] * y[l].re, F[TG_IDX(l, j, r)] * y[l].im));
    bt[j] = a;
  }
  for (int j = 0; j < q; ++j) {
    tz a = tz_c(0.0, 0.0);
    for (int l = 0; l < r; ++l) a = tz_add(a, tz_c(Cr[TG_IDX(l, j, r)] * x[l].re, Cr[TG_IDX(l, j, r)] * x[l].im));
    ct[j] = a;
  }
}
