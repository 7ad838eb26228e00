// Eigenvalues of a small real pencil (A_r, E_r), r <= 64, in FP64:
//   1. LU with partial pivoting of E_r and M = E_r^{-1} A_r,
//   2. reduction of M to upper Hessenberg form by Householder reflections
//      (Golub & Van Loan, Matrix Computations, Alg. 7.4.2),
//   3. Francis implicit double-shift QR with deflation on the Hessenberg
//      matrix (Golub & Van Loan Alg. 7.5.1 / 7.5.2); 1x1 blocks give real
//      eigenvalues, 2x2 blocks real pairs or exact complex-conjugate pairs.
// Written as plain host/device C++ so that one thread of one block runs it.
// Only eigenvalues are computed (no Schur vectors), so the transformations
// are applied inside the active window only.
#pragma once
#include <math.h>

#define SE_IDX(i, j, ld) ((i) + (size_t)(j) * (ld))

// returns 0 on success, 1 if E is singular, 2 if QR did not converge
__host__ __device__ inline int small_eig(int r, const double* Ar, const double* Er, double* M /* r*r work */,
                                         double* LU /* r*r work */, int* piv, double* wr, double* wi) {
  // ---- LU of E with partial pivoting
  for (int i = 0; i < r * r; ++i) LU[i] = Er[i];
  for (int k = 0; k < r; ++k) {
    int p = k;
    double best = fabs(LU[SE_IDX(k, k, r)]);
    for (int i = k + 1; i < r; ++i) {
      double v = fabs(LU[SE_IDX(i, k, r)]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (best == 0.0) return 1;
    if (p != k)
      for (int j = 0; j < r; ++j) { double t = LU[SE_IDX(k, j, r)]; LU[SE_IDX(k, j, r)] = LU[SE_IDX(p, j, r)]; LU[SE_IDX(p, j, r)] = t; }
    const double d = LU[SE_IDX(k, k, r)];
    for (int i = k + 1; i < r; ++i) {
      const double l = LU[SE_IDX(i, k, r)] / d;
      LU[SE_IDX(i, k, r)] = l;
      for (int j = k + 1; j < r; ++j) LU[SE_IDX(i, j, r)] -= l * LU[SE_IDX(k, j, r)];
    }
  }
  // ---- M = E^{-1} A, column by column
  for (int j = 0; j < r; ++j) {
    double* x = M + (size_t)j * r;
    for (int i = 0; i < r; ++i) x[i] = Ar[SE_IDX(i, j, r)];
    for (int k = 0; k < r; ++k) { int p = piv[k]; if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; } }
    for (int i = 0; i < r; ++i) for (int k = 0; k < i; ++k) x[i] -= LU[SE_IDX(i, k, r)] * x[k];
    for (int i = r - 1; i >= 0; --i) {
      for (int k = i + 1; k < r; ++k) x[i] -= LU[SE_IDX(i, k, r)] * x[k];
      x[i] /= LU[SE_IDX(i, i, r)];
    }
  }
  double* H = M;
  const int n = r;
  // ---- Householder reduction to Hessenberg form
  double v[64];
  for (int k = 0; k < n - 2; ++k) {
    double alpha = 0.0;
    for (int i = k + 1; i < n; ++i) alpha += H[SE_IDX(i, k, n)] * H[SE_IDX(i, k, n)];
    alpha = sqrt(alpha);
    if (alpha == 0.0) continue;
    const double x0 = H[SE_IDX(k + 1, k, n)];
    const double sgn = (x0 >= 0.0) ? 1.0 : -1.0;
    for (int i = k + 1; i < n; ++i) v[i] = H[SE_IDX(i, k, n)];
    v[k + 1] += sgn * alpha;
    double vn2 = 0.0;
    for (int i = k + 1; i < n; ++i) vn2 += v[i] * v[i];
    if (vn2 == 0.0) continue;
    const double beta = 2.0 / vn2;
    for (int j = 0; j < n; ++j) {          // H = (I - beta v v^T) H
      double s = 0.0;
      for (int i = k + 1; i < n; ++i) s += v[i] * H[SE_IDX(i, j, n)];
      s *= beta;
      for (int i = k + 1; i < n; ++i) H[SE_IDX(i, j, n)] -= s * v[i];
    }
    for (int i = 0; i < n; ++i) {          // H = H (I - beta v v^T)
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += H[SE_IDX(i, j, n)] * v[j];
      s *= beta;
      for (int j = k + 1; j < n; ++j) H[SE_IDX(i, j, n)] -= s * v[j];
    }
    for (int i = k + 2; i < n; ++i) H[SE_IDX(i, k, n)] = 0.0;
  }
  // ---- Francis double-shift QR with deflation
  int hi = n - 1;
  int its = 0, total = 0;
  const double eps = 2.220446049250313e-16;
  while (hi >= 0) {
    // find the start lo of the unreduced block ending at hi
    int lo = hi;
    while (lo > 0) {
      double s = fabs(H[SE_IDX(lo - 1, lo - 1, n)]) + fabs(H[SE_IDX(lo, lo, n)]);
      if (s == 0.0) s = 1.0;
      if (fabs(H[SE_IDX(lo, lo - 1, n)]) <= eps * s) { H[SE_IDX(lo, lo - 1, n)] = 0.0; break; }
      --lo;
    }
    if (lo == hi) {                         // 1x1 block
      wr[hi] = H[SE_IDX(hi, hi, n)];
      wi[hi] = 0.0;
      --hi;
      its = 0;
      continue;
    }
    if (lo == hi - 1) {                     // 2x2 block
      const double a = H[SE_IDX(hi - 1, hi - 1, n)], b = H[SE_IDX(hi - 1, hi, n)];
      const double c = H[SE_IDX(hi, hi - 1, n)], d = H[SE_IDX(hi, hi, n)];
      const double p = 0.5 * (a - d);
      const double disc = p * p + b * c;
      const double mid = 0.5 * (a + d);
      if (disc >= 0.0) {
        const double sq = sqrt(disc);
        const double l1 = mid + ((p >= 0.0) ? sq : -sq);
        const double det = a * d - b * c;
        const double l2 = (l1 != 0.0) ? det / l1 : mid - ((p >= 0.0) ? sq : -sq);
        wr[hi - 1] = l1; wi[hi - 1] = 0.0;
        wr[hi] = l2; wi[hi] = 0.0;
      } else {
        const double sq = sqrt(-disc);
        wr[hi - 1] = mid; wi[hi - 1] = sq;
        wr[hi] = mid; wi[hi] = -sq;
      }
      hi -= 2;
      its = 0;
      continue;
    }
    if (++total > 100 * n) return 2;
    ++its;
    // shifts: eigenvalues of the trailing 2x2 (via trace s and determinant t),
    // with an exceptional shift every 10 stagnant iterations
    double s, t;
    if (its % 10 == 0) {
      const double w = fabs(H[SE_IDX(hi, hi - 1, n)]) + fabs(H[SE_IDX(hi - 1, hi - 2, n)]);
      s = 1.5 * w;
      t = w * w;
    } else {
      s = H[SE_IDX(hi - 1, hi - 1, n)] + H[SE_IDX(hi, hi, n)];
      t = H[SE_IDX(hi - 1, hi - 1, n)] * H[SE_IDX(hi, hi, n)] - H[SE_IDX(hi - 1, hi, n)] * H[SE_IDX(hi, hi - 1, n)];
    }
    // first column of (H - s1 I)(H - s2 I) = H^2 - s H + t I
    const double h00 = H[SE_IDX(lo, lo, n)], h10 = H[SE_IDX(lo + 1, lo, n)];
    const double h01 = H[SE_IDX(lo, lo + 1, n)], h11 = H[SE_IDX(lo + 1, lo + 1, n)];
    const double h21 = H[SE_IDX(lo + 2, lo + 1, n)];
    double x = h00 * h00 + h01 * h10 - s * h00 + t;
    double y = h10 * (h00 + h11 - s);
    double z = h10 * h21;
    for (int k = lo; k <= hi - 2; ++k) {
      // 3-element reflector P = I - beta u u^T with P [x y z]^T = -sign * norm e1
      double nrm = sqrt(x * x + y * y + z * z);
      if (nrm != 0.0) {
        double u0 = x + ((x >= 0.0) ? nrm : -nrm), u1 = y, u2 = z;
        const double beta = 2.0 / (u0 * u0 + u1 * u1 + u2 * u2);
        const int q = (k > lo) ? k - 1 : lo;
        for (int j = q; j <= hi; ++j) {
          double sum = u0 * H[SE_IDX(k, j, n)] + u1 * H[SE_IDX(k + 1, j, n)] + u2 * H[SE_IDX(k + 2, j, n)];
          sum *= beta;
          H[SE_IDX(k, j, n)] -= sum * u0;
          H[SE_IDX(k + 1, j, n)] -= sum * u1;
          H[SE_IDX(k + 2, j, n)] -= sum * u2;
        }
        const int rmax = (k + 3 < hi) ? k + 3 : hi;
        for (int i = lo; i <= rmax; ++i) {
          double sum = H[SE_IDX(i, k, n)] * u0 + H[SE_IDX(i, k + 1, n)] * u1 + H[SE_IDX(i, k + 2, n)] * u2;
          sum *= beta;
          H[SE_IDX(i, k, n)] -= sum * u0;
          H[SE_IDX(i, k + 1, n)] -= sum * u1;
          H[SE_IDX(i, k + 2, n)] -= sum * u2;
        }
      }
      x = H[SE_IDX(k + 1, k, n)];
      y = H[SE_IDX(k + 2, k, n)];
      if (k < hi - 2) z = H[SE_IDX(k + 3, k, n)];
    }
    // final 2-element reflector on rows/cols hi-1, hi
    {
      double nrm = sqrt(x * x + y * y);
      if (nrm != 0.0) {
        const int k = hi - 1;
        double u0 = x + ((x >= 0.0) ? nrm : -nrm), u1 = y;
        const double beta = 2.0 / (u0 * u0 + u1 * u1);
        for (int j = k - 1; j <= hi; ++j) {
          double sum = (u0 * H[SE_IDX(k, j, n)] + u1 * H[SE_IDX(k + 1, j, n)]) * beta;
          H[SE_IDX(k, j, n)] -= sum * u0;
          H[SE_IDX(k + 1, j, n)] -= sum * u1;
        }
        for (int i = lo; i <= hi; ++i) {
          double sum = (H[SE_IDX(i, k, n)] * u0 + H[SE_IDX(i, k + 1, n)] * u1) * beta;
          H[SE_IDX(i, k, n)] -= sum * u0;
          H[SE_IDX(i, k + 1, n)] -= sum * u1;
        }
      }
    }
  }
  return 0;
}

// sigma = |Re lambda| - i Im lambda, sorted by (Re, |Im|, -Im) (insertion sort)
__host__ __device__ inline void mirror_sort(int r, const double* wr, const double* wi, double* sr, double* si) {
  for (int i = 0; i < r; ++i) { sr[i] = fabs(wr[i]); si[i] = -wi[i]; }
  for (int i = 1; i < r; ++i) {
    double a = sr[i], b = si[i];
    int j = i - 1;
    while (j >= 0) {
      bool gt;
      if (sr[j] != a) gt = sr[j] > a;
      else if (fabs(si[j]) != fabs(b)) gt = fabs(si[j]) > fabs(b);
      else gt = (-si[j]) > (-b);
      if (!gt) break;
      sr[j + 1] = sr[j]; si[j + 1] = si[j];
      --j;
    }
    sr[j + 1] = a; si[j + 1] = b;
  }
}
