// Expansion-point update of the second-order reduction (Algorithm 1 line 11
// states only that all points are updated).  Reading: the new points are the
// mirror images sigma = |Re lambda| - i Im lambda of the eigenvalues of the
// reduced quadratic eigenproblem (lambda^2 M_r + lambda D_r + K_r) x = 0,
// D_r = alpha M_r + beta K_r, of smallest modulus, as many as before, closed
// under conjugation: candidates in order of increasing |lambda| (ties by Re,
// then Im), a conjugate pair only when two places are left; one place left
// with only pairs to come takes the real point |lambda| of the first pair
// that did not fit.
// The eigenvalues come from the first companion pencil
//   [[0, I], [-K_r, -D_r]] z = lambda [[I, 0], [0, M_r]] z,  z = [x; lambda x],
// handed to small_eig.  Plain host/device C++.
#pragma once
#include <math.h>

#include "small_eig.cuh"

// A2, E2: 2r x 2r column-major
__host__ __device__ inline void qep_pencil(int r, const double* Mr, const double* Kr, double alpha, double beta,
                                           double* A2, double* E2) {
  const int n2 = 2 * r;
  for (int t = 0; t < n2 * n2; ++t) { A2[t] = 0.0; E2[t] = 0.0; }
  for (int i = 0; i < r; ++i) {
    A2[SE_IDX(i, r + i, n2)] = 1.0;
    E2[SE_IDX(i, i, n2)] = 1.0;
  }
  for (int j = 0; j < r; ++j)
    for (int i = 0; i < r; ++i) {
      const double m = Mr[SE_IDX(i, j, r)], k = Kr[SE_IDX(i, j, r)];
      A2[SE_IDX(r + i, j, n2)] = -k;
      A2[SE_IDX(r + i, r + j, n2)] = -(alpha * m + beta * k);
      E2[SE_IDX(r + i, r + j, n2)] = m;
    }
}

// count new points (pr, pi), sorted by (Re, |Im|, -Im), from ne eigenvalues
// (wr, wi; conjugate pairs exact).  work: 3 ne doubles.  Returns 0, or 1 if
// the eigenvalues cannot fill `count` places.
__host__ __device__ inline int qep_select(int ne, const double* wr, const double* wi, int count, double* pr,
                                          double* pi, double* work) {
  double* mod = work;
  double* cre = work + ne;
  double* cim = work + 2 * ne;
  int nc = 0;
  for (int e = 0; e < ne; ++e) {
    if (wi[e] < 0.0) continue;                  // the Im > 0 member stands for its pair
    mod[nc] = hypot(wr[e], wi[e]);
    cre[nc] = wr[e];
    cim[nc] = wi[e];
    ++nc;
  }
  // insertion sort of the candidates by (modulus, Re, Im)
  for (int i = 1; i < nc; ++i) {
    const double a = mod[i], b = cre[i], c = cim[i];
    int j = i - 1;
    while (j >= 0) {
      bool gt;
      if (mod[j] != a) gt = mod[j] > a;
      else if (cre[j] != b) gt = cre[j] > b;
      else gt = cim[j] > c;
      if (!gt) break;
      mod[j + 1] = mod[j]; cre[j + 1] = cre[j]; cim[j + 1] = cim[j];
      --j;
    }
    mod[j + 1] = a; cre[j + 1] = b; cim[j + 1] = c;
  }
  int np = 0, left = count;
  double skipped = -1.0;
  for (int i = 0; i < nc && left > 0; ++i) {
    const int size = (cim[i] == 0.0) ? 1 : 2;
    if (size <= left) {
      pr[np] = fabs(cre[i]);
      pi[np] = -cim[i];
      ++np;
      if (size == 2) {
        pr[np] = fabs(cre[i]);
        pi[np] = cim[i];
        ++np;
      }
      left -= size;
    } else if (skipped < 0.0) {
      skipped = mod[i];
    }
  }
  if (left > 0) {
    if (skipped < 0.0) return 1;
    pr[np] = skipped;
    pi[np] = 0.0;
    ++np;
  }
  // final order (Re, |Im|, -Im)
  for (int i = 1; i < np; ++i) {
    const double a = pr[i], b = pi[i];
    int j = i - 1;
    while (j >= 0) {
      bool gt;
      if (pr[j] != a) gt = pr[j] > a;
      else if (fabs(pi[j]) != fabs(b)) gt = fabs(pi[j]) > fabs(b);
      else gt = (-pi[j]) > (-b);
      if (!gt) break;
      pr[j + 1] = pr[j]; pi[j + 1] = pi[j];
      --j;
    }
    pr[j + 1] = a; pi[j + 1] = b;
  }
  return 0;
}
