// Reuse-or-rebuild decision of the SPAI reuse schedule.  The paper motivates
// reuse with three Frobenius ratios (Sec. IV, the table of its reuse
// experiment): reuse pays when ||I - A_new||_F / ||I||_F is large and the
// change ||A_old - A_new||_F / ||A_old||_F is small.  It fixes no thresholds;
// the reading taken here: reuse when the change ratio is below 1 and below
// the first ratio, otherwise build a fresh SPAI for the new shift.
//
// Every shifted matrix of the method has the form A(s) = c1(s) P + c2(s) Q:
//   first order   P = E, Q = A:  c1 = s,              c2 = -1
//   second order  P = M, Q = K:  c1 = s^2 + alpha s,  c2 = 1 + beta s
// so with the scalar products <P,P>, <P,Q>, <Q,Q>, tr P, tr Q (computed once
// from the stored matrices) the three quantities follow in closed form:
//   ||c1 P + c2 Q||_F^2 = |c1|^2 <P,P> + 2 Re(conj(c1) c2) <P,Q> + |c2|^2 <Q,Q>
//   ||I - A(s)||_F^2    = n - 2 Re tr A(s) + ||A(s)||_F^2,  tr A(s) = c1 tr P + c2 tr Q
//   A(s1) - A(s2)       = (c1(s1) - c1(s2)) P + (c2(s1) - c2(s2)) Q.
// Transposition changes none of them.  Plain host C++.
#pragma once
#include <cmath>
#include <cstdint>

struct FrobScalars {
  int order = 1;
  double n = 0.0;
  double PP = 0.0, PQ = 0.0, QQ = 0.0, trP = 0.0, trQ = 0.0;
  double alpha = 0.0, beta = 0.0;
};

struct frob_z { double re, im; };

inline frob_z frob_coef1(const FrobScalars& f, frob_z s) {
  if (f.order == 1) return s;
  // s^2 + alpha s
  return frob_z{s.re * s.re - s.im * s.im + f.alpha * s.re, 2.0 * s.re * s.im + f.alpha * s.im};
}
inline frob_z frob_coef2(const FrobScalars& f, frob_z s) {
  if (f.order == 1) return frob_z{-1.0, 0.0};
  return frob_z{1.0 + f.beta * s.re, f.beta * s.im};
}

// ||c1 P + c2 Q||_F^2
inline double frob_norm2(const FrobScalars& f, frob_z c1, frob_z c2) {
  const double a2 = c1.re * c1.re + c1.im * c1.im, b2 = c2.re * c2.re + c2.im * c2.im;
  const double cross = c1.re * c2.re + c1.im * c2.im;   // Re(conj(c1) c2)
  const double v = a2 * f.PP + 2.0 * cross * f.PQ + b2 * f.QQ;
  return v > 0.0 ? v : 0.0;
}

// ||I - A(s)||_F / ||I||_F
inline double frob_ratio_identity(const FrobScalars& f, frob_z s) {
  const frob_z c1 = frob_coef1(f, s), c2 = frob_coef2(f, s);
  const double tr_re = c1.re * f.trP + c2.re * f.trQ;
  const double v = f.n - 2.0 * tr_re + frob_norm2(f, c1, c2);
  return std::sqrt(v > 0.0 ? v : 0.0) / std::sqrt(f.n);
}

// ||A(s_old) - A(s_new)||_F / ||A(s_old)||_F
inline double frob_ratio_change(const FrobScalars& f, frob_z s_old, frob_z s_new) {
  const frob_z a0 = frob_coef1(f, s_old), b0 = frob_coef2(f, s_old);
  const frob_z a1 = frob_coef1(f, s_new), b1 = frob_coef2(f, s_new);
  const double den = frob_norm2(f, a0, b0);
  if (!(den > 0.0)) return INFINITY;
  const double num = frob_norm2(f, frob_z{a0.re - a1.re, a0.im - a1.im}, frob_z{b0.re - b1.re, b0.im - b1.im});
  return std::sqrt(num / den);
}

inline bool frob_reuse_ok(const FrobScalars& f, frob_z s_old, frob_z s_new) {
  const double change = frob_ratio_change(f, s_old, s_new);
  const double ident = frob_ratio_identity(f, s_new);
  return change < (ident < 1.0 ? ident : 1.0);
}

// ---- scalar products of the stored matrices (CSR with sorted, unique columns per row)
inline double frob_csr_self(int64_t n, const int32_t* rp, const double* val) {
  double s = 0.0;
  for (int64_t p = 0; p < rp[n]; ++p) s += val[p] * val[p];
  return s;
}
inline double frob_csr_trace(int64_t n, const int32_t* rp, const int32_t* col, const double* val) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
      if (col[p] == i) s += val[p];
  return s;
}
// <X, Y> = sum_ij X_ij Y_ij by merging the sorted rows
inline double frob_csr_dot(int64_t n, const int32_t* rx, const int32_t* cx, const double* vx, const int32_t* ry,
                           const int32_t* cy, const double* vy) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t p = rx[i], q = ry[i];
    while (p < rx[i + 1] && q < ry[i + 1]) {
      if (cx[p] < cy[q]) ++p;
      else if (cx[p] > cy[q]) ++q;
      else { s += vx[p] * vy[q]; ++p; ++q; }
    }
  }
  return s;
}
// <diag(d), Y> = sum_i d_i Y_ii
inline double frob_diag_dot(int64_t n, const double* d, const int32_t* ry, const int32_t* cy, const double* vy) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int32_t q = ry[i]; q < ry[i + 1]; ++q)
      if (cy[q] == i) s += d[i] * vy[q];
  return s;
}

// The scalars for A(s) = c1(s) P + c2(s) Q with Q in CSR and P either the
// identity (pdiag == nullptr and prp == nullptr), diagonal (pdiag) or CSR.
inline FrobScalars frob_scalars(int order, double alpha, double beta, int64_t n, const double* pdiag,
                                const int32_t* prp, const int32_t* pcol, const double* pval, const int32_t* qrp,
                                const int32_t* qcol, const double* qval) {
  FrobScalars f;
  f.order = order;
  f.alpha = alpha;
  f.beta = beta;
  f.n = (double)n;
  f.QQ = frob_csr_self(n, qrp, qval);
  f.trQ = frob_csr_trace(n, qrp, qcol, qval);
  if (prp) {
    f.PP = frob_csr_self(n, prp, pval);
    f.trP = frob_csr_trace(n, prp, pcol, pval);
    f.PQ = frob_csr_dot(n, prp, pcol, pval, qrp, qcol, qval);
  } else if (pdiag) {
    double pp = 0.0, tr = 0.0;
    for (int64_t i = 0; i < n; ++i) { pp += pdiag[i] * pdiag[i]; tr += pdiag[i]; }
    f.PP = pp;
    f.trP = tr;
    f.PQ = frob_diag_dot(n, pdiag, qrp, qcol, qval);
  } else {
    f.PP = (double)n;
    f.trP = (double)n;
    f.PQ = f.trQ;
  }
  return f;
}
