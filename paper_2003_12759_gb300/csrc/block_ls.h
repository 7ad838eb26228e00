// Block least-squares problem of restarted block GMRES (Saad 2003, Sec. 6.12,
// block GMRES): after k block Arnoldi steps with blocks of p columns,
//     min_Y || E_1 R_0 - Hbar_k Y ||_F,
// Hbar_k the ((k+1)p) x (kp) block upper Hessenberg matrix of the block
// Arnoldi relation A P [V_0 .. V_{k-1}] = [V_0 .. V_k] Hbar_k, and R_0 the
// p x p factor of the first block (R = V_0 R_0).  Solved incrementally: each
// new block column of Hbar gets the Householder reflectors of the earlier
// columns, then one reflector per column zeroes its part below the diagonal
// (the subdiagonal block R_{j+1} is upper triangular, so p + 1 rows are
// touched at most); the same reflectors are applied to G = E_1 R_0.  The
// least-squares residual of right-hand side b after k steps is the norm of
// rows kp .. (k+1)p - 1 of column b of the transformed G; Y comes from one
// triangular solve.  Plain host C++, FP64 complex.
#pragma once
#include <cmath>
#include <complex>
#include <vector>

struct BlockLS {
  typedef std::complex<double> cx;
  int p = 0, m = 0;
  std::vector<cx> H;     // (m+1)p x mp, column-major, leading dimension (m+1)p: R factor in place
  std::vector<cx> G;     // (m+1)p x p, column-major
  std::vector<std::vector<cx>> v;   // reflector of global column c: rows c .. c + len - 1
  std::vector<cx> tau;
  int k = 0;             // block columns added

  void reset(int p_, int m_, const cx* R0 /* p x p, column-major */) {
    p = p_;
    m = m_;
    k = 0;
    const int ldh = (m + 1) * p;
    H.assign((size_t)ldh * m * p, cx(0.0, 0.0));
    G.assign((size_t)ldh * p, cx(0.0, 0.0));
    for (int b = 0; b < p; ++b)
      for (int a = 0; a < p; ++a) G[(size_t)b * ldh + a] = R0[(size_t)b * p + a];
    v.assign((size_t)m * p, std::vector<cx>());
    tau.assign((size_t)m * p, cx(0.0, 0.0));
  }

  // apply reflector of column c, (I - tau w w^H), to column x (leading dimension ld)
  void reflect(int c, cx* x) const {
    const std::vector<cx>& w = v[c];
    cx s(0.0, 0.0);
    for (size_t i = 0; i < w.size(); ++i) s += std::conj(w[i]) * x[c + i];
    s *= tau[c];
    for (size_t i = 0; i < w.size(); ++i) x[c + i] -= s * w[i];
  }

  // Append block column j = k: hcol holds rows 0 .. (j+2)p - 1 of its p
  // columns (column-major, leading dimension (j+2)p).
  void add_block(const cx* hcol) {
    const int j = k;
    const int ldh = (m + 1) * p;
    const int rows = (j + 2) * p;
    for (int c = 0; c < p; ++c) {
      cx* col = &H[(size_t)(j * p + c) * ldh];
      for (int i = 0; i < rows; ++i) col[i] = hcol[(size_t)c * rows + i];
      for (int q = 0; q < j * p; ++q) reflect(q, col);
    }
    // new reflectors for the columns of this block (each applied at once to
    // the block's later columns and to G)
    for (int c = 0; c < p; ++c) {
      const int gc = j * p + c;
      cx* col = &H[(size_t)gc * ldh];
      const int len = rows - gc;       // rows gc .. rows - 1
      double nrm2 = 0.0;
      for (int i = 0; i < len; ++i) nrm2 += std::norm(col[gc + i]);
      const double nrm = std::sqrt(nrm2);
      std::vector<cx> w(len, cx(0.0, 0.0));
      if (nrm == 0.0) {
        tau[gc] = cx(0.0, 0.0);
        w[0] = cx(1.0, 0.0);
      } else {
        const cx x0 = col[gc];
        const double a0 = std::abs(x0);
        const cx ph = a0 > 0.0 ? x0 / a0 : cx(1.0, 0.0);
        const cx alpha = -ph * nrm;              // new diagonal
        w[0] = x0 - alpha;
        for (int i = 1; i < len; ++i) w[i] = col[gc + i];
        double wn2 = 0.0;
        for (int i = 0; i < len; ++i) wn2 += std::norm(w[i]);
        tau[gc] = wn2 > 0.0 ? cx(2.0 / wn2, 0.0) : cx(0.0, 0.0);
        col[gc] = alpha;
        for (int i = 1; i < len; ++i) col[gc + i] = cx(0.0, 0.0);
      }
      v[gc] = w;
      for (int c2 = c + 1; c2 < p; ++c2) reflect(gc, &H[(size_t)(j * p + c2) * ldh]);
      for (int b = 0; b < p; ++b) reflect(gc, &G[(size_t)b * ldh]);
    }
    k = j + 1;
  }

  // least-squares residual norm of right-hand side b after k steps
  double resnorm(int b) const {
    const int ldh = (m + 1) * p;
    double s = 0.0;
    for (int i = k * p; i < (k + 1) * p; ++i) s += std::norm(G[(size_t)b * ldh + i]);
    return std::sqrt(s);
  }

  // Y (kp x p, column-major, leading dimension kp) = R^{-1} G(0:kp, :);
  // a zero diagonal (exact rank deficiency) gives a zero component
  void solve(cx* Y) const {
    const int ldh = (m + 1) * p;
    const int kp = k * p;
    for (int b = 0; b < p; ++b)
      for (int i = kp - 1; i >= 0; --i) {
        cx s = G[(size_t)b * ldh + i];
        for (int l = i + 1; l < kp; ++l) s -= H[(size_t)l * ldh + i] * Y[(size_t)b * kp + l];
        const cx d = H[(size_t)i * ldh + i];
        Y[(size_t)b * kp + i] = (d == cx(0.0, 0.0)) ? cx(0.0, 0.0) : s / d;
      }
  }
};

// Cholesky factor of a p x p Hermitian positive definite G (column-major):
// G = R^H R, R upper triangular (column-major, zero below the diagonal).
// Returns the number of columns factored before a pivot fell to or below
// tol times the largest diagonal of G (p when G is numerically definite).
inline int block_cholesky(int p, const std::complex<double>* G, std::complex<double>* R, double tol) {
  typedef std::complex<double> cx;
  double dmax = 0.0;
  for (int i = 0; i < p; ++i) dmax = std::max(dmax, std::abs(G[(size_t)i * p + i].real()));
  for (size_t i = 0; i < (size_t)p * p; ++i) R[i] = cx(0.0, 0.0);
  for (int j = 0; j < p; ++j) {
    double d = G[(size_t)j * p + j].real();
    for (int l = 0; l < j; ++l) d -= std::norm(R[(size_t)j * p + l]);
    if (!(d > tol * dmax) || !(dmax > 0.0)) return j;
    const double rjj = std::sqrt(d);
    R[(size_t)j * p + j] = cx(rjj, 0.0);
    for (int c = j + 1; c < p; ++c) {
      cx s = G[(size_t)c * p + j];
      for (int l = 0; l < j; ++l) s -= std::conj(R[(size_t)j * p + l]) * R[(size_t)c * p + l];
      R[(size_t)c * p + j] = s / rjj;
    }
  }
  return p;
}

// inverse of a p x p upper triangular R with a nonzero diagonal (column-major)
inline void block_triu_inverse(int p, const std::complex<double>* R, std::complex<double>* Ri) {
  typedef std::complex<double> cx;
  for (size_t i = 0; i < (size_t)p * p; ++i) Ri[i] = cx(0.0, 0.0);
  for (int c = 0; c < p; ++c) {
    Ri[(size_t)c * p + c] = 1.0 / R[(size_t)c * p + c];
    for (int i = c - 1; i >= 0; --i) {
      cx s(0.0, 0.0);
      for (int l = i + 1; l <= c; ++l) s += R[(size_t)l * p + i] * Ri[(size_t)c * p + l];
      Ri[(size_t)c * p + i] = -s / R[(size_t)i * p + i];
    }
  }
}

// Rank-revealing orthonormalisation of a block W (n x p) from its Gram
// matrix G = W^H W (p x p, column-major), by Cholesky with diagonal
// pivoting: G(perm, perm) = R^H R with R upper trapezoidal of rank r (a pivot
// at or below tol times the largest diagonal ends the factor).  Returns r and
//   C (p x p): V = W C has orthonormal columns 0 .. r-1 (the pivoted columns
//              times R11^{-1}) and zero columns r .. p-1;
//   F (p x p): W = V F up to the dropped part (rows r .. p-1 of F are zero),
// both column-major.  Columns that are (numerically) combinations of others
// give zero basis columns instead of noise: the block Krylov space of the
// remaining directions continues, which is the deflation block GMRES needs
// when some right-hand sides converge or coincide.
inline int block_orth_factor(int p, const std::complex<double>* G, double tol, std::complex<double>* C,
                             std::complex<double>* F) {
  typedef std::complex<double> cx;
  std::vector<cx> A(G, G + (size_t)p * p);       // working copy, permuted in place
  std::vector<int> perm(p);
  for (int i = 0; i < p; ++i) perm[i] = i;
  double dmax = 0.0;
  for (int i = 0; i < p; ++i) dmax = std::max(dmax, A[(size_t)i * p + i].real());
  std::vector<cx> R((size_t)p * p, cx(0.0, 0.0));
  int r = 0;
  for (int j = 0; j < p; ++j) {
    // pivot: largest remaining diagonal (Schur complement)
    int q = j;
    double best = -1.0;
    for (int i = j; i < p; ++i) {
      double d = A[(size_t)i * p + i].real();
      for (int l = 0; l < j; ++l) d -= std::norm(R[(size_t)i * p + l]);
      if (d > best) { best = d; q = i; }
    }
    if (!(dmax > 0.0) || !(best > tol * dmax)) break;
    if (q != j) {
      std::swap(perm[j], perm[q]);
      for (int i = 0; i < p; ++i) std::swap(A[(size_t)j * p + i], A[(size_t)q * p + i]);   // columns
      for (int i = 0; i < p; ++i) std::swap(A[(size_t)i * p + j], A[(size_t)i * p + q]);   // rows
      for (int l = 0; l < j; ++l) std::swap(R[(size_t)j * p + l], R[(size_t)q * p + l]);
    }
    const double rjj = std::sqrt(best);
    R[(size_t)j * p + j] = cx(rjj, 0.0);
    for (int c = j + 1; c < p; ++c) {
      cx s = A[(size_t)c * p + j];
      for (int l = 0; l < j; ++l) s -= std::conj(R[(size_t)j * p + l]) * R[(size_t)c * p + l];
      R[(size_t)c * p + j] = s / rjj;
    }
    r = j + 1;
  }
  // R11^{-1} (r x r, upper triangular)
  std::vector<cx> Ri((size_t)r * r, cx(0.0, 0.0));
  for (int c = 0; c < r; ++c) {
    Ri[(size_t)c * r + c] = 1.0 / R[(size_t)c * p + c];
    for (int i = c - 1; i >= 0; --i) {
      cx s(0.0, 0.0);
      for (int l = i + 1; l <= c; ++l) s += R[(size_t)l * p + i] * Ri[(size_t)c * r + l];
      Ri[(size_t)c * r + i] = -s / R[(size_t)i * p + i];
    }
  }
  for (size_t i = 0; i < (size_t)p * p; ++i) { C[i] = cx(0.0, 0.0); F[i] = cx(0.0, 0.0); }
  // V(:, i) = sum_{b < r} W(:, perm[b]) Ri(b, i), i < r
  for (int i = 0; i < r; ++i)
    for (int b = 0; b < r; ++b) C[(size_t)i * p + perm[b]] = Ri[(size_t)i * r + b];
  // W(:, perm[c]) = sum_{i < r} V(:, i) R(i, c)
  for (int c = 0; c < p; ++c)
    for (int i = 0; i < r && i <= c; ++i) F[(size_t)perm[c] * p + i] = R[(size_t)c * p + i];
  return r;
}
