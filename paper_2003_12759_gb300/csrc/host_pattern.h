// Host-side construction of the sparsity data of the solve path, plain C++
// (no CUDA), so that it also compiles for the host tests:
//   * the static SPAI / reuse pattern S = pattern(A) + pattern(E) + diagonal
//     (Sec. III.A with a static pattern: every P and Q has the pattern of the
//     shifted matrix, diagonal included so that column j of A(sigma_old)
//     restricted to the shadow rows is exact for the reuse right-hand side),
//     with A's and E's values aligned to it;
//   * its transpose and the map between the two orders;
//   * the shadow sets I_j = union over k in J_j of the pattern of column k
//     (the rows a column least-squares problem of Eq. gen-precond-par touches);
//   * the SELL-32 layout (slices of 32 rows, column-major inside a slice);
//   * the diagonal (DIA) layout of patterns with few distinct diagonals.
#pragma once
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace mor_host {

struct HostCSR {
  int64_t n = 0;
  std::vector<int32_t> rowptr, col;
  std::vector<double> val;
};

// merged pattern of A (+ E) + diagonal, values aligned
inline void merge_pattern(const HostCSR& A, const HostCSR* E, HostCSR& S, std::vector<double>& sa, std::vector<double>& se) {
  const int64_t n = A.n;
  S.n = n;
  S.rowptr.assign(n + 1, 0);
  S.col.clear();
  sa.clear();
  se.clear();
  S.col.reserve(A.col.size() + n + (E ? E->col.size() : 0));
  sa.reserve(S.col.capacity());
  if (E) se.reserve(S.col.capacity());
  for (int64_t i = 0; i < n; ++i) {
    int32_t pa = A.rowptr[i], ea = A.rowptr[i + 1];
    int32_t pe = E ? E->rowptr[i] : 0, ee = E ? E->rowptr[i + 1] : 0;
    bool diag_done = false;
    while (pa < ea || pe < ee || !diag_done) {
      int64_t ca = pa < ea ? A.col[pa] : INT64_MAX;
      int64_t ce = pe < ee ? E->col[pe] : INT64_MAX;
      int64_t cd = diag_done ? INT64_MAX : i;
      int64_t c = std::min(ca, std::min(ce, cd));
      double va = 0.0, ve = 0.0;
      if (ca == c) { va = A.val[pa]; ++pa; }
      if (ce == c) { ve = E->val[pe]; ++pe; }
      if (cd == c) diag_done = true;
      S.col.push_back((int32_t)c);
      sa.push_back(va);
      if (E) se.push_back(ve);
    }
    S.rowptr[i + 1] = (int32_t)S.col.size();
  }
}

// transpose pattern; t2p[t] = position in S of the entry at T position t
inline void transpose_pattern(const HostCSR& S, HostCSR& T, std::vector<int64_t>& t2p) {
  const int64_t n = S.n, nnz = (int64_t)S.col.size();
  T.n = n;
  T.rowptr.assign(n + 1, 0);
  for (int64_t p = 0; p < nnz; ++p) T.rowptr[S.col[p] + 1]++;
  for (int64_t i = 0; i < n; ++i) T.rowptr[i + 1] += T.rowptr[i];
  T.col.resize(nnz);
  t2p.resize(nnz);
  std::vector<int32_t> next(T.rowptr.begin(), T.rowptr.end() - 1);
  for (int64_t i = 0; i < n; ++i)
    for (int32_t p = S.rowptr[i]; p < S.rowptr[i + 1]; ++p) {
      const int32_t t = next[S.col[p]]++;
      T.col[t] = (int32_t)i;
      t2p[t] = p;
    }
}

// shadow sets: for column j of the operator whose columns are the rows of
// `cols` (a CSR whose row j lists J_j), I_j = union over k in J_j of row k.
inline void shadow_sets(const HostCSR& cols, std::vector<int64_t>& iptr, std::vector<int32_t>& iidx, int& nImax, int& nJmax) {
  const int64_t n = cols.n;
  unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  if (n < 20000) nt = 1;
  std::vector<std::vector<int32_t>> parts(nt);
  std::vector<std::vector<int32_t>> counts(nt);
  std::vector<int> maxI(nt, 0);
  auto work = [&](unsigned t) {
    const int64_t j0 = n * t / nt, j1 = n * (t + 1) / nt;
    std::vector<int64_t> stamp(n, -1);
    std::vector<int32_t> buf;
    auto& out = parts[t];
    auto& cnt = counts[t];
    cnt.reserve(j1 - j0);
    for (int64_t j = j0; j < j1; ++j) {
      buf.clear();
      for (int32_t p = cols.rowptr[j]; p < cols.rowptr[j + 1]; ++p) {
        const int32_t k = cols.col[p];
        for (int32_t q = cols.rowptr[k]; q < cols.rowptr[k + 1]; ++q) {
          const int32_t i = cols.col[q];
          if (stamp[i] != j) { stamp[i] = j; buf.push_back(i); }
        }
      }
      std::sort(buf.begin(), buf.end());
      out.insert(out.end(), buf.begin(), buf.end());
      cnt.push_back((int32_t)buf.size());
      maxI[t] = std::max(maxI[t], (int)buf.size());
    }
  };
  std::vector<std::thread> th;
  for (unsigned t = 1; t < nt; ++t) th.emplace_back(work, t);
  work(0);
  for (auto& x : th) x.join();
  iptr.assign(n + 1, 0);
  int64_t j = 0;
  for (unsigned t = 0; t < nt; ++t)
    for (int32_t c : counts[t]) { iptr[j + 1] = iptr[j] + c; ++j; }
  iidx.resize(iptr[n]);
  int64_t off = 0;
  for (unsigned t = 0; t < nt; ++t) {
    std::memcpy(iidx.data() + off, parts[t].data(), parts[t].size() * sizeof(int32_t));
    off += (int64_t)parts[t].size();
  }
  nImax = 0;
  for (int x : maxI) nImax = std::max(nImax, x);
  nJmax = 0;
  for (int64_t jj = 0; jj < n; ++jj) nJmax = std::max(nJmax, cols.rowptr[jj + 1] - cols.rowptr[jj]);
}

// SELL-32 (sigma = 1) layout of a CSR pattern: slice offsets, padded columns,
// and the map CSR position -> layout position.
inline void sell_layout(const HostCSR& S, std::vector<int64_t>& sptr, std::vector<int32_t>& scol, std::vector<int64_t>& lay) {
  const int64_t n = S.n;
  const int64_t ns = (n + 31) / 32;
  sptr.assign(ns + 1, 0);
  for (int64_t s = 0; s < ns; ++s) {
    int w = 0;
    for (int64_t r = s * 32; r < std::min(n, s * 32 + 32); ++r) w = std::max(w, S.rowptr[r + 1] - S.rowptr[r]);
    sptr[s + 1] = sptr[s] + 32LL * w;
  }
  scol.assign(sptr[ns], 0);
  lay.resize(S.col.size());
  for (int64_t s = 0; s < ns; ++s) {
    const int64_t w = (sptr[s + 1] - sptr[s]) / 32;
    for (int64_t l = 0; l < 32; ++l) {
      const int64_t r = s * 32 + l;
      for (int64_t t = 0; t < w; ++t) {
        const int64_t pos = sptr[s] + 32 * t + l;
        if (r < n && t < S.rowptr[r + 1] - S.rowptr[r]) {
          const int64_t p = S.rowptr[r] + t;
          scol[pos] = S.col[p];
          lay[p] = pos;
        } else {
          scol[pos] = (int32_t)std::min<int64_t>(r, n - 1);   // padding: a valid index, value 0
        }
      }
    }
  }
}

// Diagonal layout: the distinct offsets c - r of the pattern, ascending, and
// every entry (r, c) at position d n + r, d the index of its offset (so the
// entries of one diagonal are contiguous and ordered by row, and a row's
// entries come in the order of its columns).  Positions of no entry are
// padding (value 0).  Returns false, with nothing set, when the pattern has
// more than max_diag offsets or its ndiag n stored entries exceed max_fill
// times its entries (or 2^31).
inline bool dia_layout(const HostCSR& S, int max_diag, double max_fill, std::vector<int32_t>& offsets,
                       std::vector<int64_t>& lay) {
  const int64_t n = S.n;
  const int64_t nnz = (int64_t)S.col.size();
  std::vector<int32_t> offs;
  for (int64_t r = 0; r < n; ++r) {
    for (int32_t p = S.rowptr[r]; p < S.rowptr[r + 1]; ++p) {
      const int32_t o = (int32_t)(S.col[p] - r);
      if (std::find(offs.begin(), offs.end(), o) == offs.end()) {
        offs.push_back(o);
        if ((int)offs.size() > max_diag) return false;
      }
    }
  }
  std::sort(offs.begin(), offs.end());
  const int64_t nlay = (int64_t)offs.size() * n;
  if (nnz == 0 || (double)nlay > max_fill * (double)nnz || nlay > (int64_t)INT32_MAX) return false;
  std::vector<int64_t> out(nnz);
  for (int64_t r = 0; r < n; ++r) {
    for (int32_t p = S.rowptr[r]; p < S.rowptr[r + 1]; ++p) {
      const int32_t o = (int32_t)(S.col[p] - r);
      const int64_t d = std::lower_bound(offs.begin(), offs.end(), o) - offs.begin();
      out[p] = d * n + r;
    }
  }
  offsets.swap(offs);
  lay.swap(out);
  return true;
}

}  // namespace mor_host
