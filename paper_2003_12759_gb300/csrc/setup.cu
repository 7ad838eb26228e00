// Handle lifecycle and system set-up (host C++ runtime).
//
// mor_set_system builds, once per system, everything the hot path reads:
//   * the SPAI pattern S = pattern(A) + pattern(E) + diagonal (the pattern of
//     sigma E - A for generic sigma) with A and E values aligned to it;
//   * the transposed pattern S^T with its values (for the W solves, which use
//     A(sigma)^T, Algorithm 2 line 5) and the position maps between the two;
//   * the shadow sets I_j (rows reached by the columns J_j) of every column,
//     which fix the size of each column least-squares problem of the SPAI;
//   * the storage layout (CSR or SELL-32), chosen by timing both (the
//     autotuner) unless the caller fixes it.
// All host work is O(nnz) or O(sum |I_j|), multi-threaded where it matters.
#include "mor_ctx.h"
#include "mor_types.cuh"
#include "host_pattern.h"
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <thread>
#include <atomic>
#include <mutex>
#include <map>

static std::atomic<long long> g_launches{0};
// launches recorded into a CUDA graph are counted when the graph is replayed
static thread_local int t_capturing = 0;
void mor_count_launches(int64_t n) { if (!t_capturing) g_launches += n; }
// SpMV launches by (kernel, vector type, real columns): process-wide, and the
// part recorded into the graph this thread is capturing
static std::atomic<long long> g_tally[2][4][MOR_KMAX + 1];
static thread_local ShapeTally t_cap_tally;
void mor_capture_mark(int on) {
  t_capturing = on;
  if (on) t_cap_tally = ShapeTally{};
}
void mor_tally(int kernel, int st, int kreal, int64_t n) {
  if (kernel < 0 || kernel > 1 || st < 0 || st > 3 || kreal < 0 || kreal > MOR_KMAX) return;
  if (t_capturing) t_cap_tally.c[kernel][st][kreal] += n;
  else g_tally[kernel][st][kreal] += n;
}
ShapeTally mor_capture_tally() { return t_cap_tally; }
void mor_replay_tally(const ShapeTally& t) {
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c <= MOR_KMAX; ++c)
        if (t.c[a][b][c]) g_tally[a][b][c] += t.c[a][b][c];
}

int mor_fail(mor_t h, int code, const char* fmt, ...) {
  if (h) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    static std::mutex mu;                 // two lanes may fail at once
    std::lock_guard<std::mutex> lk(mu);
    h->err = buf;
  }
  return code;
}

int mor_lane(mor_t h, int i, SolveLane** out) {
  SolveLane& L = h->lanes[i];
  if (!L.stream) {
    if (i == 0) L.stream = h->stream;
    else {
      if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess)
        return mor_fail(h, MOR_ECUDA, "cannot create the second solve stream");
      L.own_stream = true;
    }
  }
  if (!L.pinned) {
    L.pinned_bytes = 1 << 21;
    if (cudaHostAlloc(&L.pinned, L.pinned_bytes, cudaHostAllocDefault) != cudaSuccess) {
      L.pinned = nullptr;
      return mor_fail(h, MOR_ENOMEM, "cannot allocate pinned host memory");
    }
  }
  *out = &L;
  return MOR_OK;
}

Coef mor_coef(const mor_ctx* h, mor_c64 s) {
  Coef c;
  if (h->order == 2) {
    // (s^2 + alpha s) M + (1 + beta s) K
    c.sEr = s.re * s.re - s.im * s.im + h->alpha * s.re;
    c.sEi = 2.0 * s.re * s.im + h->alpha * s.im;
    c.sAr = 1.0 + h->beta * s.re;
    c.sAi = h->beta * s.im;
  } else {
    c.sEr = s.re; c.sEi = s.im; c.sAr = -1.0; c.sAi = 0.0;
  }
  return c;
}

int mor_build_segments(mor_t h, const std::vector<int64_t>& rows) {
  const int nseg = (int)rows.size() - 1;
  if (nseg < 1) return mor_fail(h, MOR_EINVAL, "no segments");
  const int64_t N = rows[nseg];
  // blocks of 256 threads per SM in total: a whole number of resident waves
  // for the solve kernels (override: MOR_SEG_BLOCKS_PER_SM)
  int bps = nseg == 1 ? 4 : 12;
  if (const char* ev = std::getenv("MOR_SEG_BLOCKS_PER_SM")) {
    const int v = std::atoi(ev);
    if (v >= 1 && v <= 64) bps = v;
  }
  const int64_t target = (int64_t)h->sm_count * bps;
  int64_t R = (N + target - 1) / target;
  if (R < 64) R = 64;
  std::vector<int> blk0(nseg + 1, 0);
  for (int s = 0; s < nseg; ++s) {
    const int64_t ns = rows[s + 1] - rows[s];
    blk0[s + 1] = blk0[s] + (int)std::max<int64_t>(1, (ns + R - 1) / R);
  }
  MOR_CK(h, h->seg_blk0.alloc(sizeof(int) * (nseg + 1)));
  MOR_CK(h, h->seg_row0.alloc(sizeof(int64_t) * (nseg + 1)));
  MOR_CK(h, h->seg_counters.alloc(sizeof(unsigned) * nseg));
  MOR_CK(h, h->seg_live.alloc(sizeof(int) * 2));
  MOR_CK(h, cudaMemcpyAsync(h->seg_blk0.p, blk0.data(), sizeof(int) * (nseg + 1), cudaMemcpyHostToDevice, h->stream));
  MOR_CK(h, cudaMemcpyAsync(h->seg_row0.p, rows.data(), sizeof(int64_t) * (nseg + 1), cudaMemcpyHostToDevice, h->stream));
  MOR_CK(h, cudaMemsetAsync(h->seg_counters.p, 0, sizeof(unsigned) * nseg, h->stream));
  MOR_CK(h, cudaMemsetAsync(h->seg_live.p, 0, sizeof(int) * 2, h->stream));
  MOR_CK(h, cudaStreamSynchronize(h->stream));
  h->seg.nseg = nseg;
  h->seg.nblocks = blk0[nseg];
  h->seg.rows_per_block = R;
  h->seg.nrows = N;
  h->seg.sms = h->sm_count;
  h->seg.blk0 = h->seg_blk0.as<int>();
  h->seg.row0 = h->seg_row0.as<int64_t>();
  h->seg.counters = h->seg_counters.as<unsigned>();
  h->seg.live = h->seg_live.as<int>();
  h->seg_rows_h = rows;
  return MOR_OK;
}

namespace {

using mor_host::HostCSR;
using mor_host::merge_pattern;
using mor_host::transpose_pattern;
using mor_host::shadow_sets;
using mor_host::sell_layout;
using mor_host::dia_layout;

int fetch_csr(mor_t h, const mor_csr* M, bool dev, const char* name, HostCSR& out) {
  if (!M || M->n <= 0 || M->nnz < 0 || !M->rowptr || (M->nnz > 0 && (!M->col || !M->val)))
    return mor_fail(h, MOR_EINVAL, "%s: null pointer or non-positive size", name);
  if (M->n > 0x7fffffffLL || M->nnz > 0x7fffffffLL)
    return mor_fail(h, MOR_EINVAL, "%s: n and nnz must fit int32", name);
  out.n = M->n;
  out.rowptr.resize(M->n + 1);
  out.col.resize(M->nnz);
  out.val.resize(M->nnz);
  cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  MOR_CK(h, cudaMemcpy(out.rowptr.data(), M->rowptr, sizeof(int32_t) * (M->n + 1), kind));
  if (M->nnz > 0) {
    MOR_CK(h, cudaMemcpy(out.col.data(), M->col, sizeof(int32_t) * M->nnz, kind));
    MOR_CK(h, cudaMemcpy(out.val.data(), M->val, sizeof(double) * M->nnz, kind));
  }
  // validation
  if (out.rowptr[0] != 0) return mor_fail(h, MOR_EINVAL, "%s: rowptr[0] != 0", name);
  if (out.rowptr[M->n] != M->nnz) return mor_fail(h, MOR_EINVAL, "%s: rowptr[n] != nnz", name);
  for (int64_t i = 0; i < M->n; ++i) {
    if (out.rowptr[i + 1] < out.rowptr[i]) return mor_fail(h, MOR_EINVAL, "%s: rowptr decreases at row %lld", name, (long long)i);
    for (int32_t p = out.rowptr[i]; p < out.rowptr[i + 1]; ++p) {
      const int32_t c = out.col[p];
      if (c < 0 || c >= M->n) return mor_fail(h, MOR_EINVAL, "%s: column index %d out of range in row %lld", name, c, (long long)i);
      if (p > out.rowptr[i] && c <= out.col[p - 1])
        return mor_fail(h, MOR_EINVAL, "%s: columns not strictly increasing in row %lld", name, (long long)i);
      if (!std::isfinite(out.val[p])) return mor_fail(h, MOR_EINVAL, "%s: non-finite value in row %lld", name, (long long)i);
    }
  }
  return MOR_OK;
}

template <class T>
int upload(mor_t h, DBuf& d, const std::vector<T>& v) {
  MOR_CK(h, d.alloc(sizeof(T) * std::max<size_t>(1, v.size())));
  if (!v.empty()) MOR_CK(h, cudaMemcpyAsync(d.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, h->stream));
  return MOR_OK;
}

template <class T>
std::vector<T> permute_to_layout(const std::vector<T>& csrv, const std::vector<int64_t>& lay, int64_t nlay) {
  std::vector<T> out(nlay, T(0));
  for (size_t p = 0; p < csrv.size(); ++p) out[lay[p]] = csrv[p];
  return out;
}

// Autotuner cache: the timed CSR / SELL choice of a matrix is kept for the
// process, keyed by its signature (device, rows, stored entries, kind of E,
// and an FNV-1a hash of the row pointers and column indices), so that a
// pattern set again -- a new handle, a rebuilt system, the next job on the
// same model -- skips the timing runs.
struct PatternKey {
  int dev;
  int64_t n, nnz;
  int ekind;
  uint64_t hash;
  bool operator<(const PatternKey& o) const {
    if (dev != o.dev) return dev < o.dev;
    if (n != o.n) return n < o.n;
    if (nnz != o.nnz) return nnz < o.nnz;
    if (ekind != o.ekind) return ekind < o.ekind;
    return hash < o.hash;
  }
};
std::mutex g_fmt_mu;
std::map<PatternKey, int> g_fmt_cache;

uint64_t fnv1a(const void* p, size_t bytes, uint64_t h = 1469598103934665603ull) {
  const unsigned char* c = (const unsigned char*)p;
  for (size_t i = 0; i < bytes; ++i) { h ^= c[i]; h *= 1099511628211ull; }
  return h;
}
PatternKey pattern_key(mor_t h, const HostCSR& S, int ekind) {
  uint64_t hs = fnv1a(S.rowptr.data(), S.rowptr.size() * sizeof(int32_t));
  hs = fnv1a(S.col.data(), S.col.size() * sizeof(int32_t), hs);
  return PatternKey{h->dev, S.n, (int64_t)S.col.size(), ekind, hs};
}
bool cached_format(const PatternKey& k, int* fmt) {
  std::lock_guard<std::mutex> lk(g_fmt_mu);
  auto it = g_fmt_cache.find(k);
  if (it == g_fmt_cache.end()) return false;
  *fmt = it->second;
  return true;
}
void store_format(const PatternKey& k, int fmt) {
  std::lock_guard<std::mutex> lk(g_fmt_mu);
  g_fmt_cache[k] = fmt;
}

// upload one operator in a given format
int build_op(mor_t h, OpData& op, const HostCSR& S, const std::vector<double>& sa, const std::vector<double>& se,
             int fmt, bool has_e) {
  op.fmt = fmt;
  op.n = S.n;
  op.nnz = (int64_t)S.col.size();
  op.h_rowptr = S.rowptr;
  op.h_col = S.col;
  std::vector<int64_t> sptr;
  std::vector<int32_t> scol;
  std::vector<int32_t> doffs;
  op.ndiag = 0;
  op.doff.release();
  if (fmt == FMT_SELL) {
    sell_layout(S, sptr, scol, op.h_lay);
    op.nlay = (int64_t)scol.size();
    // the kernels index stored entries with 32-bit positions
    if (op.nlay > (int64_t)INT32_MAX) return mor_fail(h, MOR_EINVAL, "SELL layout exceeds 2^31 stored entries");
  } else if (fmt == FMT_DIA) {
    if (!dia_layout(S, MOR_DIA_MAXDIAG, 1.25, doffs, op.h_lay))
      return mor_fail(h, MOR_EINVAL, "the pattern has more than %d diagonals or more than 25%% padding in the "
                                     "diagonal layout", MOR_DIA_MAXDIAG);
    op.ndiag = (int)doffs.size();
    op.nlay = (int64_t)op.ndiag * S.n;
    op.sptr.release();
    op.scol.release();
  } else {
    op.h_lay.resize(op.nnz);
    for (int64_t p = 0; p < op.nnz; ++p) op.h_lay[p] = p;
    op.nlay = op.nnz;
    op.sptr.release();
    op.scol.release();
  }
  MOR_TRY(upload(h, op.rowptr, S.rowptr));
  MOR_TRY(upload(h, op.col, S.col));
  if (fmt == FMT_SELL) {
    MOR_TRY(upload(h, op.sptr, sptr));
    MOR_TRY(upload(h, op.scol, scol));
  }
  if (fmt == FMT_DIA) MOR_TRY(upload(h, op.doff, doffs));
  op.h_doff = doffs;
  std::vector<double> la = permute_to_layout(sa, op.h_lay, op.nlay);
  std::vector<float> la32(la.begin(), la.end());
  MOR_TRY(upload(h, op.a64, la));
  MOR_TRY(upload(h, op.a32, la32));
  MOR_TRY(upload(h, op.ca64, sa));
  MOR_TRY(upload(h, op.ca32, std::vector<float>(sa.begin(), sa.end())));
  if (has_e) {
    std::vector<double> le = permute_to_layout(se, op.h_lay, op.nlay);
    std::vector<float> le32(le.begin(), le.end());
    MOR_TRY(upload(h, op.e64, le));
    MOR_TRY(upload(h, op.e32, le32));
    MOR_TRY(upload(h, op.ce64, se));
    MOR_TRY(upload(h, op.ce32, std::vector<float>(se.begin(), se.end())));
  } else {
    op.e64.release(); op.e32.release(); op.ce64.release(); op.ce32.release();
  }
  return MOR_OK;
}

// Score of a built op's layout for the autotuner: the FP32 operator SpMV
// (k = 1 real plus k = 8 complex) and four factor SpMVs in the same layout
// (complex64 values, zero, k = 1 plus k = 8 complex), CUDA-event time of the
// best of three repetitions after one untimed.  A BiCGSTAB iteration applies
// the operator twice and the preconditioner chain twice, and the chains of
// the sweeps hold several factors, so the factor SpMV carries the weight.
double time_op(mor_t h, OpData& op, int& status) {
  status = MOR_OK;
  const int64_t n = op.n;
  DBuf x, y, fv, ap;
  if (x.alloc(n * 8 * sizeof(cfloat)) != cudaSuccess || y.alloc(n * 8 * sizeof(cfloat)) != cudaSuccess ||
      fv.alloc((size_t)op.nlay * sizeof(cfloat)) != cudaSuccess || ap.alloc(8 * sizeof(int)) != cudaSuccess) {
    status = MOR_ENOMEM;
    return 1e30;
  }
  cudaMemsetAsync(x.p, 0, n * 8 * sizeof(cfloat), h->stream);
  cudaMemsetAsync(fv.p, 0, (size_t)op.nlay * sizeof(cfloat), h->stream);
  const int ones[8] = {1, 1, 1, 1, 1, 1, 1, 1};
  cudaMemcpyAsync(ap.p, ones, sizeof(ones), cudaMemcpyHostToDevice, h->stream);
  OpVals ov{h->ekind, op.a32.p, op.e32.p, h->ediag32.p};
  Coef cf[8];
  for (int c = 0; c < 8; ++c) cf[c] = mor_coef(h, mor_c64{1.0 + c, 0.5});
  PatView pv = op.view();
  cudaEvent_t e0, e1, e2;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventCreate(&e2);
  float best_op = 1e30f, best_f = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, h->stream);
    launch_op_spmv(ST_F32, h->seg, pv, ov, cf, 1, x.p, y.p, nullptr, nullptr, h->stream);
    launch_op_spmv(ST_C32, h->seg, pv, ov, cf, 8, x.p, y.p, nullptr, nullptr, h->stream);
    cudaEventRecord(e1, h->stream);
    launch_factor_spmv(ST_C32, ST_C32, h->seg, pv, fv.p, ap.as<int>(), 1, x.p, y.p, nullptr, nullptr, h->stream);
    launch_factor_spmv(ST_C32, ST_C32, h->seg, pv, fv.p, ap.as<int>(), 8, x.p, y.p, nullptr, nullptr, h->stream);
    cudaEventRecord(e2, h->stream);
    cudaEventSynchronize(e2);
    float m1 = 0.f, m2 = 0.f;
    cudaEventElapsedTime(&m1, e0, e1);
    cudaEventElapsedTime(&m2, e1, e2);
    if (rep > 0) {
      best_op = std::min(best_op, m1);
      best_f = std::min(best_f, m2);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  if (cudaGetLastError() != cudaSuccess) status = MOR_ECUDA;
  return (double)best_op + 4.0 * (double)best_f;
}

int set_system_common(mor_t h, const HostCSR& A, const HostCSR* Ecsr, const std::vector<double>* Ediag, const double* B,
                      int m, const double* C, int q, int format, bool dev,
                      const std::vector<int64_t>* seg_rows = nullptr) {
  const int64_t n = A.n;
  if (m < 1 || m > MOR_MAX_IO || q < 1 || q > MOR_MAX_IO) return mor_fail(h, MOR_EINVAL, "m and q must be in [1, %d]", MOR_MAX_IO);
  if (!B || !C) return mor_fail(h, MOR_EINVAL, "B and C are required");
  if (format < MOR_FMT_AUTO || format > MOR_FMT_DIA) return mor_fail(h, MOR_EINVAL, "unknown format %d", format);
  h->has_sys = false;
  h->P.chain.clear(); h->T.chain.clear();
  h->P.chain_prec = h->T.chain_prec = -1;
  h->irka_z = 0; h->vlen[0] = h->vlen[1] = 0;
  h->n = n;
  h->ekind = Ecsr ? EK_CSR : (Ediag ? EK_DIAG : EK_IDENTITY);
  // A(s) = c1(s) P + c2(s) Q with P = E (or M), Q = A (or K): the scalars of the
  // reuse decision's Frobenius ratios, once per system
  h->frob = frob_scalars(h->order, h->alpha, h->beta, n, Ediag ? Ediag->data() : nullptr,
                         Ecsr ? Ecsr->rowptr.data() : nullptr, Ecsr ? Ecsr->col.data() : nullptr,
                         Ecsr ? Ecsr->val.data() : nullptr, A.rowptr.data(), A.col.data(), A.val.data());
  // pattern and transpose
  HostCSR S, Tm;
  std::vector<double> sa, se, ta, te;
  merge_pattern(A, Ecsr, S, sa, se);
  std::vector<int64_t> t2p;
  transpose_pattern(S, Tm, t2p);
  const int64_t nnz = (int64_t)S.col.size();
  ta.resize(nnz);
  for (int64_t t = 0; t < nnz; ++t) ta[t] = sa[t2p[t]];
  if (Ecsr) { te.resize(nnz); for (int64_t t = 0; t < nnz; ++t) te[t] = se[t2p[t]]; }
  bool psym = (Tm.rowptr == S.rowptr) && (Tm.col == S.col);
  bool sym = psym;
  if (sym) for (int64_t t = 0; t < nnz && sym; ++t) sym = (ta[t] == sa[t]) && (!Ecsr || te[t] == se[t]);
  h->sym = sym;
  // diag of E
  if (Ediag) {
    std::vector<float> d32(Ediag->begin(), Ediag->end());
    MOR_TRY(upload(h, h->ediag64, *Ediag));
    MOR_TRY(upload(h, h->ediag32, d32));
  } else {
    h->ediag64.release(); h->ediag32.release();
  }
  // segment table (one segment unless the caller is mor_set_batch, which passes its own)
  MOR_TRY(mor_build_segments(h, seg_rows ? *seg_rows : std::vector<int64_t>{0, n}));
  // layout / autotune
  int fmt = format;
  const PatternKey key = pattern_key(h, S, h->ekind);
  if (fmt == MOR_FMT_AUTO && cached_format(key, &fmt)) {
    MOR_TRY(build_op(h, h->P, S, sa, se, fmt, Ecsr != nullptr));
  } else if (fmt == MOR_FMT_AUTO) {
    // time the operator SpMV in every layout the pattern admits: CSR, SELL-32,
    // and the diagonal layout when the pattern has few diagonals
    int st1 = 0, st2 = 0, st3 = 0, last = FMT_CSR;
    MOR_TRY(build_op(h, h->P, S, sa, se, FMT_CSR, Ecsr != nullptr));
    double tc = time_op(h, h->P, st1);
    double ts = 1e300, td = 1e300;
    if (build_op(h, h->P, S, sa, se, FMT_SELL, Ecsr != nullptr) == MOR_OK) {
      ts = time_op(h, h->P, st2);
      last = FMT_SELL;
    }
    {
      std::vector<int32_t> offs;
      std::vector<int64_t> lay;
      if (dia_layout(S, MOR_DIA_MAXDIAG, 1.25, offs, lay)) {
        MOR_TRY(build_op(h, h->P, S, sa, se, FMT_DIA, Ecsr != nullptr));
        td = time_op(h, h->P, st3);
        last = FMT_DIA;
      }
    }
    if (st1 != MOR_OK || st2 != MOR_OK || st3 != MOR_OK) return mor_fail(h, MOR_ECUDA, "format autotuning failed");
    fmt = FMT_CSR;
    if (ts <= tc && ts <= td) fmt = FMT_SELL;
    if (td < tc && td < ts) fmt = FMT_DIA;
    if (fmt != last) MOR_TRY(build_op(h, h->P, S, sa, se, fmt, Ecsr != nullptr));
    store_format(key, fmt);
  } else {
    MOR_TRY(build_op(h, h->P, S, sa, se, fmt, Ecsr != nullptr));
  }
  if (!sym) MOR_TRY(build_op(h, h->T, Tm, ta, te, fmt, Ecsr != nullptr));
  // shadows: columns of the primal operator are the rows of S^T
  std::vector<int64_t> iptr;
  std::vector<int32_t> iidx;
  int nImax = 0, nJmax = 0;
  shadow_sets(sym ? S : Tm, iptr, iidx, nImax, nJmax);
  MOR_TRY(upload(h, h->P.iptr_b, iptr));
  MOR_TRY(upload(h, h->P.iidx_b, iidx));
  h->P.iptr = h->P.iptr_b.as<int64_t>();
  h->P.iidx = h->P.iidx_b.as<int32_t>();
  h->P.nImax = nImax; h->P.nJmax = nJmax;
  // outpos for the primal SPAI: column entries = entries of S^T (positions t) -> S position t2p[t] -> layout
  {
    std::vector<int64_t> outp(nnz);
    for (int64_t t = 0; t < nnz; ++t) outp[t] = h->P.h_lay[t2p[t]];
    MOR_TRY(upload(h, h->P.outpos, outp));
  }
  if (!sym) {
    if (psym) {
      h->T.iptr = h->P.iptr; h->T.iidx = h->P.iidx;
      h->T.nImax = nImax; h->T.nJmax = nJmax;
    } else {
      std::vector<int64_t> iptr2;
      std::vector<int32_t> iidx2;
      int a2 = 0, b2 = 0;
      shadow_sets(S, iptr2, iidx2, a2, b2);
      MOR_TRY(upload(h, h->T.iptr_b, iptr2));
      MOR_TRY(upload(h, h->T.iidx_b, iidx2));
      h->T.iptr = h->T.iptr_b.as<int64_t>();
      h->T.iidx = h->T.iidx_b.as<int32_t>();
      h->T.nImax = a2; h->T.nJmax = b2;
    }
    // transposed SPAI: column entries = entries of S (positions p); T position of (i,j) is p2t[p]
    std::vector<int64_t> p2t(nnz);
    for (int64_t t = 0; t < nnz; ++t) p2t[t2p[t]] = t;
    std::vector<int64_t> outp(nnz);
    for (int64_t p = 0; p < nnz; ++p) outp[p] = h->T.h_lay[p2t[p]];
    MOR_TRY(upload(h, h->T.outpos, outp));
  } else {
    h->T.chain.clear();
  }
  // B, C
  cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  MOR_CK(h, h->B.alloc(sizeof(double) * n * m));
  MOR_CK(h, h->C.alloc(sizeof(double) * n * q));
  MOR_CK(h, cudaMemcpyAsync(h->B.p, B, sizeof(double) * n * m, kind, h->stream));
  MOR_CK(h, cudaMemcpyAsync(h->C.p, C, sizeof(double) * n * q, kind, h->stream));
  h->m = m;
  h->q = q;
  MOR_CK(h, cudaStreamSynchronize(h->stream));
  h->has_sys = true;
  return MOR_OK;
}

}  // namespace

extern "C" {

void mor_default_opts(mor_solve_opts* o) {
  if (!o) return;
  o->precision = MOR_MIXED;
  o->solver = MOR_BICGSTAB;
  o->restart = 50;
  o->precond_precision = -1;
  o->fp64_fallback = 1;
  o->concurrent_sweeps = 1;
  o->tol = 1e-8;
  o->maxit = 20000;
  o->inner_tol = 1e-4;
  o->max_refine = 10;
  o->batch = 1;
  o->use_graph = 1;
  o->graph_chunk = 16;
  o->precond = 0;
  o->max_chain = 0;
  o->reuse = MOR_REUSE_CHAIN;
  o->moments = 1;
}

int mor_create(mor_t* out, int device, void* stream) {
  if (!out) return MOR_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return MOR_ECUDA;
  if (device < 0 || device >= ndev) return MOR_EINVAL;
  mor_ctx* h = new (std::nothrow) mor_ctx();
  if (!h) return MOR_ENOMEM;
  h->dev = device;
  if (cudaSetDevice(device) != cudaSuccess) { delete h; return MOR_ECUDA; }
  cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device);
  h->grid_cap = h->sm_count * 8;
  if (stream) { h->stream = (cudaStream_t)stream; h->own_stream = false; }
  else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) { delete h; return MOR_ECUDA; }
    h->own_stream = true;
  }
  if (h->ws_counter.alloc(64 * sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(h->ws_counter.p, 0, 64 * sizeof(unsigned)) != cudaSuccess) { delete h; return MOR_ENOMEM; }
  h->pinned_bytes = 1 << 21;
  if (cudaHostAlloc(&h->pinned, h->pinned_bytes, cudaHostAllocDefault) != cudaSuccess) { delete h; return MOR_ENOMEM; }
  *out = h;
  return MOR_OK;
}

int mor_destroy(mor_t h) {
  if (!h) return MOR_OK;
  cudaSetDevice(h->dev);
  cudaStreamSynchronize(h->stream);
  if (h->pinned) cudaFreeHost(h->pinned);
  for (SolveLane& L : h->lanes) {
    if (L.own_stream) { cudaStreamSynchronize(L.stream); cudaStreamDestroy(L.stream); }
    if (L.pinned) cudaFreeHost(L.pinned);
  }
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return MOR_OK;
}

int mor_launch_count(int64_t* count) {
  if (!count) return MOR_EINVAL;
  *count = (int64_t)g_launches.load();
  return MOR_OK;
}

int mor_kernel_tally(int which, int vec_type, int64_t* counts) {
  if (which < 0 || which > 1 || vec_type < 0 || vec_type > 3 || !counts) return MOR_EINVAL;
  for (int k = 0; k <= MOR_KMAX; ++k) counts[k] = (int64_t)g_tally[which][vec_type][k].load();
  return MOR_OK;
}

const char* mor_last_error(mor_t h) { return h ? h->err.c_str() : "null handle"; }

int mor_set_system(mor_t h, const mor_csr* A, const mor_csr* E, const double* E_diag, const double* B, int m,
                   const double* C, int q, int format, unsigned flags) {
  if (!h) return MOR_EINVAL;
  cudaSetDevice(h->dev);
  const bool dev = (flags & MOR_DEVICE_PTRS) != 0;
  HostCSR Ah, Eh;
  MOR_TRY(fetch_csr(h, A, dev, "A", Ah));
  const HostCSR* Ep = nullptr;
  std::vector<double> ed;
  if (E) {
    MOR_TRY(fetch_csr(h, E, dev, "E", Eh));
    if (Eh.n != Ah.n) return mor_fail(h, MOR_EINVAL, "E and A differ in size");
    Ep = &Eh;
  } else if (E_diag) {
    ed.resize(Ah.n);
    MOR_CK(h, cudaMemcpy(ed.data(), E_diag, sizeof(double) * Ah.n, dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
    for (double v : ed) if (!std::isfinite(v)) return mor_fail(h, MOR_EINVAL, "E_diag has a non-finite value");
  }
  h->order = 1;
  h->alpha = h->beta = 0.0;
  return set_system_common(h, Ah, Ep, E_diag && !E ? &ed : nullptr, B, m, C, q, format, dev);
}

int mor_set_system_2nd(mor_t h, const mor_csr* K, const double* M_diag, double alpha, double beta, const double* F,
                       int m, const double* C, int q, int format, unsigned flags) {
  if (!h) return MOR_EINVAL;
  if (!M_diag) return mor_fail(h, MOR_EINVAL, "M_diag is required");
  if (!std::isfinite(alpha) || !std::isfinite(beta)) return mor_fail(h, MOR_EINVAL, "alpha/beta not finite");
  cudaSetDevice(h->dev);
  const bool dev = (flags & MOR_DEVICE_PTRS) != 0;
  HostCSR Kh;
  MOR_TRY(fetch_csr(h, K, dev, "K", Kh));
  std::vector<double> md(Kh.n);
  MOR_CK(h, cudaMemcpy(md.data(), M_diag, sizeof(double) * Kh.n, dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
  for (double v : md) if (!std::isfinite(v)) return mor_fail(h, MOR_EINVAL, "M_diag has a non-finite value");
  h->order = 2;
  h->alpha = alpha;
  h->beta = beta;
  return set_system_common(h, Kh, nullptr, &md, F, m, C, q, format, dev);
}

int mor_set_batch(mor_t h, int nsys, const mor_csr* A, const double* const* E_diag, const double* const* B,
                  const double* const* C, int format, unsigned flags) {
  if (!h) return MOR_EINVAL;
  if (nsys < 1 || !A || !B || !C) return mor_fail(h, MOR_EINVAL, "nsys >= 1, A, B and C are required");
  if (flags & MOR_DEVICE_PTRS) return mor_fail(h, MOR_EINVAL, "mor_set_batch takes host pointers only");
  cudaSetDevice(h->dev);
  std::vector<int64_t> rows(nsys + 1, 0);
  std::vector<HostCSR> parts(nsys);
  for (int s = 0; s < nsys; ++s) {
    MOR_TRY(fetch_csr(h, &A[s], false, "A[s]", parts[s]));
    if (!B[s] || !C[s]) return mor_fail(h, MOR_EINVAL, "B[%d] or C[%d] is null", s, s);
    rows[s + 1] = rows[s] + parts[s].n;
  }
  const int64_t N = rows[nsys];
  int64_t nnz = 0;
  for (auto& pa : parts) nnz += (int64_t)pa.col.size();
  if (N > 0x7fffffffLL || nnz > 0x7fffffffLL) return mor_fail(h, MOR_EINVAL, "batch too large for int32 indices");
  HostCSR cat;
  cat.n = N;
  cat.rowptr.resize(N + 1);
  cat.col.resize(nnz);
  cat.val.resize(nnz);
  std::vector<double> bcat(N), ccat(N), ecat;
  bool anyE = false;
  if (E_diag) for (int s = 0; s < nsys; ++s) anyE |= (E_diag[s] != nullptr);
  if (anyE) ecat.assign(N, 1.0);
  int64_t pos = 0;
  for (int s = 0; s < nsys; ++s) {
    const HostCSR& pa = parts[s];
    const int64_t r0 = rows[s];
    for (int64_t i = 0; i < pa.n; ++i) {
      cat.rowptr[r0 + i] = (int32_t)(pos + pa.rowptr[i]);
      if (anyE && E_diag[s]) {
        const double e = E_diag[s][i];
        if (!std::isfinite(e)) return mor_fail(h, MOR_EINVAL, "E_diag[%d] has a non-finite value", s);
        ecat[r0 + i] = e;
      }
      bcat[r0 + i] = B[s][i];
      ccat[r0 + i] = C[s][i];
    }
    for (size_t q = 0; q < pa.col.size(); ++q) {
      cat.col[pos + q] = (int32_t)(pa.col[q] + r0);
      cat.val[pos + q] = pa.val[q];
    }
    pos += (int64_t)pa.col.size();
  }
  cat.rowptr[N] = (int32_t)pos;
  h->order = 1;
  h->alpha = h->beta = 0.0;
  return set_system_common(h, cat, nullptr, anyE ? &ecat : nullptr, bcat.data(), 1, ccat.data(), 1, format, false,
                           &rows);
}

int mor_batch_info(mor_t h, int* nsys, int64_t* offsets) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  if (nsys) *nsys = h->seg.nseg;
  if (offsets) std::memcpy(offsets, h->seg_rows_h.data(), sizeof(int64_t) * h->seg_rows_h.size());
  return MOR_OK;
}

int mor_get_info(mor_t h, int64_t* n, int64_t* nnz, int* format, int* symmetric) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  if (n) *n = h->n;
  if (nnz) *nnz = h->P.nnz;
  if (format) *format = h->P.fmt;
  if (symmetric) *symmetric = h->sym ? 1 : 0;
  return MOR_OK;
}

int mor_get_io(mor_t h, int* m, int* q) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  if (m) *m = h->m;
  if (q) *q = h->q;
  return MOR_OK;
}

int mor_get_pattern(mor_t h, int transpose, int32_t* rowptr, int32_t* col) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  OpData& op = h->op(transpose);
  if (rowptr) std::memcpy(rowptr, op.h_rowptr.data(), sizeof(int32_t) * op.h_rowptr.size());
  if (col) std::memcpy(col, op.h_col.data(), sizeof(int32_t) * op.h_col.size());
  return MOR_OK;
}

}  // extern "C"
