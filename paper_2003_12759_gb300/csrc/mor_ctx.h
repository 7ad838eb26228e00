// Host-side runtime state of a handle (C++, not part of the C ABI).
#pragma once
#include "mor_spai.h"
#include "mor_internal.h"
#include "reuse_policy.h"
#include <cstdarg>
#include <cstdio>
#include <memory>
#include <string>
#include <vector>

// grow-only device buffer
struct DBuf {
  void* p = nullptr;
  size_t n = 0;
  DBuf() {}
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  cudaError_t alloc(size_t bytes) {
    if (p && bytes <= n) return cudaSuccess;
    release();
    if (bytes == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) n = bytes; else p = nullptr;
    return e;
  }
  void release() { if (p) cudaFree(p); p = nullptr; n = 0; }
  template <class T> T* as() const { return (T*)p; }
};

struct Factor {
  std::unique_ptr<DBuf> vals;   // layout order, type st
  int st = ST_F64;
  mor_c64 from{0, 0}, to{0, 0};
  int kind = 0;                 // 0 SPAI, 1 reuse
};

// One operator: A(s) (primal) or A(s)^T (transposed).
struct OpData {
  int fmt = FMT_CSR;
  int64_t n = 0, nnz = 0, nlay = 0;     // rows, CSR entries, stored layout entries
  DBuf rowptr, col;                      // CSR (device)
  DBuf sptr, scol;                       // SELL-32 layout (device)
  DBuf doff;                             // DIA offsets (device)
  std::vector<int32_t> h_doff;           // DIA offsets (host)
  int ndiag = 0;
  DBuf a64, a32, e64, e32;               // values in layout order
  DBuf ca64, ce64, ca32, ce32;           // values in CSR order (column data for the other op's SPAI)
  DBuf outpos;                           // int64 per column-entry: position in this op's layout
  DBuf iptr_b, iidx_b;                   // shadow sets (owned)
  const int64_t* iptr = nullptr;         // shadow sets (may point into the other op's buffers)
  const int32_t* iidx = nullptr;
  int nImax = 0, nJmax = 0;
  std::vector<int32_t> h_rowptr, h_col;  // host CSR pattern
  std::vector<int64_t> h_lay;            // CSR position -> layout position
  std::vector<Factor> chain;
  int chain_prec = -1;                   // MOR_FP64 / MOR_MIXED of the chain
  PatView view() const {
    PatView v;
    v.fmt = fmt;
    v.n = (int)n;
    v.rowptr = rowptr.as<int32_t>();
    v.col = (fmt == FMT_SELL) ? scol.as<int32_t>() : col.as<int32_t>();
    v.sptr = sptr.as<int64_t>();
    v.doff = doff.as<int32_t>();
    v.ndiag = ndiag;
    v.h_doff = h_doff.empty() ? nullptr : h_doff.data();
    return v;
  }
};

// Everything one batch solve needs besides the system and its chains: a
// stream, the Krylov / refinement / GMRES workspaces, the per-(segment)
// reduction tickets and live counter, small device state and a pinned
// staging buffer.  Lane 0 runs on the handle's stream; lane 1 (its own
// non-blocking stream) lets the transposed sweep of an IRKA step run
// concurrently with the primal one.
struct SolveLane {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  DBuf ws_vec, ws_x64, ws_r64, ws_b64, ws_part, ws_small, ws_kstate, ws_segarr, ws_sums, ws_io;
  DBuf ws_gm_vec, ws_gm_small, ws_gm_part;
  DBuf ws_fb;                        // FP64 re-solve of failed mixed columns: maps, b, x
  DBuf seg_counters, seg_live;
  int seg_alloc = 0;                 // segments the counters were zeroed for
  void* pinned = nullptr;
  size_t pinned_bytes = 0;
  SolveLane() {}
  SolveLane(const SolveLane&) = delete;
  SolveLane& operator=(const SolveLane&) = delete;
};

struct mor_ctx {
  int dev = 0;
  int sm_count = 1;          // set from the device at mor_create
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  bool has_sys = false;
  int order = 1;
  double alpha = 0.0, beta = 0.0;
  int64_t n = 0;
  int ekind = EK_IDENTITY;
  DBuf ediag64, ediag32;
  OpData P, T;
  bool sym = false;
  DBuf B, C;        // FP64 column-major
  int m = 0, q = 0;
  // workspace
  DBuf ws_vec, ws_x64, ws_r64, ws_b64, ws_part, ws_small, ws_gram, ws_basis, ws_rom;
  DBuf ws_counter;  // unsigned counters (zeroed once)
  DBuf ws_io;       // API conversions
  void* pinned = nullptr;   // small pinned host buffer
  size_t pinned_bytes = 0;
  int grid_cap = 8;          // sm_count * 8, set at mor_create
  // segment table: one segment per independent system (1 for mor_set_system)
  DBuf seg_blk0, seg_row0, seg_counters, seg_live;
  SegView seg{};
  std::vector<int64_t> seg_rows_h;   // nseg + 1 row offsets (host)
  DBuf ws_kstate, ws_segarr, ws_sums;
  SolveLane lanes[2];                        // batch-solve state per stream (lane 0: `stream`)
  // scalar products of the stored matrices for the Frobenius-ratio reuse decision
  FrobScalars frob;
  // IRKA reuse schedule
  int irka_z = 0;
  int vlen[2] = {0, 0};
  OpData& op(int transpose) { return (transpose && !sym) ? T : P; }
};

int mor_fail(mor_t h, int code, const char* fmt, ...);
// lane i ready (stream, pinned buffer); lane 0 uses the handle's stream
int mor_lane(mor_t h, int i, SolveLane** out);

#define MOR_CK(h, call)                                                                     \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return mor_fail(h, (e_ == cudaErrorMemoryAllocation) ? MOR_ENOMEM : MOR_ECUDA,        \
                      "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define MOR_CKI(h, call)                                                                    \
  do {                                                                                      \
    int e_ = (call);                                                                        \
    if (e_ != 0)                                                                            \
      return mor_fail(h, MOR_ECUDA, "%s failed: %s (%s:%d)", #call,                         \
                      cudaGetErrorString((cudaError_t)e_), __FILE__, __LINE__);             \
  } while (0)

#define MOR_TRY(call)            \
  do {                           \
    int s_ = (call);             \
    if (s_ != MOR_OK) return s_; \
  } while (0)

// shift -> operator coefficients
Coef mor_coef(const mor_ctx* h, mor_c64 s);
// (re)build the segment table for the given row offsets (nseg + 1 entries)
int mor_build_segments(mor_t h, const std::vector<int64_t>& row_offsets);
inline bool is_real_shift(mor_c64 s) { return s.im == 0.0; }
