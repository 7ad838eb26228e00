// Internal declarations shared by the translation units of the library.
// Nothing here is part of the public C ABI (include/mor_spai.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

// scalar type codes for runtime dispatch
enum ScalarType { ST_F32 = 0, ST_F64 = 1, ST_C32 = 2, ST_C64 = 3 };
inline bool st_is_cplx(int st) { return st >= ST_C32; }
inline bool st_is_f32(int st) { return st == ST_F32 || st == ST_C32; }
inline size_t st_size(int st) { return st == ST_F32 ? 4 : (st == ST_C64 ? 16 : 8); }

enum { FMT_CSR = 1, FMT_SELL = 2, FMT_DIA = 3 };
// patterns with at most this many distinct diagonals (and at most 25% padding)
// may be stored in the diagonal layout
#define MOR_DIA_MAXDIAG 32
enum { EK_IDENTITY = 0, EK_DIAG = 1, EK_CSR = 2 };

// Device view of a stored sparse pattern (CSR, or SELL-32 with sigma = 1).
// SELL: rows are cut into slices of 32; slice s holds width_s = (sptr[s+1] -
// sptr[s]) / 32 slots, slot t of row 32 s + l is at sptr[s] + 32 t + l.
// Padding slots carry col = the row itself and value 0.
// DIA: ndiag distinct offsets doff[0] < ... (column = row + doff[d]); the
// entry of row r on diagonal d is at d n + r; positions with no entry (and
// columns outside 0 .. n - 1) hold value 0.
struct PatView {
  int fmt;
  int n;
  const int32_t* rowptr;  // CSR
  const int32_t* col;     // CSR col, or SELL col (padded)
  const int64_t* sptr;    // SELL slice offsets (nslices + 1)
  const int32_t* doff;    // DIA offsets (ndiag)
  int ndiag;
  const int32_t* h_doff;  // DIA offsets, host copy (launch set-up; not read by kernels)
};

// Real-valued operator data for y = sE * (E x) + sA * (A x).
struct OpVals {
  int ekind;              // EK_IDENTITY | EK_DIAG | EK_CSR
  const void* a;          // A values in layout order (float or double)
  const void* e;          // E values in layout order (EK_CSR) or nullptr
  const void* ediag;      // E diagonal (EK_DIAG) or nullptr
};

// complex FP64 coefficient pair of one column
struct Coef { double sEr, sEi, sAr, sAi; };

#define MOR_KMAX 16

// ---------------------------------------------------------------------------
// fused reduction modes of the operator SpMV
enum {
  RED_NONE = 0,
  RED_DOT_W = 1,     // partial[c] = sum conj(w) * y           (r_hat^H v)
  RED_DOT_TT = 2,    // partial[c] = (sum conj(y) * w, sum |y|^2)   ((t, s), (t, t))
  RED_NORM = 3       // partial[c] = sum |y|^2  (and y = b + op, see b pointer)
};

// ---------------------------------------------------------------------------
// Row layout of the n x k blocks of a solve: row-major with stride ld (the k
// columns of one row contiguous).  A row of at least 16 bytes is a whole
// number of 16-byte vectors: ld = ceil(k / c) c with c = 16 / size (only FP32
// rows of k = 5..7, 9..11, 13..15 and FP64 / complex64 rows of odd k carry
// dummy columns, kept at zero).  Lane `sub` of the tpr lanes of a row owns the
// cpt = c consecutive columns sub * c ... (one 16-byte load or store); tpr is
// ld / c rounded up to a power of two so that a warp holds whole rows, and the
// lanes past the row's last vector stay idle.  Narrow rows (k * size < 16)
// use one thread per row.
inline int next_pow2(int v) { int p = 1; while (p < v) p <<= 1; return p; }
inline bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
inline int row_stride(int st, int k) {
  const int es = (int)st_size(st);
  if (k * es < 16) return k;
  const int c = 16 / es;
  return (k + c - 1) / c * c;
}
// Lanes per row (tpr) and columns per lane (cpt) for rows of stride ld.  A
// stride chosen for another type (the FP64 refinement reuses the stride of
// the FP32 inner solve) that does not make rows whole 16-byte vectors of this
// type is handled one thread per row with scalar accesses: a 16-byte access
// is only ever made at a 16-byte aligned address.
inline void lane_shape(int st, int ld, int* tpr, int* cpt) {
  const int es = (int)st_size(st);
  const int c = 16 / es;
  if (ld * es < 16 || ld % c != 0) { *tpr = 1; *cpt = ld; return; }
  *cpt = c;
  *tpr = next_pow2(ld / c);
}

#define MOR_LDMAX 16

// Independent systems stored as one block-diagonal operator ("segments").
// Every kernel of the solve runs on nblocks blocks; block b belongs to the
// segment s with blk0[s] <= b < blk0[s+1] and walks rows row0[s] + (b -
// blk0[s]) * rows_per_block ... (clipped to the segment).  Reductions are
// per (segment, column): the last block of a segment (ticket counters[s])
// finalizes that segment's columns; `live` counts segments with an active
// column.  A single system is the one-segment case.
struct SegView {
  int nseg;
  int nblocks;
  int64_t rows_per_block;
  int64_t nrows;           // total rows (row0[nseg])
  int sms;                 // SMs of the device
  const int* blk0;         // nseg + 1
  const int64_t* row0;     // nseg + 1
  unsigned* counters;      // nseg, zero between launches
  int* live;               // segments with an active column
};

// Fused reductions: `part` holds per-block FP64 partials, the last block (by
// ticket on `counter`) reduces them in a fixed order and runs the finalize
// stage `fin` on `state` (or writes the 2 * ld sums to `out`).
struct RedArgs {
  int mode;            // RED_*
  const void* w;       // second vector of the reduction
  void* part;          // nblocks * ld * 2 complex partials (doubles)
  unsigned* counter;   // unused (the segment tickets live in SegView)
  int fin;             // finalize stage id (0 = none: just write the reduced sums to `out`)
  void* state;         // solver state for the finalize stage
  void* out;           // reduced sums (nseg x 2 ld complex doubles), when fin == 0
  const int* done;     // if non-null and *done != 0 the kernel returns at once
};

// Grid of one launch.  A single system (nseg == 1) is split into one resident
// wave of the kernel `kern` (blocks of 256 threads, occupancy queried once per
// kernel), each block a contiguous range of whole passes of 256 / tpr rows;
// a batch keeps the segment table's blocks (krylov.cu).
SegView fit_grid(const SegView& sg, const void* kern, int tpr);

// GMRES(m) kernels (gmres.cu): single system, basis vectors V_i at
// V + i * vstride (n x ld blocks of type st), per-column FP64 state.
#define GM_MMAX 64
size_t gmres_state_bytes();
int gmres_state_iters(const void* state_entry);
int gmres_state_status(const void* state_entry);
int gmres_state_conv(const void* state_entry);
int gmres_launch_dot(int st, const SegView& sg, int ld, const void* V, int64_t vstride, int nv, const void* w,
                     double* part, unsigned* counter, void* out, const int* done, cudaStream_t s);
int gmres_launch_axpy(int st, const SegView& sg, int ld, const void* V, int64_t vstride, int nv, const void* coef,
                      void* w, int mode, int fin, double* part, unsigned* counter, void* state, void* H, int m,
                      const void* h1, const void* h2, int* done, cudaStream_t s);
int gmres_launch_scale(int st, const SegView& sg, int ld, const void* w, void* v, const void* state, int use_active,
                       const int* done, cudaStream_t s);
int gmres_launch_add(int st, const SegView& sg, int ld, void* x, const void* z, cudaStream_t s);
int gmres_launch_begin(int ld, const void* sums, void* state, const double* target, const int* maxit,
                       const int* enabled, int first, int* done_cycle, int* done_all, cudaStream_t s);
int gmres_launch_solve_y(int ld, int m, void* state, const void* H, void* ycoef, cudaStream_t s);

// Block GMRES kernels (bgmres.cu): stacked basis V (n x ldv row-major, K
// columns used), blocks W, Y of P <= bgmres_max_cols() columns (row stride
// ldw, ldy); out / C: K x P complex128 row-major (out[kk * P + b]).
int bgmres_max_cols();
int bgmres_dot_grid();
size_t bgmres_part_doubles(int K, int P);
int bgmres_launch_dot(int st, int64_t n, int K, int P, const void* V, int64_t ldv, const void* W, int64_t ldw,
                      double* part, unsigned* counter, void* out, cudaStream_t s);
// mode 0: Y = W - V C; mode 1: Y = V C (Y must not overlap V)
int bgmres_launch_update(int st, int64_t n, int K, int P, const void* V, int64_t ldv, const void* C, const void* W,
                         int64_t ldw, int mode, void* Y, int64_t ldy, cudaStream_t s);
int bgmres_launch_copy(int st, int64_t n, int P, const void* src, int64_t lds, void* dst, int64_t ldd, int64_t off,
                       cudaStream_t s);

// Launchers (spmv.cu).  x, y, w, b: n x ld row-major blocks of type st.
// kreal: real (non-dummy) columns of the block, for the launch tally (-1: ld)
int launch_op_spmv(int st, const SegView& sg, const PatView& pv, const OpVals& ov, const Coef* coefs, int ld,
                   const void* x, void* y, const void* b, const RedArgs* red, cudaStream_t s, int kreal = -1);
// fst: scalar type of the factor values (FP32 factors may serve FP64 vectors).
// kstate (nullable): the per-(segment, column) Krylov states of the solve the
// factor is applied in; lanes whose columns have all stopped skip their rows
// (their rows of y are left as they were).
// factor SpMV in the diagonal layout specialised to 5 or 7 diagonals and FP32 /
// complex64 vectors (spmv_dia.cu): -1 when it does not apply, else 0
int launch_factor_dia_nd(int st, int fst, const SegView& sg, const PatView& pv, const void* fvals, const int* apply,
                         int ld, const void* x, void* y, const int* done, const void* kstate, cudaStream_t s);
int launch_factor_spmv(int st, int fst, const SegView& sg, const PatView& pv, const void* fvals,
                       const int* apply, int ld, const void* x, void* y, const int* done,
                       const void* kstate, cudaStream_t s, int kreal = -1);

// Krylov helpers (krylov.cu)
int krylov_launch_update_p(int st, const SegView& sg, int ld, const void* r, void* p, const void* v,
                           const void* state, const int* done, cudaStream_t s);
int krylov_launch_update_s(int st, const SegView& sg, int ld, const void* r, const void* v, void* sv,
                           const void* state, const int* done, cudaStream_t s);
int krylov_launch_update_xr(int st, const SegView& sg, int ld, void* x, void* r, const void* phat,
                            const void* shat, const void* sv, const void* t, const void* rhat,
                            void* part, void* state, int* done, cudaStream_t s);
// stag: iterations without a 0.1% drop of the best residual after which a
// column stops as stagnated (0: never)
int krylov_launch_init(int st, const SegView& sg, int ld, const void* rhs, void* x, void* r, void* rhat,
                       void* p, void* v, void* part, void* state, const double* target, const int* maxit,
                       int stag, int* done, cudaStream_t s);
int krylov_status_stagnated(int status);
size_t krylov_state_bytes(int st);
int krylov_read_state(int st, const void* state_dev, int k, int* iters, int* status,
                      cudaStream_t s);
// outer FP64 refinement: rhs_in = r64 / ||r64|| (cast), x64 += nrm * d
int refine_launch_scale_cast(int st_in, const SegView& sg, int ld, const void* r64, const double* nrm2,
                             const int* active, void* rhs_in, cudaStream_t s);
int refine_launch_update(int st_in, const SegView& sg, int ld, void* x64, const void* d,
                         const double* nrm2, const int* active, cudaStream_t s);
// layout conversion: column-major complex128 (API, k columns) <-> row-major type st, stride ld
int conv_launch_colmajor_c128_to_rowmajor(int st, int n, int k, int ld, const void* src, void* dst,
                                          cudaStream_t s);
int conv_launch_rowmajor_to_colmajor_c128(int st, int n, int k, int ld, const void* src, void* dst,
                                          cudaStream_t s);
int conv_launch_real_col_to_rowmajor(int st, int n, int k, int ld, const double* src, int64_t lds,
                                     void* dst, cudaStream_t s);
int conv_launch_copy_cast(int st_dst, int st_src, int64_t count, const void* src, void* dst,
                          cudaStream_t s);
// active-column compaction: gather map[c] -> c into a narrower stride, scatter back
int conv_launch_gather_cols(int st, int64_t n, int ld_src, int ld_dst, int ncols, const int* map, const void* src,
                            void* dst, cudaStream_t s);
int conv_launch_scatter_cols(int st, int64_t n, int ld_src, int ld_dst, int ncols, const int* smap, const int* dmap,
                             const void* src, void* dst, cudaStream_t s);
// host access to the per-column Krylov state (opaque, krylov_state_bytes() each)
int krylov_write_state(const void* host_states, void* state_dev, int k, cudaStream_t s);
int krylov_read_states(void* host_states, const void* state_dev, int k, cudaStream_t s);
int krylov_state_active(const void* host_state);
int krylov_state_iters(const void* host_state);
int krylov_state_status(const void* host_state);
void krylov_state_make_dummy(void* host_state);

// SPAI (spai.cu)
struct SpaiArgs {
  int n;
  const int32_t* colptr;    // column lists of the operator = rows of the other op's CSR
  const int32_t* colidx;
  const double* ca;         // A values of those entries (FP64)
  const double* ce;         // E values (EK_CSR) or nullptr
  const double* ediag;      // E diagonal (EK_DIAG) or nullptr
  const float* ca32;        // FP32 copies, read when the factor is FP32 / complex64
  const float* ce32;
  const float* ediag32;
  int ekind;
  const int64_t* outpos;    // layout position of each column entry in this operator
  const int64_t* iptr;      // shadow sets I_j
  const int32_t* iidx;
  int nImax, nJmax;
  Coef cnew, cold;          // coefficients of A(sigma_new), A(sigma_old)
  int update;               // 0: rhs e_j (SPAI), 1: rhs = column j of A(sigma_old) (reuse Q)
  int* nsingular;           // count of rank-deficient columns
};
int launch_spai(int st, const SpaiArgs& a, void* out, cudaStream_t s);

// dense FP64 helpers (dense.cu)
int dense_launch_gram(int n, int a, int b, const double* X, int64_t ldx, const double* Y,
                      int64_t ldy, double* out, double* part, unsigned* counter, int grid_cap,
                      cudaStream_t s);
int dense_launch_gs_update(int n, int j, const double* V, int64_t ldv, const double* h, double* v,
                           cudaStream_t s);
int dense_launch_scale(int n, double* v, const double* nrm2, cudaStream_t s);
int dense_launch_eig(int r, const double* Ar, const double* Er, double* out /*wr,wi,sr,si,status*/,
                     cudaStream_t s);
// tangential directions of r poles (lam: r complex as 2r doubles); out gets
// r x m then r x q complex directions and a status double; work holds
// dense_tangent_work(r, m) doubles, iwork r * (r + 1) ints
size_t dense_tangent_work(int r, int m);
int dense_launch_tangent(int r, int m, int q, const double* Ar, const double* Er, const double* Br, const double* Cr,
                         const double* lam, double* out, double* work, int* iwork, cudaStream_t s);
// second-order point update: out gets 2r eigenvalues, count points (complex
// as re, im) and a status; work dense_qep_work doubles, iwork 2r ints
size_t dense_qep_work(int r, int count);
int dense_launch_qep(int r, int count, const double* Kr, const double* Mr, double alpha, double beta, double* out,
                     double* work, int* iwork, cudaStream_t s);
// H(i w) per frequency; order 2 reads (A_r, E_r) as (K_r, M_r) with D_r = alpha M_r + beta K_r
int dense_launch_tf(int r, int m, int q, const double* Ar, const double* Er, const double* Br,
                    const double* Cr, const double* omega, int nw, double* H, cudaStream_t s, int order = 1,
                    double alpha = 0.0, double beta = 0.0);
int dense_launch_diag_mul(int n, int k, const double* d, const double* X, double* Y,
                          cudaStream_t s);

// SMs of the current CUDA device (queried once per device)
int mor_device_sms();

// process-wide count of executed kernels (see mor_launch_count)
void mor_count_launches(int64_t n);
// on = 1 while this thread records a CUDA graph (its launches are counted per replay)
void mor_capture_mark(int on);
// SpMV launch tally (see mor_kernel_tally): kernel 0 operator, 1 factor; st the
// vector type; kreal the real (non-dummy) columns of the block
struct ShapeTally { int64_t c[2][4][MOR_KMAX + 1] = {}; };
void mor_tally(int kernel, int st, int kreal, int64_t n = 1);
ShapeTally mor_capture_tally();               // what the current capture recorded
void mor_replay_tally(const ShapeTally& t);   // one replay of a captured graph
