// Preconditioner chain, shifted solves, Gram-Schmidt, projection, reduced
// poles, IRKA step and transfer-function evaluation (host C++ runtime that
// drives the kernels).
//
// The solve of a batch of k <= 16 shifts:
//   outer (FP64):  r = b - A(sigma) x  (FP64 operator SpMV, fused norms);
//                  stop when ||r|| / ||b|| <= tol;
//   inner:         right-preconditioned BiCGSTAB on A(sigma) d = r / ||r||
//                  (FP32/complex64 in MOR_MIXED; FP64 in MOR_FP64, where the
//                  outer loop is the restart-on-true-residual of the FP64
//                  algorithm), all k columns in lock step, scalars and
//                  convergence on the device, iterations replayed from a
//                  CUDA graph in chunks with one 4-byte read per chunk;
//                  x += ||r|| d.
#include "mor_ctx.h"
#include "krylov_state.cuh"
#include "block_ls.h"
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <thread>

namespace {

int st_of(int precision, bool cplx) {
  if (precision == MOR_FP64) return cplx ? ST_C64 : ST_F64;
  return cplx ? ST_C32 : ST_F32;
}
bool same_shift(mor_c64 a, mor_c64 b) { return a.re == b.re && a.im == b.im; }

OpVals op_vals(mor_t h, OpData& op, bool f32) {
  OpVals v;
  v.ekind = h->ekind;
  v.a = f32 ? op.a32.p : op.a64.p;
  v.e = f32 ? op.e32.p : op.e64.p;
  v.ediag = f32 ? h->ediag32.p : h->ediag64.p;
  return v;
}

// small device scratch: [counter area][done][kstate][targets][maxit][active][nrm2][masks][sums]
struct Small {
  unsigned* counter;
  int* done;
  void* kstate;
  double* target;
  int* maxit;
  int* active;
  double* nrm2;
  int* masks;        // MOR_KMAX ints per factor
  cdouble* sums;     // 2 * MOR_KMAX
  int* nsing;
};
const int MAX_FACTORS = 4096;

// kernel launches recorded in a captured graph (counted once per replay)
int64_t kernel_nodes(cudaGraph_t g) {
  size_t nn = 0;
  if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess || nn == 0) return 0;
  std::vector<cudaGraphNode_t> nodes(nn);
  if (cudaGraphGetNodes(g, nodes.data(), &nn) != cudaSuccess) return 0;
  int64_t k = 0;
  for (size_t i = 0; i < nn; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

int get_small(mor_t h, DBuf& buf, Small& s) {
  const size_t bytes = 64 * 1024 + 4096 + (size_t)MAX_FACTORS * MOR_KMAX * sizeof(int);
  MOR_CK(h, buf.alloc(bytes));
  char* b = buf.as<char>();
  s.done = (int*)(b + 0);
  s.nsing = (int*)(b + 64);
  s.kstate = (void*)(b + 256);                          // 16 * 112 B
  s.target = (double*)(b + 256 + 4096);
  s.maxit = (int*)(b + 256 + 4096 + 256);
  s.active = (int*)(b + 256 + 4096 + 512);
  s.nrm2 = (double*)(b + 256 + 4096 + 768);
  s.sums = (cdouble*)(b + 256 + 4096 + 1024);
  s.masks = (int*)(b + 64 * 1024 + 4096);
  s.counter = h->ws_counter.as<unsigned>();
  return MOR_OK;
}

}  // namespace

// forward
static int build_factor(mor_t h, int transpose, mor_c64 s_old, mor_c64 s_new, bool update, int precision,
                        bool append = false);

// precision of the factors the schedule builds: opts.precond_precision, or
// opts.precision when that is negative (the default)
static int factor_precision(const mor_solve_opts& o) {
  return o.precond_precision >= 0 ? o.precond_precision : o.precision;
}

// blocks a per-block partial buffer must hold: the segment table's grid (a
// batch) or one resident wave of up to 8 blocks per SM (fit_grid)
static size_t part_blocks(const mor_t h) {
  return std::max<size_t>({(size_t)h->seg.nblocks, (size_t)h->sm_count * 8, (size_t)2048});
}

// ---------------------------------------------------------------------------
// preconditioner chain
// ---------------------------------------------------------------------------
// update: a reuse factor Q from s_old to s_new, appended to the chain; else a
// SPAI at s_new that replaces the chain, or (append) starts a new chain after
// the factors already held (the reuse decision's fresh build).
static int build_factor(mor_t h, int transpose, mor_c64 s_old, mor_c64 s_new, bool update, int precision,
                        bool append) {
  OpData& X = h->op(transpose);
  OpData& Y = (transpose && !h->sym) ? h->P : (h->sym ? h->P : h->T);   // column data source
  const bool cplx = !is_real_shift(s_new) || (update && !is_real_shift(s_old));
  const int st = st_of(precision, cplx);
  Factor f;
  f.vals.reset(new DBuf());
  f.st = st;
  f.from = update ? s_old : s_new;
  f.to = s_new;
  f.kind = update ? 1 : 0;
  MOR_CK(h, f.vals->alloc(st_size(st) * (size_t)X.nlay));
  MOR_CK(h, cudaMemsetAsync(f.vals->p, 0, st_size(st) * (size_t)X.nlay, h->stream));
  Small sm;
  MOR_TRY(get_small(h, h->ws_small, sm));
  MOR_CK(h, cudaMemsetAsync(sm.nsing, 0, sizeof(int), h->stream));
  SpaiArgs a;
  a.n = (int)X.n;
  a.colptr = Y.rowptr.as<int32_t>();
  a.colidx = Y.col.as<int32_t>();
  a.ca = Y.ca64.as<double>();
  a.ce = Y.ce64.as<double>();
  a.ediag = h->ediag64.as<double>();
  a.ca32 = Y.ca32.as<float>();
  a.ce32 = Y.ce32.as<float>();
  a.ediag32 = h->ediag32.as<float>();
  a.ekind = h->ekind;
  a.outpos = X.outpos.as<int64_t>();
  a.iptr = X.iptr;
  a.iidx = X.iidx;
  a.nImax = X.nImax;
  a.nJmax = X.nJmax;
  a.cnew = mor_coef(h, s_new);
  a.cold = mor_coef(h, s_old);
  a.update = update ? 1 : 0;
  a.nsingular = sm.nsing;
  MOR_CKI(h, launch_spai(st, a, f.vals->p, h->stream));
  int nsing = 0;
  MOR_CK(h, cudaMemcpyAsync(&nsing, sm.nsing, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  MOR_CK(h, cudaStreamSynchronize(h->stream));
  if (!update && !append) { X.chain.clear(); }
  X.chain.push_back(std::move(f));
  X.chain_prec = precision;
  if (nsing > 0) return mor_fail(h, MOR_ESINGULAR, "%d rank-deficient least-squares columns", nsing);
  return MOR_OK;
}

// ---------------------------------------------------------------------------
// one batch of k <= 16 columns
// ---------------------------------------------------------------------------
// The factors of the chain one shift column applies, in chain order: every f
// with a <= f < b, then f = x when x >= b.  A prefix Q_L ... Q_2 P_1 (Algorithm
// 4) is {0, L, -1}; the first approach of Table II is the vertical prefix plus
// the shift's own factor {0, v, x}; a chain restarted by a fresh SPAI at
// factor a is {a, b, -1}.
struct ColChain {
  int a = 0, b = 0, x = -1;
  int end() const { return x >= 0 ? x + 1 : b; }
  bool uses(int f) const { return (f >= a && f < b) || f == x; }
  int count() const { return (b > a ? b - a : 0) + (x >= 0 ? 1 : 0); }
};
static ColChain prefix_chain(int L) { ColChain c; c.b = L; return c; }

struct BatchIO {
  const mor_c64* sig;   // k shifts
  int k;
  int ld;               // padded row stride of the blocks
  const ColChain* L;    // factors of the chain each column applies
  void* b64;            // row-major n x k, st64
  void* x64;            // row-major n x k, st64 (out)
};

// minimum stagnation window of a mixed-precision inner BiCGSTAB solve (iterations
// without a 0.1% drop of its best residual; 0 = no stagnation test)
#ifndef MOR_MIXED_STAG
#define MOR_MIXED_STAG 200
#endif
// refinement passes in a row, each cutting the FP64 residual by less than 10%, after
// which a mixed-precision column is given up (and solved again in FP64).  Measured on
// GB300: one pass (with the 200-iteration window) gives the shortest times on the
// uneven batch, on near-resonant second-order shifts and on mixed AIRGA iterations --
// a column that needs longer FP32 solves than the rest of its batch finishes sooner
// in FP64 than by more refinement passes.
#ifndef MOR_MIXED_POOR
#define MOR_MIXED_POOR 1
#endif

static int solve_batch(mor_t h, SolveLane& ln, int transpose, const mor_solve_opts& o, bool cplx, const BatchIO& io,
                       mor_solve_stats* stats) {
  OpData& op = h->op(transpose);
  // the system's segment table with this lane's tickets and live counter
  SegView sg = h->seg;
  const int nseg = sg.nseg;
  if (ln.seg_alloc < nseg) {
    MOR_CK(h, ln.seg_counters.alloc(sizeof(unsigned) * nseg));
    MOR_CK(h, ln.seg_live.alloc(sizeof(int) * 2));
    MOR_CK(h, cudaMemsetAsync(ln.seg_counters.p, 0, sizeof(unsigned) * nseg, ln.stream));
    MOR_CK(h, cudaMemsetAsync(ln.seg_live.p, 0, sizeof(int) * 2, ln.stream));
    ln.seg_alloc = nseg;
  }
  sg.counters = ln.seg_counters.as<unsigned>();
  sg.live = ln.seg_live.as<int>();
  const int k = io.k;
  const int64_t n = op.n;
  const int prec = o.precision;
  const int st_in = st_of(prec, cplx);
  const int st64 = cplx ? ST_C64 : ST_F64;
  const int ld = io.ld;                              // padded row stride, columns k..ld-1 are dummies
  const size_t es = st_size(st_in), es64 = st_size(st64);
  int Lmax = 0;
  for (int c = 0; c < k; ++c) Lmax = std::max(Lmax, io.L[c].end());
  if (Lmax > (int)op.chain.size()) return mor_fail(h, MOR_ESTATE, "chain shorter than requested prefix");
  if (Lmax > MAX_FACTORS - 4) return mor_fail(h, MOR_EINVAL, "chain too long");
  for (int f = 0; f < Lmax; ++f) {
    const Factor& F = op.chain[f];
    bool used = false;
    for (int c = 0; c < k; ++c) used |= io.L[c].uses(f);
    if (!used) continue;
    if (!st_is_f32(F.st) && st_is_f32(st_in))
      return mor_fail(h, MOR_ESTATE, "an FP64 preconditioner chain cannot serve an FP32 inner solve");
    if (st_is_cplx(F.st) && !st_is_cplx(st_in)) return mor_fail(h, MOR_EINVAL, "internal: complex factor, real vectors");
  }
  // workspace: 12 inner vectors of n x ld
  const size_t vbytes = ((es * (size_t)n * ld) + 255) / 256 * 256;
  MOR_CK(h, ln.ws_vec.alloc(vbytes * 12));
  char* vb = ln.ws_vec.as<char>();
  auto vec = [&](int i) { return (void*)(vb + vbytes * i); };
  void *rhs = vec(0), *d = vec(1), *r = vec(2), *rhat = vec(3), *p = vec(4), *v = vec(5), *sv = vec(6),
       *t = vec(7), *ph = vec(8), *sh = vec(9), *tmp0 = vec(10), *tmp1 = vec(11);
  MOR_CK(h, ln.ws_r64.alloc(es64 * (size_t)n * ld));
  void* r64 = ln.ws_r64.p;
  MOR_CK(h, ln.ws_part.alloc(sizeof(double) * 2 * 2 * MOR_LDMAX * part_blocks(h)));
  Small sm;
  MOR_TRY(get_small(h, ln.ws_small, sm));
  const size_t ksb = krylov_state_bytes(st_in);
  const size_t nsc = (size_t)nseg * ld;                 // (segment, column) slots
  MOR_CK(h, ln.ws_kstate.alloc(ksb * (size_t)nseg * MOR_LDMAX));
  void* kstate = ln.ws_kstate.p;
  MOR_CK(h, ln.ws_segarr.alloc((sizeof(double) * 2 + sizeof(int) * 2) * (size_t)nseg * MOR_LDMAX));
  double* d_target = ln.ws_segarr.as<double>();
  double* d_nrm2 = d_target + (size_t)nseg * MOR_LDMAX;
  int* d_maxit = (int*)(d_nrm2 + (size_t)nseg * MOR_LDMAX);
  int* d_active = d_maxit + (size_t)nseg * MOR_LDMAX;
  MOR_CK(h, ln.ws_sums.alloc(sizeof(cdouble) * 2 * (size_t)nseg * MOR_LDMAX));
  cdouble* d_sums = ln.ws_sums.as<cdouble>();
  if ((sizeof(cdouble) * 2 + 64) * nsc > ln.pinned_bytes / 2) return mor_fail(h, MOR_EINVAL, "too many systems");
  // coefficients (dummy columns reuse column 0's)
  Coef cf[MOR_LDMAX], ncf[MOR_LDMAX];
  for (int c = 0; c < ld; ++c) {
    cf[c] = mor_coef(h, io.sig[c < k ? c : 0]);
    ncf[c] = Coef{-cf[c].sEr, -cf[c].sEi, -cf[c].sAr, -cf[c].sAi};
  }
  PatView pv = op.view();
  OpVals ov_in = op_vals(h, op, st_is_f32(st_in));
  OpVals ov64 = op_vals(h, op, false);
  MOR_CK(h, cudaMemsetAsync(io.x64, 0, es64 * (size_t)n * ld, ln.stream));

  // Current geometry of the batch.  When enough columns have converged that
  // the live ones fit a narrower stride, the converged columns are flushed
  // to d_full (in the original layout) and the state-carrying vectors
  // (d, r, r_hat, p, v) are repacked into the free scratch vectors (single
  // system only: with several systems a column lives while any system needs it).
  int ldc = ld;
  std::vector<int> cmap(ld);                 // current column -> original column
  void* d_full = rhs;                        // free after init: collects flushed columns
  void* dd = d;
  void *rr = r, *rh = rhat, *pp = p, *vv = v, *ssv = sv, *tt = t, *pph = ph, *ssh = sh, *t0 = tmp0, *t1 = tmp1;
  Coef cfc[MOR_LDMAX];
  // Lcur: the longest chain prefix among the columns still in the batch.
  // The high shifts carry the longest horizontal prefixes and converge
  // first, so after compaction the chain is applied only as far as the
  // remaining columns need (no copy-through launches for the dropped ones).
  int Lcur = Lmax;
  int kreal = k;                             // real columns in the current geometry (launch tally)
  auto upload_masks = [&]() -> int {
    kreal = 0;
    for (int c = 0; c < ldc; ++c) kreal += (cmap[c] >= 0 && cmap[c] < k) ? 1 : 0;
    if (Lmax == 0) return 0;
    int lc = 0;
    for (int c = 0; c < ldc; ++c)
      if (cmap[c] >= 0 && cmap[c] < k) lc = std::max(lc, io.L[cmap[c]].end());
    Lcur = lc > 0 ? lc : Lmax;
    std::vector<int> mk((size_t)Lmax * MOR_KMAX, 0);
    for (int f = 0; f < Lmax; ++f)
      for (int c = 0; c < ldc; ++c) {
        const int oc = cmap[c];
        mk[(size_t)f * MOR_KMAX + c] = (oc < 0 || oc >= k || io.L[oc].uses(f)) ? 1 : 0;
      }
    return (int)cudaMemcpyAsync(sm.masks, mk.data(), sizeof(int) * mk.size(), cudaMemcpyHostToDevice, ln.stream);
  };
  auto chain_apply_d = [&](void* src, void* dst, const int* dn, const void* ks = nullptr) -> int {
    if (Lmax == 0) return 0;
    void* s = src;
    for (int f = 0; f < Lcur; ++f) {
      void* dd2 = (f == Lcur - 1) ? dst : ((f % 2 == 0) ? t0 : t1);
      const Factor& F = op.chain[f];
      int e = launch_factor_spmv(st_in, F.st, sg, pv, F.vals->p, sm.masks + (size_t)f * MOR_KMAX, ldc, s,
                                 dd2, dn, ks, ln.stream, kreal);
      if (e) return e;
      s = dd2;
    }
    return 0;
  };
  // BiCGSTAB: stopped columns (and finished systems of a batch) skip the chain
  auto chain_apply = [&](void* src, void* dst) -> int { return chain_apply_d(src, dst, sm.done, kstate); };
  auto one_iter = [&]() -> int {
    int e;
    void* phat = (Lmax == 0) ? pp : pph;
    void* shat = (Lmax == 0) ? ssv : ssh;
    if ((e = krylov_launch_update_p(st_in, sg, ldc, rr, pp, vv, kstate, sm.done, ln.stream))) return e;
    if ((e = chain_apply(pp, pph))) return e;
    RedArgs ra{RED_DOT_W, rh, ln.ws_part.p, nullptr, FIN_ALPHA, kstate, nullptr, sm.done};
    if ((e = launch_op_spmv(st_in, sg, pv, ov_in, cfc, ldc, phat, vv, nullptr, &ra, ln.stream, kreal))) return e;
    if ((e = krylov_launch_update_s(st_in, sg, ldc, rr, vv, ssv, kstate, sm.done, ln.stream))) return e;
    if ((e = chain_apply(ssv, ssh))) return e;
    RedArgs rb{RED_DOT_TT, ssv, ln.ws_part.p, nullptr, FIN_OMEGA, kstate, nullptr, sm.done};
    if ((e = launch_op_spmv(st_in, sg, pv, ov_in, cfc, ldc, shat, tt, nullptr, &rb, ln.stream, kreal))) return e;
    if ((e = krylov_launch_update_xr(st_in, sg, ldc, dd, rr, phat, shat, ssv, tt, rh, ln.ws_part.p, kstate, sm.done,
                                     ln.stream)))
      return e;
    return 0;
  };
  const int chunk = std::max(1, o.graph_chunk);
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_nodes = 0;
  ShapeTally graph_tally;
  auto drop_graph = [&]() { if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; } };
  struct GraphGuard { std::function<void()> f; ~GraphGuard() { f(); } } guard{drop_graph};
  auto capture = [&]() -> int {
    drop_graph();
    if (!o.use_graph) return MOR_OK;
    cudaGraph_t g = nullptr;
    MOR_CK(h, cudaStreamBeginCapture(ln.stream, cudaStreamCaptureModeThreadLocal));
    mor_capture_mark(1);
    int e = 0;
    for (int it = 0; it < chunk && !e; ++it) e = one_iter();
    graph_tally = mor_capture_tally();
    mor_capture_mark(0);
    cudaError_t ce = cudaStreamEndCapture(ln.stream, &g);
    graph_nodes = (ce == cudaSuccess && g) ? kernel_nodes(g) : 0;
    if (e) { if (g) cudaGraphDestroy(g); return mor_fail(h, MOR_ECUDA, "kernel launch failed during capture: %s", cudaGetErrorString((cudaError_t)e)); }
    MOR_CK(h, ce);
    ce = cudaGraphInstantiate(&gexec, g, 0);
    cudaGraphDestroy(g);
    MOR_CK(h, ce);
    return MOR_OK;
  };

  const int max_outer = (prec == MOR_FP64) ? 4 : std::max(1, o.max_refine);
  const size_t NK = (size_t)nseg * k;                  // (segment, real column) pairs
  std::vector<double> bnorm(NK, 0.0), relres(NK, 0.0), rn2(NK, 0.0), prevrel(NK, 0.0);
  std::vector<int> iters(NK, 0), refs(NK, 0), status(NK, MOR_OK), act(NK, 0), poor(NK, 0);
  double* hp = (double*)ln.pinned;
  cdouble* h_sums = (cdouble*)hp;                                  // 2 ld per segment
  double* tg = hp + 4 * nsc;
  double* nr = tg + nsc;
  int* mi = (int*)(nr + nsc);
  int* ac = mi + nsc;
  std::vector<unsigned char> kst_host(ksb * MOR_LDMAX * std::max(nseg, 1)), kst_new(ksb * MOR_LDMAX);
  // ---- GMRES(m) inner solve of A P y = rhs, x_in = P y (single system): the
  // basis V_0..V_m, then w, z (chain output), u (V y); one captured graph per
  // cycle (m Arnoldi steps, the update x_in += P V y and the next cycle's
  // start: true inner residual, beta, v_0).
  auto gmres_inner = [&](void* xin, std::vector<int>& kit_out, std::vector<int>& kst_out) -> int {
    if (nseg != 1) return mor_fail(h, MOR_EINVAL, "GMRES solves one system (not a batch of systems)");
    const int m = o.restart;
    if (m < 1 || m > GM_MMAX) return mor_fail(h, MOR_EINVAL, "GMRES restart %d outside 1..%d", m, GM_MMAX);
    const int64_t vst = (int64_t)(vbytes / es);
    MOR_CK(h, ln.ws_gm_vec.alloc(vbytes * (size_t)(m + 4)));
    char* gb = ln.ws_gm_vec.as<char>();
    auto V = [&](int i) { return (void*)(gb + vbytes * (size_t)i); };
    void* W = V(m + 1);
    void* Z = V(m + 2);
    void* U = V(m + 3);
    size_t off = 0;
    auto take = [&](size_t b) { const size_t o2 = off; off += (b + 255) / 256 * 256; return o2; };
    const size_t hb = sizeof(cdouble) * (size_t)(m + 1) * ld;
    const size_t o_st = take(gmres_state_bytes() * ld);
    const size_t o_H = take(sizeof(cdouble) * (size_t)ld * (m + 1) * m);
    const size_t o_h1 = take(hb), o_h2 = take(hb), o_y = take(hb), o_fl = take(64);
    MOR_CK(h, ln.ws_gm_small.alloc(off));
    char* sb = ln.ws_gm_small.as<char>();
    void* gst = sb + o_st;
    void* Hm = sb + o_H;
    void *h1 = sb + o_h1, *h2 = sb + o_h2, *yc = sb + o_y;
    unsigned* gcnt = (unsigned*)(sb + o_fl);
    int* done_cycle = (int*)(sb + o_fl + 16);
    int* done_all = (int*)(sb + o_fl + 32);
    MOR_CK(h, cudaMemsetAsync(sb, 0, off, ln.stream));
    MOR_CK(h, ln.ws_gm_part.alloc(sizeof(double) * 2 * (size_t)(m + 1) * ld * (size_t)(h->sm_count * 8)));
    double* gpart = ln.ws_gm_part.as<double>();
    MOR_CK(h, cudaMemsetAsync(gb, 0, vbytes * (size_t)(m + 4), ln.stream));   // no stale values in the basis
    MOR_CK(h, cudaMemsetAsync(xin, 0, vbytes, ln.stream));
    RedArgs rn{RED_NORM, nullptr, ln.ws_part.p, nullptr, FIN_NONE, nullptr, d_sums, nullptr};
    RedArgs none{RED_NONE, nullptr, nullptr, nullptr, 0, nullptr, nullptr, done_cycle};
    auto start_cycle = [&](int first) -> int {
      int e;
      if ((e = launch_op_spmv(st_in, sg, pv, ov_in, ncf, ld, xin, W, rhs, &rn, ln.stream, k))) return e;
      if ((e = gmres_launch_begin(ld, d_sums, gst, d_target, d_maxit, d_active, first, done_cycle, done_all,
                                  ln.stream)))
        return e;
      return gmres_launch_scale(st_in, sg, ld, W, V(0), gst, 1, done_cycle, ln.stream);
    };
    auto cycle = [&]() -> int {
      int e;
      for (int j = 0; j < m; ++j) {
        void* src = V(j);
        if (Lmax > 0) {
          if ((e = chain_apply_d(V(j), Z, done_cycle))) return e;
          src = Z;
        }
        if ((e = launch_op_spmv(st_in, sg, pv, ov_in, cf, ld, src, W, nullptr, &none, ln.stream, k))) return e;
        if ((e = gmres_launch_dot(st_in, sg, ld, V(0), vst, j + 1, W, gpart, gcnt, h1, done_cycle, ln.stream))) return e;
        if ((e = gmres_launch_axpy(st_in, sg, ld, V(0), vst, j + 1, h1, W, 0, 0, gpart, gcnt, gst, Hm, m, h1, h2,
                                   done_cycle, ln.stream)))
          return e;
        if ((e = gmres_launch_dot(st_in, sg, ld, V(0), vst, j + 1, W, gpart, gcnt, h2, done_cycle, ln.stream))) return e;
        if ((e = gmres_launch_axpy(st_in, sg, ld, V(0), vst, j + 1, h2, W, 0, 1, gpart, gcnt, gst, Hm, m, h1, h2,
                                   done_cycle, ln.stream)))
          return e;
        if ((e = gmres_launch_scale(st_in, sg, ld, W, V(j + 1), gst, 1, done_cycle, ln.stream))) return e;
      }
      if ((e = gmres_launch_solve_y(ld, m, gst, Hm, yc, ln.stream))) return e;
      if ((e = gmres_launch_axpy(st_in, sg, ld, V(0), vst, m, yc, U, 1, 0, gpart, gcnt, gst, Hm, m, h1, h2, nullptr,
                                 ln.stream)))
        return e;
      void* upd = U;
      if (Lmax > 0) {
        if ((e = chain_apply_d(U, Z, nullptr))) return e;
        upd = Z;
      }
      if ((e = gmres_launch_add(st_in, sg, ld, xin, upd, ln.stream))) return e;
      return start_cycle(0);
    };
    MOR_CKI(h, start_cycle(1));
    cudaGraphExec_t gx = nullptr;
    struct GxGuard { cudaGraphExec_t* g; ~GxGuard() { if (*g) cudaGraphExecDestroy(*g); } } gxg{&gx};
    int64_t gnodes = 0;
    ShapeTally gm_tally;
    if (o.use_graph) {
      cudaGraph_t g = nullptr;
      MOR_CK(h, cudaStreamBeginCapture(ln.stream, cudaStreamCaptureModeThreadLocal));
      mor_capture_mark(1);
      const int e = cycle();
      gm_tally = mor_capture_tally();
      mor_capture_mark(0);
      const cudaError_t ce = cudaStreamEndCapture(ln.stream, &g);
      gnodes = (ce == cudaSuccess && g) ? kernel_nodes(g) : 0;
      if (e) { if (g) cudaGraphDestroy(g); return mor_fail(h, MOR_ECUDA, "launch failed during capture: %s", cudaGetErrorString((cudaError_t)e)); }
      MOR_CK(h, ce);
      const cudaError_t ie = cudaGraphInstantiate(&gx, g, 0);
      cudaGraphDestroy(g);
      MOR_CK(h, ie);
    }
    int maxrem = 0;
    for (int c = 0; c < ld; ++c) maxrem = std::max(maxrem, mi[c]);
    int* hd = (int*)(ac + nsc);
    for (int cyc = 0; cyc <= maxrem; ++cyc) {
      MOR_CK(h, cudaMemcpyAsync(hd, done_all, sizeof(int), cudaMemcpyDeviceToHost, ln.stream));
      MOR_CK(h, cudaStreamSynchronize(ln.stream));
      if (*hd) break;
      if (gx) {
        MOR_CK(h, cudaGraphLaunch(gx, ln.stream));
        mor_count_launches(gnodes);
        mor_replay_tally(gm_tally);
      } else {
        MOR_CKI(h, cycle());
      }
    }
    std::vector<unsigned char> gs(gmres_state_bytes() * ld);
    MOR_CK(h, cudaMemcpyAsync(gs.data(), gst, gs.size(), cudaMemcpyDeviceToHost, ln.stream));
    MOR_CK(h, cudaStreamSynchronize(ln.stream));
    for (int c = 0; c < k; ++c) {
      const void* e = gs.data() + gmres_state_bytes() * c;
      kit_out[c] = gmres_state_iters(e);
      const int stt = gmres_state_status(e);
      kst_out[c] = gmres_state_conv(e) ? KST_OK : (stt == KST_BREAKDOWN ? KST_BREAKDOWN : KST_NOCONV);
    }
    return MOR_OK;
  };

  // ---- block GMRES(m) inner solve of A P Y = rhs, x_in = P Y (single system):
  // the k columns (one shift, one chain) share one block Krylov space of A P
  // (Saad 2003, Sec. 6.12).  Each cycle starts from the residual block with
  // every unconverged column scaled to unit norm (converged columns are left
  // out as zero columns), block Arnoldi by block CGS2 over the stacked basis,
  // each new block orthonormalised by a rank-revealing CholQR (two passes,
  // pivoted Cholesky of the Gram matrix: dependent directions become zero
  // basis columns), the block least-squares problem incrementally on the host
  // (block_ls.h); a column stops iterating once its least-squares residual
  // meets its target.  x_in += P V Y at the end of a cycle.
  auto bgmres_inner = [&](void* xin, std::vector<int>& kit_out, std::vector<int>& kst_out) -> int {
    typedef std::complex<double> cx;
    if (nseg != 1) return mor_fail(h, MOR_EINVAL, "block GMRES solves one system (not a batch of systems)");
    const int m = o.restart;
    if (m < 1 || m > GM_MMAX) return mor_fail(h, MOR_EINVAL, "block GMRES restart %d outside 1..%d", m, GM_MMAX);
    if (k > bgmres_max_cols()) return mor_fail(h, MOR_EINVAL, "block GMRES takes at most %d columns", bgmres_max_cols());
    for (int c = 1; c < k; ++c)
      if (!same_shift(io.sig[c], io.sig[0]) || io.L[c].a != io.L[0].a || io.L[c].b != io.L[0].b ||
          io.L[c].x != io.L[0].x)
        return mor_fail(h, MOR_EINVAL, "block GMRES needs one shift and one chain for all columns of a block");
    const double gtol = st_is_f32(st_in) ? 1e-8 : 1e-20;
    const int64_t ldv = (int64_t)(m + 1) * k;
    const size_t sbytes = ((es * (size_t)n * ldv) + 255) / 256 * 256;
    MOR_CK(h, ln.ws_gm_vec.alloc(sbytes + vbytes * 5));
    char* gb = ln.ws_gm_vec.as<char>();
    void* Vst = gb;
    void* W = gb + sbytes;
    void* Wt = (char*)W + vbytes;
    void* Vj = (char*)Wt + vbytes;
    void* Z = (char*)Vj + vbytes;
    void* U = (char*)Z + vbytes;
    const int Kmax = (m + 1) * k;
    size_t off = 0;
    auto take = [&](size_t b) { const size_t o2 = off; off += (b + 255) / 256 * 256; return o2; };
    const size_t o_h1 = take(sizeof(cdouble) * Kmax * k), o_h2 = take(sizeof(cdouble) * Kmax * k);
    const size_t o_c = take(sizeof(cdouble) * Kmax * k), o_g = take(sizeof(cdouble) * k * k), o_cnt = take(64);
    MOR_CK(h, ln.ws_gm_small.alloc(off));
    char* sb = ln.ws_gm_small.as<char>();
    cdouble* h1d = (cdouble*)(sb + o_h1);
    cdouble* h2d = (cdouble*)(sb + o_h2);
    cdouble* cd = (cdouble*)(sb + o_c);
    cdouble* gd = (cdouble*)(sb + o_g);
    unsigned* bcnt = (unsigned*)(sb + o_cnt);
    MOR_CK(h, cudaMemsetAsync(sb, 0, off, ln.stream));
    MOR_CK(h, ln.ws_gm_part.alloc(sizeof(double) * bgmres_part_doubles(Kmax, k)));
    double* gpart = ln.ws_gm_part.as<double>();
    MOR_CK(h, cudaMemsetAsync(gb, 0, sbytes + vbytes * 5, ln.stream));
    MOR_CK(h, cudaMemsetAsync(xin, 0, vbytes, ln.stream));
    std::vector<cx> hh1((size_t)Kmax * k), hh2((size_t)Kmax * k), up((size_t)Kmax * k), hg((size_t)k * k);
    auto dot = [&](const void* V, int64_t ldvv, int K, const void* Wp, cdouble* outd) -> int {
      return bgmres_launch_dot(st_in, n, K, k, V, ldvv, Wp, ld, gpart, bcnt, outd, ln.stream);
    };
    auto fetch = [&](const cdouble* d, std::vector<cx>& hbuf, size_t cnt) -> int {
      MOR_CK(h, cudaMemcpyAsync(hbuf.data(), d, sizeof(cdouble) * cnt, cudaMemcpyDeviceToHost, ln.stream));
      MOR_CK(h, cudaStreamSynchronize(ln.stream));
      return MOR_OK;
    };
    // Y = V C for a K x k coefficient matrix given column-major (Cm[b K + kk])
    auto apply_coef = [&](const void* V, int64_t ldvv, int K, const std::vector<cx>& Cm, void* Y) -> int {
      for (int kk = 0; kk < K; ++kk)
        for (int b = 0; b < k; ++b) up[(size_t)kk * k + b] = Cm[(size_t)b * K + kk];
      MOR_CK(h, cudaMemcpyAsync(cd, up.data(), sizeof(cdouble) * K * k, cudaMemcpyHostToDevice, ln.stream));
      MOR_CKI(h, bgmres_launch_update(st_in, n, K, k, V, ldvv, cd, nullptr, 0, 1, Y, ld, ln.stream));
      return MOR_OK;
    };
    // rank-revealing CholQR2 of the k columns of Wsrc (stride ld) into Vout; F = R factor
    std::vector<cx> Gm((size_t)k * k), C1((size_t)k * k), F1((size_t)k * k), C2((size_t)k * k), F2((size_t)k * k);
    auto orth = [&](const void* Wsrc, void* Vout, std::vector<cx>& F, int* rank) -> int {
      MOR_CKI(h, dot(Wsrc, ld, k, Wsrc, gd));
      MOR_TRY(fetch(gd, hg, (size_t)k * k));
      for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) Gm[(size_t)b * k + a] = hg[(size_t)a * k + b];
      const int r1 = block_orth_factor(k, Gm.data(), gtol, C1.data(), F1.data());
      MOR_TRY(apply_coef(Wsrc, ld, k, C1, Wt));
      MOR_CKI(h, dot(Wt, ld, k, Wt, gd));
      MOR_TRY(fetch(gd, hg, (size_t)k * k));
      for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) Gm[(size_t)b * k + a] = hg[(size_t)a * k + b];
      const int r2 = block_orth_factor(k, Gm.data(), 1e-2, C2.data(), F2.data());
      MOR_TRY(apply_coef(Wt, ld, k, C2, Vout));
      // W = Vt F1 = Vout F2 F1
      for (int c = 0; c < k; ++c)
        for (int i = 0; i < k; ++i) {
          cx s2(0.0, 0.0);
          for (int l = 0; l < k; ++l) s2 += F2[(size_t)l * k + i] * F1[(size_t)c * k + l];
          F[(size_t)c * k + i] = s2;
        }
      *rank = std::min(r1, r2);
      return MOR_OK;
    };
    std::vector<int> itc(k, 0), conv(k, 0), brk(k, 0);
    std::vector<double> tgt(k), scale(k);
    int budget = 0;
    for (int c = 0; c < k; ++c) { tgt[c] = tg[c]; budget = std::max(budget, mi[c]); }
    BlockLS ls;
    std::vector<cx> R0((size_t)k * k), Y, hcol;
    int used = 0;
    for (;;) {
      // residual block of the inner system and its column norms
      MOR_CKI(h, launch_op_spmv(st_in, sg, pv, ov_in, ncf, ld, xin, W, rhs, nullptr, ln.stream, k));
      MOR_CKI(h, dot(W, ld, k, W, gd));
      MOR_TRY(fetch(gd, hg, (size_t)k * k));
      int nact = 0;
      for (int c = 0; c < k; ++c) {
        const double rn = std::sqrt(std::max(0.0, hg[(size_t)c * k + c].real()));
        if (!std::isfinite(rn)) brk[c] = 1;
        conv[c] = (std::isfinite(rn) && rn <= tgt[c]) ? 1 : 0;
        scale[c] = (!conv[c] && !brk[c] && itc[c] < mi[c]) ? rn : 0.0;
        nact += scale[c] > 0.0 ? 1 : 0;
      }
      if (nact == 0 || used >= budget) break;
      // unit-norm unconverged columns, zero columns for the rest
      std::vector<cx> Dm((size_t)k * k, cx(0.0, 0.0));
      for (int c = 0; c < k; ++c) Dm[(size_t)c * k + c] = scale[c] > 0.0 ? cx(1.0 / scale[c], 0.0) : cx(0.0, 0.0);
      MOR_TRY(apply_coef(W, ld, k, Dm, U));
      int rank = 0;
      MOR_TRY(orth(U, Vj, R0, &rank));
      if (rank == 0) break;
      ls.reset(k, m, R0.data());
      MOR_CKI(h, bgmres_launch_copy(st_in, n, k, Vj, ld, Vst, ldv, 0, ln.stream));
      int steps = 0;
      for (int j = 0; j < m && used < budget; ++j) {
        void* src = Vj;
        if (Lmax > 0) {
          MOR_CKI(h, chain_apply_d(Vj, Z, nullptr, nullptr));
          src = Z;
        }
        MOR_CKI(h, launch_op_spmv(st_in, sg, pv, ov_in, cf, ld, src, W, nullptr, nullptr, ln.stream, k));
        const int K = (j + 1) * k;
        MOR_CKI(h, dot(Vst, ldv, K, W, h1d));
        MOR_CKI(h, bgmres_launch_update(st_in, n, K, k, Vst, ldv, h1d, W, ld, 0, W, ld, ln.stream));
        MOR_CKI(h, dot(Vst, ldv, K, W, h2d));
        MOR_CKI(h, bgmres_launch_update(st_in, n, K, k, Vst, ldv, h2d, W, ld, 0, W, ld, ln.stream));
        MOR_CK(h, cudaMemcpyAsync(hh1.data(), h1d, sizeof(cdouble) * K * k, cudaMemcpyDeviceToHost, ln.stream));
        MOR_CK(h, cudaMemcpyAsync(hh2.data(), h2d, sizeof(cdouble) * K * k, cudaMemcpyDeviceToHost, ln.stream));
        std::vector<cx> Rs((size_t)k * k);
        int rk = 0;
        MOR_TRY(orth(W, Vj, Rs, &rk));        // synchronises the stream (hh1/hh2 are in place)
        const int rows = (j + 2) * k;
        hcol.assign((size_t)rows * k, cx(0.0, 0.0));
        for (int b = 0; b < k; ++b) {
          for (int kk = 0; kk < K; ++kk) hcol[(size_t)b * rows + kk] = hh1[(size_t)kk * k + b] + hh2[(size_t)kk * k + b];
          for (int i = 0; i < k; ++i) hcol[(size_t)b * rows + K + i] = Rs[(size_t)b * k + i];
        }
        ls.add_block(hcol.data());
        steps = j + 1;
        ++used;
        bool all = true;
        for (int c = 0; c < k; ++c) {
          if (scale[c] == 0.0) continue;
          if (!conv[c]) itc[c] += 1;
          if (ls.resnorm(c) * scale[c] <= tgt[c]) conv[c] = 1;
          all = all && (conv[c] || itc[c] >= mi[c]);
        }
        if (all || rk == 0) break;
        MOR_CKI(h, bgmres_launch_copy(st_in, n, k, Vj, ld, Vst, ldv, (int64_t)(j + 1) * k, ln.stream));
      }
      // x_in += P V Y, Y scaled back column by column
      Y.assign((size_t)steps * k * k, cx(0.0, 0.0));
      ls.solve(Y.data());
      for (int c = 0; c < k; ++c)
        for (int kk = 0; kk < steps * k; ++kk) Y[(size_t)c * steps * k + kk] *= scale[c];
      MOR_TRY(apply_coef(Vst, ldv, steps * k, Y, U));
      void* upd = U;
      if (Lmax > 0) {
        MOR_CKI(h, chain_apply_d(U, Z, nullptr, nullptr));
        upd = Z;
      }
      MOR_CKI(h, gmres_launch_add(st_in, sg, ld, xin, upd, ln.stream));
      for (int c = 0; c < k; ++c) conv[c] = 0;       // decided again on the true residual
    }
    for (int c = 0; c < k; ++c) {
      kit_out[c] = itc[c];
      kst_out[c] = conv[c] ? KST_OK : (brk[c] ? KST_BREAKDOWN : KST_NOCONV);
    }
    return MOR_OK;
  };

  for (int pass = 0;; ++pass) {
    // true residual r64 = b - A(sigma) x64 in FP64 with fused norms, per (system, column)
    RedArgs rn{RED_NORM, nullptr, ln.ws_part.p, nullptr, FIN_NONE, nullptr, d_sums, nullptr};
    MOR_CKI(h, launch_op_spmv(st64, sg, pv, ov64, ncf, ld, io.x64, r64, io.b64, &rn, ln.stream, k));
    MOR_CK(h, cudaMemcpyAsync(h_sums, d_sums, sizeof(cdouble) * 2 * nsc, cudaMemcpyDeviceToHost, ln.stream));
    MOR_CK(h, cudaStreamSynchronize(ln.stream));
    int nact = 0;
    for (int sgi = 0; sgi < nseg; ++sgi)
      for (int c = 0; c < k; ++c) {
        const size_t q = (size_t)sgi * k + c;
        rn2[q] = h_sums[(size_t)sgi * 2 * ld + 2 * c].re;
        if (pass == 0) bnorm[q] = std::sqrt(rn2[q]);
        relres[q] = bnorm[q] > 0 ? std::sqrt(rn2[q]) / bnorm[q] : 0.0;
        // mixed precision: MOR_MIXED_POOR refinement passes in a row that each cut the FP64
        // residual by less than 10% (FP32 inner solves that break down or stagnate) end the
        // column
        if (prec == MOR_MIXED && pass > 0 && refs[q] > 0 && status[q] == MOR_OK && relres[q] > o.tol) {
          poor[q] = (relres[q] > 0.9 * prevrel[q]) ? poor[q] + 1 : 0;
          if (poor[q] >= MOR_MIXED_POOR) status[q] = MOR_ENOCONV;
        }
        prevrel[q] = relres[q];
        act[q] = (bnorm[q] > 0 && relres[q] > o.tol && status[q] == MOR_OK && iters[q] < o.maxit &&
                  std::isfinite(relres[q])) ? 1 : 0;
        nact += act[q];
      }
    if (nact == 0 || pass >= max_outer) {
      for (size_t q = 0; q < NK; ++q) {
        if (!(relres[q] <= o.tol)) {
          if (status[q] == MOR_OK) status[q] = MOR_ENOCONV;
        } else status[q] = MOR_OK;
      }
      break;
    }
    // inner targets (dummy columns: inactive)
    for (int sgi = 0; sgi < nseg; ++sgi)
      for (int c = 0; c < ld; ++c) {
        const size_t z = (size_t)sgi * ld + c;
        if (c >= k) { tg[z] = 1.0; mi[z] = 0; ac[z] = 0; nr[z] = 0.0; continue; }
        const size_t q = (size_t)sgi * k + c;
        const double need = act[q] ? o.tol * bnorm[q] / std::sqrt(rn2[q]) : 1.0;
        tg[z] = (prec == MOR_FP64) ? need : std::max(o.inner_tol, 0.5 * need);
        mi[z] = act[q] ? std::max(0, o.maxit - iters[q]) : 0;
        ac[z] = act[q];
        nr[z] = rn2[q];
        if (act[q]) refs[q] += 1;
      }
    MOR_CK(h, cudaMemcpyAsync(d_target, tg, sizeof(double) * nsc, cudaMemcpyHostToDevice, ln.stream));
    MOR_CK(h, cudaMemcpyAsync(d_maxit, mi, sizeof(int) * nsc, cudaMemcpyHostToDevice, ln.stream));
    MOR_CK(h, cudaMemcpyAsync(d_active, ac, sizeof(int) * nsc, cudaMemcpyHostToDevice, ln.stream));
    MOR_CK(h, cudaMemcpyAsync(d_nrm2, nr, sizeof(double) * nsc, cudaMemcpyHostToDevice, ln.stream));
    // full geometry for this inner solve
    ldc = ld;
    for (int c = 0; c < ld; ++c) { cmap[c] = c < k ? c : -1; cfc[c] = cf[c]; }
    dd = d; rr = r; rh = rhat; pp = p; vv = v; ssv = sv; tt = t; pph = ph; ssh = sh; t0 = tmp0; t1 = tmp1;
    bool compacted = false;
    MOR_CKI(h, upload_masks());
    MOR_CKI(h, refine_launch_scale_cast(st_in, sg, ld, r64, d_nrm2, d_active, rhs, ln.stream));
    std::vector<int> kit(NK, 0), kstat(NK, KST_OK);
    void* dres = dd;
    if (o.solver == MOR_BGMRES) {
      MOR_TRY(bgmres_inner(dd, kit, kstat));
    } else if (o.solver == MOR_GMRES) {
      MOR_TRY(gmres_inner(dd, kit, kstat));
    } else {
      // mixed precision: an FP32 inner solve that stops improving hands back to the refinement
      const int stag = (prec == MOR_MIXED) ? MOR_MIXED_STAG : 0;
      MOR_CKI(h, krylov_launch_init(st_in, sg, ld, rhs, dd, rr, rh, pp, vv, ln.ws_part.p, kstate, d_target, d_maxit,
                                    stag, sm.done, ln.stream));
      MOR_TRY(capture());
      int maxrem = 0;
      for (size_t z = 0; z < nsc; ++z) maxrem = std::max(maxrem, mi[z]);
      int it = 0;
      int* hd = (int*)(ac + nsc);
      while (it < maxrem) {
        if (gexec) {
          MOR_CK(h, cudaGraphLaunch(gexec, ln.stream));
          mor_count_launches(graph_nodes);
          mor_replay_tally(graph_tally);
          it += chunk;
        } else {
          MOR_CKI(h, one_iter());
          it += 1;
          if ((it % chunk) != 0 && it < maxrem) continue;
        }
        if (nseg > 1) {
          MOR_CK(h, cudaMemcpyAsync(hd, sm.done, sizeof(int), cudaMemcpyDeviceToHost, ln.stream));
          MOR_CK(h, cudaStreamSynchronize(ln.stream));
          if (*hd) break;
          continue;
        }
        MOR_CKI(h, krylov_read_states(kst_host.data(), kstate, ldc, ln.stream));
        int nlive = 0;
        for (int c = 0; c < ldc; ++c) nlive += krylov_state_active(kst_host.data() + ksb * c) ? 1 : 0;
        if (nlive == 0) break;
        // repack when the live columns fit rows at least a quarter narrower or
        // half as many lanes (a repack and a graph capture cost about as much
        // as a few iterations)
        const int ld_new = row_stride(st_in, nlive);
        int tpr_old = 1, tpr_new = 1, cpt_ = 1;
        lane_shape(st_in, ldc, &tpr_old, &cpt_);
        lane_shape(st_in, ld_new, &tpr_new, &cpt_);
        if (ld_new >= ldc || it >= maxrem || (4 * ld_new > 3 * ldc && tpr_new >= tpr_old)) continue;
        // ---- compaction: flush dropped real columns, repack the live ones
        std::vector<int> live, drop_src, drop_dst;
        for (int c = 0; c < ldc; ++c) {
          const unsigned char* ks = kst_host.data() + ksb * c;
          if (krylov_state_active(ks)) { live.push_back(c); continue; }
          const int oc = cmap[c];
          if (oc >= 0 && oc < k) {
            drop_src.push_back(c);
            drop_dst.push_back(oc);
            kit[oc] = krylov_state_iters(ks);
            kstat[oc] = krylov_state_status(ks);
          }
        }
        int* dmaps = sm.masks + (size_t)MAX_FACTORS * MOR_KMAX - 3 * MOR_LDMAX;   // tail of the mask area
        std::vector<int> maps(3 * MOR_LDMAX, 0);
        for (size_t i = 0; i < drop_src.size(); ++i) { maps[i] = drop_src[i]; maps[MOR_LDMAX + i] = drop_dst[i]; }
        for (size_t i = 0; i < live.size(); ++i) maps[2 * MOR_LDMAX + i] = live[i];
        MOR_CK(h, cudaMemcpyAsync(dmaps, maps.data(), sizeof(int) * maps.size(), cudaMemcpyHostToDevice, ln.stream));
        if (!drop_src.empty())
          MOR_CKI(h, conv_launch_scatter_cols(st_in, n, ldc, ld, (int)drop_src.size(), dmaps, dmaps + MOR_LDMAX, dd,
                                              d_full, ln.stream));
        const int* gmap = dmaps + 2 * MOR_LDMAX;
        void* src[5] = {dd, rr, rh, pp, vv};
        void* dst[5] = {ssv, tt, pph, ssh, t0};
        for (int q = 0; q < 5; ++q)
          MOR_CKI(h, conv_launch_gather_cols(st_in, n, ldc, ld_new, (int)live.size(), gmap, src[q], dst[q], ln.stream));
        // the old state vectors become the scratch set
        dd = dst[0]; rr = dst[1]; rh = dst[2]; pp = dst[3]; vv = dst[4];
        ssv = src[0]; tt = src[1]; pph = src[2]; ssh = src[3]; t0 = src[4];
        std::vector<int> nmap(ld_new, -1);
        for (int c = 0; c < ld_new; ++c) {
          if (c < (int)live.size()) {
            nmap[c] = cmap[live[c]];
            memcpy(kst_new.data() + ksb * c, kst_host.data() + ksb * live[c], ksb);
            cfc[c] = cfc[live[c]];
          } else {
            krylov_state_make_dummy(kst_new.data() + ksb * c);
            cfc[c] = cfc[live[0]];
          }
        }
        cmap = nmap;
        ldc = ld_new;
        MOR_CKI(h, krylov_write_state(kst_new.data(), kstate, ldc, ln.stream));
        MOR_CKI(h, upload_masks());
        compacted = true;
        MOR_TRY(capture());
      }
      // final per-(system, column) state of this inner solve
      MOR_CKI(h, krylov_read_states(kst_host.data(), kstate, nseg * ldc, ln.stream));
      for (int sgi = 0; sgi < nseg; ++sgi)
        for (int c = 0; c < ldc; ++c) {
          const int oc = cmap[c];
          if (oc >= 0 && oc < k) {
            const unsigned char* ks = kst_host.data() + ksb * ((size_t)sgi * ldc + c);
            kit[(size_t)sgi * k + oc] = krylov_state_iters(ks);
            kstat[(size_t)sgi * k + oc] = krylov_state_status(ks);
          }
        }
      if (compacted) {
        // collect the remaining columns into d_full (original layout)
        std::vector<int> maps(2 * MOR_LDMAX, 0);
        int nrem = 0;
        for (int c = 0; c < ldc; ++c)
          if (cmap[c] >= 0 && cmap[c] < k) { maps[nrem] = c; maps[MOR_LDMAX + nrem] = cmap[c]; ++nrem; }
        int* dmaps = sm.masks + (size_t)MAX_FACTORS * MOR_KMAX - 3 * MOR_LDMAX;
        MOR_CK(h, cudaMemcpyAsync(dmaps, maps.data(), sizeof(int) * maps.size(), cudaMemcpyHostToDevice, ln.stream));
        if (nrem > 0)
          MOR_CKI(h, conv_launch_scatter_cols(st_in, n, ldc, ld, nrem, dmaps, dmaps + MOR_LDMAX, dd, d_full, ln.stream));
        dres = d_full;
      }
    }
    for (size_t q = 0; q < NK; ++q) {
      if (!act[q]) continue;
      iters[q] += kit[q];
      if (kstat[q] == KST_BREAKDOWN && pass + 1 >= max_outer) status[q] = MOR_EBREAKDOWN;
    }
    MOR_CKI(h, refine_launch_update(st_in, sg, ld, io.x64, dres, d_nrm2, d_active, ln.stream));
  }
  // per-column statistics: with several systems, stats has nseg x k entries
  if (stats)
    for (size_t q = 0; q < NK; ++q) {
      stats[q].iters = iters[q];
      stats[q].refinements = refs[q];
      stats[q].relres = relres[q];
      stats[q].status = status[q];
      stats[q].fallback = 0;
    }
  int worst = MOR_OK;
  for (size_t q = 0; q < NK; ++q)
    if (status[q] != MOR_OK) worst = (worst == MOR_OK || status[q] == MOR_EBREAKDOWN) ? status[q] : worst;
  if (worst != MOR_OK) return mor_fail(h, worst, "%s in at least one column", worst == MOR_EBREAKDOWN ? "breakdown" : "no convergence");
  return MOR_OK;
}

// Solve k shifts (any k), batching by 16.  rhs: either R (col-major c128, host or
// device) or the system's B/C column 0.  X out col-major c128 (host or device).
static int solve_many(mor_t h, SolveLane& ln, const mor_c64* sig, int k, int transpose, const mor_solve_opts& o,
                      const std::vector<ColChain>& L, bool cplx, const mor_c64* R, bool dev, mor_c64* X,
                      mor_solve_stats* stats) {
  const int64_t n = h->n;
  const int st64 = cplx ? ST_C64 : ST_F64;
  const int st_in = st_of(o.precision, cplx);
  const size_t es64 = st_size(st64);
  const int bmax = o.batch ? MOR_KMAX : 1;
  int ret = MOR_OK;
  for (int c0 = 0, kc = 0; c0 < k; c0 += kc) {
    kc = std::min(bmax, k - c0);
    if (o.solver == MOR_BGMRES) {
      // a block: the consecutive columns that share the shift and the chain
      kc = 1;
      while (c0 + kc < k && kc < bgmres_max_cols() && same_shift(sig[c0 + kc], sig[c0]) &&
             L[c0 + kc].a == L[c0].a && L[c0 + kc].b == L[c0].b && L[c0 + kc].x == L[c0].x)
        ++kc;
    }
    const int ld = row_stride(st_in, kc);
    MOR_CK(h, ln.ws_b64.alloc(es64 * (size_t)n * ld));
    MOR_CK(h, ln.ws_x64.alloc(es64 * (size_t)n * ld));
    void* xrow = ln.ws_x64.p;
    if (ld > kc) MOR_CK(h, cudaMemsetAsync(ln.ws_b64.p, 0, es64 * (size_t)n * ld, ln.stream));
    if (R) {
      const mor_c64* Rc = R + (size_t)n * c0;
      const void* src = Rc;
      if (!dev) {
        MOR_CK(h, ln.ws_io.alloc(sizeof(mor_c64) * (size_t)n * kc));
        MOR_CK(h, cudaMemcpyAsync(ln.ws_io.p, Rc, sizeof(mor_c64) * (size_t)n * kc, cudaMemcpyHostToDevice, ln.stream));
        src = ln.ws_io.p;
      }
      MOR_CKI(h, conv_launch_colmajor_c128_to_rowmajor(st64, (int)n, kc, ld, src, ln.ws_b64.p, ln.stream));
    } else {
      const double* col0 = transpose ? h->C.as<double>() : h->B.as<double>();
      MOR_CKI(h, conv_launch_real_col_to_rowmajor(st64, (int)n, kc, ld, col0, 0, ln.ws_b64.p, ln.stream));
    }
    BatchIO io{sig + c0, kc, ld, L.data() + c0, ln.ws_b64.p, xrow};
    const int nseg = h->seg.nseg;
    std::vector<mor_solve_stats> sb((size_t)nseg * kc);
    int s = solve_batch(h, ln, transpose, o, cplx, io, sb.data());
    if ((s == MOR_ENOCONV || s == MOR_EBREAKDOWN) && o.precision == MOR_MIXED && o.fp64_fallback) {
      // columns that failed in mixed precision before maxit: solve them again from zero with
      // FP64 Krylov iterations (same chain prefix), then put them back in place
      std::vector<int> redo;
      for (int c = 0; c < kc; ++c) {
        bool bad = false;
        for (int sgi = 0; sgi < nseg; ++sgi) {
          const mor_solve_stats& x = sb[(size_t)sgi * kc + c];
          if (x.status != MOR_OK && x.iters < o.maxit) bad = true;
        }
        if (bad) redo.push_back(c);
      }
      if (!redo.empty()) {
        const int nr = (int)redo.size();
        mor_solve_opts o64 = o;
        o64.precision = MOR_FP64;
        const int ld2 = row_stride(st_of(MOR_FP64, cplx), nr);
        const size_t vb = es64 * (size_t)n * ld2;
        MOR_CK(h, ln.ws_fb.alloc(256 + 2 * vb));
        int* dmap = ln.ws_fb.as<int>();                   // [redo columns | 0 .. nr-1]
        void* b2 = ln.ws_fb.as<char>() + 256;
        void* x2 = (char*)b2 + vb;
        std::vector<int> hmap(2 * nr);
        for (int i = 0; i < nr; ++i) { hmap[i] = redo[i]; hmap[nr + i] = i; }
        MOR_CK(h, cudaMemcpyAsync(dmap, hmap.data(), sizeof(int) * 2 * nr, cudaMemcpyHostToDevice, ln.stream));
        MOR_CK(h, cudaStreamSynchronize(ln.stream));
        MOR_CKI(h, conv_launch_gather_cols(st64, n, ld, ld2, nr, dmap, ln.ws_b64.p, b2, ln.stream));
        std::vector<mor_c64> s2(nr);
        std::vector<ColChain> L2(nr);
        for (int i = 0; i < nr; ++i) { s2[i] = sig[c0 + redo[i]]; L2[i] = L[c0 + redo[i]]; }
        BatchIO io2{s2.data(), nr, ld2, L2.data(), b2, x2};
        std::vector<mor_solve_stats> sb2((size_t)nseg * nr);
        const int s2r = solve_batch(h, ln, transpose, o64, cplx, io2, sb2.data());
        if (s2r != MOR_OK && s2r != MOR_ENOCONV && s2r != MOR_EBREAKDOWN) return s2r;
        MOR_CKI(h, conv_launch_scatter_cols(st64, n, ld2, ld, nr, dmap + nr, dmap, x2, xrow, ln.stream));
        s = MOR_OK;
        for (int sgi = 0; sgi < nseg; ++sgi)
          for (int i = 0; i < nr; ++i) {
            mor_solve_stats& a = sb[(size_t)sgi * kc + redo[i]];
            const mor_solve_stats& b = sb2[(size_t)sgi * nr + i];
            a.iters += b.iters;
            a.refinements = b.refinements;
            a.relres = b.relres;
            a.status = b.status;
            a.fallback = 1;
          }
        for (const mor_solve_stats& a : sb)
          if (a.status != MOR_OK) s = (s == MOR_OK || a.status == MOR_EBREAKDOWN) ? a.status : s;
      }
    }
    if (stats)   // stats has nseg x k entries: [seg * k + c]
      for (int sgi = 0; sgi < nseg; ++sgi)
        for (int c = 0; c < kc; ++c) stats[(size_t)sgi * k + c0 + c] = sb[(size_t)sgi * kc + c];
    if (s != MOR_OK && s != MOR_ENOCONV && s != MOR_EBREAKDOWN) return s;
    if (s != MOR_OK) ret = s;
    if (X) {
      mor_c64* Xc = X + (size_t)n * c0;
      if (dev) {
        MOR_CKI(h, conv_launch_rowmajor_to_colmajor_c128(st64, (int)n, kc, ld, xrow, Xc, ln.stream));
      } else {
        MOR_CK(h, ln.ws_io.alloc(sizeof(mor_c64) * (size_t)n * kc));
        MOR_CKI(h, conv_launch_rowmajor_to_colmajor_c128(st64, (int)n, kc, ld, xrow, ln.ws_io.p, ln.stream));
        MOR_CK(h, cudaMemcpyAsync(Xc, ln.ws_io.p, sizeof(mor_c64) * (size_t)n * kc, cudaMemcpyDeviceToHost, ln.stream));
      }
    }
  }
  MOR_CK(h, cudaStreamSynchronize(ln.stream));
  return ret;
}

static std::vector<ColChain> prefix_lengths(OpData& op, const mor_c64* sig, int k) {
  std::vector<ColChain> L(k, prefix_chain((int)op.chain.size()));
  for (int c = 0; c < k; ++c)
    for (int f = (int)op.chain.size() - 1; f >= 0; --f)
      if (same_shift(op.chain[f].to, sig[c])) { L[c] = prefix_chain(f + 1); break; }
  return L;
}

static bool chain_cplx(const OpData& op, const std::vector<ColChain>& L) {
  for (const ColChain& c : L)
    for (int f = 0; f < c.end(); ++f)
      if (c.uses(f) && st_is_cplx(op.chain[f].st)) return true;
  return false;
}

// ---------------------------------------------------------------------------
// Gram-Schmidt and projection helpers on device FP64 column-major blocks
// ---------------------------------------------------------------------------
static int orth_device(mor_t h, double* V, int64_t n, int k, int* dependent) {
  MOR_CK(h, h->ws_gram.alloc(sizeof(double) * (2 * 2 * 128 + 4096)));
  double* hbuf = h->ws_gram.as<double>();          // h coefficients (k), norms
  double* norms = hbuf + 256;                       // [2j] original, [2j+1] final
  MOR_CK(h, h->ws_part.alloc(sizeof(double) * 1024 * (size_t)h->grid_cap));
  unsigned* cnt = h->ws_counter.as<unsigned>() + 8;
  for (int j = 0; j < k; ++j) {
    double* v = V + (size_t)j * n;
    MOR_CKI(h, dense_launch_gram((int)n, 1, 1, v, n, v, n, norms + 2 * j, h->ws_part.as<double>(), cnt, h->grid_cap, h->stream));
    for (int pass = 0; pass < 2 && j > 0; ++pass) {
      MOR_CKI(h, dense_launch_gram((int)n, j, 1, V, n, v, n, hbuf, h->ws_part.as<double>(), cnt, h->grid_cap, h->stream));
      MOR_CKI(h, dense_launch_gs_update((int)n, j, V, n, hbuf, v, h->stream));
    }
    MOR_CKI(h, dense_launch_gram((int)n, 1, 1, v, n, v, n, norms + 2 * j + 1, h->ws_part.as<double>(), cnt, h->grid_cap, h->stream));
    MOR_CKI(h, dense_launch_scale((int)n, v, norms + 2 * j + 1, h->stream));
  }
  std::vector<double> nh(2 * k);
  MOR_CK(h, cudaMemcpyAsync(nh.data(), norms, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost, h->stream));
  MOR_CK(h, cudaStreamSynchronize(h->stream));
  *dependent = 0;
  for (int j = 0; j < k; ++j)
    if (!(nh[2 * j + 1] > 1e-28 * nh[2 * j]) || !std::isfinite(nh[2 * j + 1])) *dependent = 1;
  return MOR_OK;
}

// A_r = W^T A V, E_r = W^T E V, B_r = W^T B, C_r = V^T C (device V, W), into rom
static int project_device(mor_t h, const double* V, const double* W, int r, mor_reduced* rom) {
  const int64_t n = h->n;
  OpData& op = h->P;
  MOR_CK(h, h->ws_basis.alloc(sizeof(double) * (size_t)n * r * 2));
  double* AV = h->ws_basis.as<double>();
  double* EV = AV + (size_t)n * r;
  PatView pv = op.view();
  OpVals ov = op_vals(h, op, false);
  Coef ca{0, 0, 1, 0}, ce{1, 0, 0, 0};
  for (int j = 0; j < r; ++j) {
    MOR_CKI(h, launch_op_spmv(ST_F64, h->seg, pv, ov, &ca, 1, V + (size_t)j * n, AV + (size_t)j * n, nullptr, nullptr, h->stream));
    MOR_CKI(h, launch_op_spmv(ST_F64, h->seg, pv, ov, &ce, 1, V + (size_t)j * n, EV + (size_t)j * n, nullptr, nullptr, h->stream));
  }
  MOR_CK(h, h->ws_rom.alloc(sizeof(double) * 6 * MOR_MAX_R * MOR_MAX_R));
  double* dAr = h->ws_rom.as<double>();
  double* dEr = dAr + MOR_MAX_R * MOR_MAX_R;
  double* dBr = dEr + MOR_MAX_R * MOR_MAX_R;
  double* dCr = dBr + MOR_MAX_R * MOR_MAX_IO;
  MOR_CK(h, h->ws_part.alloc(sizeof(double) * 1024 * (size_t)h->grid_cap));
  unsigned* cnt = h->ws_counter.as<unsigned>() + 16;
  double* part = h->ws_part.as<double>();
  MOR_CKI(h, dense_launch_gram((int)n, r, r, W, n, AV, n, dAr, part, cnt, h->grid_cap, h->stream));
  MOR_CKI(h, dense_launch_gram((int)n, r, r, W, n, EV, n, dEr, part, cnt, h->grid_cap, h->stream));
  MOR_CKI(h, dense_launch_gram((int)n, r, h->m, W, n, h->B.as<double>(), n, dBr, part, cnt, h->grid_cap, h->stream));
  MOR_CKI(h, dense_launch_gram((int)n, r, h->q, V, n, h->C.as<double>(), n, dCr, part, cnt, h->grid_cap, h->stream));
  rom->r = r;
  rom->m = h->m;
  rom->q = h->q;
  MOR_CK(h, cudaMemcpyAsync(rom->Ar, dAr, sizeof(double) * r * r, cudaMemcpyDeviceToHost, h->stream));
  MOR_CK(h, cudaMemcpyAsync(rom->Er, dEr, sizeof(double) * r * r, cudaMemcpyDeviceToHost, h->stream));
  MOR_CK(h, cudaMemcpyAsync(rom->Br, dBr, sizeof(double) * r * h->m, cudaMemcpyDeviceToHost, h->stream));
  MOR_CK(h, cudaMemcpyAsync(rom->Cr, dCr, sizeof(double) * r * h->q, cudaMemcpyDeviceToHost, h->stream));
  MOR_CK(h, cudaStreamSynchronize(h->stream));
  return MOR_OK;
}

static int poles_device(mor_t h, const mor_reduced* rom, mor_c64* lam, mor_c64* shifts) {
  const int r = rom->r;
  MOR_CK(h, h->ws_rom.alloc(sizeof(double) * 6 * MOR_MAX_R * MOR_MAX_R));
  double* dAr = h->ws_rom.as<double>();
  double* dEr = dAr + MOR_MAX_R * MOR_MAX_R;
  double* out = dEr + MOR_MAX_R * MOR_MAX_R;   // 4r+1 + 2r^2 doubles + r ints fits in 2 * 64^2
  MOR_CK(h, cudaMemcpyAsync(dAr, rom->Ar, sizeof(double) * r * r, cudaMemcpyHostToDevice, h->stream));
  MOR_CK(h, cudaMemcpyAsync(dEr, rom->Er, sizeof(double) * r * r, cudaMemcpyHostToDevice, h->stream));
  MOR_CKI(h, dense_launch_eig(r, dAr, dEr, out, h->stream));
  std::vector<double> ho(4 * r + 1);
  MOR_CK(h, cudaMemcpyAsync(ho.data(), out, sizeof(double) * (4 * r + 1), cudaMemcpyDeviceToHost, h->stream));
  MOR_CK(h, cudaStreamSynchronize(h->stream));
  if (ho[4 * r] != 0.0) return mor_fail(h, MOR_ESINGULAR, ho[4 * r] == 1.0 ? "E_r is singular" : "QR iteration did not converge");
  for (int i = 0; i < r; ++i) {
    if (lam) lam[i] = mor_c64{ho[i], ho[r + i]};
    if (shifts) shifts[i] = mor_c64{ho[2 * r + i], ho[3 * r + i]};
  }
  return MOR_OK;
}

// out(:, i) = M b_i for i < l, M n x m FP64 column-major, b_i = coef[i m .. i m + m - 1]
// complex: the tangential right-hand sides B b_i and C c_i (complex128 columns)
__global__ void combine_kernel(int64_t n, int m, int l, const double* M, const mor_c64* coef, double* out) {
  const int64_t tot = n * l;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx % n;
    const int i = (int)(idx / n);
    double re = 0.0, im = 0.0;
    for (int j = 0; j < m; ++j) {
      const double v = M[row + (int64_t)j * n];
      re += v * coef[(size_t)i * m + j].re;
      im += v * coef[(size_t)i * m + j].im;
    }
    out[2 * idx] = re;
    out[2 * idx + 1] = im;
  }
}

// Reads n16 16-byte words (an L2 flush that leaves clean lines: evicting them
// costs the next kernel no write-back); sink is written only if the sum of
// the words hits a value that never occurs, so the reads cannot be elided.
__global__ void flush_read_kernel(const uint4* __restrict__ p, int64_t n16, unsigned* sink) {
  unsigned acc = 0u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 v = p[i];
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  if (acc == 0x9e3779b9u && threadIdx.x == 1023) *sink = acc;
}

// real (part 0) or imaginary (part 1) part of a complex128 column into an FP64 basis column
__global__ void extract_kernel(int n, int part, const double* src, double* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[2 * i + part];
}

// out(:, c) = sgn * D X(:, c) / ||X(:, g c .. g c + g - 1)||_F for the group
// of g columns containing c (nrm2: squared column norms; nullptr: no scaling);
// D diagonal (d), or the identity (d = nullptr).  n x k complex128, column-major.
__global__ void moment_rhs_kernel(int64_t n, int k, int g, const double* d, const cdouble* X, const double* nrm2,
                                  double sgn, cdouble* out) {
  const int64_t tot = n * k;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx % n;
    const int c = (int)(idx / n);
    double sc = sgn;
    if (nrm2) {
      double f = 0.0;
      for (int j = (c / g) * g; j < (c / g) * g + g; ++j) f += nrm2[j];
      sc = f > 0.0 ? sgn / sqrt(f) : 0.0;
    }
    if (d) sc *= d[row];
    out[idx] = cdouble(sc * X[idx].re, sc * X[idx].im);
  }
}

// squared norms of k complex128 columns (n rows each, column-major) into nrm2[0..k-1]
static int column_norms2(mor_t h, const mor_c64* X, int64_t n, int k, double* nrm2, cudaStream_t s) {
  if (2 * n > 0x7fffffffLL) return mor_fail(h, MOR_EINVAL, "columns too long for the norm kernel");
  MOR_CK(h, h->ws_part.alloc(sizeof(double) * 1024 * (size_t)h->grid_cap));
  unsigned* cnt = h->ws_counter.as<unsigned>() + 8;
  for (int c = 0; c < k; ++c) {
    const double* v = (const double*)(X + (size_t)n * c);
    MOR_CKI(h, dense_launch_gram((int)(2 * n), 1, 1, v, 2 * n, v, 2 * n, nrm2 + c, h->ws_part.as<double>(), cnt,
                                 h->grid_cap, s));
  }
  return MOR_OK;
}

// Y = E' X for k complex128 columns (column-major, device): E' = E (transpose
// 0) or E^T (1) of the first-order system.  Identity and diagonal E act
// elementwise; a general sparse E runs the operator SpMV with coefficients
// (1, 0) on row-major batches of at most 16 columns.
static int apply_E(mor_t h, int transpose, const mor_c64* X, mor_c64* Y, int64_t n, int k, cudaStream_t s) {
  const int g = (int)std::min<int64_t>((n * k + 255) / 256, h->grid_cap);
  if (h->ekind != EK_CSR) {
    moment_rhs_kernel<<<g, 256, 0, s>>>(n, k, 1, h->ekind == EK_DIAG ? h->ediag64.as<double>() : nullptr,
                                        (const cdouble*)X, nullptr, 1.0, (cdouble*)Y);
    mor_count_launches(1);
    MOR_CK(h, cudaGetLastError());
    return MOR_OK;
  }
  OpData& op = h->op(transpose);
  for (int c0 = 0; c0 < k; c0 += MOR_KMAX) {
    const int kc = std::min(MOR_KMAX, k - c0);
    const int ld = row_stride(ST_C64, kc);
    MOR_CK(h, h->ws_io.alloc(sizeof(mor_c64) * (size_t)n * 2 * ld));
    char* xr = h->ws_io.as<char>();
    char* yr = xr + sizeof(mor_c64) * (size_t)n * ld;
    if (ld > kc) MOR_CK(h, cudaMemsetAsync(xr, 0, sizeof(mor_c64) * (size_t)n * ld, s));
    MOR_CKI(h, conv_launch_colmajor_c128_to_rowmajor(ST_C64, (int)n, kc, ld, X + (size_t)n * c0, xr, s));
    Coef cf[MOR_LDMAX];
    for (int c = 0; c < ld; ++c) cf[c] = Coef{1.0, 0.0, 0.0, 0.0};
    MOR_CKI(h, launch_op_spmv(ST_C64, h->seg, op.view(), op_vals(h, op, false), cf, ld, xr, yr, nullptr, nullptr, s, kc));
    MOR_CKI(h, conv_launch_rowmajor_to_colmajor_c128(ST_C64, (int)n, kc, ld, yr, Y + (size_t)n * c0, s));
  }
  return MOR_OK;
}

extern "C" {

int mor_build_precond(mor_t h, mor_c64 sigma, int transpose, int precision) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  if (precision != MOR_FP64 && precision != MOR_MIXED) return mor_fail(h, MOR_EINVAL, "bad precision");
  if (!std::isfinite(sigma.re) || !std::isfinite(sigma.im)) return mor_fail(h, MOR_EINVAL, "non-finite shift");
  cudaSetDevice(h->dev);
  return build_factor(h, transpose, sigma, sigma, false, precision);
}

int mor_update_precond(mor_t h, mor_c64 sigma_new, int transpose) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  OpData& X = h->op(transpose);
  if (X.chain.empty()) return mor_fail(h, MOR_ESTATE, "update_precond before build_precond");
  if (!std::isfinite(sigma_new.re) || !std::isfinite(sigma_new.im)) return mor_fail(h, MOR_EINVAL, "non-finite shift");
  cudaSetDevice(h->dev);
  return build_factor(h, transpose, X.chain.back().to, sigma_new, true, X.chain_prec);
}

int mor_truncate_precond(mor_t h, int transpose, int length) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  OpData& X = h->op(transpose);
  if (length < 0) return mor_fail(h, MOR_EINVAL, "negative length");
  if ((size_t)length < X.chain.size()) {
    cudaStreamSynchronize(h->stream);
    X.chain.resize(length);
  }
  return MOR_OK;
}

int mor_chain_info(mor_t h, int transpose, int* length, int* precision) {
  if (!h) return MOR_EINVAL;
  OpData& X = h->op(transpose);
  if (length) *length = (int)X.chain.size();
  if (precision) *precision = X.chain_prec;
  return MOR_OK;
}

int mor_get_factor(mor_t h, int transpose, int index, mor_c64* vals, mor_c64* sfrom, mor_c64* sto) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  OpData& X = h->op(transpose);
  if (index < 0 || index >= (int)X.chain.size()) return mor_fail(h, MOR_EINVAL, "factor index out of range");
  const Factor& F = X.chain[index];
  if (sfrom) *sfrom = F.from;
  if (sto) *sto = F.to;
  if (vals) {
    DBuf tmp;
    MOR_CK(h, tmp.alloc(sizeof(mor_c64) * (size_t)X.nlay));
    MOR_CKI(h, conv_launch_copy_cast(ST_C64, F.st, X.nlay, F.vals->p, tmp.p, h->stream));
    std::vector<mor_c64> lay(X.nlay);
    MOR_CK(h, cudaMemcpyAsync(lay.data(), tmp.p, sizeof(mor_c64) * X.nlay, cudaMemcpyDeviceToHost, h->stream));
    MOR_CK(h, cudaStreamSynchronize(h->stream));
    for (int64_t p = 0; p < X.nnz; ++p) vals[p] = lay[X.h_lay[p]];
  }
  return MOR_OK;
}

int mor_apply_operator(mor_t h, const mor_c64* sigma, int k, int transpose, int precision, const mor_c64* X,
                       mor_c64* Y, unsigned flags) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  if (k < 1 || k > MOR_KMAX || !sigma || !X || !Y) return mor_fail(h, MOR_EINVAL, "bad arguments");
  cudaSetDevice(h->dev);
  const bool dev = flags & MOR_DEVICE_PTRS;
  const bool real = flags & MOR_REAL_VECTORS;
  if (real)
    for (int c = 0; c < k; ++c)
      if (!is_real_shift(sigma[c])) return mor_fail(h, MOR_EINVAL, "MOR_REAL_VECTORS needs real shifts");
  OpData& op = h->op(transpose);
  const int64_t n = h->n;
  const int st = (precision == MOR_FP64) ? (real ? ST_F64 : ST_C64) : (real ? ST_F32 : ST_C32);
  const int ld = row_stride(st, k);
  MOR_CK(h, h->ws_io.alloc(sizeof(mor_c64) * (size_t)n * (k + 2 * ld)));
  mor_c64* io = h->ws_io.as<mor_c64>();
  const void* src = X;
  if (!dev) {
    MOR_CK(h, cudaMemcpyAsync(io, X, sizeof(mor_c64) * n * k, cudaMemcpyHostToDevice, h->stream));
    src = io;
  }
  char* xr = (char*)(io + (size_t)n * k);
  char* yr = xr + st_size(st) * (size_t)n * ld;
  if (ld > k) MOR_CK(h, cudaMemsetAsync(xr, 0, st_size(st) * (size_t)n * ld, h->stream));
  MOR_CKI(h, conv_launch_colmajor_c128_to_rowmajor(st, (int)n, k, ld, src, xr, h->stream));
  Coef cf[MOR_LDMAX];
  for (int c = 0; c < ld; ++c) cf[c] = mor_coef(h, sigma[c < k ? c : 0]);
  MOR_CKI(h, launch_op_spmv(st, h->seg, op.view(), op_vals(h, op, precision != MOR_FP64), cf, ld, xr, yr, nullptr,
                            nullptr, h->stream, k));
  if (dev) {
    MOR_CKI(h, conv_launch_rowmajor_to_colmajor_c128(st, (int)n, k, ld, yr, Y, h->stream));
  } else {
    MOR_CKI(h, conv_launch_rowmajor_to_colmajor_c128(st, (int)n, k, ld, yr, io, h->stream));
    MOR_CK(h, cudaMemcpyAsync(Y, io, sizeof(mor_c64) * n * k, cudaMemcpyDeviceToHost, h->stream));
  }
  MOR_CK(h, cudaStreamSynchronize(h->stream));
  return MOR_OK;
}

int mor_apply_precond(mor_t h, const mor_c64* sigma, int k, int transpose, const mor_c64* X, mor_c64* Y,
                      unsigned flags) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  if (k < 1 || k > MOR_KMAX || !sigma || !X || !Y) return mor_fail(h, MOR_EINVAL, "bad arguments");
  OpData& op = h->op(transpose);
  if (op.chain.empty()) return mor_fail(h, MOR_ESTATE, "no preconditioner built");
  cudaSetDevice(h->dev);
  const bool dev = flags & MOR_DEVICE_PTRS;
  const bool real = flags & MOR_REAL_VECTORS;
  const int64_t n = h->n;
  const int st = (op.chain_prec == MOR_FP64) ? (real ? ST_F64 : ST_C64) : (real ? ST_F32 : ST_C32);
  std::vector<ColChain> L = prefix_lengths(op, sigma, k);
  int Lmax = 0;
  for (const ColChain& x : L) Lmax = std::max(Lmax, x.end());
  if (real)
    for (int f = 0; f < Lmax; ++f)
      if (st_is_cplx(op.chain[f].st)) return mor_fail(h, MOR_EINVAL, "MOR_REAL_VECTORS with a complex chain factor");
  const int ld = row_stride(st, k);
  MOR_CK(h, h->ws_io.alloc(sizeof(mor_c64) * (size_t)n * (k + 2 * ld)));
  mor_c64* io = h->ws_io.as<mor_c64>();
  const void* src = X;
  if (!dev) {
    MOR_CK(h, cudaMemcpyAsync(io, X, sizeof(mor_c64) * n * k, cudaMemcpyHostToDevice, h->stream));
    src = io;
  }
  char* a = (char*)(io + (size_t)n * k);
  char* b = a + st_size(st) * (size_t)n * ld;
  if (ld > k) MOR_CK(h, cudaMemsetAsync(a, 0, st_size(st) * (size_t)n * ld, h->stream));
  MOR_CKI(h, conv_launch_colmajor_c128_to_rowmajor(st, (int)n, k, ld, src, a, h->stream));
  Small sm;
  MOR_TRY(get_small(h, h->ws_small, sm));
  std::vector<int> masks((size_t)std::max(Lmax, 1) * MOR_KMAX, 0);
  for (int f = 0; f < Lmax; ++f)
    for (int c = 0; c < ld; ++c) masks[(size_t)f * MOR_KMAX + c] = (c >= k || L[c].uses(f)) ? 1 : 0;
  MOR_CK(h, cudaMemcpyAsync(sm.masks, masks.data(), sizeof(int) * masks.size(), cudaMemcpyHostToDevice, h->stream));
  char* s = a;
  char* d = b;
  for (int f = 0; f < Lmax; ++f) {
    MOR_CKI(h, launch_factor_spmv(st, op.chain[f].st, h->seg, op.view(), op.chain[f].vals->p,
                                  sm.masks + (size_t)f * MOR_KMAX, ld, s, d, nullptr, nullptr, h->stream, k));
    std::swap(s, d);
  }
  if (dev) {
    MOR_CKI(h, conv_launch_rowmajor_to_colmajor_c128(st, (int)n, k, ld, s, Y, h->stream));
  } else {
    MOR_CKI(h, conv_launch_rowmajor_to_colmajor_c128(st, (int)n, k, ld, s, io, h->stream));
    MOR_CK(h, cudaMemcpyAsync(Y, io, sizeof(mor_c64) * n * k, cudaMemcpyDeviceToHost, h->stream));
  }
  MOR_CK(h, cudaStreamSynchronize(h->stream));
  return MOR_OK;
}

int mor_solve_shifts(mor_t h, const mor_c64* sigma, int k, int transpose, const mor_solve_opts* opts,
                     const mor_c64* R, mor_c64* X, mor_solve_stats* stats, unsigned flags) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  if (k < 1 || k > 64 || !sigma || !X) return mor_fail(h, MOR_EINVAL, "bad arguments (1 <= k <= 64)");
  mor_solve_opts o;
  if (opts) o = *opts; else mor_default_opts(&o);
  if (o.precision != MOR_FP64 && o.precision != MOR_MIXED) return mor_fail(h, MOR_EINVAL, "bad precision");
  if (o.solver != MOR_BICGSTAB && o.solver != MOR_GMRES && o.solver != MOR_BGMRES)
    return mor_fail(h, MOR_EINVAL, "unknown solver %d", o.solver);
  if (o.precond_precision != -1 && o.precond_precision != MOR_FP64 && o.precond_precision != MOR_MIXED)
    return mor_fail(h, MOR_EINVAL, "bad precond_precision");
  if (o.precision == MOR_MIXED && o.precond_precision == MOR_FP64)
    return mor_fail(h, MOR_EINVAL, "FP64 factors cannot serve a mixed-precision solve");
  if (!(o.tol > 0) || o.maxit < 0) return mor_fail(h, MOR_EINVAL, "bad tolerance or maxit");
  for (int c = 0; c < k; ++c)
    if (!std::isfinite(sigma[c].re) || !std::isfinite(sigma[c].im)) return mor_fail(h, MOR_EINVAL, "non-finite shift");
  cudaSetDevice(h->dev);
  SolveLane* lane0 = nullptr;
  MOR_TRY(mor_lane(h, 0, &lane0));
  const bool dev = flags & MOR_DEVICE_PTRS;
  OpData& op = h->op(transpose);
  bool rc = false;
  if (R) {
    if (dev) rc = true;
    else for (int64_t i = 0; i < h->n * (int64_t)k && !rc; ++i) rc = (R[i].im != 0.0);
  }
  bool anyc = rc;
  for (int c = 0; c < k; ++c) anyc |= !is_real_shift(sigma[c]);
  if (o.precond == 1 && h->seg.nseg != 1) return mor_fail(h, MOR_EINVAL, "a fresh SPAI per shift needs a single system");
  if (o.precond == 1) {
    // a new SPAI per shift: one column at a time
    int ret = MOR_OK;
    for (int c = 0; c < k; ++c) {
      MOR_TRY(build_factor(h, transpose, sigma[c], sigma[c], false, factor_precision(o)));
      std::vector<ColChain> L(1, prefix_chain(1));
      bool cc = anyc || chain_cplx(op, L);
      int s = solve_many(h, *lane0, sigma + c, 1, transpose, o, L, cc, R ? R + (size_t)h->n * c : nullptr, dev,
                         X + (size_t)h->n * c, stats ? stats + c : nullptr);
      if (s != MOR_OK && s != MOR_ENOCONV && s != MOR_EBREAKDOWN) return s;
      if (s != MOR_OK) ret = s;
    }
    return ret;
  }
  std::vector<ColChain> L = (o.precond == 2) ? std::vector<ColChain>(k) : prefix_lengths(op, sigma, k);
  if (o.precond == 0 && !op.chain.empty() && op.chain_prec != o.precision &&
      !(op.chain_prec == MOR_MIXED && o.precision == MOR_FP64))
    return mor_fail(h, MOR_ESTATE, "an FP64 preconditioner chain cannot serve a mixed-precision solve");
  bool cc = anyc || chain_cplx(op, L);
  const int nseg = h->seg.nseg;
  if (nseg == 1 || !stats) return solve_many(h, *lane0, sigma, k, transpose, o, L, cc, R, dev, X, stats);
  // several systems: report, per shift, the worst over the systems
  std::vector<mor_solve_stats> all((size_t)nseg * k);
  int ret = solve_many(h, *lane0, sigma, k, transpose, o, L, cc, R, dev, X, all.data());
  for (int c = 0; c < k; ++c) {
    mor_solve_stats a = all[c];
    for (int sgi = 1; sgi < nseg; ++sgi) {
      const mor_solve_stats& b = all[(size_t)sgi * k + c];
      a.iters = std::max(a.iters, b.iters);
      a.refinements = std::max(a.refinements, b.refinements);
      a.relres = std::max(a.relres, b.relres);
      a.fallback = std::max(a.fallback, b.fallback);
      if (b.status != MOR_OK) a.status = b.status;
    }
    stats[c] = a;
  }
  return ret;
}

int mor_batch_solve(mor_t h, const mor_c64* sigma, int k, int transpose, const mor_solve_opts* opts, mor_c64* X,
                    mor_solve_stats* stats, unsigned flags) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  if (k < 1 || k > 64 || !sigma || !X) return mor_fail(h, MOR_EINVAL, "bad arguments (1 <= k <= 64)");
  mor_solve_opts o;
  if (opts) o = *opts; else mor_default_opts(&o);
  if (o.precision != MOR_FP64 && o.precision != MOR_MIXED) return mor_fail(h, MOR_EINVAL, "bad precision");
  if (o.solver != MOR_BICGSTAB && o.solver != MOR_GMRES && o.solver != MOR_BGMRES)
    return mor_fail(h, MOR_EINVAL, "unknown solver %d", o.solver);
  if (o.precond_precision != -1 && o.precond_precision != MOR_FP64 && o.precond_precision != MOR_MIXED)
    return mor_fail(h, MOR_EINVAL, "bad precond_precision");
  if (o.precision == MOR_MIXED && o.precond_precision == MOR_FP64)
    return mor_fail(h, MOR_EINVAL, "FP64 factors cannot serve a mixed-precision solve");
  if (!(o.tol > 0) || o.maxit < 0) return mor_fail(h, MOR_EINVAL, "bad tolerance or maxit");
  if (o.precond == 1) return mor_fail(h, MOR_EINVAL, "mor_batch_solve: build the preconditioner with mor_build_precond");
  for (int c = 0; c < k; ++c)
    if (!std::isfinite(sigma[c].re) || !std::isfinite(sigma[c].im)) return mor_fail(h, MOR_EINVAL, "non-finite shift");
  cudaSetDevice(h->dev);
  SolveLane* lane0 = nullptr;
  MOR_TRY(mor_lane(h, 0, &lane0));
  OpData& op = h->op(transpose);
  std::vector<ColChain> L = (o.precond == 2) ? std::vector<ColChain>(k) : prefix_lengths(op, sigma, k);
  if (o.precond == 0 && !op.chain.empty() && op.chain_prec != o.precision &&
      !(op.chain_prec == MOR_MIXED && o.precision == MOR_FP64))
    return mor_fail(h, MOR_ESTATE, "an FP64 preconditioner chain cannot serve a mixed-precision solve");
  bool cc = chain_cplx(op, L);
  for (int c = 0; c < k; ++c) cc |= !is_real_shift(sigma[c]);
  std::vector<mor_solve_stats> all((size_t)h->seg.nseg * k);
  int ret = solve_many(h, *lane0, sigma, k, transpose, o, L, cc, nullptr, (flags & MOR_DEVICE_PTRS) != 0, X,
                       all.data());
  if (stats) std::memcpy(stats, all.data(), sizeof(mor_solve_stats) * all.size());
  return ret;
}

int mor_orthonormalize(mor_t h, double* X, int k, unsigned flags) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  if (k < 1 || k > MOR_MAX_R || !X) return mor_fail(h, MOR_EINVAL, "bad arguments (1 <= k <= 64)");
  cudaSetDevice(h->dev);
  const int64_t n = h->n;
  double* V = X;
  DBuf tmp;
  if (!(flags & MOR_DEVICE_PTRS)) {
    MOR_CK(h, tmp.alloc(sizeof(double) * n * k));
    MOR_CK(h, cudaMemcpyAsync(tmp.p, X, sizeof(double) * n * k, cudaMemcpyHostToDevice, h->stream));
    V = tmp.as<double>();
  }
  int dep = 0;
  MOR_TRY(orth_device(h, V, n, k, &dep));
  if (!(flags & MOR_DEVICE_PTRS)) {
    MOR_CK(h, cudaMemcpyAsync(X, V, sizeof(double) * n * k, cudaMemcpyDeviceToHost, h->stream));
    MOR_CK(h, cudaStreamSynchronize(h->stream));
  }
  if (dep) return mor_fail(h, MOR_ESINGULAR, "numerically dependent column");
  return MOR_OK;
}

int mor_project(mor_t h, const double* V, const double* W, int r, mor_reduced* rom, unsigned flags) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  if (h->order != 1) return mor_fail(h, MOR_EINVAL, "projection of second-order systems is not available");
  if (r < 1 || r > MOR_MAX_R || !V || !W || !rom) return mor_fail(h, MOR_EINVAL, "bad arguments");
  cudaSetDevice(h->dev);
  const int64_t n = h->n;
  const double *Vd = V, *Wd = W;
  DBuf tmp;
  if (!(flags & MOR_DEVICE_PTRS)) {
    MOR_CK(h, tmp.alloc(sizeof(double) * n * r * 2));
    MOR_CK(h, cudaMemcpyAsync(tmp.p, V, sizeof(double) * n * r, cudaMemcpyHostToDevice, h->stream));
    MOR_CK(h, cudaMemcpyAsync(tmp.as<double>() + n * r, W, sizeof(double) * n * r, cudaMemcpyHostToDevice, h->stream));
    Vd = tmp.as<double>();
    Wd = Vd + n * r;
  }
  return project_device(h, Vd, Wd, r, rom);
}

int mor_reduced_poles(mor_t h, const mor_reduced* rom, mor_c64* lambda, mor_c64* shifts) {
  if (!h || !rom) return MOR_EINVAL;
  if (rom->r < 1 || rom->r > MOR_MAX_R) return mor_fail(h, MOR_EINVAL, "bad r");
  cudaSetDevice(h->dev);
  return poles_device(h, rom, lambda, shifts);
}

int mor_irka_reset(mor_t h) {
  if (!h) return MOR_EINVAL;
  h->irka_z = 0;
  h->vlen[0] = h->vlen[1] = 0;
  return MOR_OK;
}

// Reuse schedule of Algorithm 4 for the solved shifts `sol` of one iteration
// on the primal operator and, with nops == 2, the transposed one.  Vertical:
// on the first iteration (or when the chain is rebuilt) a full SPAI at
// sol[0], else a Q from the previous first shift.  Horizontal, by opts.reuse:
//   MOR_REUSE_CHAIN  a Q from sol[i-1] to sol[i] for every further shift
//                    (P_i = Q_i P_{i-1}, Table II second approach);
//   MOR_REUSE_FIRST  a Q from sol[0] to sol[i] (P_i = Q_i P_1, Table II first
//                    approach): shift i applies the vertical chain and its Q;
//   MOR_REUSE_AUTO   as MOR_REUSE_CHAIN, but a factor is built only when the
//                    Frobenius ratios allow reuse (frob_reuse_ok), otherwise
//                    a fresh SPAI at the new shift, vertically (the chain is
//                    rebuilt) or horizontally (later shifts chain from it).
// Ls[t][i] = the factors shift i applies (none without a preconditioner;
// precond 1 builds per shift at solve time).
static int schedule_chains(mor_t h, const std::vector<mor_c64>& sol, const mor_solve_opts& o, int nops,
                           std::vector<ColChain>* Ls, mor_irka_stats& st) {
  const int l = (int)sol.size();
  if (o.reuse < MOR_REUSE_CHAIN || o.reuse > MOR_REUSE_AUTO) return mor_fail(h, MOR_EINVAL, "unknown reuse variant");
  auto fz = [](mor_c64 z) { return frob_z{z.re, z.im}; };
  for (int t = 0; t < nops; ++t) {
    OpData& X = h->op(t);
    std::vector<ColChain>& L = Ls[t];
    L.assign(l, ColChain{});
    if (o.precond == 2 || o.precond == 1) continue;
    const int fp = factor_precision(o);
    bool rebuild = (h->irka_z == 0) || X.chain.empty() || X.chain_prec != fp ||
                   (o.max_chain > 0 && h->vlen[t] + 1 > o.max_chain);
    if (!rebuild) { X.chain.resize(h->vlen[t]); }
    if (!rebuild && o.reuse == MOR_REUSE_AUTO) rebuild = !frob_reuse_ok(h->frob, fz(X.chain.back().to), fz(sol[0]));
    if (rebuild) {
      MOR_TRY(build_factor(h, t, sol[0], sol[0], false, fp));
      h->vlen[t] = 1;
      st.builds_spai++;
    } else {
      MOR_TRY(build_factor(h, t, X.chain.back().to, sol[0], true, fp));
      h->vlen[t] += 1;
      st.builds_reuse++;
    }
    const int v = h->vlen[t];
    L[0] = prefix_chain(v);
    for (int i = 1; i < l; ++i) {
      if (o.reuse == MOR_REUSE_FIRST) {
        MOR_TRY(build_factor(h, t, sol[0], sol[i], true, fp));
        L[i] = ColChain{0, v, (int)X.chain.size() - 1};
        st.builds_reuse++;
      } else if (o.reuse == MOR_REUSE_AUTO && !frob_reuse_ok(h->frob, fz(sol[i - 1]), fz(sol[i]))) {
        MOR_TRY(build_factor(h, t, sol[i], sol[i], false, fp, true));
        const int a = (int)X.chain.size() - 1;
        L[i] = ColChain{a, a + 1, -1};
        st.builds_spai++;
      } else {
        MOR_TRY(build_factor(h, t, sol[i - 1], sol[i], true, fp));
        L[i] = ColChain{L[i - 1].a, (int)X.chain.size(), -1};
        st.builds_reuse++;
      }
    }
    for (int i = 0; i < l; ++i) st.chain_len = std::max(st.chain_len, L[i].count());
  }
  return MOR_OK;
}

// One IRKA iteration; btil/ctil == nullptr: SISO (input and output column
// 0), otherwise tangential with r x m / r x q directions (row-major, in and out).
static int irka_step_impl(mor_t h, mor_c64* shifts, mor_c64* btil, mor_c64* ctil, int r, const mor_solve_opts* opts,
                          mor_reduced* rom_out, mor_irka_stats* st_out) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  if (h->order != 1) return mor_fail(h, MOR_EINVAL, "IRKA of second-order systems is not available");
  if (r < 1 || r > MOR_MAX_R || !shifts) return mor_fail(h, MOR_EINVAL, "bad r");
  const bool tang = btil != nullptr;
  if (!tang && (h->m != 1 || h->q != 1))
    return mor_fail(h, MOR_EINVAL, "mor_irka_step is the SISO form (m = q = 1); use mor_irka_step_tangential");
  if (tang && !ctil) return mor_fail(h, MOR_EINVAL, "tangential directions missing");
  const int m = h->m, q = h->q;
  if (h->seg.nseg != 1) return mor_fail(h, MOR_EINVAL, "mor_irka_step needs a single system, not a batch");
  mor_solve_opts o;
  if (opts) o = *opts; else mor_default_opts(&o);
  if ((o.precision != MOR_FP64 && o.precision != MOR_MIXED) ||
      (o.precond_precision != -1 && o.precond_precision != MOR_FP64 && o.precond_precision != MOR_MIXED) ||
      (o.precision == MOR_MIXED && o.precond_precision == MOR_FP64))
    return mor_fail(h, MOR_EINVAL, "bad precision / precond_precision");
  cudaSetDevice(h->dev);
  cudaEvent_t ev[5];
  for (auto& e : ev) cudaEventCreate(&e);
  struct EvGuard { cudaEvent_t* e; ~EvGuard() { for (int i = 0; i < 5; ++i) cudaEventDestroy(e[i]); } } eg{ev};
  mor_irka_stats st;
  std::memset(&st, 0, sizeof st);
  // sort (Re, |Im|, -Im) and check conjugate closure
  for (int i = 0; i < r; ++i)
    if (!std::isfinite(shifts[i].re) || !std::isfinite(shifts[i].im)) return mor_fail(h, MOR_EINVAL, "non-finite shift");
  std::vector<int> perm(r);
  for (int i = 0; i < r; ++i) perm[i] = i;
  std::stable_sort(perm.begin(), perm.end(), [&](int ia, int ib) {
    const mor_c64 a = shifts[ia], b = shifts[ib];
    if (a.re != b.re) return a.re < b.re;
    if (std::fabs(a.im) != std::fabs(b.im)) return std::fabs(a.im) < std::fabs(b.im);
    return -a.im < -b.im;
  });
  std::vector<mor_c64> s(r);
  for (int i = 0; i < r; ++i) s[i] = shifts[perm[i]];
  std::vector<mor_c64> sol, bsol, csol;     // solved shifts and (tangential) their directions
  for (int i = 0; i < r; ++i) {
    if (s[i].im < 0) return mor_fail(h, MOR_EINVAL, "shift set not closed under conjugation");
    if (s[i].im > 0 && (i + 1 >= r || s[i + 1].re != s[i].re || s[i + 1].im != -s[i].im))
      return mor_fail(h, MOR_EINVAL, "shift set not closed under conjugation");
    sol.push_back(s[i]);
    if (tang) {
      for (int j = 0; j < m; ++j) bsol.push_back(btil[(size_t)perm[i] * m + j]);
      for (int j = 0; j < q; ++j) csol.push_back(ctil[(size_t)perm[i] * q + j]);
    }
    if (s[i].im > 0) ++i;
  }
  const int l = (int)sol.size();
  st.nsolve = l;
  cudaEventRecord(ev[0], h->stream);
  // reuse schedule (Algorithm 4) for the primal and, unless symmetric, the transposed operator
  std::vector<ColChain> Ls[2];
  MOR_TRY(schedule_chains(h, sol, o, h->sym ? 1 : 2, Ls, st));
  if (h->sym) Ls[1] = Ls[0];
  cudaEventRecord(ev[1], h->stream);
  // solves: V (primal, rhs B) and W (transposed, rhs C)
  bool cplx = false;
  for (auto& x : sol) cplx |= (x.im != 0.0);
  const int64_t n = h->n;
  for (int t = 0; t < 2; ++t) {
    OpData& X = h->op(t);
    if (o.precond == 0) cplx |= chain_cplx(X, Ls[t]);
  }
  for (const mor_c64& z : bsol) cplx |= (z.im != 0.0);
  for (const mor_c64& z : csol) cplx |= (z.im != 0.0);
  // tangential right-hand sides B b_i (primal) and C c_i (transposed), n x l complex128
  DBuf rhs[2], dcoef;
  if (tang) {
    const int g = (int)std::min<int64_t>((n * l + 255) / 256, h->grid_cap);
    MOR_CK(h, dcoef.alloc(sizeof(mor_c64) * (size_t)l * (m + q)));
    MOR_CK(h, cudaMemcpyAsync(dcoef.p, bsol.data(), sizeof(mor_c64) * l * m, cudaMemcpyHostToDevice, h->stream));
    MOR_CK(h, cudaMemcpyAsync(dcoef.as<mor_c64>() + (size_t)l * m, csol.data(), sizeof(mor_c64) * l * q,
                              cudaMemcpyHostToDevice, h->stream));
    for (int t = 0; t < 2; ++t) {
      MOR_CK(h, rhs[t].alloc(sizeof(mor_c64) * (size_t)n * l));
      combine_kernel<<<g, 256, 0, h->stream>>>(n, t == 0 ? m : q, l, (t == 0 ? h->B : h->C).as<double>(),
                                               dcoef.as<mor_c64>() + (t == 0 ? 0 : (size_t)l * m), rhs[t].as<double>());
      mor_count_launches(1);
    }
    MOR_CK(h, cudaGetLastError());
  }
  DBuf xs[2];                       // solutions, n x l complex128 column-major (device)
  std::vector<mor_solve_stats> ss[2];
  int s2v[2] = {MOR_OK, MOR_OK};
  for (int t = 0; t < 2; ++t) {
    MOR_CK(h, xs[t].alloc(sizeof(mor_c64) * (size_t)n * l));
    ss[t].resize(l);
  }
  SolveLane* lane[2];
  MOR_TRY(mor_lane(h, 0, &lane[0]));
  MOR_TRY(mor_lane(h, 1, &lane[1]));
  if (o.precond == 1) {
    // a fresh SPAI per shift: factor builds and solves alternate on the handle's stream
    for (int t = 0; t < 2; ++t)
      for (int i = 0; i < l; ++i) {
        MOR_TRY(build_factor(h, t, sol[i], sol[i], false, factor_precision(o)));
        st.builds_spai++;
        std::vector<ColChain> L1(1, prefix_chain(1));
        const mor_c64* Ri = tang ? rhs[t].as<mor_c64>() + (size_t)n * i : nullptr;
        int s3 = solve_many(h, *lane[0], &sol[i], 1, t, o, L1, cplx, Ri, true, xs[t].as<mor_c64>() + (size_t)n * i,
                            &ss[t][i]);
        if (s3 != MOR_OK && s3 != MOR_ENOCONV && s3 != MOR_EBREAKDOWN) return s3;
        if (s3 != MOR_OK) s2v[t] = s3;
      }
  } else {
    // the primal (V) and transposed (W) sweeps are independent: V on the
    // handle's stream, W on lane 1's stream from a second host thread, both
    // after the factor builds queued so far
    cudaEvent_t built;
    MOR_CK(h, cudaEventCreateWithFlags(&built, cudaEventDisableTiming));
    struct EvG { cudaEvent_t e; ~EvG() { cudaEventDestroy(e); } } evg{built};
    MOR_CK(h, cudaEventRecord(built, h->stream));
    MOR_CK(h, cudaStreamWaitEvent(lane[1]->stream, built, 0));
    auto sweep = [&](int t) {
      cudaSetDevice(h->dev);
      s2v[t] = solve_many(h, *lane[t], sol.data(), l, t, o, Ls[t], cplx, tang ? rhs[t].as<mor_c64>() : nullptr, true,
                          xs[t].as<mor_c64>(), ss[t].data());
    };
    if (o.concurrent_sweeps) {
      std::thread tw(sweep, 1);
      sweep(0);
      tw.join();
    } else {
      sweep(0);
      sweep(1);
    }
    // solve_many leaves its stream synchronised; order lane 1 before the handle's later work
    cudaEvent_t wdone;
    MOR_CK(h, cudaEventCreateWithFlags(&wdone, cudaEventDisableTiming));
    struct EvG2 { cudaEvent_t e; ~EvG2() { cudaEventDestroy(e); } } evg2{wdone};
    MOR_CK(h, cudaEventRecord(wdone, lane[1]->stream));
    MOR_CK(h, cudaStreamWaitEvent(h->stream, wdone, 0));
    for (int t = 0; t < 2; ++t)
      if (s2v[t] != MOR_OK && s2v[t] != MOR_ENOCONV && s2v[t] != MOR_EBREAKDOWN) return s2v[t];
  }
  int solve_status = MOR_OK;
  for (int t = 0; t < 2; ++t) {
    if (s2v[t] != MOR_OK) solve_status = s2v[t];
    for (int i = 0; i < l; ++i) {
      (t == 0 ? st.iters_V : st.iters_W) += ss[t][i].iters;
      st.max_relres = std::max(st.max_relres, ss[t][i].relres);
      st.fallbacks += ss[t][i].fallback;
    }
  }
  cudaEventRecord(ev[2], h->stream);
  // real bases [Re v, Im v] and CGS2
  DBuf basis;
  MOR_CK(h, basis.alloc(sizeof(double) * (size_t)n * r * 2));
  double* Vb = basis.as<double>();
  double* Wb = Vb + (size_t)n * r;
  const int g = (int)std::min<int64_t>((n + 255) / 256, h->grid_cap);
  for (int t = 0; t < 2; ++t) {
    double* dst = t == 0 ? Vb : Wb;
    int col = 0;
    for (int i = 0; i < l; ++i) {
      const double* src = (const double*)(xs[t].as<mor_c64>() + (size_t)n * i);
      extract_kernel<<<g, 256, 0, h->stream>>>((int)n, 0, src, dst + (size_t)n * col++);
      mor_count_launches(1);
      if (sol[i].im != 0.0) {
        extract_kernel<<<g, 256, 0, h->stream>>>((int)n, 1, src, dst + (size_t)n * col++);
        mor_count_launches(1);
      }
    }
    MOR_CK(h, cudaGetLastError());
  }
  if (!std::isfinite(st.max_relres)) return mor_fail(h, MOR_EBREAKDOWN, "a shifted solve broke down");
  int dep = 0, dep2 = 0;
  MOR_TRY(orth_device(h, Vb, n, r, &dep));
  MOR_TRY(orth_device(h, Wb, n, r, &dep2));
  if (dep || dep2) return mor_fail(h, MOR_ESINGULAR, "projection basis is numerically rank deficient");
  cudaEventRecord(ev[3], h->stream);
  mor_reduced rom;
  MOR_TRY(project_device(h, Vb, Wb, r, &rom));
  std::vector<mor_c64> news(r), lam(r);
  MOR_TRY(poles_device(h, &rom, lam.data(), news.data()));
  std::vector<mor_c64> bnew, cnew;
  if (tang) {
    // the pole behind each new shift (the sort permutes mirror images exactly)
    std::vector<double> lsorted(2 * r);
    std::vector<char> used(r, 0);
    for (int i = 0; i < r; ++i) {
      int e = -1;
      for (int k = 0; k < r && e < 0; ++k)
        if (!used[k] && std::fabs(lam[k].re) == news[i].re && -lam[k].im == news[i].im) e = k;
      if (e < 0) return mor_fail(h, MOR_ESINGULAR, "internal: shift without its pole");
      used[e] = 1;
      lsorted[2 * i] = lam[e].re;
      lsorted[2 * i + 1] = lam[e].im;
    }
    DBuf tw;
    const size_t nout = 2 * (size_t)r * (m + q) + 1;
    const size_t nw = dense_tangent_work(r, m);
    MOR_CK(h, tw.alloc(sizeof(double) * ((size_t)r * (m + q) + 2 * r + nout + nw) + sizeof(int) * (size_t)r * (r + 1)));
    double* dB = tw.as<double>();
    double* dC = dB + (size_t)r * m;
    double* dl = dC + (size_t)r * q;
    double* dout = dl + 2 * r;
    double* dwork = dout + nout;
    int* diwork = (int*)(dwork + nw);
    const double* dAr = h->ws_rom.as<double>();
    const double* dEr = dAr + MOR_MAX_R * MOR_MAX_R;
    MOR_CK(h, cudaMemcpyAsync(dB, rom.Br, sizeof(double) * r * m, cudaMemcpyHostToDevice, h->stream));
    MOR_CK(h, cudaMemcpyAsync(dC, rom.Cr, sizeof(double) * r * q, cudaMemcpyHostToDevice, h->stream));
    MOR_CK(h, cudaMemcpyAsync(dl, lsorted.data(), sizeof(double) * 2 * r, cudaMemcpyHostToDevice, h->stream));
    MOR_CKI(h, dense_launch_tangent(r, m, q, dAr, dEr, dB, dC, dl, dout, dwork, diwork, h->stream));
    std::vector<double> ho(nout);
    MOR_CK(h, cudaMemcpyAsync(ho.data(), dout, sizeof(double) * nout, cudaMemcpyDeviceToHost, h->stream));
    MOR_CK(h, cudaStreamSynchronize(h->stream));
    if (ho[nout - 1] != 0.0) return mor_fail(h, MOR_ESINGULAR, "E_r is singular");
    bnew.resize((size_t)r * m);
    cnew.resize((size_t)r * q);
    for (size_t i = 0; i < (size_t)r * m; ++i) bnew[i] = mor_c64{ho[2 * i], ho[2 * i + 1]};
    for (size_t i = 0; i < (size_t)r * q; ++i) cnew[i] = mor_c64{ho[2 * r * m + 2 * i], ho[2 * r * m + 2 * i + 1]};
    // the -Im member of a conjugate pair takes the conjugate directions
    for (int i = 0; i + 1 < r; ++i)
      if (news[i].im > 0) {
        for (int j = 0; j < m; ++j) bnew[(size_t)(i + 1) * m + j] = mor_c64{bnew[(size_t)i * m + j].re, -bnew[(size_t)i * m + j].im};
        for (int j = 0; j < q; ++j) cnew[(size_t)(i + 1) * q + j] = mor_c64{cnew[(size_t)i * q + j].re, -cnew[(size_t)i * q + j].im};
        ++i;
      }
  }
  cudaEventRecord(ev[4], h->stream);
  cudaEventSynchronize(ev[4]);
  float ms;
  cudaEventElapsedTime(&ms, ev[0], ev[1]); st.ms_precond = ms;
  cudaEventElapsedTime(&ms, ev[1], ev[2]); st.ms_solve = ms;
  cudaEventElapsedTime(&ms, ev[2], ev[3]); st.ms_orth = ms;
  cudaEventElapsedTime(&ms, ev[3], ev[4]); st.ms_reduce = ms;
  double chg = 0.0;
  for (int i = 0; i < r; ++i) {
    const double dr = news[i].re - s[i].re, di = news[i].im - s[i].im;
    const double a = std::hypot(news[i].re, news[i].im);
    chg = std::max(chg, std::hypot(dr, di) / (a > 0 ? a : 1.0));
  }
  st.shift_change = chg;
  h->irka_z += 1;
  st.z = h->irka_z;
  st.status = solve_status;
  for (int i = 0; i < r; ++i) shifts[i] = news[i];
  if (tang) {
    std::copy(bnew.begin(), bnew.end(), btil);
    std::copy(cnew.begin(), cnew.end(), ctil);
  }
  if (rom_out) *rom_out = rom;
  if (st_out) *st_out = st;
  if (solve_status != MOR_OK) return mor_fail(h, solve_status, "a shifted solve did not converge");
  return MOR_OK;
}

int mor_moment_blocks(mor_t h, const mor_c64* sigma, int l, int J, int transpose, const mor_solve_opts* opts,
                      const mor_c64* R, int m, mor_c64* X, mor_solve_stats* stats, unsigned flags) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  if (h->order != 1 || h->seg.nseg != 1)
    return mor_fail(h, MOR_EINVAL, "mor_moment_blocks needs a single first-order system");
  if (!sigma || !X || l < 1 || J < 1 || (transpose != 0 && transpose != 1))
    return mor_fail(h, MOR_EINVAL, "bad arguments");
  if (!R) m = transpose ? h->q : h->m;
  if (m < 1 || m > MOR_MAX_IO) return mor_fail(h, MOR_EINVAL, "1 <= m <= %d right-hand sides", MOR_MAX_IO);
  const int k = l * m;                     // lock-step columns: (shift c / m, right-hand side c % m)
  if (k > 64) return mor_fail(h, MOR_EINVAL, "l m must not exceed 64");
  mor_solve_opts o;
  if (opts) o = *opts; else mor_default_opts(&o);
  if ((o.precision != MOR_FP64 && o.precision != MOR_MIXED) ||
      (o.precond_precision != -1 && o.precond_precision != MOR_FP64 && o.precond_precision != MOR_MIXED) ||
      (o.precision == MOR_MIXED && o.precond_precision == MOR_FP64))
    return mor_fail(h, MOR_EINVAL, "bad precision / precond_precision");
  if (o.precond < 0 || o.precond > 2) return mor_fail(h, MOR_EINVAL, "bad precond");
  for (int i = 0; i < l; ++i)
    if (!std::isfinite(sigma[i].re) || !std::isfinite(sigma[i].im)) return mor_fail(h, MOR_EINVAL, "non-finite shift");
  cudaSetDevice(h->dev);
  const bool dev = flags & MOR_DEVICE_PTRS;
  const int64_t n = h->n;
  cudaStream_t s = h->stream;
  SolveLane* lane0 = nullptr;
  MOR_TRY(mor_lane(h, 0, &lane0));
  // right-hand sides: R (or B / C) repeated for every shift, n x k complex128
  DBuf rhs, lev, Rd;
  MOR_CK(h, rhs.alloc(sizeof(mor_c64) * (size_t)n * k));
  MOR_CK(h, lev.alloc(sizeof(mor_c64) * (size_t)n * k * J));     // level-major: block j at lev + j n k
  if (R) {
    const mor_c64* src = R;
    if (!dev) {
      MOR_CK(h, Rd.alloc(sizeof(mor_c64) * (size_t)n * m));
      MOR_CK(h, cudaMemcpyAsync(Rd.p, R, sizeof(mor_c64) * (size_t)n * m, cudaMemcpyHostToDevice, s));
      src = Rd.as<mor_c64>();
    }
    for (int i = 0; i < l; ++i)
      MOR_CK(h, cudaMemcpyAsync(rhs.as<mor_c64>() + (size_t)n * m * i, src, sizeof(mor_c64) * (size_t)n * m,
                                cudaMemcpyDeviceToDevice, s));
  } else {
    std::vector<mor_c64> unit((size_t)k * m, mor_c64{0.0, 0.0});
    for (int c = 0; c < k; ++c) unit[(size_t)c * m + c % m] = mor_c64{1.0, 0.0};
    DBuf dcoef;
    MOR_CK(h, dcoef.alloc(sizeof(mor_c64) * unit.size()));
    MOR_CK(h, cudaMemcpyAsync(dcoef.p, unit.data(), sizeof(mor_c64) * unit.size(), cudaMemcpyHostToDevice, s));
    const int g = (int)std::min<int64_t>((n * k + 255) / 256, h->grid_cap);
    combine_kernel<<<g, 256, 0, s>>>(n, m, k, (transpose ? h->C : h->B).as<double>(), dcoef.as<mor_c64>(),
                                     rhs.as<double>());
    mor_count_launches(1);
    MOR_CK(h, cudaGetLastError());
    MOR_CK(h, cudaStreamSynchronize(s));
  }
  bool cplx = true;                        // right-hand sides may be complex; complex arithmetic throughout
  std::vector<mor_c64> sig(k);
  for (int c = 0; c < k; ++c) sig[c] = sigma[c / m];
  std::vector<mor_solve_stats> sst((size_t)k * J);
  int worst = MOR_OK;
  auto note = [&](int st2) { if (st2 != MOR_OK) worst = (worst == MOR_OK || st2 == MOR_EBREAKDOWN) ? st2 : worst; };
  // the J levels of the columns cs .. cs + kc - 1 (one shift's m columns, or all of them)
  auto levels = [&](int cs, int kc, const std::vector<ColChain>& L) -> int {
    for (int j = 0; j < J; ++j) {
      mor_c64* Xj = lev.as<mor_c64>() + (size_t)n * k * j + (size_t)n * cs;
      const mor_c64* Rj = rhs.as<mor_c64>() + (size_t)n * cs;
      if (j > 0) {
        MOR_TRY(apply_E(h, transpose, lev.as<mor_c64>() + (size_t)n * k * (j - 1) + (size_t)n * cs,
                        rhs.as<mor_c64>() + (size_t)n * cs, n, kc, s));
      }
      const int st2 = solve_many(h, *lane0, sig.data() + cs, kc, transpose, o, L, cplx, Rj, true, Xj,
                                 sst.data() + (size_t)k * j + cs);
      if (st2 != MOR_OK && st2 != MOR_ENOCONV && st2 != MOR_EBREAKDOWN) return st2;
      note(st2);
    }
    return MOR_OK;
  };
  const int fp = factor_precision(o);
  if (o.precond == 1) {
    // a fresh SPAI per shift (the matrix of a shift is fixed for its J blocks)
    for (int i = 0; i < l; ++i) {
      MOR_TRY(build_factor(h, transpose, sigma[i], sigma[i], false, fp));
      MOR_TRY(levels(i * m, m, std::vector<ColChain>(m, prefix_chain(1))));
    }
  } else {
    std::vector<ColChain> L(k);
    if (o.precond == 0) {
      // Algorithm 4 along the shifts: SPAI at the first, a reuse factor per further shift
      MOR_TRY(build_factor(h, transpose, sigma[0], sigma[0], false, fp));
      for (int i = 1; i < l; ++i) MOR_TRY(build_factor(h, transpose, sigma[i - 1], sigma[i], true, fp));
      for (int c = 0; c < k; ++c) L[c] = prefix_chain(c / m + 1);
    }
    MOR_TRY(levels(0, k, L));
  }
  // out: block (i, j) at columns (i J + j) m .. (i J + j) m + m - 1
  for (int i = 0; i < l; ++i)
    for (int j = 0; j < J; ++j) {
      const mor_c64* src = lev.as<mor_c64>() + (size_t)n * k * j + (size_t)n * m * i;
      mor_c64* dst = X + (size_t)n * m * ((size_t)i * J + j);
      MOR_CK(h, cudaMemcpyAsync(dst, src, sizeof(mor_c64) * (size_t)n * m,
                                dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
      if (stats)
        for (int c = 0; c < m; ++c) stats[((size_t)i * J + j) * m + c] = sst[(size_t)k * j + (size_t)m * i + c];
    }
  MOR_CK(h, cudaStreamSynchronize(s));
  if (worst != MOR_OK) return mor_fail(h, worst, "a moment solve did not converge");
  return MOR_OK;
}

int mor_irka_step(mor_t h, mor_c64* shifts, int r, const mor_solve_opts* opts, mor_reduced* rom_out,
                  mor_irka_stats* st_out) {
  if (!h) return MOR_EINVAL;
  return irka_step_impl(h, shifts, nullptr, nullptr, r, opts, rom_out, st_out);
}

int mor_irka_step_tangential(mor_t h, mor_c64* shifts, mor_c64* btil, mor_c64* ctil, int r,
                             const mor_solve_opts* opts, mor_reduced* rom_out, mor_irka_stats* st_out) {
  if (!h) return MOR_EINVAL;
  if (!btil || !ctil) return mor_fail(h, MOR_EINVAL, "tangential directions required");
  return irka_step_impl(h, shifts, btil, ctil, r, opts, rom_out, st_out);
}

int mor_airga_step(mor_t h, mor_c64* points, int l, const mor_solve_opts* opts, mor_reduced2* rom_out,
                   mor_irka_stats* st_out) {
  if (!h) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  if (h->order != 2) return mor_fail(h, MOR_EINVAL, "mor_airga_step needs a second-order system (mor_set_system_2nd)");
  if (h->seg.nseg != 1) return mor_fail(h, MOR_EINVAL, "mor_airga_step needs a single system, not a batch");
  const int m = h->m, q = h->q;
  mor_solve_opts o;
  if (opts) o = *opts; else mor_default_opts(&o);
  const int J = o.moments;
  if (J < 1) return mor_fail(h, MOR_EINVAL, "moments must be >= 1");
  if (!points || l < 1 || m * J * l > MOR_MAX_R2)
    return mor_fail(h, MOR_EINVAL, "bad points: need 1 <= m moments l <= %d", MOR_MAX_R2);
  if (o.precond == 1) return mor_fail(h, MOR_EINVAL, "mor_airga_step supports precond 0 (reuse) and 2 (none)");
  if ((o.precision != MOR_FP64 && o.precision != MOR_MIXED) ||
      (o.precond_precision != -1 && o.precond_precision != MOR_FP64 && o.precond_precision != MOR_MIXED) ||
      (o.precision == MOR_MIXED && o.precond_precision == MOR_FP64))
    return mor_fail(h, MOR_EINVAL, "bad precision / precond_precision");
  cudaSetDevice(h->dev);
  cudaEvent_t ev[5];
  for (auto& e : ev) cudaEventCreate(&e);
  struct EvGuard { cudaEvent_t* e; ~EvGuard() { for (int i = 0; i < 5; ++i) cudaEventDestroy(e[i]); } } eg{ev};
  mor_irka_stats st;
  std::memset(&st, 0, sizeof st);
  for (int i = 0; i < l; ++i)
    if (!std::isfinite(points[i].re) || !std::isfinite(points[i].im)) return mor_fail(h, MOR_EINVAL, "non-finite point");
  std::vector<mor_c64> s(points, points + l);
  std::stable_sort(s.begin(), s.end(), [](mor_c64 a, mor_c64 b) {
    if (a.re != b.re) return a.re < b.re;
    if (std::fabs(a.im) != std::fabs(b.im)) return std::fabs(a.im) < std::fabs(b.im);
    return -a.im < -b.im;
  });
  std::vector<mor_c64> sol;
  for (int i = 0; i < l; ++i) {
    if (s[i].im < 0 || (s[i].im > 0 && (i + 1 >= l || s[i + 1].re != s[i].re || s[i + 1].im != -s[i].im)))
      return mor_fail(h, MOR_EINVAL, "point set not closed under conjugation");
    sol.push_back(s[i]);
    if (s[i].im > 0) ++i;
  }
  const int ls = (int)sol.size();
  const int r = m * J * l;
  st.nsolve = ls * m * J;
  cudaEventRecord(ev[0], h->stream);
  std::vector<ColChain> Ls[2];
  MOR_TRY(schedule_chains(h, sol, o, 1, Ls, st));
  cudaEventRecord(ev[1], h->stream);
  // block solves: column c = (point c / m, input c % m)
  const int k = ls * m;
  const int64_t n = h->n;
  std::vector<mor_c64> sig(k), unit((size_t)k * m, mor_c64{0.0, 0.0});
  std::vector<ColChain> L(k);
  bool cplx = false;
  for (int c = 0; c < k; ++c) {
    sig[c] = sol[c / m];
    L[c] = Ls[0][c / m];
    unit[(size_t)c * m + c % m] = mor_c64{1.0, 0.0};
    cplx |= (sig[c].im != 0.0);
  }
  if (o.precond == 0) cplx |= chain_cplx(h->op(0), Ls[0]);
  DBuf rhs, dcoef, xs;
  MOR_CK(h, dcoef.alloc(sizeof(mor_c64) * unit.size()));
  MOR_CK(h, cudaMemcpyAsync(dcoef.p, unit.data(), sizeof(mor_c64) * unit.size(), cudaMemcpyHostToDevice, h->stream));
  MOR_CK(h, rhs.alloc(sizeof(mor_c64) * (size_t)n * k));
  // moment blocks X^(0), ..., X^(J-1), each n x k (block j at xs + j n k)
  MOR_CK(h, xs.alloc(sizeof(mor_c64) * (size_t)n * k * J));
  const int g = (int)std::min<int64_t>((n * k + 255) / 256, h->grid_cap);
  combine_kernel<<<g, 256, 0, h->stream>>>(n, m, k, h->B.as<double>(), dcoef.as<mor_c64>(), rhs.as<double>());
  mor_count_launches(1);
  MOR_CK(h, cudaGetLastError());
  std::vector<mor_solve_stats> ss(k);
  SolveLane* lane0 = nullptr;
  MOR_TRY(mor_lane(h, 0, &lane0));
  const int solve_status = solve_many(h, *lane0, sig.data(), k, 0, o, L, cplx, rhs.as<mor_c64>(), true, xs.as<mor_c64>(),
                                      ss.data());
  if (solve_status != MOR_OK && solve_status != MOR_ENOCONV && solve_status != MOR_EBREAKDOWN) return solve_status;
  int solve_worst = solve_status;
  auto add_stats = [&]() {
    for (int c = 0; c < k; ++c) {
      st.iters_V += ss[c].iters;
      st.max_relres = std::max(st.max_relres, ss[c].relres);
      st.fallbacks += ss[c].fallback;
    }
  };
  add_stats();
  // inner moment loop (Algorithm 1 lines 7-12): V_j = X^(j-1) / ||X^(j-1)||_F per
  // point, X^(j) = -A(s)^{-1} M V_j with the same matrix and the same chain
  if (J > 1) {
    DBuf nrm;
    MOR_CK(h, nrm.alloc(sizeof(double) * (size_t)k));
    for (int j = 1; j < J && std::isfinite(st.max_relres); ++j) {
      const mor_c64* Xp = xs.as<mor_c64>() + (size_t)n * k * (j - 1);
      mor_c64* Xj = xs.as<mor_c64>() + (size_t)n * k * j;
      MOR_TRY(column_norms2(h, Xp, n, k, nrm.as<double>(), h->stream));
      moment_rhs_kernel<<<g, 256, 0, h->stream>>>(n, k, m, h->ediag64.as<double>(), (const cdouble*)Xp,
                                                  nrm.as<double>(), -1.0, rhs.as<cdouble>());
      mor_count_launches(1);
      MOR_CK(h, cudaGetLastError());
      const int sj = solve_many(h, *lane0, sig.data(), k, 0, o, L, cplx, rhs.as<mor_c64>(), true, Xj, ss.data());
      if (sj != MOR_OK && sj != MOR_ENOCONV && sj != MOR_EBREAKDOWN) return sj;
      if (sj != MOR_OK) solve_worst = sj;
      add_stats();
    }
  }
  const int solve_status_all = solve_worst;
  // a solve that broke down (non-finite residual) leaves no basis to project on: report it as such
  if (!std::isfinite(st.max_relres)) return mor_fail(h, MOR_EBREAKDOWN, "a block solve broke down");
  cudaEventRecord(ev[2], h->stream);
  // real basis: per solved point and moment block, Re X, then Im X for a complex
  // point; CGS2, Galerkin projection (W = V)
  DBuf basis;
  MOR_CK(h, basis.alloc(sizeof(double) * (size_t)n * r));
  double* Vb = basis.as<double>();
  const int ge = (int)std::min<int64_t>((n + 255) / 256, h->grid_cap);
  int col = 0;
  for (int i = 0; i < ls; ++i)
    for (int jm = 0; jm < J; ++jm)
      for (int part = 0; part < (sol[i].im != 0.0 ? 2 : 1); ++part)
        for (int j = 0; j < m; ++j) {
          const double* src = (const double*)(xs.as<mor_c64>() + (size_t)n * k * jm + (size_t)n * (i * m + j));
          extract_kernel<<<ge, 256, 0, h->stream>>>((int)n, part, src, Vb + (size_t)n * col++);
          mor_count_launches(1);
        }
  MOR_CK(h, cudaGetLastError());
  int dep = 0;
  MOR_TRY(orth_device(h, Vb, n, r, &dep));
  if (dep) return mor_fail(h, MOR_ESINGULAR, "projection basis is numerically rank deficient");
  cudaEventRecord(ev[3], h->stream);
  mor_reduced rom;
  MOR_TRY(project_device(h, Vb, Vb, r, &rom));        // Ar = K_r, Er = M_r, Br = F_r, Cr = C_r
  // reduced QEP and the next points (device, one thread)
  DBuf qw;
  const size_t nout = 2 * (size_t)(2 * r) + 2 * (size_t)l + 1;
  const size_t nw = dense_qep_work(r, l);
  MOR_CK(h, qw.alloc(sizeof(double) * (nout + nw) + sizeof(int) * 2 * (size_t)r));
  double* dout = qw.as<double>();
  double* dwork = dout + nout;
  int* diwork = (int*)(dwork + nw);
  const double* dKr = h->ws_rom.as<double>();
  const double* dMr = dKr + MOR_MAX_R * MOR_MAX_R;
  MOR_CKI(h, dense_launch_qep(r, l, dKr, dMr, h->alpha, h->beta, dout, dwork, diwork, h->stream));
  std::vector<double> ho(nout);
  MOR_CK(h, cudaMemcpyAsync(ho.data(), dout, sizeof(double) * nout, cudaMemcpyDeviceToHost, h->stream));
  cudaEventRecord(ev[4], h->stream);
  MOR_CK(h, cudaStreamSynchronize(h->stream));
  const int qst = (int)ho[nout - 1];
  if (qst != 0)
    return mor_fail(h, MOR_ESINGULAR, qst == 1 ? "M_r is singular" : qst == 2 ? "QR iteration did not converge"
                                                                          : "too few eigenvalues for the points");
  float ms;
  cudaEventElapsedTime(&ms, ev[0], ev[1]); st.ms_precond = ms;
  cudaEventElapsedTime(&ms, ev[1], ev[2]); st.ms_solve = ms;
  cudaEventElapsedTime(&ms, ev[2], ev[3]); st.ms_orth = ms;
  cudaEventElapsedTime(&ms, ev[3], ev[4]); st.ms_reduce = ms;
  double chg = 0.0;
  std::vector<mor_c64> news(l);
  for (int i = 0; i < l; ++i) {
    news[i] = mor_c64{ho[4 * r + 2 * i], ho[4 * r + 2 * i + 1]};
    const double a = std::hypot(news[i].re, news[i].im);
    chg = std::max(chg, std::hypot(news[i].re - s[i].re, news[i].im - s[i].im) / (a > 0 ? a : 1.0));
  }
  st.shift_change = chg;
  h->irka_z += 1;
  st.z = h->irka_z;
  st.status = solve_status_all;
  for (int i = 0; i < l; ++i) points[i] = news[i];
  if (rom_out) {
    rom_out->r = r;
    rom_out->m = m;
    rom_out->q = q;
    rom_out->alpha = h->alpha;
    rom_out->beta = h->beta;
    std::memcpy(rom_out->Mr, rom.Er, sizeof(double) * r * r);
    std::memcpy(rom_out->Kr, rom.Ar, sizeof(double) * r * r);
    std::memcpy(rom_out->Fr, rom.Br, sizeof(double) * r * m);
    std::memcpy(rom_out->Cr, rom.Cr, sizeof(double) * r * q);
  }
  if (st_out) *st_out = st;
  if (solve_status_all != MOR_OK) return mor_fail(h, solve_status_all, "a shifted solve did not converge");
  return MOR_OK;
}

int mor_eval_tf2(mor_t h, const mor_reduced2* rom, const double* omega, int nw, mor_c64* H, unsigned flags) {
  if (!h || !rom || !omega || !H) return MOR_EINVAL;
  if (rom->r < 1 || rom->r > MOR_MAX_R2 || rom->m < 1 || rom->m > MOR_MAX_IO || rom->q < 1 || rom->q > MOR_MAX_IO ||
      nw < 1)
    return mor_fail(h, MOR_EINVAL, "bad reduced system or nw");
  cudaSetDevice(h->dev);
  const int r = rom->r, m = rom->m, q = rom->q;
  DBuf d;
  const size_t nrom = (size_t)2 * r * r + (size_t)r * m + (size_t)r * q;
  MOR_CK(h, d.alloc(sizeof(double) * (nrom + nw) + sizeof(mor_c64) * (size_t)nw * m * q));
  double* dK = d.as<double>();
  double* dM = dK + r * r;
  double* dF = dM + r * r;
  double* dC = dF + r * m;
  double* dw = dC + r * q;
  mor_c64* dH = (mor_c64*)(dw + nw);
  MOR_CK(h, cudaMemcpyAsync(dK, rom->Kr, sizeof(double) * r * r, cudaMemcpyHostToDevice, h->stream));
  MOR_CK(h, cudaMemcpyAsync(dM, rom->Mr, sizeof(double) * r * r, cudaMemcpyHostToDevice, h->stream));
  MOR_CK(h, cudaMemcpyAsync(dF, rom->Fr, sizeof(double) * r * m, cudaMemcpyHostToDevice, h->stream));
  MOR_CK(h, cudaMemcpyAsync(dC, rom->Cr, sizeof(double) * r * q, cudaMemcpyHostToDevice, h->stream));
  const bool dev = flags & MOR_DEVICE_PTRS;
  const double* w = omega;
  if (!dev) {
    MOR_CK(h, cudaMemcpyAsync(dw, omega, sizeof(double) * nw, cudaMemcpyHostToDevice, h->stream));
    w = dw;
  }
  mor_c64* out = dev ? H : dH;
  MOR_CKI(h, dense_launch_tf(r, m, q, dK, dM, dF, dC, w, nw, (double*)out, h->stream, 2, rom->alpha, rom->beta));
  if (!dev) MOR_CK(h, cudaMemcpyAsync(H, dH, sizeof(mor_c64) * (size_t)nw * m * q, cudaMemcpyDeviceToHost, h->stream));
  MOR_CK(h, cudaStreamSynchronize(h->stream));
  return MOR_OK;
}

int mor_time_kernel(mor_t h, int which, const mor_c64* sigma, int k, int precision, int reps, double* ms) {
  if (!h || !sigma || !ms) return MOR_EINVAL;
  if (!h->has_sys) return mor_fail(h, MOR_ESTATE, "no system set");
  if (k < 1 || k > MOR_KMAX || reps < 1 || (which != 0 && which != 1)) return mor_fail(h, MOR_EINVAL, "bad arguments");
  OpData& op = h->P;
  if (which == 1 && op.chain.empty()) return mor_fail(h, MOR_ESTATE, "no preconditioner built");
  cudaSetDevice(h->dev);
  bool cplx = false;
  for (int c = 0; c < k; ++c) cplx |= !is_real_shift(sigma[c]);
  // the factor timed: the chain's last one of the vectors' kind (complex values
  // for complex shifts, as the solve applies them), else the last one
  int fidx = (int)op.chain.size() - 1;
  if (which == 1) {
    for (int f = fidx; f >= 0; --f)
      if (st_is_cplx(op.chain[f].st) == cplx) { fidx = f; break; }
    cplx |= st_is_cplx(op.chain[fidx].st);
    precision = op.chain_prec;
  }
  const int st = st_of(precision, cplx);
  const int ld = row_stride(st, k);
  const int64_t n = op.n;
  DBuf x, y, w;
  MOR_CK(h, x.alloc(st_size(st) * (size_t)n * ld));
  MOR_CK(h, y.alloc(st_size(st) * (size_t)n * ld));
  MOR_CK(h, w.alloc(st_size(st) * (size_t)n * ld));
  MOR_CK(h, cudaMemsetAsync(x.p, 0, st_size(st) * (size_t)n * ld, h->stream));
  MOR_CK(h, cudaMemsetAsync(w.p, 0, st_size(st) * (size_t)n * ld, h->stream));
  Small sm;
  MOR_TRY(get_small(h, h->ws_small, sm));
  MOR_CK(h, h->ws_part.alloc(sizeof(double) * 2 * 2 * MOR_LDMAX * part_blocks(h)));
  std::vector<int> ones(MOR_KMAX, 1);
  MOR_CK(h, cudaMemcpyAsync(sm.masks, ones.data(), sizeof(int) * MOR_KMAX, cudaMemcpyHostToDevice, h->stream));
  Coef cf[MOR_LDMAX];
  for (int c = 0; c < ld; ++c) cf[c] = mor_coef(h, sigma[c < k ? c : 0]);
  PatView pv = op.view();
  OpVals ov = op_vals(h, op, st_is_f32(st));
  MOR_CK(h, h->ws_sums.alloc(sizeof(cdouble) * 2 * (size_t)h->seg.nseg * MOR_LDMAX));
  RedArgs ra{RED_DOT_W, w.p, h->ws_part.p, nullptr, FIN_NONE, nullptr, h->ws_sums.p, nullptr};
  auto launch = [&]() -> int {
    if (which == 0) return launch_op_spmv(st, h->seg, pv, ov, cf, ld, x.p, y.p, nullptr, &ra, h->stream, k);
    return launch_factor_spmv(st, op.chain[fidx].st, h->seg, pv, op.chain[fidx].vals->p, sm.masks, ld,
                              x.p, y.p, nullptr, nullptr, h->stream, k);
  };
  // L2 is flushed before every timed launch by reading a buffer of twice its
  // size (clean lines: the launch pays no write-back for them), so that no
  // launch finds the previous one's matrix or vectors in L2.  The launches
  // and flushes run back to back between one pair of events, and the time of
  // the flushes alone (timed the same way) is subtracted: the per-launch
  // figure is the kernel's duration plus one inter-kernel gap, as in a
  // graph replay, without the event-recording overhead of a single launch.
  int l2 = 0;
  MOR_CK(h, cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->dev));
  DBuf flush;
  const size_t fbytes = std::max<size_t>((size_t)2 * (size_t)l2, (size_t)64 << 20) / 16 * 16;
  MOR_CK(h, flush.alloc(fbytes + 256));
  MOR_CK(h, cudaMemsetAsync(flush.p, 0, fbytes + 256, h->stream));
  unsigned* sink = (unsigned*)((char*)flush.p + fbytes);
  const int fgrid = h->sm_count * 8;
  auto do_flush = [&]() -> int {
    flush_read_kernel<<<fgrid, 256, 0, h->stream>>>((const uint4*)flush.p, (int64_t)(fbytes / 16), sink);
    return (int)cudaGetLastError();
  };
  for (int i = 0; i < 3; ++i) { MOR_CKI(h, do_flush()); MOR_CKI(h, launch()); }
  cudaEvent_t e[4];
  for (auto& x : e) MOR_CK(h, cudaEventCreate(&x));
  struct EvQ { cudaEvent_t* e; ~EvQ() { for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]); } } evq{e};
  MOR_CK(h, cudaEventRecord(e[0], h->stream));
  for (int i = 0; i < reps; ++i) { MOR_CKI(h, do_flush()); MOR_CKI(h, launch()); }
  MOR_CK(h, cudaEventRecord(e[1], h->stream));
  MOR_CK(h, cudaEventRecord(e[2], h->stream));
  for (int i = 0; i < reps; ++i) MOR_CKI(h, do_flush());
  MOR_CK(h, cudaEventRecord(e[3], h->stream));
  MOR_CK(h, cudaEventSynchronize(e[3]));
  float ta = 0.f, tb = 0.f;
  MOR_CK(h, cudaEventElapsedTime(&ta, e[0], e[1]));
  MOR_CK(h, cudaEventElapsedTime(&tb, e[2], e[3]));
  *ms = std::max(0.0, (double)(ta - tb)) / reps;
  return MOR_OK;
}

int mor_eval_tf(mor_t h, const mor_reduced* rom, const double* omega, int nw, mor_c64* H, unsigned flags) {
  if (!h || !rom || !omega || !H) return MOR_EINVAL;
  if (rom->r < 1 || rom->r > MOR_MAX_R || rom->m < 1 || rom->m > MOR_MAX_IO || rom->q < 1 || rom->q > MOR_MAX_IO || nw < 1)
    return mor_fail(h, MOR_EINVAL, "bad reduced system or nw");
  cudaSetDevice(h->dev);
  const int r = rom->r, m = rom->m, q = rom->q;
  DBuf d;
  const size_t nrom = (size_t)2 * r * r + (size_t)r * m + (size_t)r * q;
  MOR_CK(h, d.alloc(sizeof(double) * (nrom + nw) + sizeof(mor_c64) * (size_t)nw * m * q));
  double* dA = d.as<double>();
  double* dE = dA + r * r;
  double* dB = dE + r * r;
  double* dC = dB + r * m;
  double* dw = dC + r * q;
  mor_c64* dH = (mor_c64*)(dw + nw);
  MOR_CK(h, cudaMemcpyAsync(dA, rom->Ar, sizeof(double) * r * r, cudaMemcpyHostToDevice, h->stream));
  MOR_CK(h, cudaMemcpyAsync(dE, rom->Er, sizeof(double) * r * r, cudaMemcpyHostToDevice, h->stream));
  MOR_CK(h, cudaMemcpyAsync(dB, rom->Br, sizeof(double) * r * m, cudaMemcpyHostToDevice, h->stream));
  MOR_CK(h, cudaMemcpyAsync(dC, rom->Cr, sizeof(double) * r * q, cudaMemcpyHostToDevice, h->stream));
  const bool dev = flags & MOR_DEVICE_PTRS;
  const double* w = omega;
  if (!dev) {
    MOR_CK(h, cudaMemcpyAsync(dw, omega, sizeof(double) * nw, cudaMemcpyHostToDevice, h->stream));
    w = dw;
  }
  mor_c64* out = dev ? H : dH;
  MOR_CKI(h, dense_launch_tf(r, m, q, dA, dE, dB, dC, w, nw, (double*)out, h->stream));
  if (!dev) MOR_CK(h, cudaMemcpyAsync(H, dH, sizeof(mor_c64) * (size_t)nw * m * q, cudaMemcpyDeviceToHost, h->stream));
  MOR_CK(h, cudaStreamSynchronize(h->stream));
  return MOR_OK;
}

}  // extern "C"
