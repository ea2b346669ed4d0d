// engine.cu -- host side of the RBiCG library: handles, the solve loop of Algorithm 2, the
// Section 4 recycle-space refresh schedule, FP32 inner solves under FP64 refinement, and the
// C ABI declared in include/rbicg.h.
#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/rbicg.h"
#include "internal.cuh"

namespace rb {

static thread_local std::string g_last_error;

void set_global_error(const char* msg) { g_last_error = msg; }

static bool debug_on() {
  static int v = -1;
  if (v < 0) { const char* e = getenv("RBICG_DEBUG"); v = (e && *e && *e != '0') ? 1 : 0; }
  return v == 1;
}

struct Err {
  rbicg_status st;
  std::string msg;
};

#define RB_CUDA(call)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      throw Err{e_ == cudaErrorMemoryAllocation ? RBICG_ERR_OOM : RBICG_ERR_CUDA,     \
                std::string(#call) + ": " + cudaGetErrorString(e_)};                  \
  } while (0)

template <class P>
static P* dmalloc(size_t count) {
  void* p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&p, count * sizeof(P));
  if (e != cudaSuccess)
    throw Err{e == cudaErrorMemoryAllocation ? RBICG_ERR_OOM : RBICG_ERR_CUDA,
              std::string("cudaMalloc: ") + cudaGetErrorString(e)};
  return static_cast<P*>(p);
}

int64_t dense_work_elems();
static int64_t dense_work_elems_fwd() { return dense_work_elems(); }

static int kt_for(int k) {
  if (k <= 0) return 0;
  if (k <= 8) return 8;
  if (k <= 16) return 16;
  if (k <= 24) return 24;
  return 32;
}

static int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// Host copy of the leading DevState fields (same layout), read with one copy per sync.
struct HostView {
  int iter, done, kc, restart, kk, pcyc, eig_status, max_itn;
  double rnorm, rtnorm, bnorm, btnorm, true_rnorm, true_rtnorm;
};
static_assert(offsetof(HostView, true_rtnorm) == offsetof(DevState, true_rtnorm), "HostView layout");

struct OpKey {
  const void* rp = nullptr; const void* ci = nullptr; const void* va = nullptr;
  int64_t n = 0, nnz = 0;
  int has_shift = 0, val_complex = 0;
  double sr = 0, si = 0;
  bool operator==(const OpKey& o) const {
    return rp == o.rp && ci == o.ci && va == o.va && n == o.n && nnz == o.nnz && has_shift == o.has_shift &&
           val_complex == o.val_complex && sr == o.sr && si == o.si;
  }
};

// ------------------------------------------------------------------------------------
// Per-step device timing with CUDA events on the solver's stream (measurement hooks).
// Slots: 0 phase 1 (dual SpMV + projections), 1 phase 2 (q, (pt, q)), 2 phase 3 (x, r
// updates and dots), 3 refresh Gram, 4 refresh dense eigen solve, 5 refresh basis update
// (combine, SpMM, small Gram, SVD, rotation), 6 system start, 7 init / finish / A^H.
// ------------------------------------------------------------------------------------
struct Profiler {
  bool on = false;
  bool serial = false;   // refreshes run alone: no overlap with the iteration stream
  double ms[RBICG_NPROF] = {};
  int64_t cnt[RBICG_NPROF] = {};
  int64_t pcols = 0;   // projection columns summed over the slot-0 launches
  int64_t gpairs = 0;  // column pairs (mx x my) summed over the slot-3 (pencil Gram) launches
  std::vector<cudaEvent_t> pool;
  struct Pend { int slot, nl; cudaEvent_t a, b; };
  std::vector<Pend> pending;
  cudaEvent_t get() {
    if (pool.empty()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      return e;
    }
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  int begin(int slot, cudaStream_t s) {
    if (!on) return -1;
    Pend p{slot, 0, get(), get()};
    cudaEventRecord(p.a, s);
    pending.push_back(p);
    return (int)pending.size() - 1;
  }
  void end(int idx, int nl, cudaStream_t s) {
    if (idx < 0) return;
    pending[idx].nl = nl;
    cudaEventRecord(pending[idx].b, s);
  }
  void harvest() {   // call after a stream sync
    for (auto& p : pending) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) { ms[p.slot] += t; cnt[p.slot] += p.nl; }
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  void reset() {
    pcols = 0;
    gpairs = 0;
    for (int i = 0; i < RBICG_NPROF; ++i) { ms[i] = 0; cnt[i] = 0; }
  }
  ~Profiler() {
    for (auto& p : pending) { pool.push_back(p.a); pool.push_back(p.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// ------------------------------------------------------------------------------------
// Solver<V, T>: one precision of the iteration (V operator value type, T vector type)
// ------------------------------------------------------------------------------------
struct SolverBase {
  virtual ~SolverBase() {}
};

template <class V, class T>
struct Solver : SolverBase {
  typedef typename traits<T>::acc A;
  rbicg_params prm;
  int64_t n;
  int ldk, R, grid, gram_grid;
  cudaStream_t s;
  // The cycle refresh (Sections 4.1-4.3) reads only the finished cycle's ring columns and
  // scalar histories and writes only the next system's U_j, C_j: it runs on its own stream,
  // concurrently with the next cycle's iterations.  The ring holds two cycles for that.
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_cycle = nullptr, ev_ref = nullptr;
  cudaStream_t gs = nullptr;                        // graph capture / launch stream
  cudaEvent_t ev_g0 = nullptr, ev_g1 = nullptr;
  bool ref_pending = false;
  // solve() launches a cycle's refresh after the next cycle's iterations (one graph launch)
  // instead of before them (about twenty launches): ev_cycle marks the cycle's end at once, the
  // refresh kernels follow the graph launch
  bool defer_refresh = false, ref_deferred = false;
  int def_j = 0, def_kp = 0;
  void* gpart = nullptr;        // Gram partials of the refresh (part belongs to the iteration)
  int64_t* launches;
  // operator (values in V; A^H values owned here)
  OpArgs<V> op{};
  V* tva = nullptr;
  int* trp_own = nullptr;
  int* tci_own = nullptr;
  V* va_own = nullptr;          // converted copy of A's values (inner FP32 solver)
  int64_t nnz_cap = 0;
  int op_ready = 0;
  // vectors
  T *ring = nullptr, *ringt = nullptr, *p[2] = {}, *pt[2] = {}, *z = nullptr, *zt = nullptr;
  // recycle space of the next system (U, Ut with kU columns) and of the current system
  T *U = nullptr, *Ut = nullptr, *C = nullptr, *Ct = nullptr;
  T *Uc[2] = {}, *Utc[2] = {}, *Cc[2] = {}, *Ctc[2] = {};
  int kU = 0;         // valid columns in U for the next system start
  int kc = 0;         // columns of C in the current system
  int last_plain_iters = 0;   // iterations of the last solve without a recycle space (guard)
  double diverge = 0.0;       // > 0: stop once ||r|| > diverge ||b|| (inner FP32 solves)
  int stall_window = 0;       // > 0: stop once ||r|| has not reached a new minimum for this
                              // many iterations (inner FP32 solves)
  T *x_save = nullptr, *xt_save = nullptr;   // initial guesses kept while the guard is armed
  // inner FP32 solves (stall_window > 0): the iterate with the smallest residual seen at a cycle
  // end, with its zeta_c, is kept and returned when the solve ends without converging (a BiCG
  // iterate after a residual spike can be far worse than one a cycle earlier)
  T *x_best = nullptr, *xt_best = nullptr;
  zd* zc_best = nullptr;
  double best_metric = 0.0;
  bool have_best = false;
  int pending_start = 0;
  // device scratch
  DevState* st = nullptr;
  void* part = nullptr;
  T *Cq = nullptr, *Ctq = nullptr;   // compact copies of C, Ct (row stride VecArgs::ldc)
  A* G = nullptr;
  zd* work = nullptr;
  zd *Wphi = nullptr, *Wphit = nullptr, *Nmat = nullptr, *Mmat = nullptr;
  double* sig = nullptr;
  zd* s2in = nullptr;           // input of the Section 4.3 SVD (Ct^H C and column norms)
  int* iflag = nullptr;
  HostView* hv = nullptr;       // pinned

  Profiler* prof;

  Solver(const rbicg_params& p_, int64_t n_, cudaStream_t s_, int64_t* launches_, Profiler* prof_)
      : prm(p_), n(n_), s(s_), launches(launches_), prof(prof_) {
    ldk = std::max(1, ((prm.k + 3) / 4) * 4);
    // ring of residuals r_m at slot m % R: a refresh after iteration j s reads r_{(j-1)s-1} ..
    // r_{js} while cycle j+1 writes r_{js+1} .. r_{(j+1)s}
    R = prm.recycle ? 2 * (prm.s + 2) : prm.s + 2;
    int lo_prio = 0, hi_prio = 0;
    RB_CUDA(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
    RB_CUDA(cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, hi_prio));
    RB_CUDA(cudaEventCreateWithFlags(&ev_cycle, cudaEventDisableTiming));
    RB_CUDA(cudaEventCreateWithFlags(&ev_ref, cudaEventDisableTiming));
    RB_CUDA(cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
    RB_CUDA(cudaEventCreateWithFlags(&ev_g0, cudaEventDisableTiming));
    RB_CUDA(cudaEventCreateWithFlags(&ev_g1, cudaEventDisableTiming));
    const int sms = num_sms();
    // default: 3 blocks per SM (one wave of the phase-1 kernel, which then fills the register
    // file) without recycling; 2 per SM with it, so that the cycle refresh, which runs concurrently
    // on its own stream and is bound by the same FP64 units, finds room on every SM (512^2
    // benchmark sequence: 189 us per iteration in all against 228 us with 3 per SM and 202 us with
    // 1).  Every block walks an equal share of whole 32-row chunks, so each SM gets the same rows.
    const int per_sm = prm.recycle ? 2 : 3;
    grid = prm.grid_blocks > 0
               ? (int)std::min<int64_t>(prm.grid_blocks, std::max<int64_t>(1, (n + NTHREADS - 1) / NTHREADS))
               : (int)std::max<int64_t>(1, std::min<int64_t>((n + NTHREADS - 1) / NTHREADS, (int64_t)sms * per_sm));
    // blocks of the refresh's Gram products (rbicg_params.setup_blocks; default 8 x SMs: a Gram
    // block's work depends on how many of its column tiles' warps are active, and several waves
    // of short blocks let the scheduler even that out across the SMs -- 512^2 benchmark sequence,
    // the Gram run alone: 0.73 TFLOP/s at 2 x SMs, 0.82 at 4 x, 0.92 at 8 x, 0.93 at 12 x)
    gram_grid = prm.setup_blocks > 0 ? prm.setup_blocks : 8 * sms;
    const int64_t ldv = ((n + 31) / 32) * 32;   // padded vector stride (256-byte aligned slots)
    ring = dmalloc<T>(ldv * R);
    ringt = dmalloc<T>(ldv * R);
    for (int i = 0; i < 2; ++i) { p[i] = dmalloc<T>(n); pt[i] = dmalloc<T>(n); }
    z = dmalloc<T>(n);
    zt = dmalloc<T>(n);
    const size_t bsz = (size_t)n * ldk;
    U = dmalloc<T>(bsz); Ut = dmalloc<T>(bsz); C = dmalloc<T>(bsz); Ct = dmalloc<T>(bsz);
    for (int i = 0; i < 2; ++i) {
      Uc[i] = dmalloc<T>(bsz); Utc[i] = dmalloc<T>(bsz); Cc[i] = dmalloc<T>(bsz); Ctc[i] = dmalloc<T>(bsz);
    }
    RB_CUDA(cudaMemsetAsync(U, 0, bsz * sizeof(T), s));
    RB_CUDA(cudaMemsetAsync(Ut, 0, bsz * sizeof(T), s));
    ring_ld = ldv;
    st = dmalloc<DevState>(1);
    RB_CUDA(cudaMemsetAsync(st, 0, sizeof(DevState), s));
    // Gram partials: one 32 x 32 tile per (row chunk, tile) with at most max(grid, tiles) of them
    // (36 tiles at 176 x 176 columns), then the SVD input's 64 column-norm partials per block
    const size_t gelems = (size_t)std::max(gram_grid, 64) * (32 * 32 + 64);
    const size_t part_elems = std::max<size_t>(part_elems_for(grid), gelems);
    part = dmalloc<A>(part_elems);
    gpart = dmalloc<A>(gelems);
    G = dmalloc<A>((size_t)GRAM_MAXCOLS * GRAM_MAXCOLS);
    work = dmalloc<zd>(dense_work_elems_fwd());
    Wphi = dmalloc<zd>(MMAX * KMAX); Wphit = dmalloc<zd>(MMAX * KMAX);
    Nmat = dmalloc<zd>(KMAX * KMAX); Mmat = dmalloc<zd>(KMAX * KMAX);
    sig = dmalloc<double>(KMAX);
    s2in = dmalloc<zd>((size_t)4 * KMAX * KMAX);
    iflag = dmalloc<int>(4);
    RB_CUDA(cudaMallocHost(&hv, sizeof(HostView)));
  }
  int64_t ring_ld = 0;

  ~Solver() override {
    cudaStreamSynchronize(s);
    if (s2) cudaStreamSynchronize(s2);
    if (gs) cudaStreamSynchronize(gs);
    drop_graph();
    T* bufs[] = {ring, ringt, p[0], p[1], pt[0], pt[1], z, zt, U, Ut, C, Ct,
                 Uc[0], Uc[1], Utc[0], Utc[1], Cc[0], Cc[1], Ctc[0], Ctc[1]};
    for (T* b : bufs) cudaFree(b);
    cudaFree(Cq); cudaFree(Ctq);
    cudaFree(st); cudaFree(part); cudaFree(gpart); cudaFree(G); cudaFree(work); cudaFree(Wphi); cudaFree(Wphit);
    cudaFree(Nmat); cudaFree(Mmat); cudaFree(sig); cudaFree(s2in); cudaFree(iflag);
    if (x_save) cudaFree(x_save);
    if (xt_save) cudaFree(xt_save);
    if (x_best) cudaFree(x_best);
    if (xt_best) cudaFree(xt_best);
    if (zc_best) cudaFree(zc_best);
    free_op();
    if (hv) cudaFreeHost(hv);
    if (ev_cycle) cudaEventDestroy(ev_cycle);
    if (ev_ref) cudaEventDestroy(ev_ref);
    if (s2) cudaStreamDestroy(s2);
    if (ev_g0) cudaEventDestroy(ev_g0);
    if (ev_g1) cudaEventDestroy(ev_g1);
    if (gs) cudaStreamDestroy(gs);
  }

  void free_op() {
    if (tva) cudaFree(tva);
    if (trp_own) cudaFree(trp_own);
    if (tci_own) cudaFree(tci_own);
    if (va_own) cudaFree(va_own);
    tva = nullptr; trp_own = nullptr; tci_own = nullptr; va_own = nullptr;
    op_ready = 0;
  }

  void count(int k) { *launches += k; }

  // Make the iteration stream wait for the refresh in flight (if any).
  void join_refresh() {
    if (!ref_pending) return;
    RB_CUDA(cudaStreamWaitEvent(s, ev_ref, 0));
    ref_pending = false;
  }

  // Fetch the host view of the device state (one sync, after the refresh in flight).
  void fetch() {
    fetch_async();
    RB_CUDA(cudaStreamSynchronize(s));
    prof->harvest();
  }
  // the copy of fetch() without the sync (a batch syncs once for all its requests)
  void fetch_async() {
    RB_CUDA(cudaGetLastError());   // a failed launch must not leave the host loop waiting
    join_refresh();
    RB_CUDA(cudaMemcpyAsync(hv, st, sizeof(HostView), cudaMemcpyDeviceToHost, s));
  }

  template <class F>
  void set_field(F DevState::*field, const F& value) {
    RB_CUDA(cudaMemcpyAsync(&(st->*field), &value, sizeof(F), cudaMemcpyHostToDevice, s));
  }

  // ------------------------------------------------------------------ operator
  // va_src: values in V (already converted for an inner solver)
  void set_operator(const rbicg_csr& A, const V* va_src) {
    free_op();
    op.n = (int)A.n;
    op.rp = A.row_ptr;
    op.ci = A.col_idx;
    op.va = va_src;
    op.has_shift = A.has_shift;
    op.sh_re = A.shift_re;
    op.sh_im = A.shift_im;
    tva = dmalloc<V>(std::max<int64_t>(1, A.nnz));
    int* trp = nullptr;
    int* tci = nullptr;
    int shared = 0;
    const int pi = prof->begin(7, s);
    int e = build_adjoint<V>(op.n, op.rp, op.ci, op.va, &trp, &tci, &tva, &shared, iflag, s);
    prof->end(pi, 1, s);
    if (e) throw Err{RBICG_ERR_CUDA, std::string("adjoint: ") + cudaGetErrorString((cudaError_t)e)};
    count(shared ? 1 : 5);
    op.trp = trp;
    op.tci = tci;
    op.tva = tva;
    op.shared = shared;
    if (!shared) { trp_own = trp; tci_own = tci; }
    // bandwidth for phase 1's staging of p (-1 when it cannot be read: no staging)
    int bw = -1;
    if (csr_bandwidth(op.n, op.rp, op.ci, iflag, s, &bw) != 0) bw = -1;
    op.bw = bw;
    op.stage_rows = 0;
    prepare_phase1<V, T>();
    op_ready = 1;
    pending_start = 1;
  }

  VecArgs<T> vec(const T* b, const T* bt, T* x, T* xt, const T* Cp, const T* Ctp, const T* Up, const T* Utp) {
    VecArgs<T> v{};
    v.n = n;
    v.ring = ring; v.ringt = ringt; v.ld = ring_ld; v.R = R;
    v.p[0] = p[0]; v.p[1] = p[1]; v.pt[0] = pt[0]; v.pt[1] = pt[1];
    v.z = z; v.zt = zt; v.x = x; v.xt = xt; v.b = b; v.bt = bt;
    v.C = Cp; v.Ct = Ctp; v.U = Up; v.Ut = Utp; v.ldk = ldk; v.ldc = ldk;
    return v;
  }

  ColList<T> block_cols(const T* B, int k) {
    ColList<T> l{};
    append_block(l, B, k);
    return l;
  }
  void append_block(ColList<T>& l, const T* B, int k) {
    for (int c = 0; c < k; ++c) { l.c[l.m].p = B + c; l.c[l.m].ld = ldk; ++l.m; }
  }
  void append_ring(ColList<T>& l, const T* rg, int m0, int m1) {   // residuals r_m0 .. r_m1
    for (int m = m0; m <= m1; ++m) { l.c[l.m].p = rg + (int64_t)(m % R) * ring_ld; l.c[l.m].ld = 1; ++l.m; }
  }

  // ------------------------------------------------------------------ Section 4.3, system start
  // C = Op U, Ct = Op^H Ut, SVD of Ct^H C after column scaling, truncation, rotation.
  void system_start() {
    pending_start = 0;
    kc = 0;
    set_field(&DevState::kc, 0);
    if (!prm.recycle || kU <= 0) return;
    int* kdev = iflag + 1;
    RB_CUDA(cudaMemcpyAsync(kdev, &kU, sizeof(int), cudaMemcpyHostToDevice, s));
    const int pi = prof->begin(6, s);
    launch_spmm<V, T>(op, 0, U, ldk, kdev, KMAX, C, 0, s);
    launch_spmm<V, T>(op, 1, Ut, ldk, kdev, KMAX, Ct, 0, s);
    launch_svd_input<T>(C, Ct, ldk, prm.k, prm.k, n, part, gram_grid, G, s2in, s);
    launch_dense_svd(!traits<T>::cx, kdev, prm.k, s2in, nullptr, nullptr, prm.svd_tol, Nmat, Mmat, sig, &st->kc,
                     st->Dc, iflag + 2, s);
    // U <- U N_p, Ut <- Ut M_p, then C = A U, Ct = A^H Ut for the rotated bases (as the paper
    // defines them; an SpMM of the kept columns costs less than rotating C and Ct as well)
    launch_rotate<T>(U, ldk, Nmat, kdev, &st->kc, prm.k, n, 0, s);
    launch_rotate<T>(Ut, ldk, Mmat, kdev, &st->kc, prm.k, n, 0, s);
    launch_spmm<V, T>(op, 0, U, ldk, &st->kc, KMAX, C, 0, s);
    launch_spmm<V, T>(op, 1, Ut, ldk, &st->kc, KMAX, Ct, 0, s);
    prof->end(pi, 11, s);
    count(11);
    fetch();
    kc = hv->kc;
  }

  // ------------------------------------------------------------------ Section 4.1-4.3 refresh
  // Runs after iteration j*s.  kp = columns of U_{j-1}.  Returns nothing; results are read
  // at the next sync (st->pcyc, st->eig_status).
  void refresh(int j, int kp, bool cycle_end_recorded = false) {
    if (!cycle_end_recorded) RB_CUDA(cudaEventRecord(ev_cycle, s));
    // serialised profiling: the refresh also waits for everything queued on the iteration
    // stream so far (a next cycle launched before it), and that stream waits for the refresh
    if (prof->on && prof->serial) RB_CUDA(cudaEventRecord(ev_cycle, s));
    RB_CUDA(cudaStreamWaitEvent(s2, ev_cycle, 0));
    cudaStream_t q = s2;
    const bool first = kc == 0;
    RefreshInfo f{};
    f.case_id = first ? (j == 1 ? 0 : 1) : (j == 1 ? 2 : 3);
    f.j = j; f.s = prm.s; f.k = prm.k; f.kc = kc; f.kp = kp; f.real_path = !traits<T>::cx; f.R = R;
    const int jp = (j - 1) & 1, jc = j & 1;
    const int ss = prm.s;
    ColList<T> X{}, Y{}, Ph{}, Pht{};
    if (f.case_id == 0) {
      append_ring(Ph, ring, 0, ss - 1);
      append_ring(Pht, ringt, 0, ss - 1);
    } else {
      if (f.case_id == 3) { append_block(Y, C, kc); append_block(X, Ct, kc); }
      if (f.case_id == 2) { append_block(Y, C, kc); append_block(X, Ct, kc); }
      if (f.case_id == 1 || f.case_id == 3) { append_block(Y, Cc[jp], kp); append_block(X, Ctc[jp], kp); }
      const int m0 = f.case_id == 2 ? 0 : (j - 1) * ss - 1, m1 = j * ss;
      append_ring(Y, ring, m0, m1);
      append_ring(X, ringt, m0, m1);
      const T* Ub = f.case_id == 2 ? U : Uc[jp];
      const T* Utb = f.case_id == 2 ? Ut : Utc[jp];
      const int kb = f.case_id == 2 ? kc : kp;
      append_block(Y, Ub, kb);
      f.mx = X.m; f.my = Y.m;
      append_block(Ph, Ub, kb);
      append_block(Pht, Utb, kb);
      append_ring(Ph, ring, (j - 1) * ss, j * ss - 1);
      append_ring(Pht, ringt, (j - 1) * ss, j * ss - 1);
      const int pg = prof->begin(3, q);
      if (prof->on) prof->gpairs += (int64_t)X.m * Y.m;
      launch_gram<T>(X, Y, n, prm.setup_fp32, gpart, gram_grid, G, q);
      prof->end(pg, 2, q);
      count(2);
    }
    const int pd = prof->begin(4, q);
    launch_dense_refresh<T>(f, st, G, work, Wphi, Wphit, KMAX, nullptr, q);
    prof->end(pd, f.case_id == 0 ? 2 : 4, q);
    count(f.case_id == 0 ? 2 : 4);
    const int pb = prof->begin(5, q);
    int* kk = &st->kk;
    launch_combine<T>(Ph, Wphi, KMAX, kk, prm.k, Uc[jc], ldk, n, prm.setup_fp32, q);
    launch_combine<T>(Pht, Wphit, KMAX, kk, prm.k, Utc[jc], ldk, n, prm.setup_fp32, q);
    launch_spmm<V, T>(op, 0, Uc[jc], ldk, kk, prm.k, Cc[jc], prm.setup_fp32, q);
    launch_spmm<V, T>(op, 1, Utc[jc], ldk, kk, prm.k, Ctc[jc], prm.setup_fp32, q);
    launch_svd_input<T>(Cc[jc], Ctc[jc], ldk, prm.k, prm.k, n, gpart, gram_grid, G, s2in, q);
    launch_dense_svd(!traits<T>::cx, kk, prm.k, s2in, nullptr, nullptr, prm.svd_tol, Nmat, Mmat, sig, &st->pcyc,
                     nullptr, iflag + 3, q);
    // eq. (equationForUC): U_j = Phi_j W_j N_j, C_j = A U_j (and the duals)
    launch_rotate<T>(Uc[jc], ldk, Nmat, kk, &st->pcyc, prm.k, n, prm.setup_fp32, q);
    launch_rotate<T>(Utc[jc], ldk, Mmat, kk, &st->pcyc, prm.k, n, prm.setup_fp32, q);
    launch_spmm<V, T>(op, 0, Uc[jc], ldk, &st->pcyc, prm.k, Cc[jc], prm.setup_fp32, q);
    launch_spmm<V, T>(op, 1, Utc[jc], ldk, &st->pcyc, prm.k, Ctc[jc], prm.setup_fp32, q);
    prof->end(pb, 13, q);
    count(13);
    RB_CUDA(cudaEventRecord(ev_ref, q));
    ref_pending = true;
    if (prof->on && prof->serial) join_refresh();
  }

  // ------------------------------------------------------------------ Algorithm 2
  struct PairOut {
    int iters = 0, cycles = 0, recycle_dim = 0, status = 0, fallback = 0;
    double relres = 0, relres_dual = 0, true_relres = 0, true_relres_dual = 0;
  };

  // ---- one pair solve as a resumable state machine: begin(), then per cycle launch_cycle()
  // (single) or a batched launch, fetch() and after_cycle(), then end().  solve() and the
  // batched runner share every decision.
  struct Run {
    const T *b = nullptr, *bt = nullptr;
    T *x = nullptr, *xt = nullptr;
    double tol = 0;
    int max_itn = 0;
    uint64_t seed = 0;
    int kU_in = 0, kc_start = 0, kt = 0;
    VecArgs<T> v{};
    PairOut out;
    bool recycle = false, broken = false;
    int j = 0, kp = 0, last_refresh = 0, good_refresh = 0, good_p = 0;
    int done = 0, iter = 0, iter_before = 0, best_at = 0, guard_limit = 0x7fffffff, restarts_used = 0;
    double best_r = 0;
  } run;

  // CUDA graph of one cycle (todo iterations x 3 phases), captured on first use and replayed
  // while its launch parameters stay the same
  cudaGraphExec_t cyc_exec = nullptr;
  int cyc_todo = -1, cyc_kt = -1;
  VecArgs<T> cyc_v{};
  OpArgs<V> cyc_op{};
  // cycles as CUDA graphs unless rbicg_params.graphs = 0 or RBICG_NO_GRAPHS is set (profilers
  // then see plain launches)
  bool use_graphs = prm.graphs != 0 && getenv("RBICG_NO_GRAPHS") == nullptr;

  void drop_graph() {
    if (cyc_exec) cudaGraphExecDestroy(cyc_exec);
    cyc_exec = nullptr;
    cyc_todo = -1;
  }

  void begin(const T* b, const T* bt, T* x, T* xt, double tol, int max_itn, uint64_t seed) {
    Run& R_ = run;
    R_ = Run{};
    defer_refresh = false;   // solve() turns it on after begin(); batched engine steps never do
    ref_deferred = false;
    R_.b = b; R_.bt = bt; R_.x = x; R_.xt = xt; R_.tol = tol; R_.max_itn = max_itn; R_.seed = seed;
    R_.kU_in = prm.recycle ? kU : 0;
    if (pending_start) system_start();
    R_.kc_start = kc;
    R_.kt = kt_for(kc);
    set_field(&DevState::tol, tol);
    set_field(&DevState::max_itn, max_itn);
    set_field(&DevState::done, 0);
    set_field(&DevState::eig_status, 0);
    set_field(&DevState::pcyc, 0);
    R_.v = vec(b, bt, x, xt, C, Ct, U, Ut);
    // compact copies of C, Ct for the iteration kernels: the projections then run over the
    // kc columns the system start kept (rounded up to 4), not the k columns of storage
    const int ldc = std::max(4, ((kc + 3) / 4) * 4);
    if (kc > 0 && ldc < ldk) {
      if (!Cq) { Cq = dmalloc<T>((size_t)n * ldk); Ctq = dmalloc<T>((size_t)n * ldk); }
      launch_pack_cols<T>(C, ldk, Cq, ldc, kc, n, s);
      launch_pack_cols<T>(Ct, ldk, Ctq, ldc, kc, n, s);
      count(2);
      R_.v.C = Cq; R_.v.Ct = Ctq; R_.v.ldc = ldc;
    }
    const int pi = prof->begin(7, s);
    launch_init<V, T>(op, R_.v, st, part, R_.kt, grid, 0, s);
    prof->end(pi, 2, s);
    count(2);
    fetch();
    if (hv->restart) {
      // Algorithm 2 step 3: xt_{-1} <- random (Philox4x32-10), recompute the dual start
      launch_philox<T>(xt, n, seed, s);
      launch_init<V, T>(op, R_.v, st, part, R_.kt, grid, 1, s);
      count(3);
      fetch();
    }
    R_.recycle = prm.recycle != 0;
    R_.done = hv->done;
    R_.best_r = hv->rnorm;
    have_best = false;
    best_metric = 1e300;
    // stagnation guard (not in the paper): see rbicg_params.guard
    R_.guard_limit = (kc > 0 && prm.guard > 0.0 && last_plain_iters > 0)
                         ? (int)std::min<double>(2e9, prm.guard * last_plain_iters) : 0x7fffffff;
    if (R_.guard_limit != 0x7fffffff) {
      if (!x_save) { x_save = dmalloc<T>(n); xt_save = dmalloc<T>(n); }
      RB_CUDA(cudaMemcpyAsync(x_save, x, sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
      RB_CUDA(cudaMemcpyAsync(xt_save, xt, sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
    }
  }

  // iterations of the next cycle
  int cycle_len() const { return std::min(prm.s, run.max_itn - run.iter_before - run.iter); }

  void launch_phases(int todo) {
    if (prof->on) prof->pcols += (int64_t)todo * (run.kt > 0 ? kc : 0);
    for (int t = 0; t < todo; ++t) {
      int pp = prof->begin(0, s);
      launch_phase1<V, T>(op, run.v, st, part, run.kt, grid, s);
      prof->end(pp, 1, s);
      if (run.kt > 0) {   // without a recycle space phase 1 also finishes alpha
        pp = prof->begin(1, s);
        launch_phase2<V, T>(op, run.v, st, part, run.kt, grid, s);
        prof->end(pp, 1, s);
      }
      pp = prof->begin(2, s);
      launch_phase3<V, T>(op, run.v, st, part, grid, s);
      prof->end(pp, 1, s);
    }
  }

  // The graph is captured on, and launched into, the private stream gs (the caller's stream may
  // be the legacy default stream, which cannot be captured), ordered after and before the work
  // of s by two events.  If capture or instantiation fails, the cycle runs as plain launches.
  void launch_cycle(int todo) {
    count((run.kt > 0 ? 3 : 2) * todo);
    if (!use_graphs || prof->on || todo <= 0) { launch_phases(todo); return; }
    if (!cyc_exec || cyc_todo != todo || cyc_kt != run.kt || memcmp(&cyc_v, &run.v, sizeof(cyc_v)) != 0 ||
        memcmp(&cyc_op, &op, sizeof(cyc_op)) != 0) {
      drop_graph();
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        use_graphs = false;
        launch_phases(todo);
        return;
      }
      const cudaStream_t keep = s;
      s = gs;
      launch_phases(todo);
      s = keep;
      const cudaError_t ec = cudaStreamEndCapture(gs, &g);
      const cudaError_t ei = ec == cudaSuccess ? cudaGraphInstantiate(&cyc_exec, g, 0) : ec;
      if (g) cudaGraphDestroy(g);
      if (ei != cudaSuccess) {
        cudaGetLastError();
        cyc_exec = nullptr;
        use_graphs = false;
        launch_phases(todo);
        return;
      }
      cyc_todo = todo; cyc_kt = run.kt; cyc_v = run.v; cyc_op = op;
    }
    RB_CUDA(cudaEventRecord(ev_g0, s));
    RB_CUDA(cudaStreamWaitEvent(gs, ev_g0, 0));
    RB_CUDA(cudaGraphLaunch(cyc_exec, gs));
    RB_CUDA(cudaEventRecord(ev_g1, gs));
    RB_CUDA(cudaStreamWaitEvent(s, ev_g1, 0));
  }

  // after a cycle and fetch(): statuses, stopping rules, guard, next refresh
  void after_cycle() {
    Run& R_ = run;
    // status of the refresh launched after the previous cycle
    if (R_.last_refresh > 0 && !R_.broken) {
      if (hv->eig_status != 0) R_.broken = true;
      else { R_.good_refresh = R_.last_refresh; R_.good_p = hv->pcyc; R_.kp = hv->pcyc; }
    }
    if (!hv->done && hv->iter <= R_.iter)
      throw Err{RBICG_ERR_CUDA, "iteration made no progress (device state not advancing)"};
    R_.iter = hv->iter;
    R_.done = hv->done;
    const int total = R_.iter_before + R_.iter;
    if (!R_.done && total >= R_.max_itn) R_.done = DONE_MAXIT;
    if (!R_.done && diverge > 0.0 && hv->rnorm > diverge * (hv->bnorm > 0 ? hv->bnorm : 1.0)) R_.done = DONE_MAXIT;
    if (hv->rnorm < R_.best_r) { R_.best_r = hv->rnorm; R_.best_at = total; }
    if (!R_.done && stall_window > 0 && total - R_.best_at > stall_window) R_.done = DONE_MAXIT;
    if (stall_window > 0 && R_.done != DONE_NONFINITE) {
      const double m = std::max(hv->rnorm / (hv->bnorm > 0 ? hv->bnorm : 1.0),
                                hv->btnorm > 0 ? hv->rtnorm / hv->btnorm : 0.0);
      if (m < best_metric) {
        best_metric = m;
        if (!x_best) {
          x_best = dmalloc<T>(n); xt_best = dmalloc<T>(n);
          zc_best = dmalloc<zd>(2 * KMAX);
        }
        RB_CUDA(cudaMemcpyAsync(x_best, R_.x, sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
        RB_CUDA(cudaMemcpyAsync(xt_best, R_.xt, sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
        RB_CUDA(cudaMemcpyAsync(zc_best, st->zeta_c, sizeof(zd) * KMAX, cudaMemcpyDeviceToDevice, s));
        RB_CUDA(cudaMemcpyAsync(zc_best + KMAX, st->zetat_c, sizeof(zd) * KMAX, cudaMemcpyDeviceToDevice, s));
        have_best = true;
      }
    }
    const bool breakdown = R_.done == DONE_BREAK_RHO || R_.done == DONE_BREAK_PQ;
    const bool bad_end = breakdown || R_.done == DONE_NONFINITE;
    const bool stalled = !R_.done && R_.iter >= R_.guard_limit;
    const bool armed = R_.guard_limit != 0x7fffffff;
    // the guard (armed for a pair solved with a recycle space) or a restart after a breakdown
    // (rbicg_params.restarts): step 7, then plain BiCG from the current iterate
    const bool restart = !armed && breakdown && R_.restarts_used < prm.restarts &&
                         R_.iter_before + R_.iter < R_.max_itn;
    if ((armed && (stalled || bad_end)) || restart) {
      if (restart) ++R_.restarts_used;
      join_refresh();   // the restart rewrites ring slots and histories a refresh may read
      if (R_.done == DONE_NONFINITE) {
        // the iterate may hold non-finite values: restart from the saved initial guess
        RB_CUDA(cudaMemcpyAsync(R_.x, x_save, sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
        RB_CUDA(cudaMemcpyAsync(R_.xt, xt_save, sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
      } else {
        // step 7 on the current iterate, then restart from it without the recycle space
        launch_finish_a<T>(R_.v, st, R_.kt, grid, s);
        count(1);
      }
      R_.iter_before += R_.iter;
      kc = 0;
      set_field(&DevState::kc, 0);
      set_field(&DevState::max_itn, std::max(1, R_.max_itn - R_.iter_before));
      R_.out.fallback = 1;
      R_.guard_limit = 0x7fffffff;
      have_best = false;   // the kept iterate belongs to the abandoned leg
      best_metric = 1e300;
      const int pi2 = prof->begin(7, s);
      launch_init<V, T>(op, R_.v, st, part, 0, grid, 0, s);
      prof->end(pi2, 2, s);
      count(2);
      fetch();
      if (hv->restart) {
        launch_philox<T>(R_.xt, n, R_.seed, s);
        launch_init<V, T>(op, R_.v, st, part, 0, grid, 1, s);
        count(3);
        fetch();
      }
      R_.kt = 0;
      R_.j = 0; R_.kp = 0; R_.last_refresh = 0; R_.good_refresh = 0; R_.good_p = 0; R_.broken = false;
      R_.iter = 0;
      R_.done = hv->done;
      return;
    }
    if (R_.recycle && prm.refresh && !R_.broken && R_.iter == (R_.j + 1) * prm.s) {
      ++R_.j;
      if (defer_refresh) {
        RB_CUDA(cudaEventRecord(ev_cycle, s));
        ref_deferred = true;
        def_j = R_.j;
        def_kp = R_.kp;
      } else {
        refresh(R_.j, R_.kp);
      }
      R_.last_refresh = R_.j;
    }
  }
  void launch_deferred_refresh() {
    if (!ref_deferred) return;
    ref_deferred = false;
    refresh(def_j, def_kp, true);
  }

  PairOut end() {
    Run& R_ = run;
    PairOut out = R_.out;
    if (stall_window > 0 && have_best && R_.done != DONE_CONVERGED) {
      // an inner solve that did not converge returns the best iterate it reached at a cycle end
      RB_CUDA(cudaMemcpyAsync(R_.x, x_best, sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
      RB_CUDA(cudaMemcpyAsync(R_.xt, xt_best, sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
      RB_CUDA(cudaMemcpyAsync(st->zeta_c, zc_best, sizeof(zd) * KMAX, cudaMemcpyDeviceToDevice, s));
      RB_CUDA(cudaMemcpyAsync(st->zetat_c, zc_best + KMAX, sizeof(zd) * KMAX, cudaMemcpyDeviceToDevice, s));
    }
    const int pf = prof->begin(7, s);
    launch_finish<V, T>(op, R_.v, st, part, R_.kt, grid, s);
    prof->end(pf, 2, s);
    count(2);
    fetch();
    if (R_.last_refresh > R_.good_refresh && !R_.broken) {
      if (hv->eig_status != 0) R_.broken = true;
      else { R_.good_refresh = R_.last_refresh; R_.good_p = hv->pcyc; }
    }
    out.iters = R_.iter_before + hv->iter;
    out.cycles = R_.good_refresh;
    out.recycle_dim = out.fallback ? 0 : kc;
    // the guard's baseline: the full count of the last pair solved from its start without a
    // recycle space (a leg that continued a stalled or broken solve starts from a nearly
    // converged iterate and would shrink it)
    if (R_.kc_start == 0) last_plain_iters = out.iters;
    const double nb = hv->bnorm > 0 ? hv->bnorm : 1.0, nbt = hv->btnorm > 0 ? hv->btnorm : 1.0;
    out.relres = hv->rnorm / nb;
    out.relres_dual = hv->rtnorm / nbt;
    out.true_relres = hv->true_rnorm / nb;
    out.true_relres_dual = hv->true_rtnorm / nbt;
    switch (hv->done) {
      case DONE_CONVERGED: out.status = RBICG_OK; break;
      case DONE_BREAK_RHO: out.status = RBICG_BREAKDOWN_RHO; break;
      case DONE_BREAK_PQ: out.status = RBICG_BREAKDOWN_PQ; break;
      case DONE_NONFINITE: out.status = RBICG_ERR_NONFINITE; break;
      default: out.status = RBICG_NOT_CONVERGED; break;
    }
    if (hv->iter == 0 && hv->done == DONE_CONVERGED) out.status = RBICG_OK;
    if (debug_on())
      fprintf(stderr, "[rbicg] solve n=%lld T=%zu kc=%d iters=%d done=%d relres=%.3e/%.3e true=%.3e/%.3e cycles=%d p=%d\n",
              (long long)n, sizeof(T), kc, hv->iter, hv->done, out.relres, out.relres_dual, out.true_relres,
              out.true_relres_dual, R_.good_refresh, R_.good_p);
    // recycle space for the next system (Section 4: the final U_j; Section 6.2: keep the
    // previous space if no cycle completed)
    if (R_.recycle) {
      if (R_.good_refresh > 0) {
        const int jc = R_.good_refresh & 1;
        std::swap(U, Uc[jc]); std::swap(Ut, Utc[jc]); std::swap(C, Cc[jc]); std::swap(Ct, Ctc[jc]);
        kU = R_.good_p;
      } else if (kc > 0) {
        kU = kc;
      } else {
        kU = 0;
      }
    }
    pending_start = 1;   // the next solve re-derives C, Ct for the (possibly new) operator
    // only the system start's truncation empties the space (a guard fallback is reported by
    // out.fallback alone)
    if (R_.kU_in > 0 && R_.kc_start == 0 && out.status == RBICG_OK) out.status = RBICG_RECYCLE_EMPTY;
    return out;
  }

  PairOut solve(const T* b, const T* bt, T* x, T* xt, double tol, int max_itn, uint64_t seed) {
    begin(b, bt, x, xt, tol, max_itn, seed);
    return run_to_end();
  }
  // the cycles of a begun solve, then step 7 (a solve that begin() finished goes straight to end)
  PairOut run_to_end() {
    defer_refresh = true;
    while (!run.done) {
      launch_cycle(cycle_len());
      launch_deferred_refresh();
      fetch();
      after_cycle();
    }
    launch_deferred_refresh();
    defer_refresh = false;
    return end();
  }

};


// residual kernel for the refinement loop: r = b - Op x (FP64), norms via a small reduction
template <class V, class T>
__global__ void k_residual(OpArgs<V> op, const T* b, const T* x, T* r, int adjoint) {
  const int* rp = adjoint ? op.trp : op.rp;
  const int* ci = adjoint ? op.tci : op.ci;
  const V* va = adjoint ? op.tva : op.va;
  T sh = from_zd<T>(zd(op.sh_re, adjoint ? -op.sh_im : op.sh_im));
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < op.n; row += gridDim.x * blockDim.x) {
    T acc = T(0);
    for (int e = rp[row]; e < rp[row + 1]; ++e) acc += vmul(va[e], x[ci[e]]);
    if (op.has_shift) acc = sh * x[row] - acc;
    r[row] = b[row] - acc;
  }
}
template <class T>
__global__ void k_norm2(const T* a, int64_t n, double* out) {
  __shared__ double red[8];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += (double)abs2(a[i]);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[blockIdx.x] = t;
  }
}

// ------------------------------------------------------------------------------------
// the handle
// ------------------------------------------------------------------------------------
template <class T> struct lowp;
template <> struct lowp<double> { typedef float type; };
template <> struct lowp<cplx<double>> { typedef cplx<float> type; };

struct Ctx;

struct Impl {
  virtual ~Impl() {}
  virtual void set_operator(const rbicg_csr& A) = 0;
  virtual rbicg_result solve(const void* b, const void* bt, void* x, void* xt) = 0;
  virtual void reset() = 0;
  virtual void export_recycle(void* U, void* Ut, int* p) = 0;
  virtual void import_recycle(const void* U, const void* Ut, int p) = 0;
  virtual void set_refresh(int v) = 0;
  virtual void history(double* out, int max, int* count) = 0;
  // FP32-refined handles in the engine: begin the refinement / continue it after the solver that
  // the engine stepped (kind) finished its cycles; both return 1 with the next solver to step
  // (*solver, *kind) or 0 when refine_result() holds the result
  virtual int refine_begin(const void* b, const void* bt, void* x, void* xt, void** solver, int* kind) = 0;
  virtual int refine_after(int kind, void** solver, int* kindout) = 0;
  virtual rbicg_result refine_result() = 0;
  // run this handle's work (refinement kernels and both solvers) on st; returns the previous stream
  virtual cudaStream_t swap_stream(cudaStream_t st) = 0;
  // FP64 handles: the solver that a batch drives directly, and the kind of its (V, T)
  virtual void* batch_solver(int* kind) = 0;
};

template <class V, class T>
struct ImplT : Impl {
  typedef typename lowp<T>::type T32;
  typedef typename lowp<V>::type V32;
  rbicg_params prm;
  int64_t n;
  cudaStream_t s;
  int64_t* launches;
  std::unique_ptr<Solver<V, T>> hi;
  std::unique_ptr<Solver<V32, T32>> lo;
  V32* va32 = nullptr;
  T *r64 = nullptr, *rt64 = nullptr;
  T32 *r32 = nullptr, *rt32 = nullptr, *d32 = nullptr, *dt32 = nullptr;
  T *d64 = nullptr, *dt64 = nullptr;
  double* nrm = nullptr;
  double* hnrm = nullptr;

  Profiler* prof;
  ImplT(const rbicg_params& p, int64_t n_, cudaStream_t s_, int64_t* l, Profiler* pr)
      : prm(p), n(n_), s(s_), launches(l), prof(pr) {
    if (prm.precision == RBICG_FP64) {
      hi.reset(new Solver<V, T>(prm, n, s, launches, prof));
    } else {
      // hi: the FP64 operator for the residuals, and the FP64 RBiCG solver this handle falls
      // back to when the FP32 inner recurrence cannot reach inner_tol
      rbicg_params ph = prm;
      ph.precision = RBICG_FP64;
      hi.reset(new Solver<V, T>(ph, n, s, launches, prof));
      rbicg_params pl = prm;
      pl.svd_tol = std::max(prm.svd_tol, prm.inner_svd_tol);
      lo.reset(new Solver<V32, T32>(pl, n, s, launches, prof));
      // an inner residual this far above ||b||, or no new minimum for this long, means the FP32
      // recurrence has lost its way (FP64 BiCG residuals of these problems peak near 1e3 ||b||)
      lo->diverge = 1e6;
      lo->stall_window = std::max(1000, 25 * prm.s);
      r64 = dmalloc<T>(n); rt64 = dmalloc<T>(n); d64 = dmalloc<T>(n); dt64 = dmalloc<T>(n);
      r32 = dmalloc<T32>(n); rt32 = dmalloc<T32>(n); d32 = dmalloc<T32>(n); dt32 = dmalloc<T32>(n);
      nrm = dmalloc<double>(1024);
      RB_CUDA(cudaMallocHost(&hnrm, sizeof(double) * 1024));
    }
  }
  ~ImplT() override {
    cudaStreamSynchronize(s);
    if (va32) cudaFree(va32);
    void* bufs[] = {r64, rt64, d64, dt64, r32, rt32, d32, dt32, nrm};
    for (void* b : bufs) if (b) cudaFree(b);
    if (hnrm) cudaFreeHost(hnrm);
  }

  void set_operator(const rbicg_csr& A) override {
    hi->set_operator(A, reinterpret_cast<const V*>(A.val));
    if (lo) {
      if (va32) cudaFree(va32);
      va32 = dmalloc<V32>(std::max<int64_t>(1, A.nnz));
      launch_convert<V, V32>(reinterpret_cast<const V*>(A.val), va32, A.nnz, s);
      *launches += 1;
      lo->set_operator(A, va32);
    }
  }

  double norm(const T* a) {
    const int blocks = 256;
    k_norm2<T><<<blocks, 256, 0, s>>>(a, n, nrm);
    *launches += 1;
    RB_CUDA(cudaMemcpyAsync(hnrm, nrm, sizeof(double) * blocks, cudaMemcpyDeviceToHost, s));
    RB_CUDA(cudaStreamSynchronize(s));
    double t = 0.0;
    for (int i = 0; i < blocks; ++i) t += hnrm[i];
    return sqrt(t);
  }

  // ---- FP64 iterative refinement around FP32 inner RBiCG solves, as a resumable state machine:
  // refine_begin() / refine_after() return what runs next (REF_DONE, REF_INNER: the FP32 solver
  // lo has begun an inner solve, REF_FP64: the FP64 solver hi has begun the fallback solve).
  // solve() drives it to the end on the handle's stream; the batching engine drives the same
  // states one cycle at a time, so a served FP32-refined request overlaps the others.
  enum { REF_DONE = 0, REF_INNER = 1, REF_FP64 = 2 };
  struct RefState {
    const T* b = nullptr; const T* bt = nullptr; T* x = nullptr; T* xt = nullptr;
    double nb = 0, nbt = 0, rr = 0, rtr = 0;
    int step = 0, total_iters = 0, cycles = 0, rdim = 0, first_inner = -1, inner_cap = 0, status = 0;
    double prev_rr = -1.0, prev_rtr = -1.0;   // residual norms before the last FP64 correction
    bool retried_plain = false, pc = false, dc = false;
    rbicg_result res{};
  } rs;

  rbicg_result solve(const void* bv, const void* btv, void* xv, void* xtv) override {
    if (!lo) {
      return solve_fp64(reinterpret_cast<const T*>(bv), reinterpret_cast<const T*>(btv), reinterpret_cast<T*>(xv),
                        reinterpret_cast<T*>(xtv), 0, 0);
    }
    int what = refine_begin_t(reinterpret_cast<const T*>(bv), reinterpret_cast<const T*>(btv),
                              reinterpret_cast<T*>(xv), reinterpret_cast<T*>(xtv));
    while (what != REF_DONE) {
      if (what == REF_INNER) what = after_inner(lo->run_to_end());
      else what = after_fp64(hi->run_to_end());
    }
    return rs.res;
  }

  int refine_begin_t(const T* b, const T* bt, T* x, T* xt) {
    rs = RefState{};
    rs.b = b; rs.bt = bt; rs.x = x; rs.xt = xt;
    rs.nb = norm(b);
    rs.nbt = norm(bt);
    rs.status = RBICG_NOT_CONVERGED;
    rs.inner_cap = prm.max_itn;
    return advance();
  }

  // residual of the refined iterate; converged, out of steps, or the next inner solve
  int advance() {
    const int grid = std::max(1, std::min((int)((n + 255) / 256), num_sms() * 8));
    k_residual<V, T><<<grid, 256, 0, s>>>(hi->op, rs.b, rs.x, r64, 0);
    k_residual<V, T><<<grid, 256, 0, s>>>(hi->op, rs.bt, rs.xt, rt64, 1);
    *launches += 2;
    rs.rr = norm(r64);
    rs.rtr = norm(rt64);
    if (debug_on())
      fprintf(stderr, "[rbicg] refine step %d relres %.3e dual %.3e\n", rs.step, rs.rr / (rs.nb > 0 ? rs.nb : 1.0),
              rs.rtr / (rs.nbt > 0 ? rs.nbt : 1.0));
    rs.pc = rs.rr <= prm.tol * (rs.nb > 0 ? rs.nb : 1.0) || (rs.nb == 0 && rs.rr == 0);
    rs.dc = rs.nbt == 0.0 || rs.rtr <= prm.tol * rs.nbt;
    if (rs.pc && rs.dc) { rs.status = RBICG_OK; return finish_refined(); }
    if (rs.step >= prm.refine_max) return finish_refined();
    if (fp64_only) {
      // an FP64 correction made no progress on either side: stop (status NOT_CONVERGED)
      if (rs.prev_rr >= 0.0 && !(rs.rr < 0.9 * rs.prev_rr) && !(rs.rtr < 0.9 * rs.prev_rtr)) return finish_refined();
      return begin_fp64_correction();
    }
    launch_convert<T, T32>(r64, r32, n, s);
    launch_convert<T, T32>(rt64, rt32, n, s);
    RB_CUDA(cudaMemsetAsync(d32, 0, sizeof(T32) * n, s));
    RB_CUDA(cudaMemsetAsync(dt32, 0, sizeof(T32) * n, s));
    *launches += 2;
    lo->begin(r32, rt32, d32, dt32, prm.inner_tol, rs.inner_cap, prm.seed + rs.step);
    if (!lo->run.done) return REF_INNER;
    return after_inner(lo->run_to_end());
  }

  // an inner solve ended (its step 7 applied): use its correction or retry / fall back
  int after_inner(const typename Solver<V32, T32>::PairOut& o) {
    rs.total_iters += o.iters;
    rs.cycles += o.cycles;
    rs.rdim = o.recycle_dim;
    // a non-finite inner solve is treated like an unusable correction (retried as plain BiCG)
    if (o.status < 0 && o.status != RBICG_ERR_NONFINITE) { rs.status = o.status; return finish_refined(); }
    if (rs.first_inner < 0) {
      rs.first_inner = o.iters;
      rs.inner_cap = std::min(prm.max_itn, std::max(200, 4 * rs.first_inner + 100));
    }
    // A correction is used only if the inner solve reduced its own residual; otherwise the
    // inner recycle space is dropped and the step is retried once as plain FP32 BiCG.
    const bool usable = o.status != RBICG_ERR_NONFINITE &&
                        (o.status == RBICG_OK || o.status == RBICG_RECYCLE_EMPTY ||
                         (o.true_relres < 0.5 && (rs.dc || o.true_relres_dual < 0.5)));
    if (debug_on())
      fprintf(stderr, "[rbicg] inner step %d status %d iters %d relres %.3e/%.3e usable %d\n", rs.step, o.status,
              o.iters, o.true_relres, o.true_relres_dual, (int)usable);
    if (!usable) {
      if (rs.retried_plain) {
        // the FP32 recurrence does not converge on this problem even without a recycle space:
        // this handle continues the refinement with FP64 RBiCG correction solves
        fp64_only = true;
        return begin_fp64_correction();   // the residual of this step is unchanged
      }
      rs.retried_plain = true;
      lo->kU = 0;
      lo->pending_start = 1;
      return advance();   // the same step again (the residual is unchanged)
    }
    rs.retried_plain = false;
    if (!rs.pc) {
      launch_convert<T32, T>(d32, d64, n, s);
      launch_axpy_inplace<T>(rs.x, d64, n, s);
      *launches += 2;
    }
    if (!rs.dc) {
      launch_convert<T32, T>(dt32, d64, n, s);
      launch_axpy_inplace<T>(rs.xt, d64, n, s);
      *launches += 2;
    }
    ++rs.step;
    return advance();
  }

  // FP64 correction solve of a handle that fell back: A d = r, A^H dt = rt (r, rt: the FP64
  // residuals of the refined iterate, left in r64, rt64 by advance()) with FP64 RBiCG from d = 0,
  // to the relative tolerance that brings the unconverged side(s) to tol (half of it, for margin;
  // at least 1e-13, at most 0.5).  A correction solve's attainable accuracy is relative to ||r||,
  // so repeated steps reach tol in the true residual where one FP64 solve of the whole system
  // stalls at the gap between its recurrence and its true residual.
  int begin_fp64_correction() {
    double need = 0.5;
    if (!rs.pc && rs.rr > 0) need = std::min(need, 0.5 * prm.tol * (rs.nb > 0 ? rs.nb : 1.0) / rs.rr);
    if (!rs.dc && rs.rtr > 0) need = std::min(need, 0.5 * prm.tol * rs.nbt / rs.rtr);
    const double tc = std::max(1e-13, need);
    RB_CUDA(cudaMemsetAsync(d64, 0, sizeof(T) * n, s));
    RB_CUDA(cudaMemsetAsync(dt64, 0, sizeof(T) * n, s));
    rs.prev_rr = rs.rr;
    rs.prev_rtr = rs.rtr;
    hi->begin(r64, rt64, d64, dt64, tc, prm.max_itn, prm.seed + rs.step);
    if (!hi->run.done) return REF_FP64;
    return after_fp64(hi->run_to_end());
  }

  // an FP64 correction solve ended: apply its correction (if it reduced its own residual) and
  // go on with the next refinement step
  int after_fp64(const typename Solver<V, T>::PairOut& o) {
    rs.total_iters += o.iters;
    rs.cycles += o.cycles;
    rs.rdim = o.recycle_dim;
    if (o.status < 0 && o.status != RBICG_ERR_NONFINITE) { rs.status = o.status; return finish_refined(); }
    const bool usable = o.status != RBICG_ERR_NONFINITE &&
                        (o.status == RBICG_OK || o.status == RBICG_RECYCLE_EMPTY ||
                         (o.true_relres < 0.5 && (rs.dc || o.true_relres_dual < 0.5)));
    if (debug_on())
      fprintf(stderr, "[rbicg] fp64 correction %d status %d iters %d relres %.3e/%.3e usable %d\n", rs.step,
              o.status, o.iters, o.true_relres, o.true_relres_dual, (int)usable);
    if (!usable) return finish_refined();
    if (!rs.pc) { launch_axpy_inplace<T>(rs.x, d64, n, s); *launches += 1; }
    if (!rs.dc) { launch_axpy_inplace<T>(rs.xt, dt64, n, s); *launches += 1; }
    ++rs.step;
    return advance();
  }

  // an FP64 handle's solve ended (no refinement): its result as it stands
  int after_plain(const typename Solver<V, T>::PairOut& o) {
    rbicg_result& res = rs.res;
    res = rbicg_result{};
    res.iters = o.iters; res.cycles = o.cycles; res.recycle_dim = o.recycle_dim;
    res.relres = o.relres; res.relres_dual = o.relres_dual;
    res.true_relres = o.true_relres; res.true_relres_dual = o.true_relres_dual;
    res.status = o.status;
    res.fallback = o.fallback;
    return REF_DONE;
  }

  int finish_refined() {
    rbicg_result& res = rs.res;
    res = rbicg_result{};
    res.iters = rs.total_iters;
    res.cycles = rs.cycles;
    res.recycle_dim = rs.rdim;
    res.refine_steps = rs.step;
    res.relres = rs.rr / (rs.nb > 0 ? rs.nb : 1.0);
    res.relres_dual = rs.rtr / (rs.nbt > 0 ? rs.nbt : 1.0);
    res.true_relres = res.relres;
    res.true_relres_dual = res.relres_dual;
    res.status = rs.status;
    res.fallback = fp64_only ? 2 : 0;
    return REF_DONE;
  }

  // engine entry points: kinds 0..2 are the FP64 solvers, 3..5 the FP32 ones
  static int kind_of_hi() { return traits<T>::cx ? (traits<V>::cx ? 2 : 1) : 0; }
  static int kind_of_lo() { return traits<T>::cx ? (traits<V>::cx ? 5 : 4) : 3; }
  int refine_begin(const void* b, const void* bt, void* x, void* xt, void** solver, int* kind) override {
    int w;
    if (!lo) {
      rs = RefState{};
      hi->begin(reinterpret_cast<const T*>(b), reinterpret_cast<const T*>(bt), reinterpret_cast<T*>(x),
                reinterpret_cast<T*>(xt), prm.tol, prm.max_itn, prm.seed);
      w = hi->run.done ? after_plain(hi->run_to_end()) : REF_FP64;
    } else {
      w = refine_begin_t(reinterpret_cast<const T*>(b), reinterpret_cast<const T*>(bt), reinterpret_cast<T*>(x),
                         reinterpret_cast<T*>(xt));
    }
    return route(w, solver, kind);
  }
  int refine_after(int kind, void** solver, int* kindout) override {
    const int w = kind >= 3 ? after_inner(lo->end()) : (lo ? after_fp64(hi->end()) : after_plain(hi->end()));
    return route(w, solver, kindout);
  }
  int route(int w, void** solver, int* kind) {
    if (w == REF_INNER) { *solver = lo.get(); *kind = kind_of_lo(); return 1; }
    if (w == REF_FP64) { *solver = hi.get(); *kind = kind_of_hi(); return 1; }
    return 0;
  }
  rbicg_result refine_result() override { return rs.res; }
  cudaStream_t swap_stream(cudaStream_t st) override {
    const cudaStream_t old = s;
    s = st;
    hi->s = st;
    if (lo) lo->s = st;
    return old;
  }

  bool fp64_only = false;   // FP32_REFINED handle that fell back to FP64 (until rbicg_reset)

  void* batch_solver(int* kind) override {
    if (lo) return nullptr;   // FP32-refined handles go through refine_begin / refine_after
    *kind = traits<T>::cx ? (traits<V>::cx ? 2 : 1) : 0;
    return hi.get();
  }

  rbicg_result solve_fp64(const T* b, const T* bt, T* x, T* xt, int iters_before, int steps_before) {
    rbicg_result res{};
    auto o = hi->solve(b, bt, x, xt, prm.tol, prm.max_itn, prm.seed);
    res.iters = iters_before + o.iters; res.cycles = o.cycles; res.recycle_dim = o.recycle_dim;
    res.refine_steps = steps_before;
    res.relres = o.relres; res.relres_dual = o.relres_dual;
    res.true_relres = o.true_relres; res.true_relres_dual = o.true_relres_dual;
    res.status = o.status;
    res.fallback = lo ? 2 : o.fallback;
    return res;
  }

  void reset() override {
    hi->kU = 0; hi->pending_start = 1;
    if (lo) { lo->kU = 0; lo->pending_start = 1; }
    fp64_only = false;
  }

  void set_refresh(int v) override {
    prm.refresh = v;
    hi->prm.refresh = v;
    if (lo) lo->prm.refresh = v;
  }

  // ||r_m|| of the FP64 solver's last solve for its last min(max, HR) iterations (device ring)
  void history(double* out, int max, int* count) override {
    DevState h;
    RB_CUDA(cudaMemcpyAsync(&h, hi->st, sizeof h, cudaMemcpyDeviceToHost, s));
    RB_CUDA(cudaStreamSynchronize(s));
    const int last = h.iter;
    const int cnt = std::min(std::min(max, HR), last + 1);
    for (int q = 0; q < cnt; ++q) out[q] = h.h_rnorm[(last - cnt + 1 + q) % HR];
    *count = cnt;
  }

  void export_recycle(void* Uo, void* Uto, int* p) override {
    if (lo && !fp64_only) {
      // the recycle space lives in the FP32 inner solver; export it widened to FP64
      const int64_t m = n * lo->ldk;
      T* tmp = reinterpret_cast<T*>(Uo);
      T* tmpt = reinterpret_cast<T*>(Uto);
      std::vector<int> dummy;
      (void)dummy;
      widen_rows(lo->U, tmp, lo->ldk);
      widen_rows(lo->Ut, tmpt, lo->ldk);
      (void)m;
      *p = lo->kU;
      return;
    }
    copy_rows(hi->U, reinterpret_cast<T*>(Uo), hi->ldk);
    copy_rows(hi->Ut, reinterpret_cast<T*>(Uto), hi->ldk);
    *p = hi->kU;
  }
  void copy_rows(const T* src, T* dst, int ldk) {
    RB_CUDA(cudaMemcpy2DAsync(dst, sizeof(T) * prm.k, src, sizeof(T) * ldk, sizeof(T) * prm.k, n,
                              cudaMemcpyDeviceToDevice, s));
    RB_CUDA(cudaStreamSynchronize(s));
  }
  void widen_rows(const T32* src, T* dst, int ldk) {
    T* tmp = dmalloc<T>((size_t)n * ldk);
    launch_convert<T32, T>(src, tmp, (int64_t)n * ldk, s);
    copy_rows(tmp, dst, ldk);
    cudaFree(tmp);
  }
  void import_recycle(const void* Ui, const void* Uti, int p) override {
    if (lo && !fp64_only) {
      T32* tmp = dmalloc<T32>((size_t)n * p);
      for (int side = 0; side < 2; ++side) {
        launch_convert<T, T32>(reinterpret_cast<const T*>(side ? Uti : Ui), tmp, (int64_t)n * p, s);
        RB_CUDA(cudaMemsetAsync(side ? lo->Ut : lo->U, 0, sizeof(T32) * n * lo->ldk, s));
        RB_CUDA(cudaMemcpy2DAsync(side ? lo->Ut : lo->U, sizeof(T32) * lo->ldk, tmp, sizeof(T32) * p,
                                  sizeof(T32) * p, n, cudaMemcpyDeviceToDevice, s));
      }
      RB_CUDA(cudaStreamSynchronize(s));
      cudaFree(tmp);
      lo->kU = p; lo->pending_start = 1;
      return;
    }
    for (int side = 0; side < 2; ++side) {
      T* dst = side ? hi->Ut : hi->U;
      RB_CUDA(cudaMemsetAsync(dst, 0, sizeof(T) * n * hi->ldk, s));
      RB_CUDA(cudaMemcpy2DAsync(dst, sizeof(T) * hi->ldk, side ? Uti : Ui, sizeof(T) * p, sizeof(T) * p, n,
                                cudaMemcpyDeviceToDevice, s));
    }
    RB_CUDA(cudaStreamSynchronize(s));
    hi->kU = p; hi->pending_start = 1;
  }
};

}  // namespace rb

// ------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------
using namespace rb;

struct rbicg_ctx {
  rbicg_params prm;
  int64_t n;
  rbicg_dtype dtype;
  cudaStream_t s;
  int val_complex = -1;
  std::unique_ptr<Impl> impl;
  OpKey key;
  std::string err;
  int64_t launches = 0;
  Profiler prof;
};

static rbicg_status fail(rbicg_handle h, rbicg_status st, const std::string& msg) {
  if (h) h->err = msg;
  g_last_error = msg;
  return st;
}

#define RB_GUARD(h, ...)                                                                      \
  try {                                                                                       \
    __VA_ARGS__                                                                               \
  } catch (const Err& e) {                                                                    \
    return fail(h, e.st, e.msg);                                                              \
  } catch (const std::exception& e) {                                                         \
    return fail(h, RBICG_ERR_CUDA, e.what());                                                 \
  }

extern "C" void rbicg_default_params(rbicg_params* p) {
  if (!p) return;
  p->k = 10; p->s = 40; p->max_itn = 20000; p->tol = 1e-8; p->svd_tol = 1e-6; p->inner_tol = 1e-5;
  p->refine_max = 12; p->precision = RBICG_FP64; p->seed = 0; p->setup_fp32 = 1; p->recycle = 1;
  p->inner_svd_tol = 1e-3;
  p->guard = 1.5;
  p->restarts = 0;
  p->grid_blocks = 0;
  p->refresh = 1;
  p->setup_blocks = 0;
  p->graphs = 1;
}

static std::string check_params(const rbicg_params* p, int64_t n) {
  if (!p) return "params is NULL";
  if (n <= 0 || n > (int64_t)0x7fffffff - 1) return "n out of range";
  if (p->k < 1 || p->k > KMAX) return "k must be in 1..32";
  if (p->s < 2 || p->s > SMAX) return "s must be in 2..64";
  if (p->k + p->s > MMAX) return "k + s must be <= 80";
  if (!(p->tol > 0.0)) return "tol must be positive";
  if (p->max_itn < 1) return "max_itn must be positive";
  if (!(p->svd_tol >= 0.0)) return "svd_tol must be >= 0";
  if (!(p->guard >= 0.0)) return "guard must be >= 0";
  if (p->grid_blocks < 0 || p->grid_blocks > (1 << 20)) return "grid_blocks must be in 0..2^20";
  if (p->restarts < 0 || p->restarts > 1000) return "restarts must be in 0..1000";
  if (p->refresh != 0 && p->refresh != 1) return "refresh must be 0 or 1";
  if (p->setup_blocks < 0 || p->setup_blocks > 8192) return "setup_blocks must be in 0..8192";
  if (p->graphs != 0 && p->graphs != 1) return "graphs must be 0 or 1";
  if (p->precision == RBICG_FP32_REFINED && !(p->inner_tol > 0.0 && p->inner_tol < 1.0))
    return "inner_tol must be in (0, 1)";
  if (p->precision != RBICG_FP64 && p->precision != RBICG_FP32_REFINED) return "unknown precision";
  return "";
}

extern "C" rbicg_status rbicg_create(const rbicg_params* params, int64_t n, rbicg_dtype dtype, void* stream,
                                     rbicg_handle* out) {
  if (!out) return fail(nullptr, RBICG_ERR_ARG, "out is NULL");
  *out = nullptr;
  const std::string m = check_params(params, n);
  if (!m.empty()) return fail(nullptr, RBICG_ERR_ARG, m);
  if (dtype != RBICG_R64 && dtype != RBICG_C128) return fail(nullptr, RBICG_ERR_ARG, "unknown dtype");
  rbicg_ctx* h = new rbicg_ctx();
  h->prm = *params;
  h->n = n;
  h->dtype = dtype;
  h->s = reinterpret_cast<cudaStream_t>(stream);
  *out = h;
  return RBICG_OK;
}

static void ensure_impl(rbicg_handle h, int val_complex) {
  if (h->impl && h->val_complex == val_complex) return;
  if (h->impl && h->val_complex != val_complex)
    throw Err{RBICG_ERR_ARG, "operator value type (real/complex) changed on this handle"};
  if (h->dtype == RBICG_R64) {
    if (val_complex) throw Err{RBICG_ERR_ARG, "complex operator on a real (R64) handle"};
    h->impl.reset(new ImplT<double, double>(h->prm, h->n, h->s, &h->launches, &h->prof));
  } else if (val_complex) {
    h->impl.reset(new ImplT<cplx<double>, cplx<double>>(h->prm, h->n, h->s, &h->launches, &h->prof));
  } else {
    h->impl.reset(new ImplT<double, cplx<double>>(h->prm, h->n, h->s, &h->launches, &h->prof));
  }
  h->val_complex = val_complex;
}

static std::string check_csr(rbicg_handle h, const rbicg_csr* A) {
  if (!A) return "A is NULL";
  if (A->n != h->n) return "A->n does not match the handle";
  if (A->nnz < 0 || A->nnz > (int64_t)0x7fffffff) return "nnz out of range";
  if (!A->row_ptr || (A->nnz > 0 && (!A->col_idx || !A->val))) return "null CSR array";
  if (h->dtype == RBICG_R64 && A->has_shift && A->shift_im != 0.0) return "complex shift on a real handle";
  return "";
}

static void do_update(rbicg_handle h, const rbicg_csr* A) {
  ensure_impl(h, A->val_complex ? 1 : 0);
  int* flag = nullptr;
  RB_CUDA(cudaMalloc(&flag, sizeof(int)));
  validate_csr((int)A->n, A->nnz, A->row_ptr, A->col_idx, flag, h->s);
  int hf = 0;
  RB_CUDA(cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  RB_CUDA(cudaStreamSynchronize(h->s));
  cudaFree(flag);
  h->launches += 1;
  if (hf) {
    char buf[160];
    snprintf(buf, sizeof buf, "malformed CSR (flags 0x%x: 1 row_ptr[0], 2 row_ptr[n], 4 order, 8 column range, "
                              "16 unsorted/duplicate columns)", hf);
    throw Err{RBICG_ERR_ARG, buf};
  }
  h->impl->set_operator(*A);
  h->key.rp = A->row_ptr; h->key.ci = A->col_idx; h->key.va = A->val; h->key.n = A->n; h->key.nnz = A->nnz;
  h->key.has_shift = A->has_shift; h->key.val_complex = A->val_complex; h->key.sr = A->shift_re;
  h->key.si = A->shift_im;
}

extern "C" rbicg_status rbicg_update_recycle(rbicg_handle h, const rbicg_csr* A) {
  if (!h) return fail(nullptr, RBICG_ERR_ARG, "handle is NULL");
  const std::string m = check_csr(h, A);
  if (!m.empty()) return fail(h, RBICG_ERR_ARG, m);
  RB_GUARD(h, { do_update(h, A); return RBICG_OK; })
}

extern "C" rbicg_status rbicg_solve_pair(rbicg_handle h, const rbicg_csr* A, const void* b, const void* bt,
                                         void* x, void* xt, rbicg_result* res) {
  if (!h) return fail(nullptr, RBICG_ERR_ARG, "handle is NULL");
  if (!b || !bt || !x || !xt) return fail(h, RBICG_ERR_ARG, "null vector pointer");
  RB_GUARD(h, {
    if (A) {
      const std::string m = check_csr(h, A);
      if (!m.empty()) return fail(h, RBICG_ERR_ARG, m);
      OpKey k;
      k.rp = A->row_ptr; k.ci = A->col_idx; k.va = A->val; k.n = A->n; k.nnz = A->nnz; k.has_shift = A->has_shift;
      k.val_complex = A->val_complex; k.sr = A->shift_re; k.si = A->shift_im;
      if (!h->impl || !(k == h->key)) do_update(h, A);
    }
    if (!h->impl) return fail(h, RBICG_ERR_ARG, "no operator set (pass A or call rbicg_update_recycle)");
    rbicg_result r = h->impl->solve(b, bt, x, xt);
    if (res) *res = r;
    if (r.status < 0) return fail(h, (rbicg_status)r.status, "non-finite value in the iteration");
    h->err.clear();
    return (rbicg_status)r.status;
  })
}

template <class P>
static rbicg_result to_result(const P& o) {
  rbicg_result r{};
  r.iters = o.iters; r.cycles = o.cycles; r.recycle_dim = o.recycle_dim; r.refine_steps = 0;
  r.relres = o.relres; r.relres_dual = o.relres_dual;
  r.true_relres = o.true_relres; r.true_relres_dual = o.true_relres_dual;
  r.status = o.status; r.fallback = o.fallback;
  return r;
}

extern "C" rbicg_status rbicg_export_recycle(rbicg_handle h, void* U, void* Ut, int* p) {
  if (!h || !U || !Ut || !p) return fail(h, RBICG_ERR_ARG, "null argument");
  if (!h->impl) { *p = 0; return RBICG_OK; }
  RB_GUARD(h, { h->impl->export_recycle(U, Ut, p); return RBICG_OK; })
}

extern "C" rbicg_status rbicg_import_recycle(rbicg_handle h, const void* U, const void* Ut, int p) {
  if (!h || (p > 0 && (!U || !Ut))) return fail(h, RBICG_ERR_ARG, "null argument");
  if (p < 0 || p > h->prm.k) return fail(h, RBICG_ERR_ARG, "p must be in 0..k");
  if (!h->impl) return fail(h, RBICG_ERR_ARG, "set an operator before importing a recycle space");
  RB_GUARD(h, { h->impl->import_recycle(U, Ut, p); return RBICG_OK; })
}

extern "C" rbicg_status rbicg_reset(rbicg_handle h) {
  if (!h) return fail(nullptr, RBICG_ERR_ARG, "handle is NULL");
  if (h->impl) h->impl->reset();
  return RBICG_OK;
}

extern "C" rbicg_status rbicg_residual_history(rbicg_handle h, double* out, int max, int* count) {
  if (!h || !out || !count || max < 1) return fail(h, RBICG_ERR_ARG, "null argument or max < 1");
  if (!h->impl) return fail(h, RBICG_ERR_ARG, "no solve on this handle yet");
  RB_GUARD(h, { h->impl->history(out, max, count); return RBICG_OK; })
}

extern "C" rbicg_status rbicg_set_refresh(rbicg_handle h, int refresh) {
  if (!h) return fail(nullptr, RBICG_ERR_ARG, "handle is NULL");
  if (refresh != 0 && refresh != 1) return fail(h, RBICG_ERR_ARG, "refresh must be 0 or 1");
  h->prm.refresh = refresh;
  if (h->impl) h->impl->set_refresh(refresh);
  return RBICG_OK;
}

extern "C" rbicg_status rbicg_destroy(rbicg_handle h) {
  if (!h) return RBICG_OK;
  try {
    h->impl.reset();
  } catch (...) {
  }
  delete h;
  return RBICG_OK;
}

extern "C" const char* rbicg_last_error(rbicg_handle h) { return h ? h->err.c_str() : g_last_error.c_str(); }

extern "C" int64_t rbicg_launch_count(rbicg_handle h) { return h ? h->launches : 0; }

extern "C" rbicg_status rbicg_profile(rbicg_handle h, int enable, double* ms_out, int64_t* launches_out) {
  if (!h) return fail(nullptr, RBICG_ERR_ARG, "handle is NULL");
  cudaStreamSynchronize(h->s);
  h->prof.harvest();
  for (int i = 0; i < RBICG_NPROF; ++i) {
    if (ms_out) ms_out[i] = h->prof.ms[i];
    if (launches_out) launches_out[i] = h->prof.cnt[i];
  }
  if (enable >= 0) {
    if (enable && !h->prof.on) h->prof.reset();
    h->prof.on = enable != 0;
    h->prof.serial = enable == 2;
  }
  return RBICG_OK;
}

extern "C" rbicg_status rbicg_profile_gram_pairs(rbicg_handle h, int64_t* pairs) {
  if (!h || !pairs) return fail(h, RBICG_ERR_ARG, "null argument");
  *pairs = h->prof.gpairs;
  return RBICG_OK;
}

extern "C" rbicg_status rbicg_profile_columns(rbicg_handle h, int64_t* cols) {
  if (!h || !cols) return fail(h, RBICG_ERR_ARG, "null argument");
  *cols = h->prof.pcols;
  return RBICG_OK;
}

// ------------------------------------------------------------------------------------
// component entry points
// ------------------------------------------------------------------------------------
namespace rb {
int64_t dense_state_offset();
int64_t dense_work_elems();
int64_t dense_off_L();
int64_t dense_off_R();

template <class V, class T>
static void op_spmv_project_impl(const rbicg_csr* A, const void* r, const void* rt, const void* p_old,
                                 const void* pt_old, double bre, double bim, const void* C, const void* Ct, int k,
                                 int ldc, const double* Dc_host, void* p_out, void* pt_out, void* z, void* zt,
                                 void* zeta_host, void* zetat_host, cudaStream_t s) {
  typedef typename traits<T>::acc Acc;
  OpArgs<V> op{};
  op.n = (int)A->n; op.rp = A->row_ptr; op.ci = A->col_idx; op.va = reinterpret_cast<const V*>(A->val);
  op.has_shift = A->has_shift; op.sh_re = A->shift_re; op.sh_im = A->shift_im;
  V* tva = dmalloc<V>(std::max<int64_t>(1, A->nnz));
  int* flag = dmalloc<int>(1);
  int* trp = nullptr;
  int* tci = nullptr;
  int shared = 0;
  int e = build_adjoint<V>(op.n, op.rp, op.ci, op.va, &trp, &tci, &tva, &shared, flag, s);
  if (e) throw Err{RBICG_ERR_CUDA, "adjoint construction failed"};
  op.trp = trp; op.tci = tci; op.tva = tva; op.shared = shared;
  DevState hst;
  std::memset(&hst, 0, sizeof hst);
  hst.beta = zd(bre, bim);
  hst.kc = k;
  for (int c = 0; c < k; ++c) hst.Dc[c] = Dc_host[c];
  DevState* st = dmalloc<DevState>(1);
  RB_CUDA(cudaMemcpyAsync(st, &hst, sizeof hst, cudaMemcpyHostToDevice, s));
  const int grid = std::max(1, std::min((op.n + NTHREADS - 1) / NTHREADS, num_sms() * 8));
  Acc* part = dmalloc<Acc>(part_elems_for(grid));
  VecArgs<T> v{};
  v.n = A->n;
  v.ring = const_cast<T*>(reinterpret_cast<const T*>(r));
  v.ringt = const_cast<T*>(reinterpret_cast<const T*>(rt));
  v.ld = A->n; v.R = 1;
  v.p[0] = const_cast<T*>(reinterpret_cast<const T*>(p_old)); v.p[1] = reinterpret_cast<T*>(p_out);
  v.pt[0] = const_cast<T*>(reinterpret_cast<const T*>(pt_old)); v.pt[1] = reinterpret_cast<T*>(pt_out);
  v.z = reinterpret_cast<T*>(z); v.zt = reinterpret_cast<T*>(zt);
  // the projection pass walks the bases with a row stride that is a multiple of 4: repack
  // (zero-padded columns) when the caller's stride is not that
  const int ldp = std::max(4, ((k + 3) / 4) * 4);
  T *Cp = nullptr, *Ctp = nullptr;
  if (k > 0) {
    Cp = dmalloc<T>((size_t)A->n * ldp);
    Ctp = dmalloc<T>((size_t)A->n * ldp);
    RB_CUDA(cudaMemsetAsync(Cp, 0, sizeof(T) * A->n * ldp, s));
    RB_CUDA(cudaMemsetAsync(Ctp, 0, sizeof(T) * A->n * ldp, s));
    RB_CUDA(cudaMemcpy2DAsync(Cp, sizeof(T) * ldp, C, sizeof(T) * ldc, sizeof(T) * k, A->n, cudaMemcpyDeviceToDevice, s));
    RB_CUDA(cudaMemcpy2DAsync(Ctp, sizeof(T) * ldp, Ct, sizeof(T) * ldc, sizeof(T) * k, A->n, cudaMemcpyDeviceToDevice, s));
  }
  v.C = Cp; v.Ct = Ctp; v.ldk = ldp; v.ldc = ldp;
  launch_phase1<V, T>(op, v, st, part, kt_for(k), grid, s);
  RB_CUDA(cudaGetLastError());
  RB_CUDA(cudaMemcpyAsync(&hst, st, sizeof hst, cudaMemcpyDeviceToHost, s));
  RB_CUDA(cudaStreamSynchronize(s));
  for (int c = 0; c < k; ++c) {
    if (traits<T>::cx) {
      reinterpret_cast<zd*>(zeta_host)[c] = hst.zeta[c];
      reinterpret_cast<zd*>(zetat_host)[c] = hst.zetat[c];
    } else {
      reinterpret_cast<double*>(zeta_host)[c] = hst.zeta[c].re;
      reinterpret_cast<double*>(zetat_host)[c] = hst.zetat[c].re;
    }
  }
  cudaFree(part); cudaFree(st); cudaFree(tva); cudaFree(flag);
  if (Cp) cudaFree(Cp);
  if (Ctp) cudaFree(Ctp);
  if (!shared) { cudaFree(trp); cudaFree(tci); }
}

template <class T>
static void op_gram_impl(int64_t n, const void* X, int mx, int ldx, const void* Y, int my, int ldy, int fp32,
                         void* G_host, cudaStream_t s) {
  typedef typename traits<T>::acc Acc;
  ColList<T> xl{}, yl{};
  for (int c = 0; c < mx; ++c) { xl.c[c].p = reinterpret_cast<const T*>(X) + c; xl.c[c].ld = ldx; }
  for (int c = 0; c < my; ++c) { yl.c[c].p = reinterpret_cast<const T*>(Y) + c; yl.c[c].ld = ldy; }
  xl.m = mx; yl.m = my;
  const int gg = 2 * num_sms();
  Acc* part = dmalloc<Acc>((size_t)gg * 64 * 64);
  Acc* G = dmalloc<Acc>((size_t)mx * my);
  launch_gram<T>(xl, yl, n, fp32, part, gg, G, s);
  RB_CUDA(cudaGetLastError());
  RB_CUDA(cudaMemcpyAsync(G_host, G, sizeof(Acc) * mx * my, cudaMemcpyDeviceToHost, s));
  RB_CUDA(cudaStreamSynchronize(s));
  cudaFree(part); cudaFree(G);
}
}  // namespace rb

extern "C" rbicg_status rbicg_op_dual_spmv_project(const rbicg_csr* A, rbicg_dtype dtype, const void* r,
                                                   const void* rt, const void* p_old, const void* pt_old,
                                                   double beta_re, double beta_im, const void* C, const void* Ct,
                                                   int k, int ldc, const double* Dc_host, void* p_out, void* pt_out,
                                                   void* z, void* zt, void* zeta_host, void* zetat_host,
                                                   void* stream) {
  if (!A || !A->row_ptr || A->n <= 0 || !r || !rt || !p_old || !pt_old || !p_out || !pt_out || !z || !zt)
    return fail(nullptr, RBICG_ERR_ARG, "null argument");
  if (k < 0 || k > KMAX || (k > 0 && (!C || !Ct || !Dc_host || ldc < k || !zeta_host || !zetat_host)))
    return fail(nullptr, RBICG_ERR_ARG, "bad projection arguments");
  if (dtype == RBICG_R64 && A->val_complex) return fail(nullptr, RBICG_ERR_ARG, "complex operator, real dtype");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RB_GUARD(nullptr, {
    if (dtype == RBICG_R64)
      op_spmv_project_impl<double, double>(A, r, rt, p_old, pt_old, beta_re, beta_im, C, Ct, k, ldc, Dc_host,
                                           p_out, pt_out, z, zt, zeta_host, zetat_host, s);
    else if (A->val_complex)
      op_spmv_project_impl<cplx<double>, cplx<double>>(A, r, rt, p_old, pt_old, beta_re, beta_im, C, Ct, k, ldc,
                                                       Dc_host, p_out, pt_out, z, zt, zeta_host, zetat_host, s);
    else
      op_spmv_project_impl<double, cplx<double>>(A, r, rt, p_old, pt_old, beta_re, beta_im, C, Ct, k, ldc,
                                                 Dc_host, p_out, pt_out, z, zt, zeta_host, zetat_host, s);
    return RBICG_OK;
  })
}

extern "C" rbicg_status rbicg_op_gram(rbicg_dtype dtype, int64_t n, const void* X, int mx, int ldx, const void* Y,
                                      int my, int ldy, int fp32, void* G_host, void* stream) {
  if (n <= 0 || !X || !Y || !G_host || mx < 1 || my < 1 || mx > GRAM_MAXCOLS || my > GRAM_MAXCOLS || ldx < mx ||
      ldy < my)
    return fail(nullptr, RBICG_ERR_ARG, "bad Gram arguments (1 <= mx, my <= 176, ld >= columns)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RB_GUARD(nullptr, {
    if (dtype == RBICG_R64) op_gram_impl<double>(n, X, mx, ldx, Y, my, ldy, fp32, G_host, s);
    else op_gram_impl<cplx<double>>(n, X, mx, ldx, Y, my, ldy, fp32, G_host, s);
    return RBICG_OK;
  })
}

extern "C" rbicg_status rbicg_op_eig_select(rbicg_dtype dtype, int m, const void* L_host, const void* R_host, int k,
                                            void* W_host, void* Wt_host, double* lam_host, int* kk, void* stream) {
  if (m < 2 || m > MMAX || k < 1 || k > KMAX || k > m || !L_host || !W_host || !Wt_host || !kk)
    return fail(nullptr, RBICG_ERR_ARG, "bad eigen arguments (2 <= m <= 80, 1 <= k <= min(32, m))");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RB_GUARD(nullptr, {
    const bool cx = dtype == RBICG_C128;
    const int64_t welems = dense_work_elems();
    zd* work = dmalloc<zd>(welems);
    RB_CUDA(cudaMemsetAsync(work, 0, sizeof(zd) * welems, s));
    std::vector<zd> Lh((size_t)MMAX * MMAX), Rh((size_t)MMAX * MMAX);
    for (int c = 0; c < m; ++c)
      for (int r = 0; r < m; ++r) {
        const size_t i = (size_t)r + (size_t)c * m;
        Lh[r + (size_t)c * MMAX] = cx ? reinterpret_cast<const zd*>(L_host)[i]
                                      : zd(reinterpret_cast<const double*>(L_host)[i], 0.0);
        if (R_host)
          Rh[r + (size_t)c * MMAX] = cx ? reinterpret_cast<const zd*>(R_host)[i]
                                        : zd(reinterpret_cast<const double*>(R_host)[i], 0.0);
      }
    // work layout offsets of L and R are those of kernels_dense.cu (W_L, W_R)
    RB_CUDA(cudaMemcpyAsync(work + dense_off_L(), Lh.data(), sizeof(zd) * MMAX * MMAX, cudaMemcpyHostToDevice, s));
    if (R_host)
      RB_CUDA(cudaMemcpyAsync(work + dense_off_R(), Rh.data(), sizeof(zd) * MMAX * MMAX, cudaMemcpyHostToDevice, s));
    zd* W = dmalloc<zd>(MMAX * KMAX);
    zd* Wt = dmalloc<zd>(MMAX * KMAX);
    double* lam = dmalloc<double>(2 * KMAX + 2);
    launch_dense_eig_host(!cx, m, nullptr, nullptr, R_host != nullptr, k, W, Wt, lam, nullptr, nullptr, work, s);
    RB_CUDA(cudaGetLastError());
    DevState hst;
    std::vector<zd> Wh((size_t)MMAX * KMAX), Wth((size_t)MMAX * KMAX);
    std::vector<double> lamh(2 * KMAX + 2);
    RB_CUDA(cudaMemcpyAsync(&hst, reinterpret_cast<DevState*>(work + dense_state_offset()), sizeof hst,
                            cudaMemcpyDeviceToHost, s));
    RB_CUDA(cudaMemcpyAsync(Wh.data(), W, sizeof(zd) * MMAX * KMAX, cudaMemcpyDeviceToHost, s));
    RB_CUDA(cudaMemcpyAsync(Wth.data(), Wt, sizeof(zd) * MMAX * KMAX, cudaMemcpyDeviceToHost, s));
    RB_CUDA(cudaMemcpyAsync(lamh.data(), lam, sizeof(double) * (2 * KMAX + 2), cudaMemcpyDeviceToHost, s));
    RB_CUDA(cudaStreamSynchronize(s));
    cudaFree(work); cudaFree(W); cudaFree(Wt); cudaFree(lam);
    if (hst.eig_status != 0) {
      char buf[200];
      snprintf(buf, sizeof buf, "dense eigen solve failed: stage %d (1 LU of R, 2 QR), window [%d, %d], sweeps %d / %d",
               hst.eig_status, hst.dbg[1], hst.dbg[2], hst.dbg[3], hst.dbg[4]);
      return fail(nullptr, RBICG_ERR_EIG, buf);
    }
    *kk = hst.kk;
    for (int c = 0; c < hst.kk; ++c) {
      for (int r = 0; r < m; ++r) {
        const zd w = Wh[(size_t)r * KMAX + c], wt = Wth[(size_t)r * KMAX + c];
        if (cx) {
          reinterpret_cast<zd*>(W_host)[r + (size_t)c * m] = w;
          reinterpret_cast<zd*>(Wt_host)[r + (size_t)c * m] = wt;
        } else {
          reinterpret_cast<double*>(W_host)[r + (size_t)c * m] = w.re;
          reinterpret_cast<double*>(Wt_host)[r + (size_t)c * m] = wt.re;
        }
      }
      if (lam_host) { lam_host[2 * c] = lamh[2 * c]; lam_host[2 * c + 1] = lamh[2 * c + 1]; }
    }
    return RBICG_OK;
  })
}

extern "C" rbicg_status rbicg_op_svd(rbicg_dtype dtype, int k, const void* S_host, void* M_host, double* sigma,
                                     void* N_host, void* stream) {
  if (k < 1 || k > KMAX || !S_host || !M_host || !sigma || !N_host)
    return fail(nullptr, RBICG_ERR_ARG, "bad SVD arguments (1 <= k <= 32)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RB_GUARD(nullptr, {
    const bool cx = dtype == RBICG_C128;
    const int ld2 = 2 * k;
    std::vector<zd> S2((size_t)ld2 * ld2, zd(0.0));
    for (int c = 0; c < k; ++c) {
      for (int r = 0; r < k; ++r) {
        const size_t i = (size_t)r + (size_t)c * k;
        S2[(size_t)r * ld2 + c] = cx ? reinterpret_cast<const zd*>(S_host)[i]
                                     : zd(reinterpret_cast<const double*>(S_host)[i], 0.0);
      }
      S2[(size_t)c * ld2 + k + c] = zd(1.0);     // unit column norms: no scaling
      S2[(size_t)(k + c) * ld2 + c] = zd(1.0);
    }
    zd* S2d = dmalloc<zd>(S2.size());
    zd* Nd = dmalloc<zd>(KMAX * KMAX);
    zd* Md = dmalloc<zd>(KMAX * KMAX);
    double* sd = dmalloc<double>(KMAX);
    int* ints = dmalloc<int>(4);
    RB_CUDA(cudaMemcpyAsync(S2d, S2.data(), sizeof(zd) * S2.size(), cudaMemcpyHostToDevice, s));
    RB_CUDA(cudaMemcpyAsync(ints, &k, sizeof(int), cudaMemcpyHostToDevice, s));
    launch_dense_svd(!cx, ints, k, S2d, nullptr, nullptr, 0.0, Nd, Md, sd, ints + 1, nullptr, ints + 2, s);
    RB_CUDA(cudaGetLastError());
    std::vector<zd> Nh(KMAX * KMAX), Mh(KMAX * KMAX);
    RB_CUDA(cudaMemcpyAsync(Nh.data(), Nd, sizeof(zd) * KMAX * KMAX, cudaMemcpyDeviceToHost, s));
    RB_CUDA(cudaMemcpyAsync(Mh.data(), Md, sizeof(zd) * KMAX * KMAX, cudaMemcpyDeviceToHost, s));
    RB_CUDA(cudaMemcpyAsync(sigma, sd, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    RB_CUDA(cudaStreamSynchronize(s));
    cudaFree(S2d); cudaFree(Nd); cudaFree(Md); cudaFree(sd); cudaFree(ints);
    for (int c = 0; c < k; ++c)
      for (int r = 0; r < k; ++r) {
        const zd nv = Nh[(size_t)r * KMAX + c], mv = Mh[(size_t)r * KMAX + c];
        if (cx) {
          reinterpret_cast<zd*>(N_host)[r + (size_t)c * k] = nv;
          reinterpret_cast<zd*>(M_host)[r + (size_t)c * k] = mv;
        } else {
          reinterpret_cast<double*>(N_host)[r + (size_t)c * k] = nv.re;
          reinterpret_cast<double*>(M_host)[r + (size_t)c * k] = mv.re;
        }
      }
    return RBICG_OK;
  })
}

// ------------------------------------------------------------------ continuous batching engine
// Requests (one dual pair each, on their own handle) join and leave at cycle boundaries; every
// step advances all in-flight FP64 requests of a kind by one cycle with one batched launch per
// iteration phase.  A request's arithmetic is exactly its solo solve's (its own grid, partial
// sums and reduction order), whatever else is in flight.
struct EngineReq {
  rbicg_handle h = nullptr;
  int kind = -1;             // 0..2 FP64 solvers, 3..5 FP32 (inner solves of FP32-refined requests)
  void* solver = nullptr;    // the solver the engine steps
  cudaStream_t saved = nullptr;
  int refine = 0;            // FP32-refined request: its refinement state machine picks the solvers
  int64_t tag = 0;
};

// A cycle's batched launches (todo iterations x 2 or 3 phases) captured as a CUDA graph and
// replayed while the launch shape stays the same: the kernels read the requests' arguments from
// the stride group's device BatchArgs, which is refreshed before every replay, so a graph depends
// only on (kind, stride group, blocks, ld, kt, todo).
struct EngineGraph {
  int kind = -1, g = -1, blocks = 0, ld = 0, kt = 0, todo = 0;
  cudaGraphExec_t exec = nullptr;
  int64_t last_use = 0;
};

struct rbicg_engine_s {
  cudaStream_t s = nullptr;
  std::vector<EngineReq> active;
  std::vector<std::pair<int64_t, rbicg_result>> finished;
  std::vector<std::pair<void*, void*>> bufs[6];   // per kind: (device BatchArgs, pinned staging)
  std::string err;
  int64_t steps = 0;
  // graph capture and replay (a private stream: the engine's may be the legacy default stream)
  cudaStream_t gs = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<EngineGraph> graphs;
  bool use_graphs = getenv("RBICG_NO_GRAPHS") == nullptr;
  ~rbicg_engine_s() {
    if (s) cudaStreamSynchronize(s);
    if (gs) cudaStreamSynchronize(gs);
    for (auto& gr : graphs)
      if (gr.exec) cudaGraphExecDestroy(gr.exec);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (gs) cudaStreamDestroy(gs);
    for (auto& pool : bufs)
      for (auto& b : pool) {
        cudaFree(b.first);
        cudaFreeHost(b.second);
      }
  }
};

// Launch one stride group's cycle: replay a cached graph of the same shape, capture a new one,
// or (graphs off, or capture refused) launch the kernels one by one on the engine's stream.
template <class V, class T>
static void engine_launch_cycle(rbicg_engine e, int kind, int g, BatchArgs<V, T>* dba, int blocks, int ld, int kt,
                                int todo) {
  auto launch_all = [&](cudaStream_t st) {
    for (int t = 0; t < todo; ++t) {
      launch_phase1_batch<V, T>(dba, blocks, ld, st);
      if (kt > 0) launch_phase2_batch<V, T>(dba, blocks, kt, st);
      launch_phase3_batch<V, T>(dba, blocks, st);
    }
  };
  if (!e->use_graphs || todo <= 0) { launch_all(e->s); return; }
  if (!e->gs) {
    RB_CUDA(cudaStreamCreateWithFlags(&e->gs, cudaStreamNonBlocking));
    RB_CUDA(cudaEventCreateWithFlags(&e->ev0, cudaEventDisableTiming));
    RB_CUDA(cudaEventCreateWithFlags(&e->ev1, cudaEventDisableTiming));
  }
  EngineGraph* gr = nullptr;
  for (auto& x : e->graphs)
    if (x.kind == kind && x.g == g && x.blocks == blocks && x.ld == ld && x.kt == kt && x.todo == todo) gr = &x;
  if (!gr) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(e->gs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      e->use_graphs = false;
      launch_all(e->s);
      return;
    }
    launch_all(e->gs);
    const cudaError_t ec = cudaStreamEndCapture(e->gs, &graph);
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = ec == cudaSuccess ? cudaGraphInstantiate(&exec, graph, 0) : ec;
    if (graph) cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      cudaGetLastError();
      e->use_graphs = false;
      launch_all(e->s);
      return;
    }
    if (e->graphs.size() >= 16) {   // keep the 16 most recently used shapes
      auto old = std::min_element(e->graphs.begin(), e->graphs.end(),
                                  [](const EngineGraph& a, const EngineGraph& b) { return a.last_use < b.last_use; });
      cudaGraphExecDestroy(old->exec);
      e->graphs.erase(old);
    }
    EngineGraph ng;
    ng.kind = kind; ng.g = g; ng.blocks = blocks; ng.ld = ld; ng.kt = kt; ng.todo = todo; ng.exec = exec;
    e->graphs.push_back(ng);
    gr = &e->graphs.back();
  }
  gr->last_use = e->steps;
  RB_CUDA(cudaEventRecord(e->ev0, e->s));
  RB_CUDA(cudaStreamWaitEvent(e->gs, e->ev0, 0));
  RB_CUDA(cudaGraphLaunch(gr->exec, e->gs));
  RB_CUDA(cudaEventRecord(e->ev1, e->gs));
  RB_CUDA(cudaStreamWaitEvent(e->s, e->ev1, 0));
}

template <class V, class T>
static Solver<V, T>* as_solver(const EngineReq& q) { return static_cast<Solver<V, T>*>(q.solver); }

// A request whose solver finished its cycles: an FP64 request ends (step 7, result); an
// FP32-refined one continues its refinement and may go on with another solver (returns true:
// keep it in flight).
template <class V, class T>
static bool engine_finish(rbicg_engine e, EngineReq& q) {
  if (q.refine) {
    if (q.h->impl->refine_after(q.kind, &q.solver, &q.kind)) return true;
    q.h->impl->swap_stream(q.saved);
    q.h->err.clear();
    e->finished.push_back({q.tag, q.h->impl->refine_result()});
    return false;
  }
  Solver<V, T>* sv = as_solver<V, T>(q);
  const rbicg_result r = to_result(sv->end());
  sv->s = q.saved;
  q.h->err.clear();
  e->finished.push_back({q.tag, r});
  return false;
}

// one cycle for every in-flight request of kind (V, T): one batched launch sequence per
// basis stride (the slab projection's stride is a template parameter), one sync for all
template <class V, class T>
static void engine_step_kind(rbicg_engine e, int kind) {
  std::vector<int> idx;
  for (size_t i = 0; i < e->active.size(); ++i)
    if (e->active[i].kind == kind) idx.push_back((int)i);
  if (idx.empty()) return;
  std::vector<int> strides;
  for (int i : idx) {
    const int l = as_solver<V, T>(e->active[i])->run.v.ldc;
    if (std::find(strides.begin(), strides.end(), l) == strides.end()) strides.push_back(l);
  }
  auto& pool = e->bufs[kind];
  while (pool.size() < strides.size()) {
    void* d = dmalloc<BatchArgs<V, T>>(1);
    void* hp = nullptr;
    if (cudaMallocHost(&hp, sizeof(BatchArgs<V, T>)) != cudaSuccess) {
      cudaFree(d);
      throw Err{RBICG_ERR_OOM, "pinned batch arguments"};
    }
    pool.push_back({d, hp});
  }
  int launched = 0;
  for (size_t g = 0; g < strides.size(); ++g) {
    // the previous step's copies from these staging buffers have completed: every step ends
    // with a stream sync
    BatchArgs<V, T>* hb = static_cast<BatchArgs<V, T>*>(pool[g].second);
    auto* dba = static_cast<BatchArgs<V, T>*>(pool[g].first);
    int kt = 0, todo = 0, blocks = 0, nreq = 0;
    hb->start[0] = 0;
    for (int i : idx) {
      Solver<V, T>* q = as_solver<V, T>(e->active[i]);
      if (q->run.v.ldc != strides[g]) continue;
      hb->op[nreq] = q->op;
      hb->v[nreq] = q->run.v;
      hb->st[nreq] = q->st;
      hb->part[nreq] = q->part;
      blocks += q->grid;
      hb->start[nreq + 1] = blocks;
      ++nreq;
      kt = std::max(kt, q->run.kt);
      todo = std::max(todo, q->cycle_len());
    }
    hb->nreq = nreq;
    const int ld = kt == 0 ? 0 : strides[g];
    RB_CUDA(cudaMemcpyAsync(dba, hb, sizeof(BatchArgs<V, T>), cudaMemcpyHostToDevice, e->s));
    engine_launch_cycle<V, T>(e, kind, (int)g, dba, blocks, ld, kt, todo);
    launched += (kt > 0 ? 3 : 2) * todo;
  }
  as_solver<V, T>(e->active[idx[0]])->count(launched);
  for (int i : idx) as_solver<V, T>(e->active[i])->fetch_async();
  RB_CUDA(cudaStreamSynchronize(e->s));
  for (int i : idx) {
    Solver<V, T>* q = as_solver<V, T>(e->active[i]);
    q->prof->harvest();
    q->after_cycle();
  }
  std::vector<EngineReq> keep;
  for (size_t i = 0; i < e->active.size(); ++i) {
    EngineReq& q = e->active[i];
    if (q.kind == kind && as_solver<V, T>(q)->run.done) {
      if (engine_finish<V, T>(e, q)) keep.push_back(q);
    } else {
      keep.push_back(q);
    }
  }
  e->active.swap(keep);
}

extern "C" rbicg_status rbicg_engine_create(void* stream, rbicg_engine* out) {
  if (!out) return fail(nullptr, RBICG_ERR_ARG, "out is NULL");
  rbicg_engine e = new (std::nothrow) rbicg_engine_s();
  if (!e) return fail(nullptr, RBICG_ERR_OOM, "engine allocation failed");
  e->s = reinterpret_cast<cudaStream_t>(stream);
  *out = e;
  return RBICG_OK;
}

extern "C" rbicg_status rbicg_engine_submit(rbicg_engine e, rbicg_handle h, const rbicg_csr* A, const void* b,
                                           const void* bt, void* x, void* xt, int64_t tag) {
  if (!e || !h) return fail(h, RBICG_ERR_ARG, "engine or handle is NULL");
  if (!b || !bt || !x || !xt) return fail(h, RBICG_ERR_ARG, "null vector pointer");
  for (const EngineReq& q : e->active)
    if (q.h == h) return fail(h, RBICG_ERR_ARG, "this handle already has a request in flight");
  if ((int)e->active.size() >= BMAX) return fail(h, RBICG_ERR_ARG, "engine full (32 requests in flight)");
  RB_GUARD(h, {
    if (A) {
      const std::string m = check_csr(h, A);
      if (!m.empty()) return fail(h, RBICG_ERR_ARG, m);
      OpKey k;
      k.rp = A->row_ptr; k.ci = A->col_idx; k.va = A->val; k.n = A->n; k.nnz = A->nnz; k.has_shift = A->has_shift;
      k.val_complex = A->val_complex; k.sr = A->shift_re; k.si = A->shift_im;
      if (!h->impl || !(k == h->key)) do_update(h, A);
    }
    if (!h->impl) return fail(h, RBICG_ERR_ARG, "no operator set (pass A or call rbicg_update_recycle)");
    EngineReq q;
    q.h = h;
    q.tag = tag;
    q.solver = h->impl->batch_solver(&q.kind);
    if (!q.solver) {
      // FP32-refined request: its refinement steps run on the engine's stream; the engine steps
      // its inner FP32 solves (and a FP64 fallback solve) one cycle at a time with the others
      q.refine = 1;
      q.saved = h->impl->swap_stream(e->s);
      if (!h->impl->refine_begin(b, bt, x, xt, &q.solver, &q.kind)) {
        h->impl->swap_stream(q.saved);
        e->finished.push_back({tag, h->impl->refine_result()});
        return RBICG_OK;
      }
      e->active.push_back(q);
      return RBICG_OK;
    }
    const rbicg_params& p = h->prm;
    switch (q.kind) {
      case 0: {
        auto* sv = static_cast<Solver<double, double>*>(q.solver);
        q.saved = sv->s; sv->s = e->s;
        sv->begin((const double*)b, (const double*)bt, (double*)x, (double*)xt, p.tol, p.max_itn, p.seed);
        if (sv->run.done) { engine_finish<double, double>(e, q); return RBICG_OK; }
        break;
      }
      case 1: {
        auto* sv = static_cast<Solver<double, cplx<double>>*>(q.solver);
        q.saved = sv->s; sv->s = e->s;
        sv->begin((const zd*)b, (const zd*)bt, (zd*)x, (zd*)xt, p.tol, p.max_itn, p.seed);
        if (sv->run.done) { engine_finish<double, cplx<double>>(e, q); return RBICG_OK; }
        break;
      }
      default: {
        auto* sv = static_cast<Solver<cplx<double>, cplx<double>>*>(q.solver);
        q.saved = sv->s; sv->s = e->s;
        sv->begin((const zd*)b, (const zd*)bt, (zd*)x, (zd*)xt, p.tol, p.max_itn, p.seed);
        if (sv->run.done) { engine_finish<cplx<double>, cplx<double>>(e, q); return RBICG_OK; }
        break;
      }
    }
    e->active.push_back(q);
    return RBICG_OK;
  })
}

extern "C" rbicg_status rbicg_engine_step(rbicg_engine e, int* in_flight) {
  if (!e) return fail(nullptr, RBICG_ERR_ARG, "engine is NULL");
  try {
    engine_step_kind<double, double>(e, 0);
    engine_step_kind<double, cplx<double>>(e, 1);
    engine_step_kind<cplx<double>, cplx<double>>(e, 2);
    engine_step_kind<float, float>(e, 3);
    engine_step_kind<float, cplx<float>>(e, 4);
    engine_step_kind<cplx<float>, cplx<float>>(e, 5);
  } catch (const Err& x) {
    e->err = x.msg;
    return fail(nullptr, x.st, x.msg);
  }
  ++e->steps;
  if (in_flight) *in_flight = (int)e->active.size();
  return RBICG_OK;
}

extern "C" rbicg_status rbicg_engine_poll(rbicg_engine e, int64_t* tags, rbicg_result* res, int max, int* count) {
  if (!e || !count || max < 0 || (max > 0 && (!tags || !res))) return fail(nullptr, RBICG_ERR_ARG, "bad poll arguments");
  const int c = std::min<int>(max, (int)e->finished.size());
  for (int i = 0; i < c; ++i) {
    tags[i] = e->finished[i].first;
    res[i] = e->finished[i].second;
  }
  e->finished.erase(e->finished.begin(), e->finished.begin() + c);
  *count = c;
  return RBICG_OK;
}

extern "C" rbicg_status rbicg_engine_destroy(rbicg_engine e) {
  if (!e) return RBICG_OK;
  // requests still in flight are finished (their handles get their streams back)
  try {
    while (!e->active.empty()) {
      int n = 0;
      if (rbicg_engine_step(e, &n) != RBICG_OK) break;
    }
  } catch (...) {
  }
  delete e;
  return RBICG_OK;
}

extern "C" rbicg_status rbicg_solve_batch(rbicg_handle* hs, const rbicg_csr* const* As, const void* const* bs,
                                          const void* const* bts, void* const* xs, void* const* xts, int count,
                                          rbicg_result* res) {
  if (!hs || count < 0 || count > BMAX || (count > 0 && (!bs || !bts || !xs || !xts)))
    return fail(nullptr, RBICG_ERR_ARG, "bad batch arguments (count must be 0..32, arrays non-null)");
  if (count == 0) return RBICG_OK;
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return fail(nullptr, RBICG_ERR_ARG, "handle is NULL");
    for (int q = 0; q < i; ++q)
      if (hs[q] == hs[i]) return fail(hs[i], RBICG_ERR_ARG, "a handle appears twice in the batch");
  }
  // the whole batch through a continuous-batching engine on the first handle's stream
  rbicg_engine e = nullptr;
  rbicg_status st = rbicg_engine_create(hs[0]->s, &e);
  if (st != RBICG_OK) return st;
  std::vector<rbicg_result> out(count);
  std::vector<int> got(count, 0);
  rbicg_status err = RBICG_OK;
  for (int i = 0; i < count && err == RBICG_OK; ++i) {
    st = rbicg_engine_submit(e, hs[i], As ? As[i] : nullptr, bs[i], bts[i], xs[i], xts[i], i);
    if (st < 0) err = st;
  }
  int in_flight = 1;
  while (err == RBICG_OK && in_flight > 0) {
    st = rbicg_engine_step(e, &in_flight);
    if (st < 0) err = st;
  }
  std::vector<int64_t> tags(count);
  std::vector<rbicg_result> rr(count);
  int c = 0;
  rbicg_engine_poll(e, tags.data(), rr.data(), count, &c);
  for (int i = 0; i < c; ++i) {
    out[tags[i]] = rr[i];
    got[tags[i]] = 1;
  }
  const std::string keep = g_last_error;
  rbicg_engine_destroy(e);
  if (err < 0) {
    g_last_error = keep;
    return err;
  }
  rbicg_status worst = RBICG_OK;
  for (int i = 0; i < count; ++i) {
    if (res) res[i] = out[i];
    if (!got[i]) return fail(hs[i], RBICG_ERR_CUDA, "batch request did not finish");
    if (out[i].status < 0) return fail(hs[i], (rbicg_status)out[i].status, "non-finite value in the iteration");
    if (out[i].status > worst) worst = (rbicg_status)out[i].status;
  }
  return worst;
}


// ------------------------------------------------------------------ autotuner
struct TuneKey {
  int64_t n, nnz;
  int dtype, vc, k;
  bool operator<(const TuneKey& o) const {
    if (n != o.n) return n < o.n;
    if (nnz != o.nnz) return nnz < o.nnz;
    if (dtype != o.dtype) return dtype < o.dtype;
    if (vc != o.vc) return vc < o.vc;
    return k < o.k;
  }
};
static std::map<TuneKey, std::pair<int, double>> g_tune;
static std::mutex g_tune_mu;

extern "C" rbicg_status rbicg_autotune(const rbicg_params* params, rbicg_dtype dtype, const rbicg_csr* A,
                                       int trial_iters, int* grid_blocks, double* us_per_iter) {
  if (!params || !A || !grid_blocks) return fail(nullptr, RBICG_ERR_ARG, "null argument");
  if (dtype != RBICG_R64 && dtype != RBICG_C128) return fail(nullptr, RBICG_ERR_ARG, "unknown dtype");
  const std::string m = check_params(params, A->n);
  if (!m.empty()) return fail(nullptr, RBICG_ERR_ARG, m);
  if (trial_iters < 4 || trial_iters > 100000) return fail(nullptr, RBICG_ERR_ARG, "trial_iters must be in 4..100000");
  const TuneKey key{A->n, A->nnz, (int)dtype, A->val_complex ? 1 : 0, params->k};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      *grid_blocks = it->second.first;
      if (us_per_iter) *us_per_iter = it->second.second;
      return RBICG_OK;
    }
  }
  const int64_t n = A->n;
  const size_t w = dtype == RBICG_C128 ? sizeof(zd) : sizeof(double);
  cudaStream_t s = nullptr;
  void* buf = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return fail(nullptr, RBICG_ERR_CUDA, "autotune stream");
  if (cudaMalloc(&buf, 4 * w * (size_t)n) != cudaSuccess) {
    cudaStreamDestroy(s);
    return fail(nullptr, RBICG_ERR_OOM, "autotune vectors");
  }
  char* b = static_cast<char*>(buf);
  char* bt = b + w * n;
  char* x = bt + w * n;
  char* xt = x + w * n;
  if (dtype == RBICG_C128) {
    launch_philox<cplx<double>>(reinterpret_cast<zd*>(b), n, 1, s);
    launch_philox<cplx<double>>(reinterpret_cast<zd*>(bt), n, 2, s);
  } else {
    launch_philox<double>(reinterpret_cast<double*>(b), n, 1, s);
    launch_philox<double>(reinterpret_cast<double*>(bt), n, 2, s);
  }
  const int sms = num_sms();
  const int64_t cap = std::max<int64_t>(1, (n + NTHREADS - 1) / NTHREADS);
  std::vector<int> cand;
  for (int f : {1, 2, 3, 4, 6, 8, 16}) {
    const int g = (int)std::min<int64_t>(cap, (int64_t)f * sms);
    if (std::find(cand.begin(), cand.end(), g) == cand.end()) cand.push_back(g);
  }
  int best = 0;
  double best_us = 1e300;
  rbicg_status err = RBICG_OK;
  for (int g : cand) {
    rbicg_params q = *params;
    q.grid_blocks = g;
    q.recycle = 0;                 // plain iterations: the phases' SpMV and vector sweeps
    q.tol = 1e-300;                // never met: exactly trial_iters iterations
    q.max_itn = trial_iters;
    q.precision = RBICG_FP64;
    rbicg_handle h = nullptr;
    rbicg_status st = rbicg_create(&q, n, dtype, s, &h);
    if (st != RBICG_OK) { err = st; break; }
    double t = 0.0;
    for (int rep = 0; rep < 2 && st >= 0; ++rep) {   // the first solve warms up (and builds A^H)
      cudaMemsetAsync(x, 0, 2 * w * (size_t)n, s);
      cudaStreamSynchronize(s);
      const auto t0 = std::chrono::steady_clock::now();
      rbicg_result r{};
      st = rbicg_solve_pair(h, A, b, bt, x, xt, &r);
      cudaStreamSynchronize(s);
      t = std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count() /
          std::max(1, r.iters);
    }
    rbicg_destroy(h);
    if (st < 0) { err = st; break; }
    if (t < best_us) { best_us = t; best = g; }
  }
  cudaFree(buf);
  cudaStreamDestroy(s);
  if (err < 0) return err;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = {best, best_us};
  }
  *grid_blocks = best;
  if (us_per_iter) *us_per_iter = best_us;
  return RBICG_OK;
}

extern "C" rbicg_status rbicg_autotune_params(const rbicg_params* params, rbicg_dtype dtype, const rbicg_csr* A,
                                              int trial_iters, rbicg_params* out, double* us_per_iter) {
  if (!params || !A || !out) return fail(nullptr, RBICG_ERR_ARG, "null argument");
  if (dtype != RBICG_R64 && dtype != RBICG_C128) return fail(nullptr, RBICG_ERR_ARG, "unknown dtype");
  const std::string m = check_params(params, A->n);
  if (!m.empty()) return fail(nullptr, RBICG_ERR_ARG, m);
  int g = 0;
  double us = 0.0;
  rbicg_status st = rbicg_autotune(params, dtype, A, std::max(4, trial_iters), &g, &us);
  if (st < 0) return st;
  rbicg_params best = *params;
  best.grid_blocks = g;
  const int64_t n = A->n;
  const size_t w = dtype == RBICG_C128 ? sizeof(zd) : sizeof(double);
  cudaStream_t s = nullptr;
  void* buf = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return fail(nullptr, RBICG_ERR_CUDA, "autotune stream");
  if (cudaMalloc(&buf, 4 * w * (size_t)n) != cudaSuccess) {
    cudaStreamDestroy(s);
    return fail(nullptr, RBICG_ERR_OOM, "autotune vectors");
  }
  char* b = static_cast<char*>(buf);
  char* bt = b + w * n;
  char* x = bt + w * n;
  char* xt = x + w * n;
  if (dtype == RBICG_C128) {
    launch_philox<cplx<double>>(reinterpret_cast<zd*>(b), n, 1, s);
    launch_philox<cplx<double>>(reinterpret_cast<zd*>(bt), n, 2, s);
  } else {
    launch_philox<double>(reinterpret_cast<double*>(b), n, 1, s);
    launch_philox<double>(reinterpret_cast<double*>(bt), n, 2, s);
  }
  const int sms = num_sms();
  double best_us = 1e300;
  rbicg_status err = RBICG_OK;
  for (int f : {8, 4, 12}) {
    for (int gr : {1, 0}) {
      rbicg_params q = best;
      q.setup_blocks = f * sms;
      q.graphs = gr;
      q.recycle = 1;
      q.refresh = 1;
      q.guard = 0.0;
      q.tol = 1e-300;            // never met: exactly three cycles per solve
      q.max_itn = 3 * q.s;
      q.precision = RBICG_FP64;
      rbicg_handle h = nullptr;
      st = rbicg_create(&q, n, dtype, s, &h);
      if (st != RBICG_OK) { err = st; break; }
      double t = 0.0;
      // the first solve builds A^H and a recycle space; the second runs recycled iterations and
      // their refreshes, and is timed
      for (int rep = 0; rep < 2 && st >= 0; ++rep) {
        cudaMemsetAsync(x, 0, 2 * w * (size_t)n, s);
        cudaStreamSynchronize(s);
        const auto t0 = std::chrono::steady_clock::now();
        rbicg_result r{};
        st = rbicg_solve_pair(h, A, b, bt, x, xt, &r);
        cudaStreamSynchronize(s);
        t = std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count() /
            std::max(1, r.iters);
      }
      rbicg_destroy(h);
      if (st < 0) { err = st; break; }
      if (t < best_us) {
        best_us = t;
        best.setup_blocks = q.setup_blocks;
        best.graphs = gr;
      }
    }
    if (err < 0) break;
  }
  cudaFree(buf);
  cudaStreamDestroy(s);
  if (err < 0) return err;
  *out = best;
  if (us_per_iter) *us_per_iter = best_us;
  return RBICG_OK;
}
