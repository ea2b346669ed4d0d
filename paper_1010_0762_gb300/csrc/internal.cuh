// internal.cuh -- device state, kernel argument blocks and launcher declarations.
#pragma once
#include "common.cuh"

namespace rb {

constexpr int KMAX = 32;          // largest recycle dimension k
constexpr int SMAX = 64;          // largest cycle length s
constexpr int MMAX = 80;          // largest pencil order (k + s)
constexpr int HR = 2 * SMAX + 4;  // history ring length (iteration scalars)
constexpr int NTHREADS = 256;     // threads per block of the streaming kernels
constexpr double BREAKDOWN_EPS = 1e-14;
constexpr int GMAX = 1024;        // block groups of the two-level grid reduction (iteration kernels)
constexpr int RCNT = 2 * KMAX + 2;  // widest row of per-block partial sums

// Blocks of one solve form groups of consecutive ids for the two-level grid reduction: 32 a
// group, or more when the grid has more than 32 * GMAX blocks.
RB_HD int group_size(int nblk) {
  return nblk <= 32 * GMAX ? 32 : ((nblk + GMAX - 1) / GMAX + 31) / 32 * 32;
}
RB_HD int group_count(int nblk) { return (nblk + group_size(nblk) - 1) / group_size(nblk); }
// Elements of the per-solve partial-sum buffer of the iteration kernels: one row per block and
// one per group, RCNT wide.
inline size_t part_elems_for(int nblk) { return ((size_t)nblk + group_count(nblk)) * RCNT; }

// done codes (DevState::done)
enum { RUNNING = 0, DONE_CONVERGED = 1, DONE_BREAK_RHO = 2, DONE_BREAK_PQ = 3, DONE_MAXIT = 4,
       DONE_NONFINITE = 5 };

typedef cplx<double> zd;

// Per-solve device state: iteration scalars of Algorithm 2, the projection coefficients and
// the scalar histories that the Section 4 refresh needs (indexed by iteration mod HR).
struct DevState {
  // ---- fields read by the host after a sync: kept first and contiguous (one copy) ----
  int iter;           // completed iterations
  int done;           // RUNNING or a DONE_* code
  int kc;             // columns of C, Ct in use (recycle dimension p of this system)
  int restart;        // 1 when (r_0, rt_0) ~ 0 (Algorithm 2 step 3)
  int kk;             // eigenvectors selected by the last refresh
  int pcyc;           // columns kept by the last refresh's SVD truncation
  int eig_status;     // 0 ok, else the dense solve failed
  int max_itn;
  double rnorm, rtnorm;          // recurrence residual norms of the last iteration
  double bnorm, btnorm;
  double true_rnorm, true_rtnorm;
  // ---- device-only ----
  double tol;
  zd rho;             // rho_{i} of the last completed iteration: (rt_i, r_i)
  zd alpha;           // alpha_i of the iteration in flight
  zd beta;            // beta of the last completed iteration (used by the next p update)
  int refresh_ok;
  int nonfinite;
  int dbg[8];                    // diagnostics of the last dense failure (stage, window, counts)
  unsigned int cnt[8];           // last-block counters (one-level reductions)
  unsigned int gcnt[GMAX + 1];   // group counters and the final counter of the two-level reduction
  zd zeta[KMAX], zetat[KMAX];    // zeta_i, zetat_i (Algorithm 2)
  zd zeta_c[KMAX], zetat_c[KMAX];
  zd coef[KMAX], coeft[KMAX];    // initial projection coefficients (eq. (minusXR))
  double Dc[KMAX];               // D_c = Ct^H C (real, positive)
  zd h_alpha[HR], h_beta[HR], h_rho[HR];
  double h_rnorm[HR];
  zd h_zeta[HR][KMAX], h_zetat[HR][KMAX];
};

template <class T> RB_HD T from_zd(zd v);
template <> RB_HD double from_zd<double>(zd v) { return v.re; }
template <> RB_HD float from_zd<float>(zd v) { return (float)v.re; }
template <> RB_HD cplx<double> from_zd<cplx<double>>(zd v) { return v; }
template <> RB_HD cplx<float> from_zd<cplx<float>>(zd v) { return cplx<float>((float)v.re, (float)v.im); }
RB_HD zd to_zd(double v) { return zd(v, 0.0); }
RB_HD zd to_zd(zd v) { return v; }

// Operator description used by every kernel that applies Op = A or (shift I - A) and Op^H.
template <class V>
struct OpArgs {
  int n;
  const int* rp; const int* ci; const V* va;     // A, CSR
  const int* trp; const int* tci; const V* tva;  // A^H, CSR (conjugated transposed values)
  int shared;                                    // trp == rp and tci == ci
  int has_shift; double sh_re, sh_im;
  int bw = -1;          // bandwidth max |j - i| over the nonzeros (the same for A^H); <= 0: unknown
  int stage_rows = 0;   // phase 1 (one solve's launch, real types): rows of p and pt its dynamic
                        // shared memory holds per side; 0: no staging
};

// Vectors of one solve.
template <class T>
struct VecArgs {
  int64_t n;                                     // rows
  T* ring; T* ringt; int64_t ld; int R;          // residual rings: r_m at slot m mod R
  T* p[2]; T* pt[2];                             // p_i at p[i & 1]
  T* z; T* zt;                                   // z_i (overwritten by q_i)
  T* x; T* xt;                                   // iterates (caller buffers)
  const T* b; const T* bt;
  const T* C; const T* Ct; const T* U; const T* Ut; int ldk;   // n x ldk row-major bases U, Ut
  int ldc;   // row stride of C, Ct as the iteration kernels see them: the system's kc columns
             // rounded up to 4 (a compact copy when that is below ldk), so the projections
             // skip the columns the Section 4.3 truncation dropped
};

// Per-request arguments of a batched iteration launch: request r owns the blocks
// [start[r], start[r + 1]) of the grid.  Lives in device memory.
constexpr int BMAX = 32;
template <class V, class T>
struct BatchArgs {
  OpArgs<V> op[BMAX];
  VecArgs<T> v[BMAX];
  DevState* st[BMAX];
  void* part[BMAX];
  int start[BMAX + 1];
  int nreq;
};

// Column source of a tall-skinny product: column c of a row-major block (stride ld) or a
// plain vector (stride 1), scaled on the dense side.
template <class T>
struct ColSrc { const T* p; int ld; };

constexpr int GRAM_MAXCOLS = 176;   // columns of X or Y in one Gram call

template <class T>
struct ColList { int m; ColSrc<T> c[GRAM_MAXCOLS]; };

// ---- launchers (kernels_iter.cu) ----
template <class V, class T>
void launch_phase1_batch(const BatchArgs<V, T>* ba, int blocks, int ld, cudaStream_t s);
template <class V, class T>
void launch_phase2_batch(const BatchArgs<V, T>* ba, int blocks, int kt, cudaStream_t s);
template <class V, class T>
void launch_phase3_batch(const BatchArgs<V, T>* ba, int blocks, cudaStream_t s);
template <class V, class T>
void launch_phase1(const OpArgs<V>& op, const VecArgs<T>& v, DevState* st, void* part, int kt, int grid,
                   cudaStream_t s);
template <class V, class T>
void launch_phase2(const OpArgs<V>& op, const VecArgs<T>& v, DevState* st, void* part, int kt, int grid,
                   cudaStream_t s);
template <class V, class T>
void launch_phase3(const OpArgs<V>& op, const VecArgs<T>& v, DevState* st, void* part, int grid,
                   cudaStream_t s);
template <class V, class T>
void launch_init(const OpArgs<V>& op, const VecArgs<T>& v, DevState* st, void* part, int kt, int grid,
                 int dual_only, cudaStream_t s);
template <class V, class T>
void launch_finish(const OpArgs<V>& op, const VecArgs<T>& v, DevState* st, void* part, int kt, int grid,
                   cudaStream_t s);
template <class T>
void launch_finish_a(const VecArgs<T>& v, DevState* st, int kt, int grid, cudaStream_t s);   // x -= U zeta_c
template <class T>
void launch_philox(T* out, int64_t n, uint64_t seed, cudaStream_t s);
template <class V>
int build_adjoint(int n, const int* rp, const int* ci, const V* va, int** trp, int** tci, V** tva,
                  int* shared, int* flag_dev, cudaStream_t s);   // returns 0 or a cuda error
int validate_csr(int n, int64_t nnz, const int* rp, const int* ci, int* flag_dev, cudaStream_t s);
// bandwidth of a CSR pattern (max |col - row| over its nonzeros) into *bw; returns 0 or a cuda error
int csr_bandwidth(int n, const int* rp, const int* ci, int* flag_dev, cudaStream_t s, int* bw);
// sets the phase-1 kernels' dynamic shared memory limit (call outside stream capture)
template <class V, class T>
void prepare_phase1();

// ---- launchers (kernels_basis.cu) ----
template <class T>
void launch_gram(const ColList<T>& X, const ColList<T>& Y, int64_t n, int fp32, void* part, int grid,
                 typename traits<T>::acc* G, cudaStream_t s);
template <class T>
void launch_combine(const ColList<T>& src, const zd* W, int ldw, const int* ncols_dev, int ncols_max, T* out,
                    int ldo, int64_t n, int fp32, cudaStream_t s);
template <class V, class T>
void launch_spmm(const OpArgs<V>& op, int adjoint, const T* U, int ldu, const int* ncols_dev, int ncols_max,
                 T* out, int fp32, cudaStream_t s);
template <class T>
void launch_rotate(T* B, int ld, const zd* Nmat, const int* kin_dev, const int* kout_dev, int kmax, int64_t n,
                   int fp32, cudaStream_t s);
// SVD input of Section 4.3: S = Ct^H C (k x k, FP64) and the column norms of C and Ct, packed into
// the 2 kmax x 2 kmax array the dense SVD reads.  part: Gram partials (grid x 32 x 32 accumulators)
// followed by 64 x grid doubles.
template <class T>
void launch_svd_input(const T* C, const T* Ct, int ld, int k, int kmax, int64_t n, void* part, int grid,
                      typename traits<T>::acc* G, zd* S2, cudaStream_t s);
template <class Tfrom, class Tto>
void launch_convert(const Tfrom* a, Tto* b, int64_t n, cudaStream_t s);
template <class T>
void launch_pack_cols(const T* src, int lds, T* dst, int ldd, int kc, int64_t n, cudaStream_t s);   // dst[:, :ldd] = [src[:, :kc] 0]
template <class T>
void launch_axpy_inplace(T* y, const T* x, int64_t n, cudaStream_t s);   // y += x

// ---- dense (kernels_dense.cu) ----
struct RefreshInfo {
  int case_id;       // 0 first system/first cycle (T_1); 1 first system j>=2; 2 later j=1; 3 later j>=2
  int j, s, k;       // cycle index, cycle length, requested recycle dimension
  int kc;            // columns of C (system)
  int kp;            // columns of U_{j-1}
  int real_path;
  int R;             // residual ring length
  int mx, my;        // Gram dimensions (Psit columns, [Psi U_{j-1}] columns)
};
template <class T>
void launch_dense_refresh(const RefreshInfo& info, DevState* st, const typename traits<T>::acc* G, zd* work,
                          zd* Wphi, zd* Wphit, int ldw, double* lam_out, cudaStream_t s);
void launch_dense_svd(int real_path, const int* k_dev, int kmax, const zd* S, const double* nC, const double* nCt,
                      double svd_tol, zd* Nmat, zd* Mmat, double* sigma, int* p_dev, double* Dc_dev,
                      int* status_dev, cudaStream_t s);
void launch_dense_eig_host(int real_path, int m, const zd* L, const zd* R, int has_R, int k, zd* W, zd* Wt,
                          double* lam, int* kk, int* status, zd* work, cudaStream_t s);

}  // namespace rb
