// apps.cu -- what the paper builds on top of solved dual pairs: bilinear forms u^H A^{-1} w
// (Section 1) and the IRKA outer loop of Algorithm 3 (Section 5) with the recycling strategies
// of Section 5.3.  The shifted dual solves go through the library's own entry points
// (rbicg_solve_batch / rbicg_solve_pair on handles that carry the recycle spaces); the reduced
// model and its eigenvalues are formed on the device (SpMV, Gram and dense eigen kernels).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rbicg.h"
#include "internal.cuh"

namespace rb {

void set_global_error(const char* msg);   // engine.cu: message of rbicg_last_error(NULL)
int64_t dense_state_offset();
int64_t dense_work_elems();
int64_t dense_off_L();
int64_t dense_off_R();

// ------------------------------------------------------------------------------------
// Bilinear forms (Section 1): per block, the three sums u^H x, xt^H w and xt^H (w - Op x)
// over a grid-stride range of rows; then one block adds the block rows in id order.
// ------------------------------------------------------------------------------------
template <class V, class T>
__global__ void __launch_bounds__(256) k_bilinear(OpArgs<V> op, const T* __restrict__ u, const T* __restrict__ w,
                                                  const T* __restrict__ x, const T* __restrict__ xt,
                                                  typename traits<T>::acc* part) {
  typedef typename traits<T>::acc A;
  __shared__ A sm[3 * (256 / 32)];
  A v[3] = {A(0.0), A(0.0), A(0.0)};
  const T sh = from_zd<T>(zd(op.sh_re, op.sh_im));
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < op.n; row += gridDim.x * blockDim.x) {
    T ax = T(0);
    for (int e = op.rp[row]; e < op.rp[row + 1]; ++e) ax += vmul(op.va[e], x[op.ci[e]]);
    if (op.has_shift) ax = sh * x[row] - ax;
    const T r = w[row] - ax;
    v[0] += cvt<A>(cmul(u[row], x[row]));
    v[1] += cvt<A>(cmul(xt[row], w[row]));
    v[2] += cvt<A>(cmul(xt[row], r));
  }
  block_sum_vec(v, 3, sm);
  if (threadIdx.x < 3) part[blockIdx.x * 3 + threadIdx.x] = sm[threadIdx.x];
}

// one thread adds the block rows in id order: out = (u^H x, xt^H w, u^H x + xt^H (w - Op x))
template <class A>
__global__ void k_bilinear_final(const A* part, int nblk, A* out) {
  if (threadIdx.x == 0) {
    A t[3] = {A(0.0), A(0.0), A(0.0)};
    for (int b = 0; b < nblk; ++b)
      for (int i = 0; i < 3; ++i) t[i] += part[b * 3 + i];
    out[0] = t[0];
    out[1] = t[1];
    out[2] = t[0] + t[2];
  }
}

static int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

template <class V, class T>
static cudaError_t bilinear_impl(const rbicg_csr* A, const void* u, const void* w, const void* x, const void* xt,
                                 double* out_host, cudaStream_t s) {
  typedef typename traits<T>::acc Acc;
  OpArgs<V> op{};
  op.n = (int)A->n; op.rp = A->row_ptr; op.ci = A->col_idx; op.va = reinterpret_cast<const V*>(A->val);
  op.has_shift = A->has_shift; op.sh_re = A->shift_re; op.sh_im = A->shift_im;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((A->n + 255) / 256, 2 * sm_count()));
  Acc* part = nullptr;
  cudaError_t e = cudaMalloc(&part, sizeof(Acc) * (3 * grid + 3));
  if (e != cudaSuccess) return e;
  Acc* out = part + 3 * grid;
  k_bilinear<V, T><<<grid, 256, 0, s>>>(op, reinterpret_cast<const T*>(u), reinterpret_cast<const T*>(w),
                                        reinterpret_cast<const T*>(x), reinterpret_cast<const T*>(xt), part);
  k_bilinear_final<Acc><<<1, 32, 0, s>>>(part, grid, out);
  Acc h[3];
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(part);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < 3; ++i) {
    const zd z = to_zd(h[i]);
    out_host[2 * i] = z.re;
    out_host[2 * i + 1] = z.im;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------------------------------
// IRKA (Algorithm 3) device helpers
// ------------------------------------------------------------------------------------
// dst = conj(src): the solution of the conjugate shift (real A, b, c)
__global__ void k_conj_copy(const zd* src, zd* dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = conjg(src[i]);
}

__global__ void k_widen(const double* a, zd* b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = zd(a[i], 0.0);
}

// AV[:, c] = A V[:, c] for c < r (V, AV column-major n x r; A real CSR)
__global__ void k_apply_cols(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                             const double* __restrict__ va, const zd* __restrict__ V, zd* __restrict__ AV, int r) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * r;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / n), row = (int)(e % n);
    const zd* v = V + (int64_t)c * n;
    zd acc(0.0);
    for (int q = rp[row]; q < rp[row + 1]; ++q) acc += vmul(va[q], v[ci[q]]);
    AV[(int64_t)c * n + row] = acc;
  }
}

// G (row-major 2r x (2r+2): rows W^H, V^H; columns AV, V, b, c) -> the pencil (A_r, E_r) in the
// dense work area (column-major, leading dimension MMAX), and b_r, c_r
__global__ void k_pencil(const zd* G, int r, zd* L, zd* R, zd* br, zd* cr) {
  const int w = 2 * r + 2;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int a = e / r, b = e % r;
    L[a + (size_t)b * MMAX] = G[a * w + b];
    R[a + (size_t)b * MMAX] = G[a * w + r + b];
  }
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    br[a] = G[a * w + 2 * r];
    cr[a] = G[(r + a) * w + 2 * r + 1];
  }
}

typedef std::complex<double> cd;

// Reading of "appropriately ordered" shifts (Section 5.3): ascending modulus, the larger
// imaginary part first among equal moduli (a conjugate pair is adjacent, + before -).
static std::vector<int> shift_order(const std::vector<cd>& s) {
  std::vector<int> idx(s.size());
  for (size_t i = 0; i < s.size(); ++i) idx[i] = (int)i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
    const double ma = std::abs(s[a]), mb = std::abs(s[b]);
    if (ma != mb) return ma < mb;
    if (s[a].imag() != s[b].imag()) return s[a].imag() > s[b].imag();
    return s[a].real() < s[b].real();
  });
  return idx;
}

// For real A, b, c the shift set is closed under conjugation in exact arithmetic.  An
// eigenvalue whose nearest other eigenvalue to its conjugate lies closer to that conjugate than
// the eigenvalue lies to the real axis is paired with it (both become the mean of one and the
// conjugate of the other); an eigenvalue without such a partner becomes its real part.
static std::vector<cd> conjugate_close(const std::vector<cd>& lam) {
  const size_t m = lam.size();
  std::vector<cd> out(m);
  std::vector<char> done(m, 0);
  for (size_t i = 0; i < m; ++i) {
    if (done[i]) continue;
    int best = -1;
    double bd = 0.0;
    for (size_t j = 0; j < m; ++j) {
      if (done[j] || j == i) continue;
      const double d = std::abs(lam[j] - std::conj(lam[i]));
      if (d < std::fabs(lam[i].imag()) && (best < 0 || d < bd)) { best = (int)j; bd = d; }
    }
    if (best < 0) {
      out[i] = cd(lam[i].real(), 0.0);
      done[i] = 1;
      continue;
    }
    const cd mean = 0.5 * (lam[i] + std::conj(lam[best]));
    out[i] = mean;
    out[best] = std::conj(mean);
    done[i] = done[best] = 1;
  }
  return out;
}

struct IrkaErr {
  rbicg_status st;
  std::string msg;
};

#define IR_CUDA(call)                                                                         \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      throw IrkaErr{e_ == cudaErrorMemoryAllocation ? RBICG_ERR_OOM : RBICG_ERR_CUDA,         \
                    std::string(#call) + ": " + cudaGetErrorString(e_)};                      \
  } while (0)
#define IR_CALL(call, h)                                                                      \
  do {                                                                                        \
    rbicg_status s_ = (call);                                                                 \
    if (s_ < 0) throw IrkaErr{s_, std::string(#call) + ": " + rbicg_last_error(h)};           \
  } while (0)

template <class P>
static P* ir_alloc(size_t count) {
  void* p = nullptr;
  IR_CUDA(cudaMalloc(&p, std::max<size_t>(1, count) * sizeof(P)));
  return static_cast<P*>(p);
}

// Device buffers and handles of one IRKA run; frees everything on destruction.
struct IrkaRun {
  std::vector<void*> bufs;
  std::vector<rbicg_handle> handles;
  template <class P>
  P* alloc(size_t count) {
    P* p = ir_alloc<P>(count);
    bufs.push_back(p);
    return p;
  }
  ~IrkaRun() {
    for (rbicg_handle h : handles) rbicg_destroy(h);
    for (void* p : bufs) cudaFree(p);
  }
};

}  // namespace rb

using namespace rb;

extern "C" void rbicg_irka_default_params(rbicg_irka_params* p) {
  if (!p) return;
  p->r = 8;
  p->max_steps = 10;
  p->shift_tol = 1e-6;
  p->strategy = 1;
  p->recycle_count = 0;
  p->refresh_every = 1;
  p->pool_tol = 0.5;
  p->batched = 1;
  p->conj_pairs = 1;
}

extern "C" rbicg_status rbicg_bilinear_form(const rbicg_csr* A, rbicg_dtype dtype, const void* u, const void* w,
                                            const void* x, const void* xt, double* out_host, void* stream) {
  if (!A || !A->row_ptr || A->n <= 0 || (A->nnz > 0 && (!A->col_idx || !A->val)) || !u || !w || !x || !xt ||
      !out_host) {
    set_global_error("rbicg_bilinear_form: null argument or n <= 0");
    return RBICG_ERR_ARG;
  }
  if (dtype == RBICG_R64 && (A->val_complex || (A->has_shift && A->shift_im != 0.0))) {
    set_global_error("rbicg_bilinear_form: complex operator or shift with real vectors");
    return RBICG_ERR_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (dtype == RBICG_R64) e = bilinear_impl<double, double>(A, u, w, x, xt, out_host, s);
  else if (A->val_complex) e = bilinear_impl<zd, zd>(A, u, w, x, xt, out_host, s);
  else e = bilinear_impl<double, zd>(A, u, w, x, xt, out_host, s);
  if (e != cudaSuccess) {
    set_global_error(cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? RBICG_ERR_OOM : RBICG_ERR_CUDA;
  }
  return RBICG_OK;
}

extern "C" rbicg_status rbicg_irka(const rbicg_params* sp, const rbicg_irka_params* ip, const rbicg_csr* A,
                                   const double* b, const double* c, const double* shifts_in, void* stream,
                                   double* shifts_out, double* Ar_out, double* Er_out, double* br_out, double* cr_out,
                                   int* iters_out, rbicg_irka_result* res) {
  if (!sp || !ip || !A || !A->row_ptr || A->n <= 0 || !A->col_idx || !A->val || !b || !c || !shifts_in ||
      !shifts_out || !res) {
    set_global_error("rbicg_irka: null argument");
    return RBICG_ERR_ARG;
  }
  const int r = ip->r;
  if (r < 1 || r > KMAX || ip->max_steps < 1 || !(ip->shift_tol > 0.0) || ip->strategy < 0 || ip->strategy > 4 ||
      ip->recycle_count < 0 || ip->refresh_every < 1 || !(ip->pool_tol > 0.0) ||
      (ip->conj_pairs != 0 && ip->conj_pairs != 1)) {
    set_global_error("rbicg_irka: need 1 <= r <= 32, max_steps >= 1, shift_tol > 0, strategy 0..4, "
                     "recycle_count >= 0, refresh_every >= 1, pool_tol > 0, conj_pairs 0 or 1");
    return RBICG_ERR_ARG;
  }
  if (A->val_complex || A->has_shift) {
    set_global_error("rbicg_irka: A must be a real operator without a shift (the solves use sigma I - A)");
    return RBICG_ERR_ARG;
  }
  std::memset(res, 0, sizeof(*res));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = A->n;
  try {
    IrkaRun run;
    // device buffers: V, W (n x r column-major, also the initial guesses of the next step's
    // solves, Section 6.2), A V, b and c widened to complex
    zd* V = run.alloc<zd>((size_t)n * r);
    zd* W = run.alloc<zd>((size_t)n * r);
    zd* AV = run.alloc<zd>((size_t)n * r);
    zd* bz = run.alloc<zd>(n);
    zd* cz = run.alloc<zd>(n);
    IR_CUDA(cudaMemsetAsync(V, 0, sizeof(zd) * n * r, s));
    IR_CUDA(cudaMemsetAsync(W, 0, sizeof(zd) * n * r, s));
    const int g1 = (int)std::min<int64_t>((n + 255) / 256, 4 * sm_count());
    k_widen<<<g1, 256, 0, s>>>(b, bz, n);
    k_widen<<<g1, 256, 0, s>>>(c, cz, n);
    const int gram_grid = 2 * sm_count();
    zd* gpart = run.alloc<zd>((size_t)gram_grid * 64 * 64);
    zd* G = run.alloc<zd>((size_t)(2 * r) * (2 * r + 2));
    const int64_t welems = dense_work_elems();
    zd* work = run.alloc<zd>(welems);
    IR_CUDA(cudaMemsetAsync(work, 0, sizeof(zd) * welems, s));
    zd* Wev = run.alloc<zd>(MMAX * KMAX);
    zd* Wtev = run.alloc<zd>(MMAX * KMAX);
    double* lam = run.alloc<double>(2 * KMAX + 2);
    zd* brc = run.alloc<zd>(2 * KMAX);

    // handles: strategies 0, 1 and 4 one per shift index; strategies 2 and 3 one that carries (or
    // receives) the recycle space from solve to solve, plus one without recycling for the shift
    // indices beyond recycle_count
    rbicg_params pr = *sp;
    rbicg_params pp = *sp;
    pp.recycle = 0;
    const int nrec = ip->recycle_count > 0 ? std::min(ip->recycle_count, r) : r;
    auto make = [&](const rbicg_params& q) {
      rbicg_handle h = nullptr;
      IR_CALL(rbicg_create(&q, n, RBICG_C128, stream, &h), nullptr);
      run.handles.push_back(h);
      return h;
    };
    std::vector<rbicg_handle> hidx(r, nullptr);
    rbicg_handle hrec = nullptr, hplain = nullptr;
    const bool per_index = ip->strategy <= 1 || ip->strategy == 4;
    if (per_index) {
      for (int i = 0; i < r; ++i) hidx[i] = make((ip->strategy == 1 || ip->strategy == 4) && i < nrec ? pr : pp);
    } else {
      hrec = make(pr);
      if (nrec < r) hplain = make(pp);
    }
    // strategy 3: pooled spaces of the previous step and of the current step so far
    const int kk = sp->k;
    struct Slot { cd sigma; int p; zd* U; zd* Ut; };
    std::vector<Slot> pool_prev, pool_cur;
    std::vector<zd*> slot_bufs;
    zd* tmpU = nullptr;
    zd* tmpUt = nullptr;
    if (ip->strategy == 3) {
      for (int i = 0; i < 2 * r; ++i) slot_bufs.push_back(run.alloc<zd>((size_t)n * kk * 2));
    }
    if (ip->strategy == 3 || ip->strategy == 4) {
      tmpU = run.alloc<zd>((size_t)n * kk);
      tmpUt = run.alloc<zd>((size_t)n * kk);
    }
    zd* shU = ip->strategy == 4 ? run.alloc<zd>((size_t)n * kk) : nullptr;
    zd* shUt = ip->strategy == 4 ? run.alloc<zd>((size_t)n * kk) : nullptr;

    std::vector<char> has_op(r, 0);   // handle hidx[i] has been given an operator
    std::vector<cd> sig(r);
    for (int i = 0; i < r; ++i) sig[i] = cd(shifts_in[2 * i], shifts_in[2 * i + 1]);
    {
      const std::vector<int> o = shift_order(sig);
      std::vector<cd> t(r);
      for (int i = 0; i < r; ++i) t[i] = sig[o[i]];
      sig = t;
    }
    std::vector<rbicg_csr> ops(r);
    std::vector<rbicg_result> rs(r);
    std::vector<zd> Gh((size_t)(2 * r) * (2 * r + 2));
    std::vector<double> lamh(2 * KMAX + 2);
    double change = 1e300;
    int steps = 0;
    for (int step = 0; step < ip->max_steps; ++step) {
      const int refresh = step % ip->refresh_every == 0 ? 1 : 0;
      for (rbicg_handle h : run.handles) IR_CALL(rbicg_set_refresh(h, refresh), h);
      for (int i = 0; i < r; ++i) {
        ops[i] = *A;
        ops[i].has_shift = 1;
        ops[i].shift_re = sig[i].real();
        ops[i].shift_im = sig[i].imag();
      }
      // conj_pairs: of a conjugate pair (adjacent, + first) only the + shift is solved; the other
      // column is its conjugate (real A, b, c)
      std::vector<int> partner(r, -1), solve_idx;
      for (int i = 0; i < r; ++i) {
        if (ip->conj_pairs && i > 0 && partner[i - 1] == i) continue;
        if (ip->conj_pairs && i + 1 < r && sig[i].imag() > 0.0 && sig[i + 1] == std::conj(sig[i])) partner[i] = i + 1;
        solve_idx.push_back(i);
      }
      if (ip->strategy == 4) {
        // one recycle space shared by all shifts (E = I: sigma I - A has A's eigenvectors): the
        // solve of shift index 0 computes it, the other shifts use the one it computed last step
        for (int i = 1; i < nrec; ++i) IR_CALL(rbicg_set_refresh(hidx[i], 0), hidx[i]);
        if (step > 0 && nrec > 1) {
          int p = 0;
          IR_CALL(rbicg_export_recycle(hidx[0], shU, shUt, &p), hidx[0]);
          if (p > 0) {
            IR_CUDA(cudaMemcpy2DAsync(tmpU, sizeof(zd) * p, shU, sizeof(zd) * kk, sizeof(zd) * p, n,
                                      cudaMemcpyDeviceToDevice, s));
            IR_CUDA(cudaMemcpy2DAsync(tmpUt, sizeof(zd) * p, shUt, sizeof(zd) * kk, sizeof(zd) * p, n,
                                      cudaMemcpyDeviceToDevice, s));
          }
          for (int i : solve_idx) {
            if (i == 0 || i >= nrec) continue;
            if (p > 0) {
              // a handle whose index was a conjugate partner so far has no operator yet
              if (!has_op[i]) IR_CALL(rbicg_update_recycle(hidx[i], &ops[i]), hidx[i]);
              IR_CALL(rbicg_import_recycle(hidx[i], tmpU, tmpUt, p), hidx[i]);
            } else {
              IR_CALL(rbicg_reset(hidx[i]), hidx[i]);
            }
          }
        }
      }
      for (int i = 0; i < r; ++i) rs[i] = rbicg_result{};
      // Algorithm 3 steps 2-3 (and the loop's solves): v_i = (sigma_i I - A)^{-1} b,
      // w_i = (sigma_i I - A)^{-H} c, each from the previous step's solution for index i
      const int nsolve = (int)solve_idx.size();
      if (per_index && ip->batched && nsolve > 1) {
        std::vector<const rbicg_csr*> pa(nsolve);
        std::vector<const void*> pb(nsolve), pc(nsolve);
        std::vector<void*> px(nsolve), pxt(nsolve);
        std::vector<rbicg_handle> hb(nsolve);
        std::vector<rbicg_result> rb(nsolve);
        for (int q = 0; q < nsolve; ++q) {
          const int i = solve_idx[q];
          hb[q] = hidx[i];
          pa[q] = &ops[i]; pb[q] = bz; pc[q] = cz;
          px[q] = V + (int64_t)i * n; pxt[q] = W + (int64_t)i * n;
        }
        IR_CALL(rbicg_solve_batch(hb.data(), pa.data(), pb.data(), pc.data(), px.data(), pxt.data(), nsolve,
                                  rb.data()),
                hb[0]);
        for (int q = 0; q < nsolve; ++q) rs[solve_idx[q]] = rb[q];
        for (int i : solve_idx) has_op[i] = 1;
      } else {
        pool_cur.clear();
        for (int i : solve_idx) {
          rbicg_handle h = per_index ? hidx[i] : (i < nrec ? hrec : hplain);
          if (ip->strategy == 3 && i < nrec) {
            // reading of strategy 3: the pooled space with the smallest relative shift change,
            // if below pool_tol; otherwise none
            const Slot* best = nullptr;
            double bd = 0.0;
            for (const std::vector<Slot>* pl : {&pool_prev, &pool_cur})
              for (const Slot& sl : *pl) {
                if (sl.p <= 0) continue;
                const double d = std::abs(sig[i] - sl.sigma) / std::abs(sig[i]);
                if (!best || d < bd) { best = &sl; bd = d; }
              }
            if (best && bd < ip->pool_tol) {
              IR_CUDA(cudaMemcpy2DAsync(tmpU, sizeof(zd) * best->p, best->U, sizeof(zd) * kk, sizeof(zd) * best->p,
                                        n, cudaMemcpyDeviceToDevice, s));
              IR_CUDA(cudaMemcpy2DAsync(tmpUt, sizeof(zd) * best->p, best->Ut, sizeof(zd) * kk,
                                        sizeof(zd) * best->p, n, cudaMemcpyDeviceToDevice, s));
              IR_CALL(rbicg_import_recycle(h, tmpU, tmpUt, best->p), h);
            } else {
              IR_CALL(rbicg_reset(h), h);
            }
          }
          IR_CALL(rbicg_solve_pair(h, &ops[i], bz, cz, V + (int64_t)i * n, W + (int64_t)i * n, &rs[i]), h);
          has_op[i] = 1;
          if (ip->strategy == 3 && i < nrec) {
            zd* buf = slot_bufs[(step & 1) * r + i];
            Slot sl{sig[i], 0, buf, buf + (size_t)n * kk};
            IR_CALL(rbicg_export_recycle(h, sl.U, sl.Ut, &sl.p), h);
            pool_cur.push_back(sl);
          }
        }
        if (ip->strategy == 3) pool_prev = pool_cur;
      }
      for (int i = 0; i < r; ++i)
        if (partner[i] >= 0) {
          const int g = (int)std::min<int64_t>((n + 255) / 256, 4 * sm_count());
          k_conj_copy<<<g, 256, 0, s>>>(V + (int64_t)i * n, V + (int64_t)partner[i] * n, n);
          k_conj_copy<<<g, 256, 0, s>>>(W + (int64_t)i * n, W + (int64_t)partner[i] * n, n);
        }
      int64_t its = 0;
      for (int i : solve_idx) {
        its += rs[i].iters;
        if (rs[i].status != RBICG_OK && rs[i].status != RBICG_RECYCLE_EMPTY) ++res->failed_solves;
      }
      if (iters_out)
        for (int i = 0; i < r; ++i) iters_out[(int64_t)step * r + i] = rs[i].iters;   // 0: taken by conjugation
      res->iters += its;
      // Algorithm 3 step 4: A_r = W^H A V, E_r = W^H V (E = I), b_r = W^H b, c_r = V^H c
      k_apply_cols<<<(int)std::min<int64_t>((n * r + 255) / 256, 8 * sm_count()), 256, 0, s>>>(
          (int)n, A->row_ptr, A->col_idx, reinterpret_cast<const double*>(A->val), V, AV, r);
      ColList<zd> X{}, Y{};
      for (int i = 0; i < r; ++i) { X.c[X.m].p = W + (int64_t)i * n; X.c[X.m].ld = 1; ++X.m; }
      for (int i = 0; i < r; ++i) { X.c[X.m].p = V + (int64_t)i * n; X.c[X.m].ld = 1; ++X.m; }
      for (int i = 0; i < r; ++i) { Y.c[Y.m].p = AV + (int64_t)i * n; Y.c[Y.m].ld = 1; ++Y.m; }
      for (int i = 0; i < r; ++i) { Y.c[Y.m].p = V + (int64_t)i * n; Y.c[Y.m].ld = 1; ++Y.m; }
      Y.c[Y.m].p = bz; Y.c[Y.m].ld = 1; ++Y.m;
      Y.c[Y.m].p = cz; Y.c[Y.m].ld = 1; ++Y.m;
      launch_gram<zd>(X, Y, n, 0, gpart, gram_grid, G, s);
      k_pencil<<<1, 256, 0, s>>>(G, r, work + dense_off_L(), work + dense_off_R(), brc, brc + KMAX);
      // sigma_i <- -lambda_i(A_r, E_r): all r eigenvalues of the pencil on the device
      launch_dense_eig_host(0, r, nullptr, nullptr, 1, r, Wev, Wtev, lam, nullptr, nullptr, work, s);
      IR_CUDA(cudaGetLastError());
      DevState hst;
      IR_CUDA(cudaMemcpyAsync(&hst, reinterpret_cast<DevState*>(work + dense_state_offset()), sizeof hst,
                              cudaMemcpyDeviceToHost, s));
      IR_CUDA(cudaMemcpyAsync(lamh.data(), lam, sizeof(double) * (2 * KMAX + 2), cudaMemcpyDeviceToHost, s));
      IR_CUDA(cudaMemcpyAsync(Gh.data(), G, sizeof(zd) * Gh.size(), cudaMemcpyDeviceToHost, s));
      IR_CUDA(cudaStreamSynchronize(s));
      ++steps;
      // the reduced model of this step (returned for the last step)
      const int w2 = 2 * r + 2;
      for (int a = 0; a < r; ++a) {
        for (int bb = 0; bb < r; ++bb) {
          const zd ar = Gh[(size_t)a * w2 + bb], er = Gh[(size_t)a * w2 + r + bb];
          if (Ar_out) { Ar_out[2 * (a + (size_t)bb * r)] = ar.re; Ar_out[2 * (a + (size_t)bb * r) + 1] = ar.im; }
          if (Er_out) { Er_out[2 * (a + (size_t)bb * r)] = er.re; Er_out[2 * (a + (size_t)bb * r) + 1] = er.im; }
        }
        const zd bv = Gh[(size_t)a * w2 + 2 * r], cv = Gh[(size_t)(r + a) * w2 + 2 * r + 1];
        if (br_out) { br_out[2 * a] = bv.re; br_out[2 * a + 1] = bv.im; }
        if (cr_out) { cr_out[2 * a] = cv.re; cr_out[2 * a + 1] = cv.im; }
      }
      for (int i = 0; i < r; ++i) {   // the shifts this model interpolates at
        res->model_shifts[2 * i] = sig[i].real();
        res->model_shifts[2 * i + 1] = sig[i].imag();
      }
      if (hst.eig_status != 0 || hst.kk != r) {
        char buf[160];
        snprintf(buf, sizeof buf, "rbicg_irka: eigenvalues of the reduced pencil (step %d): status %d, %d of %d values",
                 step, hst.eig_status, hst.kk, r);
        throw IrkaErr{RBICG_ERR_EIG, buf};
      }
      std::vector<cd> nl(r);
      for (int i = 0; i < r; ++i) nl[i] = -cd(lamh[2 * i], lamh[2 * i + 1]);
      nl = conjugate_close(nl);
      const std::vector<int> o = shift_order(nl);
      std::vector<cd> ns(r);
      for (int i = 0; i < r; ++i) ns[i] = nl[o[i]];
      change = 0.0;
      for (int i = 0; i < r; ++i) change = std::max(change, std::abs(ns[i] - sig[i]) / std::abs(sig[i]));
      sig = ns;
      if (change < ip->shift_tol) { res->converged = 1; break; }
    }
    for (int i = 0; i < r; ++i) { shifts_out[2 * i] = sig[i].real(); shifts_out[2 * i + 1] = sig[i].imag(); }
    res->steps = steps;
    res->last_change = change;
    return RBICG_OK;
  } catch (const IrkaErr& e) {
    set_global_error(e.msg.c_str());
    return e.st;
  } catch (const std::exception& e) {
    set_global_error(e.what());
    return RBICG_ERR_CUDA;
  }
}
