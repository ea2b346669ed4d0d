// kernels_dense.cu -- the small FP64 problems of the recycle-space refresh, on the GPU.
//
//  * k_build: H_j, Ht_j of Section 4.1 / 4.2 from the iteration scalars (T of Section 4.1,
//    B_j = Chat^H A V_j, Bt_j = Ccheck^H A^H Vt_j from the zeta histories), the Lanczos
//    scalings v_m = r_{m-1}/||r_{m-1}||, vt_m = rt_{m-1}/(v_m, rt_{m-1}) applied to the raw
//    Gram, and the pencil L = Ht^H (Psit^H Psi) H, R = Ht^H (Psit^H Phi) of eq.
//    (finalGenEigValue).  Many blocks (plain dense products of order <= 130).
//  * k_eig: one block.  M = R^{-1} L (complex LU with partial pivoting), Householder
//    reduction to Hessenberg form, shifted QR to Schur form M = Q T Q^H, selection of the
//    eigenvalues closest to the origin, right eigenvectors W = Q y and left eigenvectors of
//    the pencil Wt = R^{-H} Q yl (y, yl eigenvectors of the triangular T).
//  * k_svd: one block.  One-sided (Hestenes) Jacobi SVD of Ct_j^H C_j after unit-norm column
//    scaling (Section 4.3, eq. (equationSVD)); truncation at svd_tol; rotation coefficients.
#include <algorithm>

#include "internal.cuh"

namespace rb {

constexpr int PSIMAX = 2 * KMAX + SMAX + 2;   // rows of H (columns of Psi)

// ------------------------------------------------------------------------------------
// T of Section 4.1 from the histories: T(m,m) = 1/a_m + b_{m-1}/a_{m-1};
// T(m+1,m) = -(|r_m|/|r_{m-1}|)/a_m; T(m,m+1) = -(|r_{m-1}|/|r_m|) b_m/a_m.
// ------------------------------------------------------------------------------------
__device__ zd T_entry(const DevState* st, int gr, int gc) {
  const int m = gc;
  if (gr == m) {
    zd v = zd(1.0) / st->h_alpha[m % HR];
    if (m >= 2) v += st->h_beta[(m - 1) % HR] / st->h_alpha[(m - 1) % HR];
    return v;
  }
  if (gr == m + 1) return -(st->h_rnorm[m % HR] / st->h_rnorm[(m - 1) % HR]) * (zd(1.0) / st->h_alpha[m % HR]);
  if (gr == m - 1) {
    const int q = m - 1;
    return -(st->h_rnorm[(q - 1) % HR] / st->h_rnorm[q % HR]) * (st->h_beta[q % HR] / st->h_alpha[q % HR]);
  }
  return zd();
}

struct Layout {
  // column ranges of Psi (rows of H) and Phi (columns of H)
  int nC, nCp, nUps, nPsi;     // C block, C_{j-1} block, ring block; total
  int nUphi, nV, nPhi;         // U block of Phi, V block; total
  int g0;                      // global Lanczos index of the first ring column (v_{g0})
  int v_off;                   // offset of V_j inside the ring block
};

__device__ Layout make_layout(const RefreshInfo& f) {
  Layout L;
  L.nV = f.s;
  switch (f.case_id) {
    case 1: L.nC = 0; L.nCp = f.kp; L.nUps = f.s + 2; L.nUphi = f.kp; L.g0 = (f.j - 1) * f.s; L.v_off = 1; break;
    case 2: L.nC = f.kc; L.nCp = 0; L.nUps = f.s + 1; L.nUphi = f.kc; L.g0 = 1; L.v_off = 0; break;
    case 3: L.nC = f.kc; L.nCp = f.kp; L.nUps = f.s + 2; L.nUphi = f.kp; L.g0 = (f.j - 1) * f.s; L.v_off = 1; break;
    default: L.nC = 0; L.nCp = 0; L.nUps = f.s + 1; L.nUphi = 0; L.g0 = 1; L.v_off = 0; break;
  }
  L.nPsi = L.nC + L.nCp + L.nUps;
  L.nPhi = L.nUphi + L.nV;
  return L;
}

// scale of Psi column a (primal: 1 or 1/||r_{g-1}||) and Psit column a (1 or ||r||/conj(rho))
__device__ void psi_scale(const DevState* st, const Layout& L, int a, zd* sc, zd* sct) {
  if (a < L.nC + L.nCp) { *sc = zd(1.0); *sct = zd(1.0); return; }
  const int g = L.g0 + (a - L.nC - L.nCp);   // Lanczos index, column holds r_{g-1}
  const double rn = st->h_rnorm[(g - 1) % HR];
  *sc = zd(1.0 / rn);
  *sct = zd(rn) / conjg(st->h_rho[(g - 1) % HR]);
}

// H (primal) / Ht (dual) entry at (row a of Psi, column b of Phi)
__device__ zd H_entry(const DevState* st, const RefreshInfo& f, const Layout& L, int a, int b, bool dual) {
  const bool bU = b < L.nUphi;
  if (f.case_id == 2) {
    // [[I, B_1], [0, T_1 underlined]]
    if (a < L.nC) {
      if (bU) return a == b ? zd(1.0) : zd();
      const int m = 1 + (b - L.nUphi);   // column v_m
      const zd zm = dual ? st->h_zetat[m % HR][a] : st->h_zeta[m % HR][a];
      const zd zm1 = (m >= 2) ? (dual ? st->h_zetat[(m - 1) % HR][a] : st->h_zeta[(m - 1) % HR][a]) : zd();
      const zd bm1 = (m >= 2) ? st->h_beta[(m - 1) % HR] : zd();
      if (!dual) return (zm - bm1 * zm1) * (1.0 / st->h_rnorm[(m - 1) % HR]);
      return (zm - conjg(bm1) * zm1) * (zd(st->h_rnorm[(m - 1) % HR]) / conjg(st->h_rho[(m - 1) % HR]));
    }
    if (bU) return zd();
    const int gr = L.g0 + (a - L.nC), gc = 1 + (b - L.nUphi);
    if (gr < gc - 1 || gr > gc + 1) return zd();
    return dual ? conjg(T_entry(st, gc, gr)) : T_entry(st, gr, gc);
  }
  // cases 1 and 3: [[0, B_j], [I, 0], [0, Gamma_j]] (case 1 has no C block)
  if (a < L.nC) {
    if (bU) return zd();
    const int m = L.g0 + L.v_off + (b - L.nUphi);
    const zd zm = dual ? st->h_zetat[m % HR][a] : st->h_zeta[m % HR][a];
    const zd zm1 = dual ? st->h_zetat[(m - 1) % HR][a] : st->h_zeta[(m - 1) % HR][a];
    const zd bm1 = st->h_beta[(m - 1) % HR];
    if (!dual) return (zm - bm1 * zm1) * (1.0 / st->h_rnorm[(m - 1) % HR]);
    return (zm - conjg(bm1) * zm1) * (zd(st->h_rnorm[(m - 1) % HR]) / conjg(st->h_rho[(m - 1) % HR]));
  }
  if (a < L.nC + L.nCp) return (bU && (a - L.nC) == b) ? zd(1.0) : zd();
  if (bU) return zd();
  const int gr = L.g0 + (a - L.nC - L.nCp);
  const int gc = L.g0 + L.v_off + (b - L.nUphi);
  if (gr < gc - 1 || gr > gc + 1) return zd();
  return dual ? conjg(T_entry(st, gc, gr)) : T_entry(st, gr, gc);
}

// Gram column (Y side) holding Phi column b: U block after Psi's columns, V inside the ring
__device__ int phi_ycol(const Layout& L, int b) {
  if (b < L.nUphi) return L.nPsi + b;
  return L.nC + L.nCp + L.v_off + (b - L.nUphi);
}

// work layout (zd): Hd [PSIMAX x MMAX], Htd [PSIMAX x MMAX], GH [PSIMAX x MMAX],
// Lm [MMAX x MMAX], Rm [MMAX x MMAX] (column-major), then eig scratch.
constexpr int64_t W_HD = 0, W_HTD = W_HD + PSIMAX * MMAX, W_GH = W_HTD + PSIMAX * MMAX,
                  W_L = W_GH + PSIMAX * MMAX, W_R = W_L + MMAX * MMAX,
                  W_Y = W_R + MMAX * MMAX, W_YL = W_Y + MMAX * (KMAX + 8), W_LAM = W_YL + MMAX * (KMAX + 8),
                  W_LAM2 = W_LAM + KMAX + 8, W_INT = W_LAM2 + KMAX + 8,
                  W_END = W_INT + (MMAX + 2 * KMAX + 8 + 3) / 4 + 1;
static_assert(PSIMAX * MMAX >= 2 * MMAX * KMAX, "k_eig_c keeps the selected vectors in the GH area");
// integer area at W_INT: piv[MMAX], sel[KMAX], pair[KMAX], units, cols, ncand
constexpr int NCAND_EXTRA = 8;   // candidates beyond k refined before the final selection

template <class A>
__global__ void k_build_h(RefreshInfo f, const DevState* st, zd* work) {
  const Layout L = make_layout(f);
  zd* Hd = work + W_HD;
  zd* Htd = work + W_HTD;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L.nPsi * L.nPhi; e += gridDim.x * blockDim.x) {
    const int a = e % L.nPsi, b = e / L.nPsi;
    Hd[a + b * PSIMAX] = H_entry(st, f, L, a, b, false);
    Htd[a + b * PSIMAX] = H_entry(st, f, L, a, b, true);
  }
}

// GH[a, b] = sum_c Gs[a, c] H[c, b], Gs[a, c] = conj(sct_a) G[a, c] sc_c  (a, c over Psi)
// Lanczos scalings of all Psi columns, once per block (shared memory)
__device__ void load_psi_scales(const DevState* st, const Layout& L, zd* sc, zd* sct) {
  for (int a = threadIdx.x; a < L.nPsi; a += blockDim.x) psi_scale(st, L, a, &sc[a], &sct[a]);
  __syncthreads();
}

template <class A>
__global__ void k_gh(RefreshInfo f, const DevState* st, const A* G, zd* work) {
  __shared__ zd sc[PSIMAX], sct[PSIMAX];
  const Layout L = make_layout(f);
  load_psi_scales(st, L, sc, sct);
  const zd* Hd = work + W_HD;
  zd* GH = work + W_GH;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L.nPsi * L.nPhi; e += gridDim.x * blockDim.x) {
    const int a = e % L.nPsi, b = e / L.nPsi;
    zd s = zd();
    for (int c = 0; c < L.nPsi; ++c) {
      const zd h = Hd[c + b * PSIMAX];
      if (h.re == 0.0 && h.im == 0.0) continue;
      s += to_zd(G[(int64_t)a * f.my + c]) * sc[c] * h;
    }
    GH[a + b * PSIMAX] = conjg(sct[a]) * s;
  }
}

// L[c, b] = sum_a conj(Ht[a, c]) GH[a, b];  R[c, b] = sum_a conj(Ht[a, c]) Gs[a, phi(b)]
template <class A>
__global__ void k_lr(RefreshInfo f, const DevState* st, const A* G, zd* work) {
  const Layout L = make_layout(f);
  const zd* Htd = work + W_HTD;
  const zd* GH = work + W_GH;
  zd* Lm = work + W_L;
  zd* Rm = work + W_R;
  const int m = L.nPhi;
  __shared__ zd sc[PSIMAX], sct[PSIMAX];
  load_psi_scales(st, L, sc, sct);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int c = e % m, b = e / m;
    const int yc = phi_ycol(L, b);
    const zd sy = yc < L.nPsi ? sc[yc] : zd(1.0);
    zd sl = zd(), sr = zd();
    for (int a = 0; a < L.nPsi; ++a) {
      const zd h = Htd[a + c * PSIMAX];
      if (h.re == 0.0 && h.im == 0.0) continue;
      const zd hc = conjg(h);
      sl += hc * GH[a + b * PSIMAX];
      sr += hc * (conjg(sct[a]) * to_zd(G[(int64_t)a * f.my + yc]) * sy);
    }
    Lm[c + b * MMAX] = sl;
    Rm[c + b * MMAX] = sr;
  }
}

// First cycle of the first system (Section 4.2): L = T_1 (s x s), no R.
__global__ void k_t1(RefreshInfo f, const DevState* st, zd* work) {
  zd* Lm = work + W_L;
  const int s = f.s;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < s * s; e += gridDim.x * blockDim.x) {
    const int a = e % s, b = e / s;
    Lm[a + b * MMAX] = (a >= b - 1 && a <= b + 1) ? T_entry(st, a + 1, b + 1) : zd();
  }
}

// ------------------------------------------------------------------------------------
// one-block dense eigen solver (complex FP64)
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double cabs_(zd a) { return hypot(a.re, a.im); }
typedef cplx<float> zf;
__device__ __forceinline__ float cabs_(zf a) { return hypotf(a.re, a.im); }

template <class S> struct real_t;
template <> struct real_t<zd> { typedef double t; };
template <> struct real_t<zf> { typedef float t; };

// Block-wide LU with partial pivoting of A (m x m, leading dimension ld) in place;
// piv[k] = pivot row of step k.  Returns false on an exactly zero pivot column.
template <class S>
__device__ bool lu_block(S* A, int m, int ld, int* piv, typename real_t<S>::t* dsc) {
  typedef typename real_t<S>::t Rl;
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x < 32) {
      Rl best = -1;
      int bi = k;
      for (int r = k + threadIdx.x; r < m; r += 32) {
        const Rl v = cabs_(A[r + k * ld]);
        if (v > best) { best = v; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const Rl ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) { piv[k] = bi; dsc[0] = best; }
    }
    __syncthreads();
    const int p = piv[k];
    if (dsc[0] == Rl(0)) return false;
    if (p != k)
      for (int c = threadIdx.x; c < m; c += blockDim.x) {
        const S t = A[k + c * ld]; A[k + c * ld] = A[p + c * ld]; A[p + c * ld] = t;
      }
    __syncthreads();
    const S inv = S(Rl(1)) / A[k + k * ld];
    for (int r = k + 1 + threadIdx.x; r < m; r += blockDim.x) A[r + k * ld] = A[r + k * ld] * inv;
    __syncthreads();
    const int rem = m - k - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int r = k + 1 + e % rem, c = k + 1 + e / rem;
      A[r + c * ld] -= A[r + k * ld] * A[k + c * ld];
    }
    __syncthreads();
  }
  return true;
}

// Block-wide: columns of B (stride ldb) <- A^{-1} B for the LU of A (one thread per column)
template <class S>
__device__ void lu_solve_block(const S* LU, int m, int ld, const int* piv, S* B, int nb, int ldb) {
  for (int col = threadIdx.x; col < nb; col += blockDim.x) {
    S* b = B + col * ldb;
    for (int k = 0; k < m; ++k) { const int p = piv[k]; if (p != k) { const S t = b[k]; b[k] = b[p]; b[p] = t; } }
    for (int r = 0; r < m; ++r) { S s = b[r]; for (int c = 0; c < r; ++c) s -= LU[r + c * ld] * b[c]; b[r] = s; }
    for (int r = m - 1; r >= 0; --r) {
      S s = b[r];
      for (int c = r + 1; c < m; ++c) s -= LU[r + c * ld] * b[c];
      b[r] = s / LU[r + r * ld];
    }
  }
  __syncthreads();
}

// One warp: y <- A^{-1} y (A = P^T Lw U stored as LU, pivots piv), column-oriented substitution
__device__ void lu_solve_warp(const zd* LU, int m, int ld, const int* piv, zd* y) {
  const int lane = threadIdx.x & 31;
  if (lane == 0)
    for (int k = 0; k < m; ++k) { const int p = piv[k]; if (p != k) { const zd t = y[k]; y[k] = y[p]; y[p] = t; } }
  __syncwarp();
  for (int c = 0; c < m; ++c) {          // unit lower triangular
    const zd yc = y[c];
    __syncwarp();
    for (int r = c + 1 + lane; r < m; r += 32) y[r] -= LU[r + c * ld] * yc;
    __syncwarp();
  }
  for (int c = m - 1; c >= 0; --c) {     // upper triangular
    const zd yc = y[c] / LU[c + c * ld];
    __syncwarp();
    if (lane == 0) y[c] = yc;
    for (int r = lane; r < c; r += 32) y[r] -= LU[r + c * ld] * yc;
    __syncwarp();
  }
}

// One warp: y <- A^{-H} y.  A^H = U^H Lw^H P: solve U^H z = y, Lw^H w = z, y = P^T w.
__device__ void lu_solve_adj_warp(const zd* LU, int m, int ld, const int* piv, zd* y) {
  const int lane = threadIdx.x & 31;
  for (int c = 0; c < m; ++c) {          // U^H lower triangular: column c of U^H = conj(U[c, :])
    const zd yc = y[c] / conjg(LU[c + c * ld]);
    __syncwarp();
    if (lane == 0) y[c] = yc;
    for (int r = c + 1 + lane; r < m; r += 32) y[r] -= conjg(LU[c + r * ld]) * yc;
    __syncwarp();
  }
  for (int c = m - 1; c >= 0; --c) {     // Lw^H unit upper triangular: column c = conj(Lw[c, :])
    const zd yc = y[c];
    __syncwarp();
    for (int r = lane; r < c; r += 32) y[r] -= conjg(LU[c + r * ld]) * yc;
    __syncwarp();
  }
  if (lane == 0)
    for (int k = m - 1; k >= 0; --k) { const int p = piv[k]; if (p != k) { const zd t = y[k]; y[k] = y[p]; y[p] = t; } }
  __syncwarp();
}

// Block-wide Householder reduction of T (m x m, ld) to upper Hessenberg form (no vectors)
template <class S>
__device__ void hessenberg_block(S* T, int m, int ld, S* v, typename real_t<S>::t* dsc) {
  typedef typename real_t<S>::t Rl;
  for (int j = 0; j < m - 2; ++j) {
    const int len = m - j - 1;
    if (threadIdx.x < 32) {
      Rl sacc = 0;
      for (int r = threadIdx.x; r < len; r += 32) sacc += abs2(T[j + 1 + r + j * ld]);
      for (int o = 16; o > 0; o >>= 1) sacc += __shfl_down_sync(0xffffffffu, sacc, o);
      if (threadIdx.x == 0) dsc[0] = sacc;
    }
    __syncthreads();
    const Rl nx2 = dsc[0];
    const S x0 = T[j + 1 + j * ld];
    const Rl tail = nx2 - abs2(x0);
    if (!(tail > Rl(0)) || tail <= nx2 * Rl(1e-30)) { __syncthreads(); continue; }
    const Rl nx = sqrt(nx2);
    const Rl ax0 = cabs_(x0);
    const S ph = ax0 > Rl(0) ? x0 * (Rl(1) / ax0) : S(Rl(1));
    const S alpha = -(ph * nx);
    for (int r = threadIdx.x; r < len; r += blockDim.x) v[r] = T[j + 1 + r + j * ld];
    __syncthreads();
    if (threadIdx.x == 0) v[0] = v[0] - alpha;
    __syncthreads();
    const Rl f = Rl(2) / (tail + abs2(x0 - alpha));
    for (int c = j + threadIdx.x; c < m; c += blockDim.x) {
      S w = S(Rl(0));
      for (int r = 0; r < len; ++r) w += cmul(v[r], T[j + 1 + r + c * ld]);
      w = w * f;
      for (int r = 0; r < len; ++r) T[j + 1 + r + c * ld] -= v[r] * w;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
      S u = S(Rl(0));
      for (int c = 0; c < len; ++c) u += T[r + (j + 1 + c) * ld] * v[c];
      u = u * f;
      for (int c = 0; c < len; ++c) T[r + (j + 1 + c) * ld] -= u * conjg(v[c]);
    }
    __syncthreads();
    for (int r = j + 2 + threadIdx.x; r < m; r += blockDim.x) T[r + j * ld] = S(Rl(0));
    __syncthreads();
  }
}

// Selection of eigenvalue indices (reading: k closest to the origin; on a real problem a
// conjugate pair is one unit of two columns, k-1 columns if it straddles the cut).
// Writes sel[u] = index, pairflag[u]; returns number of units; *ncols = columns.
__device__ int select_units(const zd* lam, int m, int k, int real_path, int* sel, int* pairflag, int* ncols) {
  // thread 0 only
  int order[MMAX];
  int cnt = 0;
  for (int i = 0; i < m; ++i)
    if (isfinite(lam[i].re) && isfinite(lam[i].im)) order[cnt++] = i;
  // insertion sort by (|lam|, index)
  for (int a = 1; a < cnt; ++a) {
    const int v = order[a];
    const double av = cabs_(lam[v]);
    int b = a - 1;
    while (b >= 0 && (cabs_(lam[order[b]]) > av || (cabs_(lam[order[b]]) == av && order[b] > v))) { order[b + 1] = order[b]; --b; }
    order[b + 1] = v;
  }
  bool used[MMAX];
  for (int i = 0; i < m; ++i) used[i] = false;
  int units = 0, cols = 0;
  for (int t = 0; t < cnt; ++t) {
    const int i = order[t];
    if (used[i]) continue;
    const double al = cabs_(lam[i]);
    const bool isreal = !real_path || fabs(lam[i].im) <= 1e-10 * (al > 0.0 ? al : 1.0);
    if (!real_path || isreal) {
      if (cols + 1 > k) break;
      sel[units] = i; pairflag[units] = 0; ++units; ++cols; used[i] = true;
      continue;
    }
    // conjugate partner: nearest unused to conj(lam[i])
    int pj = -1;
    double best = 1e300;
    for (int q = 0; q < m; ++q) {
      if (used[q] || q == i) continue;
      const double dd = cabs_(lam[q] - conjg(lam[i]));
      if (dd < best) { best = dd; pj = q; }
    }
    if (cols + 2 > k) break;
    // keep the member with positive imaginary part as the representative
    int rep = i;
    if (lam[i].im < 0.0 && pj >= 0) rep = pj;
    sel[units] = rep; pairflag[units] = 1; ++units; cols += 2;
    used[i] = true;
    if (pj >= 0) used[pj] = true;
  }
  *ncols = cols;
  return units;
}

// ------------------------------------------------------------------------------------
// Eigen pipeline (three kernels).
//   k_eig_a (one block): M = R^{-1} L (FP64 LU with partial pivoting), FP64 Householder
//     reduction to Hessenberg form, eigenvalues by an FP32 implicit single-shift QR restricted
//     to the active window, and the k + NCAND_EXTRA eigenvalues closest to 0 as candidates
//     (shifts for the FP64 refinement).
//   k_eig_b (one block per candidate, FP64): inverse iteration on the pencil itself,
//     (L - sigma R) y+ = R y and (L - sigma R)^H yl+ = R^H yl (dense LU with partial pivoting),
//     then the two-sided Rayleigh quotient yl^H L y / yl^H R y; when that quotient has moved
//     away from the FP32 shift, one more factorisation at the quotient (a Rayleigh step).
//   k_eig_c (one block): candidates that refined to the same eigenvalue are merged, final
//     selection on the refined eigenvalues (real / complex decided in FP64), unit norm,
//     conjugate pairs split into real and imaginary parts, Phi scalings.
// The QR iteration is long and sequential; on this part FP64 runs at about 2 FMA per clock per
// SM and FP32 at 64x that, so it runs in FP32 and the eigenpairs are refined in FP64.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ float cabsf_(zf a) { return hypotf(a.re, a.im); }

__device__ __forceinline__ float cabs1f_(zf a) { return fabsf(a.re) + fabsf(a.im); }

// Plane rotation [c, s; -conj(s), c] with c real that zeroes b against a.  The matrix is scaled
// to entries of order one before the QR iteration, so the squares neither overflow nor lose
// anything that matters; reciprocal square roots replace hypot and division.
__device__ void givens_f(zf a, zf b, float* c, zf* s) {
  const float ab2 = abs2(b);
  if (ab2 == 0.f) { *c = 1.f; *s = zf(0.f, 0.f); return; }
  const float aa2 = abs2(a);
  if (aa2 == 0.f) { *c = 0.f; *s = conjg(b) * rsqrtf(ab2); return; }
  const float ria = rsqrtf(aa2), rn = rsqrtf(aa2 + ab2);
  *c = aa2 * ria * rn;
  *s = (a * ria) * conjg(b) * rn;
}

// Warp 0: eigenvalues of the Hessenberg H (FP32, ld) by implicit single-shift QR with Wilkinson
// shifts, updating only the active window.  Returns false (with diagnostics) on failure.
__device__ bool qr_eigs_warp_f32(zf* T, int m, int ld, int* dbg) {
  const int lane = threadIdx.x & 31;
  const float eps = 1.1920929e-07f;
  int hi = m - 1, iter = 0, total = 0;
  while (hi > 0) {
    int lo = hi;
    while (lo > 0) {
      const float sub = cabs1f_(T[lo + (lo - 1) * ld]);
      const float dsum = cabs1f_(T[lo + lo * ld]) + cabs1f_(T[lo - 1 + (lo - 1) * ld]);
      if (sub <= eps * (dsum > 0.f ? dsum : 1.f)) {
        __syncwarp();
        if (lane == 0) T[lo + (lo - 1) * ld] = zf(0.f, 0.f);
        __syncwarp();
        break;
      }
      --lo;
    }
    if (lo == hi) { --hi; iter = 0; continue; }
    if (!finite_of(T[hi + hi * ld].re) || !finite_of(T[hi + (hi - 1) * ld].re) ||
        !isfinite(T[hi + hi * ld].im) || !isfinite(T[hi + (hi - 1) * ld].im)) {
      if (lane == 0) { dbg[0] = 3; dbg[1] = lo; dbg[2] = hi; dbg[3] = iter; dbg[4] = total; }
      return false;
    }
    if (++total > 60 * m) {
      if (lane == 0) { dbg[0] = 2; dbg[1] = lo; dbg[2] = hi; dbg[3] = iter; dbg[4] = total; }
      return false;
    }
    ++iter;
    const zf a = T[hi - 1 + (hi - 1) * ld], b = T[hi - 1 + hi * ld], c = T[hi + (hi - 1) * ld], d = T[hi + hi * ld];
    zf mu;
    if (iter % 11 == 10) {
      mu = d + zf(cabsf_(c) * 0.75f, 0.f);   // exceptional shift
    } else {
      const zf tr = a + d, det = a * d - b * c;
      const zf half = tr * 0.5f;
      const zf disc = half * half - det;
      const float rdisc = cabsf_(disc);
      // radicands clamped: hypotf's rounding can put |disc| + Re(disc) below zero
      float sr = sqrtf(fmaxf(0.f, 0.5f * (rdisc + disc.re))), si = sqrtf(fmaxf(0.f, 0.5f * (rdisc - disc.re)));
      if (disc.im < 0.f) si = -si;
      const zf sq(sr, si);
      const zf l1 = half + sq, l2 = half - sq;
      mu = cabsf_(l1 - d) < cabsf_(l2 - d) ? l1 : l2;
    }
    const zf x = T[lo + lo * ld] - mu, y = T[lo + 1 + lo * ld];
    for (int k = lo; k < hi; ++k) {
      float cs;
      zf sn;
      if (k == lo) givens_f(x, y, &cs, &sn);
      else givens_f(T[k + (k - 1) * ld], T[k + 1 + (k - 1) * ld], &cs, &sn);
      __syncwarp();   // all lanes have read the rotation's defining entries
      const int c0 = k > lo ? k - 1 : lo;
      for (int col = c0 + lane; col <= hi; col += 32) {
        const zf p = T[k + col * ld], q = T[k + 1 + col * ld];
        T[k + col * ld] = cs * p + sn * q;
        T[k + 1 + col * ld] = cs * q - conjg(sn) * p;
      }
      __syncwarp();
      const int r1 = k + 2 < hi ? k + 2 : hi;
      for (int row = lo + lane; row <= r1; row += 32) {
        const zf p = T[row + k * ld], q = T[row + (k + 1) * ld];
        T[row + k * ld] = cs * p + conjg(sn) * q;
        T[row + (k + 1) * ld] = cs * q - sn * p;
      }
      __syncwarp();
      if (k > lo && lane == 0) T[k + 1 + (k - 1) * ld] = zf(0.f, 0.f);
      __syncwarp();
    }
  }
  return true;
}

struct EigInts {   // integer area of the dense work buffer
  int* piv; int* sel; int* pair; int* units; int* cols; int* ncand;
};
__device__ __host__ inline EigInts eig_ints(zd* work) {
  int* b = reinterpret_cast<int*>(work + W_INT);
  EigInts e;
  e.piv = b; e.sel = b + MMAX; e.pair = b + MMAX + KMAX; e.units = b + MMAX + 2 * KMAX; e.cols = e.units + 1;
  e.ncand = e.units + 2;
  return e;
}

__global__ void __launch_bounds__(256) k_eig_a(RefreshInfo f, DevState* st, zd* work, int has_R, int m) {
  extern __shared__ unsigned char smraw[];
  const int ld = m | 1;   // odd leading dimension: conflict-free row access
  zd* A = reinterpret_cast<zd*>(smraw);
  zd* B = A + m * ld;
  zd* v = B + m * ld;
  double* dsc = reinterpret_cast<double*>(v + MMAX);
  int* piv = reinterpret_cast<int*>(dsc + 4);
  zf* H = reinterpret_cast<zf*>(A);   // FP32 copy of the Hessenberg form, over R's LU
  __shared__ int s_ok;
  __shared__ double s_red[8];
  const zd* Lm = work + W_L;
  const zd* Rm = work + W_R;
  const EigInts ei = eig_ints(work);
  if (threadIdx.x == 0) s_ok = 1;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int r = e % m, c = e / m;
    B[r + c * ld] = Lm[r + c * MMAX];
    if (has_R) A[r + c * ld] = Rm[r + c * MMAX];
  }
  __syncthreads();
  if (has_R) {
    if (!lu_block(A, m, ld, piv, dsc)) { if (threadIdx.x == 0) s_ok = 0; }
    __syncthreads();
    if (!s_ok) { if (threadIdx.x == 0) { st->eig_status = 1; st->kk = 0; *ei.ncand = 0; } return; }
    lu_solve_block(A, m, ld, piv, B, m, ld);   // B <- R^{-1} L
  }
  // The reduction to Hessenberg form stays in FP64: the harmonic Ritz pencils of these cycles are
  // so ill-conditioned (R carries Lanczos and recycle vectors of very different norms) that an
  // FP32 reduction moves their small eigenvalues by O(1); FP32 QR on the FP64 Hessenberg form
  // still gives shifts to about 1e-4, which the FP64 refinement needs.
  hessenberg_block(B, m, ld, v, dsc);
  // FP32 copy scaled to entries of order one (the eigenvalues scale with it)
  double amax = 0.0;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const zd h = B[(e % m) + (e / m) * ld];
    amax = fmax(amax, fabs(h.re) + fabs(h.im));
  }
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = amax;
  __syncthreads();
  amax = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) amax = fmax(amax, s_red[w]);
  if (!(amax > 0.0) || !isfinite(amax)) {
    if (threadIdx.x == 0) { st->eig_status = 1; st->kk = 0; *ei.ncand = 0; }
    return;
  }
  const double inv = 1.0 / amax;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int r = e % m, c = e / m;
    const zd h = B[r + c * ld];
    H[r + c * ld] = zf((float)(h.re * inv), (float)(h.im * inv));
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool ok = qr_eigs_warp_f32(H, m, ld, st->dbg);
    if (threadIdx.x == 0 && !ok) s_ok = 0;
  }
  __syncthreads();
  if (!s_ok) { if (threadIdx.x == 0) { st->eig_status = 2; st->kk = 0; *ei.ncand = 0; } return; }
  if (threadIdx.x == 0) {
    // candidates: the k + NCAND_EXTRA finite FP32 eigenvalues closest to the origin; real /
    // complex classification and the final selection wait for the FP64 refinement
    int order[MMAX];
    int cnt = 0;
    for (int i = 0; i < m; ++i) {
      const zf h = H[i + i * ld];
      if (isfinite(h.re) && isfinite(h.im)) order[cnt++] = i;
    }
    for (int a = 1; a < cnt; ++a) {
      const int vv = order[a];
      const float av = cabs_(H[vv + vv * ld]);
      int b = a - 1;
      while (b >= 0 && cabs_(H[order[b] + order[b] * ld]) > av) { order[b + 1] = order[b]; --b; }
      order[b + 1] = vv;
    }
    const int nc = min(cnt, f.k + NCAND_EXTRA);
    for (int c = 0; c < nc; ++c) {
      const zf h = H[order[c] + order[c] * ld];
      work[W_LAM + c] = zd((double)h.re * amax, (double)h.im * amax);
    }
    *ei.ncand = nc;
    st->eig_status = 0;
  }
}

__global__ void __launch_bounds__(256) k_eig_b(zd* work, int m, int has_R) {
  extern __shared__ unsigned char smraw[];
  const EigInts ei = eig_ints(work);
  const int cand = blockIdx.x;
  if (cand >= *ei.ncand) return;
  const int ld = m | 1;
  zd* A = reinterpret_cast<zd*>(smraw);   // L - sigma R, then its LU
  zd* yr = A + m * ld;
  zd* yl = yr + MMAX;
  zd* tr = yl + MMAX;
  zd* tl = tr + MMAX;
  double* dsc = reinterpret_cast<double*>(tl + MMAX);
  int* piv = reinterpret_cast<int*>(dsc + 4);
  __shared__ int s_ok;
  __shared__ zd s_lam;
  const zd* Lm = work + W_L;
  const zd* Rm = work + W_R;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto Rat = [&](int r, int c) -> zd { return has_R ? Rm[r + c * MMAX] : (r == c ? zd(1.0) : zd()); };
  zd sigma = work[W_LAM + cand];
  for (int e = threadIdx.x; e < m; e += blockDim.x) {
    const double t = 1.0 + 0.5 * sin(1.7 * e + 0.3);   // fixed start: no zero entries, no structure
    yr[e] = zd(t, 0.0);
    yl[e] = zd(t, 0.0);
  }
  zd lam = sigma;
  for (int pass = 0; pass < 2; ++pass) {
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int r = e % m, c = e / m;
      A[r + c * ld] = Lm[r + c * MMAX] - sigma * Rat(r, c);
    }
    if (threadIdx.x == 0) s_ok = 1;
    __syncthreads();
    if (!lu_block(A, m, ld, piv, dsc)) { if (threadIdx.x == 0) s_ok = 0; }
    __syncthreads();
    if (!s_ok) {
      // sigma is an eigenvalue to working precision: nudge the zero pivots instead
      if (threadIdx.x == 0) {
        double an = 0.0;
        for (int e = 0; e < m * m; ++e) an = fmax(an, cabs_(Lm[(e % m) + (e / m) * MMAX]));
        for (int k = 0; k < m; ++k)
          if (cabs_(A[k + k * ld]) == 0.0) A[k + k * ld] = zd(1e-15 * (an > 0 ? an : 1.0));
      }
      __syncthreads();
    }
    const int steps = pass == 0 ? 4 : 2;
    for (int it = 0; it < steps; ++it) {
      // right-hand sides R y (warp 0) and R^H yl (warp 1)
      if (warp == 0)
        for (int r = lane; r < m; r += 32) { zd acc = zd(); for (int c = 0; c < m; ++c) acc += Rat(r, c) * yr[c]; tr[r] = acc; }
      if (warp == 1)
        for (int r = lane; r < m; r += 32) { zd acc = zd(); for (int c = 0; c < m; ++c) acc += cmul(Rat(c, r), yl[c]); tl[r] = acc; }
      __syncthreads();
      if (warp == 0) lu_solve_warp(A, m, ld, piv, tr);
      if (warp == 1) lu_solve_adj_warp(A, m, ld, piv, tl);
      __syncthreads();
      if (warp < 2) {   // normalise (largest entry 1 in modulus)
        zd* t = warp == 0 ? tr : tl;
        zd* y = warp == 0 ? yr : yl;
        double big = 0.0;
        for (int i = lane; i < m; i += 32) big = fmax(big, cabs_(t[i]));
        for (int o = 16; o > 0; o >>= 1) big = fmax(big, __shfl_xor_sync(0xffffffffu, big, o));
        const double sc = big > 0.0 ? 1.0 / big : 1.0;
        for (int i = lane; i < m; i += 32) y[i] = t[i] * sc;
      }
      __syncthreads();
    }
    // two-sided Rayleigh quotient of the pencil: (yl^H L y) / (yl^H R y)
    if (warp == 0) {
      zd num = zd(), den = zd();
      for (int r = lane; r < m; r += 32) {
        zd ly = zd(), ry = zd();
        for (int c = 0; c < m; ++c) { ly += Lm[r + c * MMAX] * yr[c]; ry += Rat(r, c) * yr[c]; }
        num += cmul(yl[r], ly);
        den += cmul(yl[r], ry);
      }
      num = warp_sum(num);
      den = warp_sum(den);
      if (lane == 0) s_lam = (cabs_(den) > 0.0) ? num / den : sigma;
    }
    __syncthreads();
    lam = s_lam;
    const bool finite = isfinite(lam.re) && isfinite(lam.im);
    // the FP32 shift was close enough: the quotient did not move
    if (!finite || cabs_(lam - sigma) <= 1e-6 * cabs_(lam)) break;
    sigma = lam;
  }
  zd* Y = work + W_Y + cand * MMAX;
  zd* YL = work + W_YL + cand * MMAX;
  for (int e = threadIdx.x; e < m; e += blockDim.x) { Y[e] = yr[e]; YL[e] = yl[e]; }
  if (threadIdx.x == 0) work[W_LAM2 + cand] = lam;
}

__global__ void __launch_bounds__(256) k_eig_c(RefreshInfo f, DevState* st, zd* work, zd* Wphi, zd* Wphit, int ldw,
                                               double* lam_out, int m, int raw) {
  const Layout Lay = make_layout(f);
  const EigInts ei = eig_ints(work);
  __shared__ int s_units;
  if (threadIdx.x == 0) {
    int units = 0, cols = 0;
    if (st->eig_status == 0 && *ei.ncand > 0) {
      zd lam[KMAX + NCAND_EXTRA];
      for (int c = 0; c < *ei.ncand; ++c) {
        // a candidate that refined to the eigenvalue of an earlier one is dropped
        lam[c] = work[W_LAM2 + c];
        for (int q = 0; q < c; ++q)
          if (cabs_(lam[c] - work[W_LAM2 + q]) <= 1e-8 * cabs_(lam[c])) { lam[c] = zd(nan(""), 0.0); break; }
      }
      units = select_units(lam, *ei.ncand, f.k, f.real_path, ei.sel, ei.pair, &cols);
    }
    *ei.units = units;
    *ei.cols = cols;
    st->kk = cols;
    s_units = units;
  }
  __syncthreads();
  const int units = s_units;
  if (st->eig_status != 0 || units <= 0) {
    for (int e = threadIdx.x; e < m * 2; e += blockDim.x) {
      zd* out = e >= m ? Wphit : Wphi;
      for (int c = 0; c < ldw; ++c) out[(e % m) * ldw + c] = zd();
    }
    return;
  }
  zd* Lv = work + W_GH;           // scratch: selected left vectors (stride MMAX)
  zd* Rv = Lv + MMAX * KMAX;      // selected right vectors
  for (int e = threadIdx.x; e < m * units; e += blockDim.x) {
    const int r = e % m, u = e / m;
    Rv[r + u * MMAX] = work[W_Y + ei.sel[u] * MMAX + r];
    Lv[r + u * MMAX] = work[W_YL + ei.sel[u] * MMAX + r];
  }
  __syncthreads();
  if (threadIdx.x < 2 * units) {   // unit norm, largest component real and positive
    const int u = threadIdx.x % units;
    const bool left = threadIdx.x >= units;
    zd* w = (left ? Lv : Rv) + u * MMAX;
    double nrm = 0.0, big = -1.0;
    int bi = 0;
    for (int r = 0; r < m; ++r) { const double a2 = abs2(w[r]); nrm += a2; if (a2 > big) { big = a2; bi = r; } }
    nrm = sqrt(nrm);
    const zd ph = nrm > 0.0 && big > 0.0 ? conjg(w[bi]) * (1.0 / (cabs_(w[bi]) * nrm)) : zd(1.0);
    for (int r = 0; r < m; ++r) w[r] = w[r] * ph;
  }
  __syncthreads();
  if (threadIdx.x == 0 && lam_out) {
    int col = 0;
    for (int u = 0; u < units; ++u) {
      const zd lam = work[W_LAM2 + ei.sel[u]];
      lam_out[2 * col] = lam.re; lam_out[2 * col + 1] = lam.im;
      if (ei.pair[u]) { lam_out[2 * col + 2] = lam.re; lam_out[2 * col + 3] = -lam.im; }
      col += ei.pair[u] ? 2 : 1;
    }
  }
  // W (right) and Wt (left), row r = Phi column r, Phi scaling folded in (v_m = r_{m-1} /
  // ||r_{m-1}||, vt_m = rt_{m-1} ||r_{m-1}|| / conj(rho_{m-1})); a conjugate pair of a real
  // problem contributes its real and imaginary parts
  for (int e = threadIdx.x; e < m * 2; e += blockDim.x) {
    const int r = e % m;
    const bool left = e >= m;
    zd* out = left ? Wphit : Wphi;
    zd sc = zd(1.0);
    if (!raw && (f.case_id == 0 || r >= Lay.nUphi)) {
      const int g = (f.case_id == 0 ? 1 + (f.j - 1) * f.s + r : Lay.g0 + Lay.v_off + (r - Lay.nUphi));
      const double rn = st->h_rnorm[(g - 1) % HR];
      sc = left ? zd(rn) / conjg(st->h_rho[(g - 1) % HR]) : zd(1.0 / rn);
    }
    int col = 0;
    for (int u = 0; u < units; ++u) {
      const zd wv = (left ? Lv : Rv)[r + u * MMAX];
      if (f.real_path) {
        out[r * ldw + col] = zd(sc.re * wv.re, 0.0);
        if (ei.pair[u]) { out[r * ldw + col + 1] = zd(sc.re * wv.im, 0.0); col += 2; } else col += 1;
      } else {
        out[r * ldw + col] = sc * wv;
        col += 1;
      }
    }
    for (int c = col; c < ldw; ++c) out[r * ldw + c] = zd();
  }
}

static void launch_eig3(const RefreshInfo& info, DevState* st, zd* work, zd* Wphi, zd* Wphit, int ldw,
                        double* lam_out, int has_R, int m, int raw, cudaStream_t s) {
  const int ld = m | 1;
  const size_t smem_a = (size_t)(2 * m * ld + MMAX) * sizeof(zd) + 4 * sizeof(double) + MMAX * sizeof(int);
  const size_t smem_b = (size_t)(m * ld + 4 * MMAX) * sizeof(zd) + 4 * sizeof(double) + MMAX * sizeof(int);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_eig_a, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * MMAX * (MMAX + 1) * sizeof(zd) + 8192);
    cudaFuncSetAttribute(k_eig_b, cudaFuncAttributeMaxDynamicSharedMemorySize, MMAX * (MMAX + 1) * sizeof(zd) + 8192);
    attr_set = true;
  }
  k_eig_a<<<1, 256, smem_a, s>>>(info, st, work, has_R, m);
  k_eig_b<<<KMAX + NCAND_EXTRA, 256, smem_b, s>>>(work, m, has_R);
  k_eig_c<<<1, 256, 0, s>>>(info, st, work, Wphi, Wphit, ldw, lam_out, m, raw);
}

template <class T>
void launch_dense_refresh(const RefreshInfo& info, DevState* st, const typename traits<T>::acc* G, zd* work,
                          zd* Wphi, zd* Wphit, int ldw, double* lam_out, cudaStream_t s) {
  typedef typename traits<T>::acc A;
  int m;
  int has_R = 1;
  if (info.case_id == 0) {
    k_t1<<<8, 256, 0, s>>>(info, st, work);
    m = info.s;
    has_R = 0;
  } else {
    k_build_h<A><<<32, 256, 0, s>>>(info, st, work);
    k_gh<A><<<64, 256, 0, s>>>(info, st, G, work);
    k_lr<A><<<64, 256, 0, s>>>(info, st, G, work);
    m = (info.case_id == 2 ? info.kc : info.kp) + info.s;
  }
  launch_eig3(info, st, work, Wphi, Wphit, ldw, lam_out, has_R, m, 0, s);
}

// Component entry: L (and R) already in work (W_L, W_R, ld MMAX); st is a scratch state that
// receives kk and eig_status.  Eigenvectors are written unscaled (W, Wt: m x KMAX rows).
void launch_dense_eig_host(int real_path, int m, const zd* L, const zd* R, int has_R, int k, zd* W, zd* Wt,
                           double* lam, int* kk, int* status, zd* work, cudaStream_t s) {
  (void)L; (void)R; (void)kk; (void)status;
  RefreshInfo info{};
  info.case_id = 0;
  info.j = 1;
  info.s = m;
  info.k = k;
  info.real_path = real_path;
  DevState* st = reinterpret_cast<DevState*>(work + W_END);
  launch_eig3(info, st, work, W, Wt, KMAX, lam, has_R, m, 1, s);
}

// ------------------------------------------------------------------------------------
// SVD of Ct_j^H C_j (Section 4.3).  Input: S2 = [Ct C]^H [C Ct] (2 kmax x 2 kmax, row-major)
// holding Ct^H C (top-left), Ct^H Ct (top-right), C^H C (bottom-left).  k = *k_dev columns.
// Output: Nmat = D^{-1} N_p, Mmat = Dt^{-1} M_p (kmax x KMAX row-major), sigma, *p_dev.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_svd(int real_path, const int* k_dev, int kmax, const zd* S2, double svd_tol,
                                             zd* Nmat, zd* Mmat, double* sigma, int* p_dev, double* Dc_dev,
                                             int* status) {
  __shared__ zd A[KMAX * KMAX];   // column-major k x k: A = S_norm, rotated to M Sigma
  __shared__ zd V[KMAX * KMAX];   // accumulated right rotations (N)
  __shared__ double dn[KMAX], dtn[KMAX], sg[KMAX];
  __shared__ int ord[KMAX], s_rot, s_p;
  const int k = min(*k_dev, kmax);
  const int ld2 = 2 * kmax;
  if (k <= 0) {
    if (threadIdx.x == 0) { *p_dev = 0; *status = 0; }
    return;
  }
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    dn[c] = sqrt(fmax(S2[(kmax + c) * ld2 + c].re, 0.0));          // ||C e_c||   (C^H C diag)
    dtn[c] = sqrt(fmax(S2[c * ld2 + kmax + c].re, 0.0));           // ||Ct e_c||  (Ct^H Ct diag)
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int r = e % k, c = e / k;
    const double sr = dtn[r] > 0.0 ? 1.0 / dtn[r] : 0.0, scc = dn[c] > 0.0 ? 1.0 / dn[c] : 0.0;
    zd a = S2[r * ld2 + c] * (sr * scc);
    if (real_path) a.im = 0.0;
    A[r + c * k] = a;
    V[r + c * k] = r == c ? zd(1.0) : zd();
  }
  __syncthreads();
  // one-sided Jacobi, round-robin pairs (kk even), warp w handles pair w
  const int kk = (k + 1) & ~1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < kk - 1; ++round) {
      for (int pr = warp; pr < kk / 2; pr += nw) {
        // circle method: position 0 fixed, positions 1..kk-1 rotate by `round`
        int a = pr == 0 ? 0 : 1 + (pr - 1 + round) % (kk - 1);
        const int pb = kk - 1 - pr;
        int b = 1 + (pb - 1 + round) % (kk - 1);
        if (a > b) { const int t = a; a = b; b = t; }
        if (b >= k || a == b) continue;
        double app = 0.0, aqq = 0.0;
        zd apq = zd();
        for (int r = lane; r < k; r += 32) {
          const zd x = A[r + a * k], y = A[r + b * k];
          app += abs2(x); aqq += abs2(y); apq += cmul(x, y);
        }
        app = warp_sum(app); aqq = warp_sum(aqq); apq = warp_sum(apq);
        app = __shfl_sync(0xffffffffu, app, 0); aqq = __shfl_sync(0xffffffffu, aqq, 0);
        apq = zd(__shfl_sync(0xffffffffu, apq.re, 0), __shfl_sync(0xffffffffu, apq.im, 0));
        const double g = cabs_(apq);
        if (g <= 1e-15 * sqrt(app * aqq) || g == 0.0) continue;
        if (lane == 0) s_rot = 1;
        // rotate columns a, b so that they become orthogonal
        const double zeta = (aqq - app) / (2.0 * g);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        const zd e = apq * (1.0 / g);   // phase of a^H b
        __syncwarp();                    // all lanes' reads of columns a, b precede the writes
        for (int r = lane; r < k; r += 32) {
          const zd x = A[r + a * k], y = A[r + b * k];
          A[r + a * k] = cs * x - sn * (conjg(e) * y);
          A[r + b * k] = sn * (e * x) + cs * y;
          const zd vx = V[r + a * k], vy = V[r + b * k];
          V[r + a * k] = cs * vx - sn * (conjg(e) * vy);
          V[r + b * k] = sn * (e * vx) + cs * vy;
        }
      }
      __syncthreads();
    }
    if (!s_rot) break;
    __syncthreads();
  }
  // singular values, order
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < k; ++r) s += abs2(A[r + c * k]);
    sg[c] = sqrt(s);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < k; ++c) ord[c] = c;
    for (int a = 1; a < k; ++a) {
      const int v = ord[a];
      int b = a - 1;
      while (b >= 0 && (sg[ord[b]] < sg[v] || (sg[ord[b]] == sg[v] && ord[b] > v))) { ord[b + 1] = ord[b]; --b; }
      ord[b + 1] = v;
    }
    int p = 0;
    while (p < k && sg[ord[p]] >= svd_tol) ++p;
    s_p = p;
    *p_dev = p;
    *status = 0;
  }
  __syncthreads();
  const int p = s_p;
  // Nmat[a, c] = (1/dn[a]) N[a, ord c]; Mmat[a, c] = (1/dtn[a]) M[a, ord c], M = A / sigma
  for (int e = threadIdx.x; e < kmax * KMAX; e += blockDim.x) {
    const int a = e / KMAX, c = e % KMAX;
    zd nv = zd(), mv = zd();
    if (a < k && c < p) {
      const int oc = ord[c];
      nv = V[a + oc * k] * (dn[a] > 0.0 ? 1.0 / dn[a] : 0.0);
      mv = A[a + oc * k] * ((dtn[a] > 0.0 ? 1.0 / dtn[a] : 0.0) / sg[oc]);
    }
    Nmat[e] = nv;
    Mmat[e] = mv;
  }
  for (int c = threadIdx.x; c < KMAX; c += blockDim.x) {
    const double sv = c < p ? sg[ord[c]] : 0.0;
    if (sigma) sigma[c] = sv;
    if (Dc_dev) Dc_dev[c] = c < p ? sv : 1.0;
  }
}

void launch_dense_svd(int real_path, const int* k_dev, int kmax, const zd* S, const double* nC, const double* nCt,
                      double svd_tol, zd* Nmat, zd* Mmat, double* sigma, int* p_dev, double* Dc_dev, int* status_dev,
                      cudaStream_t s) {
  (void)nC; (void)nCt;
  k_svd<<<1, 256, 0, s>>>(real_path, k_dev, kmax, S, svd_tol, Nmat, Mmat, sigma, p_dev, Dc_dev, status_dev);
}

template void launch_dense_refresh<double>(const RefreshInfo&, DevState*, const double*, zd*, zd*, zd*, int, double*,
                                           cudaStream_t);
template void launch_dense_refresh<float>(const RefreshInfo&, DevState*, const double*, zd*, zd*, zd*, int, double*,
                                          cudaStream_t);
template void launch_dense_refresh<cplx<double>>(const RefreshInfo&, DevState*, const zd*, zd*, zd*, zd*, int,
                                                 double*, cudaStream_t);
template void launch_dense_refresh<cplx<float>>(const RefreshInfo&, DevState*, const zd*, zd*, zd*, zd*, int,
                                                double*, cudaStream_t);

}  // namespace rb

namespace rb {
int64_t dense_state_offset() { return W_END; }
int64_t dense_work_elems() { return W_END + (int64_t)(sizeof(DevState) + sizeof(zd) - 1) / (int64_t)sizeof(zd) + 1; }
int64_t dense_off_L() { return W_L; }
int64_t dense_off_R() { return W_R; }
}  // namespace rb
