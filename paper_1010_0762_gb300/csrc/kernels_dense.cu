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
                  W_L = W_GH + PSIMAX * MMAX, W_R = W_L + MMAX * MMAX, W_LU = W_R + MMAX * MMAX,
                  W_Y = W_LU + MMAX * MMAX, W_YL = W_Y + MMAX * KMAX, W_END = W_YL + MMAX * KMAX;

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
template <class A>
__global__ void k_gh(RefreshInfo f, const DevState* st, const A* G, zd* work) {
  const Layout L = make_layout(f);
  const zd* Hd = work + W_HD;
  zd* GH = work + W_GH;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L.nPsi * L.nPhi; e += gridDim.x * blockDim.x) {
    const int a = e % L.nPsi, b = e / L.nPsi;
    zd sa, sta;
    psi_scale(st, L, a, &sa, &sta);
    zd s = zd();
    for (int c = 0; c < L.nPsi; ++c) {
      const zd h = Hd[c + b * PSIMAX];
      if (h.re == 0.0 && h.im == 0.0) continue;
      zd sc, stc;
      psi_scale(st, L, c, &sc, &stc);
      s += to_zd(G[(int64_t)a * f.my + c]) * sc * h;
    }
    GH[a + b * PSIMAX] = conjg(sta) * s;
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
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int c = e % m, b = e / m;
    const int yc = phi_ycol(L, b);
    zd sy, sty;
    if (yc < L.nPsi) psi_scale(st, L, yc, &sy, &sty); else sy = zd(1.0);
    zd sl = zd(), sr = zd();
    for (int a = 0; a < L.nPsi; ++a) {
      const zd h = Htd[a + c * PSIMAX];
      if (h.re == 0.0 && h.im == 0.0) continue;
      zd sa, sta;
      psi_scale(st, L, a, &sa, &sta);
      const zd hc = conjg(h);
      sl += hc * GH[a + b * PSIMAX];
      sr += hc * (conjg(sta) * to_zd(G[(int64_t)a * f.my + yc]) * sy);
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

// Givens G = [[c, s], [-conj(s), c]] with G [a; b] = [r; 0]
__device__ void givens(zd a, zd b, double* c, zd* s) {
  const double ab = cabs_(b);
  if (ab == 0.0) { *c = 1.0; *s = zd(); return; }
  const double aa = cabs_(a);
  if (aa == 0.0) { *c = 0.0; *s = conjg(b) * (1.0 / ab); return; }
  const double nr = hypot(aa, ab);
  *c = aa / nr;
  *s = (a * (1.0 / aa)) * conjg(b) * (1.0 / nr);
}

struct EigSmem {
  zd* T;   // m x m, column-major, ld = m
  zd* Q;
  int* piv;
  zd* vec;  // scratch MMAX
  double* dsc;
  int* ish;
};

// Block-wide: LU with partial pivoting of A (m x m, ld m) in place; piv[k] = pivot row.
__device__ bool lu_block(zd* A, int m, int* piv, double* dsc, int* ish) {
  for (int k = 0; k < m; ++k) {
    // pivot search (warp 0)
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = k;
      for (int r = k + threadIdx.x; r < m; r += 32) {
        const double v = cabs_(A[r + k * m]);
        if (v > best) { best = v; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) { piv[k] = bi; dsc[0] = best; }
    }
    __syncthreads();
    const int p = piv[k];
    if (dsc[0] == 0.0) return false;
    if (p != k)
      for (int c = threadIdx.x; c < m; c += blockDim.x) {
        const zd t = A[k + c * m]; A[k + c * m] = A[p + c * m]; A[p + c * m] = t;
      }
    __syncthreads();
    const zd inv = zd(1.0) / A[k + k * m];
    for (int r = k + 1 + threadIdx.x; r < m; r += blockDim.x) A[r + k * m] = A[r + k * m] * inv;
    __syncthreads();
    const int rem = m - k - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int r = k + 1 + e % rem, c = k + 1 + e / rem;
      A[r + c * m] -= A[r + k * m] * A[k + c * m];
    }
    __syncthreads();
  }
  (void)ish;
  return true;
}

// Block-wide: B <- A^{-1} B for the LU of A (B: m x nb, ld m)
__device__ void lu_solve_block(const zd* LU, int m, const int* piv, zd* B, int nb) {
  for (int col = threadIdx.x; col < nb; col += blockDim.x) {
    zd* b = B + col * m;
    for (int k = 0; k < m; ++k) { const int p = piv[k]; if (p != k) { const zd t = b[k]; b[k] = b[p]; b[p] = t; } }
    for (int r = 0; r < m; ++r) { zd s = b[r]; for (int c = 0; c < r; ++c) s -= LU[r + c * m] * b[c]; b[r] = s; }
    for (int r = m - 1; r >= 0; --r) {
      zd s = b[r];
      for (int c = r + 1; c < m; ++c) s -= LU[r + c * m] * b[c];
      b[r] = s / LU[r + r * m];
    }
  }
  __syncthreads();
}

// Block-wide: columns of B (stride ldb) <- A^{-H} B for the LU of A = P^T Lw U
__device__ void lu_solve_adj_block(const zd* LU, int m, const int* piv, zd* B, int nb, int ldb) {
  for (int col = threadIdx.x; col < nb; col += blockDim.x) {
    zd* b = B + col * ldb;
    // A = P^T Lw U  =>  A^H = U^H Lw^H P ;  solve U^H y = b, Lw^H z = y, x = P^T z
    for (int r = 0; r < m; ++r) {
      zd s = b[r];
      for (int c = 0; c < r; ++c) s -= conjg(LU[c + r * m]) * b[c];
      b[r] = s / conjg(LU[r + r * m]);
    }
    for (int r = m - 1; r >= 0; --r) {
      zd s = b[r];
      for (int c = r + 1; c < m; ++c) s -= conjg(LU[c + r * m]) * b[c];
      b[r] = s;
    }
    for (int k = m - 1; k >= 0; --k) { const int p = piv[k]; if (p != k) { const zd t = b[k]; b[k] = b[p]; b[p] = t; } }
  }
  __syncthreads();
}

// Block-wide Householder reduction of T (m x m) to upper Hessenberg, Q <- Q P_1 ... P_{m-2}
__device__ void hessenberg_block(zd* T, zd* Q, int m, zd* v, double* dsc) {
  for (int j = 0; j < m - 2; ++j) {
    const int len = m - j - 1;
    // norm of x = T[j+1.., j]
    if (threadIdx.x < 32) {
      double s = 0.0;
      for (int r = threadIdx.x; r < len; r += 32) s += abs2(T[j + 1 + r + j * m]);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0) dsc[0] = s;
    }
    __syncthreads();
    const double nx2 = dsc[0];
    const zd x0 = T[j + 1 + j * m];
    const double tail = nx2 - abs2(x0);
    if (tail <= 1e-300) { __syncthreads(); continue; }
    const double nx = sqrt(nx2);
    const double ax0 = cabs_(x0);
    const zd ph = ax0 > 0.0 ? x0 * (1.0 / ax0) : zd(1.0);
    const zd alpha = -(ph * nx);                 // x - alpha e1 avoids cancellation
    for (int r = threadIdx.x; r < len; r += blockDim.x) v[r] = T[j + 1 + r + j * m];
    __syncthreads();
    if (threadIdx.x == 0) v[0] = v[0] - alpha;
    __syncthreads();
    const double vv = tail + abs2(x0 - alpha);
    const double f = 2.0 / vv;
    // left: T[j+1.., c] -= f v (v^H T[j+1.., c]) for c >= j
    for (int c = j + threadIdx.x; c < m; c += blockDim.x) {
      zd w = zd();
      for (int r = 0; r < len; ++r) w += cmul(v[r], T[j + 1 + r + c * m]);
      w = w * f;
      for (int r = 0; r < len; ++r) T[j + 1 + r + c * m] -= v[r] * w;
    }
    __syncthreads();
    // right: T[r, j+1..] -= f (T[r, j+1..] v) v^H for all rows; Q likewise
    for (int r = threadIdx.x; r < 2 * m; r += blockDim.x) {
      zd* M = r < m ? T : Q;
      const int rr = r < m ? r : r - m;
      zd u = zd();
      for (int c = 0; c < len; ++c) u += M[rr + (j + 1 + c) * m] * v[c];
      u = u * f;
      for (int c = 0; c < len; ++c) M[rr + (j + 1 + c) * m] -= u * conjg(v[c]);
    }
    __syncthreads();
    for (int r = j + 2 + threadIdx.x; r < m; r += blockDim.x) T[r + j * m] = zd();
    __syncthreads();
  }
}

// Warp 0: shifted QR (single shift, Wilkinson, implicit via Givens) on the Hessenberg T
// to upper triangular (Schur) form, accumulating Q.  Returns false if it does not converge.
__device__ bool schur_warp(zd* T, zd* Q, int m, int* dbg) {
  const int lane = threadIdx.x & 31;
  const double eps = 2.220446049250313e-16;
  int hi = m - 1, iter = 0, total = 0;
  while (hi > 0) {
    // find lo: deflate small subdiagonals
    int lo = hi;
    while (lo > 0) {
      const double sub = cabs_(T[lo + (lo - 1) * m]);
      const double dsum = cabs_(T[lo + lo * m]) + cabs_(T[lo - 1 + (lo - 1) * m]);
      if (sub <= eps * (dsum > 0.0 ? dsum : 1.0)) { __syncwarp(); if (lane == 0) T[lo + (lo - 1) * m] = zd(); __syncwarp(); break; }
      --lo;
    }
    if (lo == hi) { --hi; iter = 0; continue; }
    if (!finite_of(T[hi + hi * m]) || !finite_of(T[hi + (hi - 1) * m])) {
      if (lane == 0) { dbg[0] = 3; dbg[1] = lo; dbg[2] = hi; dbg[3] = iter; dbg[4] = total; }
      return false;
    }
    if (++total > 60 * m) {
      if (lane == 0) { dbg[0] = 2; dbg[1] = lo; dbg[2] = hi; dbg[3] = iter; dbg[4] = total; }
      return false;
    }
    ++iter;
    // Wilkinson shift from the trailing 2x2 of the window
    const zd a = T[hi - 1 + (hi - 1) * m], b = T[hi - 1 + hi * m], c = T[hi + (hi - 1) * m], d = T[hi + hi * m];
    zd mu;
    if (iter % 11 == 10) {
      mu = d + zd(cabs_(c) * 0.75);   // exceptional shift
    } else {
      const zd tr = a + d, det = a * d - b * c;
      const zd half = tr * 0.5;
      const zd disc = half * half - det;
      // complex sqrt
      const double rdisc = cabs_(disc);
      // clamp both radicands: hypot carries up to 2 ulp of error, so |disc| + Re(disc) can
      // round below zero when disc is (nearly) a negative real, as it is for the conjugate
      // eigenvalue pairs of a real matrix
      double sr = sqrt(fmax(0.0, 0.5 * (rdisc + disc.re))), si = sqrt(fmax(0.0, 0.5 * (rdisc - disc.re)));
      if (disc.im < 0.0) si = -si;
      const zd sq(sr, si);
      const zd l1 = half + sq, l2 = half - sq;
      mu = cabs_(l1 - d) < cabs_(l2 - d) ? l1 : l2;
    }
    // implicit single-shift sweep on [lo, hi]
    zd x = T[lo + lo * m] - mu, y = T[lo + 1 + lo * m];
    for (int k = lo; k < hi; ++k) {
      double cs;
      zd sn;
      if (k == lo) givens(x, y, &cs, &sn);
      else givens(T[k + (k - 1) * m], T[k + 1 + (k - 1) * m], &cs, &sn);
      // every lane has read the entries that define the rotation (and, for k == lo, the
      // shift) before any lane overwrites them below
      __syncwarp();
      const int c0 = k > lo ? k - 1 : lo;
      // rows k, k+1, columns c0..m-1
      for (int col = c0 + lane; col < m; col += 32) {
        const zd p = T[k + col * m], q = T[k + 1 + col * m];
        T[k + col * m] = cs * p + sn * q;
        T[k + 1 + col * m] = cs * q - conjg(sn) * p;
      }
      __syncwarp();
      // columns k, k+1, rows 0..min(k+2, hi)
      const int r1 = k + 2 < hi ? k + 2 : hi;
      for (int row = lane; row <= r1; row += 32) {
        const zd p = T[row + k * m], q = T[row + (k + 1) * m];
        T[row + k * m] = cs * p + conjg(sn) * q;
        T[row + (k + 1) * m] = cs * q - sn * p;
      }
      for (int row = lane; row < m; row += 32) {
        const zd p = Q[row + k * m], q = Q[row + (k + 1) * m];
        Q[row + k * m] = cs * p + conjg(sn) * q;
        Q[row + (k + 1) * m] = cs * q - sn * p;
      }
      __syncwarp();
      if (k > lo && lane == 0) T[k + 1 + (k - 1) * m] = zd();
      __syncwarp();
    }
  }
  return true;
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

// Full eigen pipeline in one block; writes Wphi / Wphit (m x ldw, row a = Phi column) with
// the Phi scalings folded in, the selected eigenvalues, st->kk and st->eig_status.
__global__ void __launch_bounds__(256) k_eig(RefreshInfo f, DevState* st, zd* work, zd* Wphi, zd* Wphit, int ldw,
                                             double* lam_out, int has_R, int m_in, int raw) {
  extern __shared__ unsigned char smraw[];
  const Layout Lay = make_layout(f);
  const int m = m_in > 0 ? m_in : (f.case_id == 0 ? f.s : Lay.nPhi);
  zd* T = reinterpret_cast<zd*>(smraw);
  zd* Q = T + m * m;
  zd* v = Q + m * m;
  double* dsc = reinterpret_cast<double*>(v + MMAX);
  int* piv = reinterpret_cast<int*>(dsc + 4);
  __shared__ int s_sel[KMAX], s_pair[KMAX], s_units, s_cols, s_ok;
  zd* Lm = work + W_L;
  zd* Rm = work + W_R;
  zd* LU = work + W_LU;
  zd* Y = work + W_Y;
  zd* YL = work + W_YL;
  if (threadIdx.x == 0) s_ok = 1;
  // M = R^{-1} L   (T <- R, LU; Q <- L, solve)
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int r = e % m, c = e / m;
    Q[e] = Lm[r + c * MMAX];
    if (has_R) T[e] = Rm[r + c * MMAX];
  }
  __syncthreads();
  if (has_R) {
    if (!lu_block(T, m, piv, dsc, nullptr)) { if (threadIdx.x == 0) s_ok = 0; }
    __syncthreads();
    if (!s_ok) { if (threadIdx.x == 0) { st->eig_status = 1; st->kk = 0; } return; }
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) LU[e] = T[e];
    __syncthreads();
    lu_solve_block(T, m, piv, Q, m);
  }
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) { T[e] = Q[e]; Q[e] = (e % m == e / m) ? zd(1.0) : zd(); }
  __syncthreads();
  hessenberg_block(T, Q, m, v, dsc);
  if (threadIdx.x < 32) {
    const bool ok = schur_warp(T, Q, m, st->dbg);
    if (threadIdx.x == 0 && !ok) s_ok = 0;
  }
  __syncthreads();
  if (!s_ok) { if (threadIdx.x == 0) { st->eig_status = 2; st->kk = 0; } return; }
  // eigenvalues and selection
  if (threadIdx.x == 0) {
    zd lam[MMAX];
    for (int i = 0; i < m; ++i) lam[i] = T[i + i * m];
    int cols = 0;
    s_units = select_units(lam, m, f.k, f.real_path, s_sel, s_pair, &cols);
    s_cols = cols;
  }
  __syncthreads();
  const int units = s_units;
  // eigenvectors of the triangular T: right y (back substitution), left yl (forward)
  double tn = 0.0;
  for (int e = 0; e < m; ++e) tn = fmax(tn, cabs_(T[e + e * m]));
  const double small = 1e-14 * (tn > 0.0 ? tn : 1.0);
  for (int u = threadIdx.x; u < 2 * units; u += blockDim.x) {
    const int unit = u % units;
    const bool left = u >= units;
    const int i = s_sel[unit];
    const zd lam = T[i + i * m];
    zd* y = (left ? YL : Y) + unit * MMAX;
    for (int r = 0; r < m; ++r) y[r] = zd();
    y[i] = zd(1.0);
    if (!left) {
      for (int r = i - 1; r >= 0; --r) {
        zd s = zd();
        for (int c = r + 1; c <= i; ++c) s += T[r + c * m] * y[c];
        zd d = T[r + r * m] - lam;
        if (cabs_(d) < small) d = zd(small);
        y[r] = -(s / d);
      }
    } else {
      // y^H T = lam y^H  <=>  (T - lam I)^H y = 0, y_i = 1, y_r = 0 for r < i
      for (int l = i + 1; l < m; ++l) {
        zd s = zd();
        for (int p = i; p < l; ++p) s += conjg(T[p + l * m]) * y[p];
        zd d = conjg(lam) - conjg(T[l + l * m]);
        if (cabs_(d) < small) d = zd(small);
        y[l] = s / d;
      }
    }
  }
  __syncthreads();
  // back-transform: w = Q y -> Rm columns, u = Q yl -> Lm columns (L, R already consumed)
  for (int e = threadIdx.x; e < m * units * 2; e += blockDim.x) {
    const int r = e % m, u = (e / m) % units;
    const bool left = e >= m * units;
    const zd* y = (left ? YL : Y) + u * MMAX;
    zd s = zd();
    for (int c = 0; c < m; ++c) s += Q[r + c * m] * y[c];
    if (left) Lm[r + u * MMAX] = s; else Rm[r + u * MMAX] = s;
  }
  __syncthreads();
  // left vectors of the pencil: x = R^{-H} u
  if (has_R) lu_solve_adj_block(LU, m, piv, Lm, units, MMAX);
  // unit norm, largest component real and positive
  if (threadIdx.x < 2 * units) {
    const int u = threadIdx.x % units;
    const bool left = threadIdx.x >= units;
    zd* w = (left ? Lm : Rm) + u * MMAX;
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
      const zd lam = T[s_sel[u] + s_sel[u] * m];
      lam_out[2 * col] = lam.re; lam_out[2 * col + 1] = lam.im;
      if (s_pair[u]) { lam_out[2 * col + 2] = lam.re; lam_out[2 * col + 3] = -lam.im; }
      col += s_pair[u] ? 2 : 1;
    }
  }
  // write W (right) and Wt (left), row r = Phi column r, with the Phi scaling folded in
  // (v_m = r_{m-1}/||r_{m-1}||, vt_m = rt_{m-1} ||r_{m-1}|| / conj(rho_{m-1})); a conjugate
  // pair of a real problem contributes its real and imaginary parts.
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
      const zd wv = (left ? Lm : Rm)[r + u * MMAX];
      if (f.real_path) {
        out[r * ldw + col] = zd(sc.re * wv.re, 0.0);
        if (s_pair[u]) { out[r * ldw + col + 1] = zd(sc.re * wv.im, 0.0); col += 2; } else col += 1;
      } else {
        out[r * ldw + col] = sc * wv;
        col += 1;
      }
    }
    for (int c = col; c < ldw; ++c) out[r * ldw + c] = zd();
  }
  if (threadIdx.x == 0) { st->kk = s_cols; st->eig_status = 0; }
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
  const size_t smem = (size_t)(2 * m * m + MMAX) * sizeof(zd) + 4 * sizeof(double) + MMAX * sizeof(int);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * MMAX * MMAX * sizeof(zd) + 8192);
    attr_set = true;
  }
  k_eig<<<1, 256, smem, s>>>(info, st, work, Wphi, Wphit, ldw, lam_out, has_R, m, 0);
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
  const size_t smem = (size_t)(2 * m * m + MMAX) * sizeof(zd) + 4 * sizeof(double) + MMAX * sizeof(int);
  cudaFuncSetAttribute(k_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * MMAX * MMAX * sizeof(zd) + 8192);
  k_eig<<<1, 256, smem, s>>>(info, st, work, W, Wt, KMAX, lam, has_R, m, 1);
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
