// kernels_dense.cu -- the small FP64 problems of the recycle-space refresh, on the GPU.
//
//  * k_build: H_j, Ht_j of Section 4.1 / 4.2 from the iteration scalars (T of Section 4.1,
//    B_j = Chat^H A V_j, Bt_j = Ccheck^H A^H Vt_j from the zeta histories), the Lanczos
//    scalings v_m = r_{m-1}/||r_{m-1}||, vt_m = rt_{m-1}/(v_m, rt_{m-1}) applied to the raw
//    Gram, and the pencil L = Ht^H (Psit^H Psi) H, R = Ht^H (Psit^H Phi) of eq.
//    (finalGenEigValue).  Many blocks (plain dense products of order <= 130).
//  * k_eig_cl / k_eig_h / k_eig_c: the eigen pipeline of the pencil (L, R) -- FP64 Gauss-Jordan
//    and Householder reduction on a thread-block cluster, FP32 QR eigenvalues as shifts, FP64
//    inverse iteration per candidate, selection of the eigenvalues closest to the origin with
//    their right and left eigenvectors (described in full above k_eig_cl).
//  * k_svd: one block.  One-sided (Hestenes) Jacobi SVD of Ct_j^H C_j after unit-norm column
//    scaling (Section 4.3, eq. (equationSVD)): FP32 sweeps, FP64 Newton-Schulz
//    re-orthonormalisation, FP64 polish sweeps; truncation at svd_tol; rotation coefficients.
#include <algorithm>

#include <cooperative_groups.h>

#include "internal.cuh"

namespace rb {

namespace cg = cooperative_groups;

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
// Lm [MMAX x MMAX], Rm [MMAX x MMAX] (column-major), then the eigen pipeline's data:
// H (Hessenberg form of R^{-1} L), QV / QF (Householder vectors and factors), RI (R^{-1}),
// Y / YL (candidate eigenvectors), LAM / LAM2 (FP32 shifts, refined eigenvalues), integers.
constexpr int64_t W_HD = 0, W_HTD = W_HD + PSIMAX * MMAX, W_GH = W_HTD + PSIMAX * MMAX,
                  W_L = W_GH + PSIMAX * MMAX, W_R = W_L + MMAX * MMAX,
                  W_H = W_R + MMAX * MMAX, W_QV = W_H + MMAX * MMAX, W_QF = W_QV + MMAX * MMAX,
                  W_RI = W_QF + MMAX, W_Q = W_RI + MMAX * MMAX,
                  W_Y = W_Q + MMAX * MMAX, W_YL = W_Y + MMAX * (KMAX + 8), W_LAM = W_YL + MMAX * (KMAX + 8),
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
// dense eigen pipeline: shared helpers and the eigenvalue selection
// ------------------------------------------------------------------------------------
typedef cplx<float> zf;
// |re| + |im|: the pivot and scale measure of complex LU (no square root; within a factor
// sqrt(2) of the modulus).  FP64 hypot costs dozens of FP64 instructions on this part.
__device__ __forceinline__ double cabs1_(zd a) { return fabs(a.re) + fabs(a.im); }
__device__ __forceinline__ float cabs1_(zf a) { return fabsf(a.re) + fabsf(a.im); }

// Selection of eigenvalue indices (reading: k closest to the origin; on a real problem a
// conjugate pair is one unit of two columns, k-1 columns if it straddles the cut).
// Writes sel[u] = index, pairflag[u]; returns number of units; *ncols = columns.
__device__ int select_units(const zd* lam, int m, int k, int real_path, int* sel, int* pairflag, int* ncols) {
  // thread 0 only
  int order[MMAX];
  int cnt = 0;
  for (int i = 0; i < m; ++i)
    if (isfinite(lam[i].re) && isfinite(lam[i].im)) order[cnt++] = i;
  // insertion sort by (|lam|, index); |lam|^2 orders the same way without square roots
  double mag[MMAX];
  for (int i = 0; i < m; ++i) mag[i] = abs2(lam[i]);
  for (int a = 1; a < cnt; ++a) {
    const int v = order[a];
    const double av = mag[v];
    int b = a - 1;
    while (b >= 0 && (mag[order[b]] > av || (mag[order[b]] == av && order[b] > v))) { order[b + 1] = order[b]; --b; }
    order[b + 1] = v;
  }
  bool used[MMAX];
  for (int i = 0; i < m; ++i) used[i] = false;
  int units = 0, cols = 0;
  for (int t = 0; t < cnt; ++t) {
    const int i = order[t];
    if (used[i]) continue;
    const bool isreal = !real_path || lam[i].im * lam[i].im <= 1e-20 * (mag[i] > 0.0 ? mag[i] : 1.0);
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
      const double dd = abs2(lam[q] - conjg(lam[i]));
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
// Eigen pipeline of eq. (finalGenEigValue), three kernels.
//   k_eig_cl (one cluster of ECL CTAs, FP64, columns of [R | L | I] dealt round-robin to the
//     CTAs): Gauss-Jordan elimination with partial pivoting, [R | L | I] -> [I | M | R^{-1}],
//     M = R^{-1} L; Householder reduction of M to Hessenberg form H = Q^H M Q (Householder
//     vectors kept); then CTA 0 runs an FP32 implicit single-shift QR on the scaled H for the
//     eigenvalues and nominates the k + NCAND_EXTRA closest to 0 as candidates.
//   k_eig_h (one block per candidate, FP64): inverse iteration on H for the right and left
//     eigenvectors z, zl of H (O(m^2) per step: H - sigma I is upper Hessenberg, so its LU
//     with partial pivoting only exchanges neighbouring rows), one Rayleigh-quotient update of
//     the shift; then y = Q z, yl = R^{-H} Q zl are the pencil's right and left eigenvectors and
//     yl^H L y / yl^H R y its eigenvalue.
//   k_eig_c (one block): candidates that refined to the same eigenvalue are merged, final
//     selection on the refined eigenvalues (real / complex decided in FP64), unit norm,
//     conjugate pairs split into real and imaginary parts, Phi scalings.
// GB300 executes FP64 at about 1.75 FMA per clock per SM, and the pencils of these cycles are so
// ill-conditioned (R carries Lanczos and recycle vectors of very different norms) that the
// reduction must stay in FP64: it is spread over a cluster of SMs (distributed shared memory
// for the per-step broadcasts and reductions).  The QR iteration is long and sequential and
// runs in FP32 (64x the FP64 rate); its eigenvalues are only shifts for the FP64 refinement.
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

// Block-wide (all threads): eigenvalues of the Hessenberg H (FP32, ld) by implicit QR with
// several shifts per sweep, each chased as its own bulge by one warp, the bulges three rows
// apart and advanced in lockstep: step t moves bulge w to rotation k = lo + t - 3 w.  Within a
// step the bulges' row (left) updates touch disjoint row pairs and their column (right) updates
// disjoint column pairs, and left and right rotations commute, so a sweep equals the sweeps of
// the single shifts one after another while taking (hi - lo) + 3 (nb - 1) steps instead of
// nb (hi - lo).  Shifts: eigenvalues of the trailing 2 x 2 blocks, nearest ones first; an
// exceptional shift after 10 sweeps without deflation.  Returns false (with diagnostics) on a
// non-finite entry or after 60 m sweeps.
__device__ bool qr_eigs_block_f32(zf* T, int m, int ld, int* dbg) {
  __shared__ int s_lo, s_hi, s_nb, s_fail, s_hmax, s_lmax;
  __shared__ zf s_mu[8];
  __shared__ unsigned char s_neg[MMAX];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int NB = nwarp < 8 ? nwarp : 8;
  const float eps = 1.1920929e-07f;
  int stall = 0, total = 0;   // thread 0's counters
  if (threadIdx.x == 0) { s_hi = m - 1; s_fail = 0; }
  __syncthreads();
  for (;;) {
    // Deflation, all threads at once: row i (1 <= i <= hi) is split off when its subdiagonal
    // is negligible against its two diagonal neighbours (such entries are set to zero).  The
    // window's bottom moves up past split-off 1 x 1 blocks (hi' = the largest i <= hi whose
    // subdiagonal is not negligible, 0 if none) and its top is the largest split point below
    // hi' (lo, 0 if none) -- what a scan from hi downwards finds.
    const int hi0 = s_hi;
    if (threadIdx.x == 0) { s_hmax = 0; s_lmax = 0; }
    __syncthreads();
    for (int i = 1 + threadIdx.x; i <= hi0; i += blockDim.x) {
      const float sub = cabs1f_(T[i + (i - 1) * ld]);
      const float dsum = cabs1f_(T[i + i * ld]) + cabs1f_(T[i - 1 + (i - 1) * ld]);
      const bool neg = sub <= eps * (dsum > 0.f ? dsum : 1.f);
      s_neg[i] = neg;
      if (neg) T[i + (i - 1) * ld] = zf(0.f, 0.f);
      else atomicMax(&s_hmax, i);
    }
    __syncthreads();
    const int hi1 = s_hmax;
    for (int i = 1 + threadIdx.x; i < hi1; i += blockDim.x)
      if (s_neg[i]) atomicMax(&s_lmax, i);
    __syncthreads();
    const int lo1 = s_lmax;
    // shifts: eigenvalues of the 2 x 2 blocks ending at rows hi1, hi1 - 2, ..., the one nearer
    // the block's bottom entry first, one thread per block
    const int w = hi1 - lo1 + 1;
    int nb1 = (w - 1) / 3 + 1;
    if (nb1 > NB) nb1 = NB;
    if (w <= 4) nb1 = 1;
    if (hi1 > 0 && threadIdx.x < (nb1 + 1) / 2) {
      const int r = hi1 - 2 * threadIdx.x;
      const int c0 = 2 * threadIdx.x;
      if (r - 1 >= lo1) {
        const zf a = T[r - 1 + (r - 1) * ld], b = T[r - 1 + r * ld], c = T[r + (r - 1) * ld], d = T[r + r * ld];
        const zf half = (a + d) * 0.5f;
        const zf disc = half * half - (a * d - b * c);
        const float rdisc = cabsf_(disc);
        // radicands clamped: hypotf's rounding can put |disc| + Re(disc) below zero
        float sr = sqrtf(fmaxf(0.f, 0.5f * (rdisc + disc.re))), si = sqrtf(fmaxf(0.f, 0.5f * (rdisc - disc.re)));
        if (disc.im < 0.f) si = -si;
        const zf l1 = half + zf(sr, si), l2 = half - zf(sr, si);
        const bool first1 = cabsf_(l1 - d) < cabsf_(l2 - d);
        s_mu[c0] = first1 ? l1 : l2;
        if (c0 + 1 < nb1) s_mu[c0 + 1] = first1 ? l2 : l1;
      } else {
        s_mu[c0] = T[hi1 + hi1 * ld];
        if (c0 + 1 < nb1) s_mu[c0 + 1] = T[hi1 + hi1 * ld];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (hi1 < hi0) stall = 0;
      s_hi = hi1;
      s_lo = lo1;
      s_nb = nb1;
      if (hi1 > 0) {
        ++stall;
        const zf dd = T[hi1 + hi1 * ld], cc = T[hi1 + (hi1 - 1) * ld];
        if (!isfinite(dd.re) || !isfinite(dd.im) || !isfinite(cc.re) || !isfinite(cc.im)) {
          dbg[0] = 3; dbg[1] = lo1; dbg[2] = hi1; dbg[3] = stall; dbg[4] = total;
          s_fail = 1;
        } else if (++total > 60 * m) {
          dbg[0] = 2; dbg[1] = lo1; dbg[2] = hi1; dbg[3] = stall; dbg[4] = total;
          s_fail = 1;
        }
        if (stall % 11 == 10) s_mu[0] = T[hi1 + hi1 * ld] + zf(cabsf_(T[hi1 + (hi1 - 1) * ld]) * 0.75f, 0.f);
      }
    }
    __syncthreads();
    if (s_fail) return false;
    const int hi = s_hi;
    if (hi <= 0) break;
    const int lo = s_lo, nb = s_nb;
    const int nsteps = (hi - lo) + 3 * (nb - 1);
    for (int t = 0; t < nsteps; ++t) {
      const int k = lo + t - 3 * warp;
      const bool active = warp < nb && k >= lo && k < hi;
      float cs = 1.f;
      zf sn = zf(0.f, 0.f);
      if (active) {
        if (k == lo) givens_f(T[lo + lo * ld] - s_mu[warp], T[lo + 1 + lo * ld], &cs, &sn);
        else givens_f(T[k + (k - 1) * ld], T[k + 1 + (k - 1) * ld], &cs, &sn);
        __syncwarp();   // all lanes have read the rotation's defining entries
        const int c0 = k > lo ? k - 1 : lo;
        for (int col = c0 + lane; col <= hi; col += 32) {
          const zf p = T[k + col * ld], q = T[k + 1 + col * ld];
          T[k + col * ld] = cs * p + sn * q;
          T[k + 1 + col * ld] = cs * q - conjg(sn) * p;
        }
      }
      __syncthreads();   // every bulge's row update before any column update
      if (active) {
        const int r1 = k + 2 < hi ? k + 2 : hi;
        for (int row = lo + lane; row <= r1; row += 32) {
          const zf p = T[row + k * ld], q = T[row + (k + 1) * ld];
          T[row + k * ld] = cs * p + conjg(sn) * q;
          T[row + (k + 1) * ld] = cs * q - sn * p;
        }
        __syncwarp();
        if (k > lo && lane == 0) T[k + 1 + (k - 1) * ld] = zf(0.f, 0.f);
      }
      __syncthreads();
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

// Scalar helpers of the cluster kernel, real (double: a real pencil) or complex (zd).
__device__ __forceinline__ double cabs1_(double a) { return fabs(a); }
__device__ __forceinline__ double crcp(double a) { return 1.0 / a; }
__device__ __forceinline__ bool nonzero(double a) { return a != 0.0; }
__device__ __forceinline__ bool nonzero(zd a) { return a.re != 0.0 || a.im != 0.0; }
__device__ __forceinline__ double bcast0(double v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ zd bcast0(zd v) { return zd(__shfl_sync(0xffffffffu, v.re, 0), __shfl_sync(0xffffffffu, v.im, 0)); }
__device__ __forceinline__ float bcast0(float v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ zf bcast0(zf v) { return zf(__shfl_sync(0xffffffffu, v.re, 0), __shfl_sync(0xffffffffu, v.im, 0)); }

constexpr int ECL = 8;                                   // CTAs of the eigen cluster (portable size)
constexpr int ECL_COLS = (3 * MMAX + ECL - 1) / ECL;     // local columns of [R | L | I] per CTA

template <class S>
struct EclBcast {   // one elimination / reflection step, written by the CTA owning its column
  S col[MMAX];      // Gauss-Jordan: pivot column after the row exchange; Householder: v
  S f;              // Householder: 2 / ||v||^2
  int piv, flag;    // Gauss-Jordan: pivot row, 1 = zero pivot; Householder: 1 = no reflection
};

// S = double for a real pencil (real problems: L, R, the Hessenberg form and the reflectors are
// real, so the reduction runs in real arithmetic, a quarter of the complex FP64 work), zd else.
template <class S>
__global__ void __cluster_dims__(ECL, 1, 1) __launch_bounds__(256)
k_eig_cl(RefreshInfo f, DevState* st, zd* work, int has_R, int m) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  S* cols = reinterpret_cast<S*>(smraw);   // local column lc at cols + lc * MMAX
  __shared__ EclBcast<S> bc[2];
  __shared__ S up[2][MMAX];    // this CTA's part of T v (right Householder update)
  __shared__ S lv[MMAX];       // local copy of the broadcast column
  __shared__ S uvec[MMAX];
  __shared__ S tv[ECL_COLS];
  __shared__ double s_red[8];
  __shared__ int s_piv, s_skip;
  __shared__ S s_inva, s_f;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const zd* Lm = work + W_L;
  const zd* Rm = work + W_R;
  const EigInts ei = eig_ints(work);
  // global columns: has_R: [0, m) R, [m, 2m) L -> M, [2m, 3m) I -> R^{-1}; else [0, m) L = M.
  // Local column lc of CTA `rank` is global column rank + lc ECL.
  const int ncol = has_R ? 3 * m : m;
  const int mcol0 = has_R ? m : 0;
  const int nloc = ncol > rank ? (ncol - rank + ECL - 1) / ECL : 0;
  for (int e = tid; e < nloc * m; e += blockDim.x) {
    const int lc = e / m, r = e % m, g = rank + lc * ECL;
    S v;
    if (!has_R) v = from_zd<S>(Lm[r + g * MMAX]);
    else if (g < m) v = from_zd<S>(Rm[r + g * MMAX]);
    else if (g < 2 * m) v = from_zd<S>(Lm[r + (g - m) * MMAX]);
    else v = (r == g - 2 * m) ? S(1.0) : S();
    cols[lc * MMAX + r] = v;
  }
  if (tid == 0) s_skip = 1;
  bool failed = false;   // per thread, always equal in all threads: every thread reads the flags
  __syncthreads();
  // Every CTA runs the same sequence of cluster barriers whatever the data (a failed pivot only
  // switches the arithmetic off), so no CTA can wait at a barrier that another never reaches.
  // ---- Gauss-Jordan with partial pivoting: one cluster barrier per column
  for (int k = 0; has_R && k < m; ++k) {
    const int owner = k % ECL;
    if (rank == owner && warp == 0 && !failed) {
      const S* c = cols + (k / ECL) * MMAX;
      double best = -1.0;
      int bi = k;
      for (int r = k + lane; r < m; r += 32) {
        const double v = cabs1_(c[r]);
        if (v > best) { best = v; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      bi = __shfl_sync(0xffffffffu, bi, 0);
      best = __shfl_sync(0xffffffffu, best, 0);
      EclBcast<S>& B = bc[k & 1];
      for (int r = lane; r < m; r += 32) B.col[r] = c[r == k ? bi : (r == bi ? k : r)];
      if (lane == 0) { B.piv = bi; B.flag = (best > 0.0 && isfinite(best)) ? 0 : 1; }
    }
    cl.sync();
    if (!failed) {
      const EclBcast<S>* rb = cl.map_shared_rank(&bc[k & 1], owner);
      for (int r = tid; r < m; r += blockDim.x) lv[r] = rb->col[r];
      if (tid == 0) s_piv = rb->piv;
      if (rb->flag) failed = true;
      __syncthreads();
      if (!failed) {
        const int p = s_piv;
        if (tid == 0) s_inva = crcp(lv[k]);
        __syncthreads();
        const S inva = s_inva;
        for (int lc = tid; lc < nloc; lc += blockDim.x) {   // row exchange, pivot row scaled
          S* c = cols + lc * MMAX;
          if (rank + lc * ECL == k) { tv[lc] = S(); continue; }
          if (p != k) { const S t = c[k]; c[k] = c[p]; c[p] = t; }
          const S t = c[k] * inva;
          c[k] = t;
          tv[lc] = t;
        }
        __syncthreads();
        for (int e = tid; e < nloc * m; e += blockDim.x) {   // elimination in every other row
          const int lc = e / m, r = e % m;
          S* c = cols + lc * MMAX;
          const S t = tv[lc];
          if (rank + lc * ECL == k) c[r] = r == k ? S(1.0) : S();
          else if (r != k && nonzero(t)) c[r] -= lv[r] * t;   // unit columns stay
        }
        __syncthreads();
      }
    }
  }
  cl.sync();   // the last elimination broadcast is read before the reflections reuse bc
  // ---- Householder reduction of M to Hessenberg form: two cluster barriers per column
  zd* QV = work + W_QV;
  zd* QF = work + W_QF;
  for (int j = 0; j + 2 < m; ++j) {
    const int gj = mcol0 + j, owner = gj % ECL, len = m - j - 1;
    if (rank == owner && warp == 0 && !failed) {
      S* c = cols + (gj / ECL) * MMAX;
      EclBcast<S>& B = bc[j & 1];
      double nx2 = 0.0;
      for (int i = lane; i < len; i += 32) nx2 += abs2(c[j + 1 + i]);
      nx2 = __shfl_sync(0xffffffffu, warp_sum(nx2), 0);
      const S x0 = c[j + 1];
      const double tail = nx2 - abs2(x0);
      const bool skip = !(tail > 0.0) || tail <= nx2 * 1e-30;
      if (!skip) {
        const double nx = sqrt(nx2), a2 = abs2(x0);
        const S ph = a2 > 0.0 ? x0 * rsqrt(a2) : S(1.0);
        const S alpha = -(ph * nx);
        const S fct = S(2.0 / (tail + abs2(x0 - alpha)));
        for (int i = lane; i < len; i += 32) {
          const S vi = i == 0 ? x0 - alpha : c[j + 1 + i];
          B.col[i] = vi;
          QV[i + j * MMAX] = to_zd(vi);
        }
        __syncwarp();
        for (int i = lane; i < len; i += 32) c[j + 1 + i] = i == 0 ? alpha : S();   // P x = alpha e_1
        if (lane == 0) { B.f = fct; QF[j] = to_zd(fct); }
      } else if (lane == 0) {
        B.f = S();
        QF[j] = zd();
      }
      if (lane == 0) B.flag = skip ? 1 : 0;
    }
    cl.sync();
    if (!failed) {
      const EclBcast<S>* rb = cl.map_shared_rank(&bc[j & 1], owner);
      for (int i = tid; i < len; i += blockDim.x) lv[i] = rb->col[i];
      if (tid == 0) { s_skip = rb->flag; s_f = rb->f; }
      __syncthreads();
      if (!s_skip) {
        const S fct = s_f;
        // left: T[j+1:, c] -= f v (v^H T[j+1:, c]) for this CTA's columns c > j (warp per column)
        for (int lc = warp; lc < nloc; lc += nwarp) {
          const int cc = rank + lc * ECL - mcol0;
          if (cc <= j || cc >= m) continue;
          S* c = cols + lc * MMAX;
          S w = S();
          for (int i = lane; i < len; i += 32) w += cmul(lv[i], c[j + 1 + i]);
          w = warp_sum(w);
          w = bcast0(w) * fct;
          for (int i = lane; i < len; i += 32) c[j + 1 + i] -= lv[i] * w;
        }
        __syncthreads();
        // right, this CTA's part of u = T[:, j+1:] v: four threads per row (a quarter of the
        // local columns each, lanes 8 apart in one warp), combined in a fixed order
        for (int base = 0; base < m; base += blockDim.x / 4) {
          const int r = base + (warp * 8 + (lane & 7)), qtr = (lane >> 3) & 3;
          S acc = S();
          if (r < m)
            for (int lc = qtr; lc < nloc; lc += 4) {
              const int cc = rank + lc * ECL - mcol0;
              if (cc > j && cc < m) acc += cols[lc * MMAX + r] * lv[cc - j - 1];
            }
          acc += shfl_xor(acc, 8);
          acc += shfl_xor(acc, 16);
          if (r < m && qtr == 0) up[j & 1][r] = acc;
        }
      }
    }
    cl.sync();
    if (!failed && !s_skip) {
      for (int r = tid; r < m; r += blockDim.x) {
        S acc = S();
        for (int q = 0; q < ECL; ++q) acc += cl.map_shared_rank(&up[j & 1][0], q)[r];
        uvec[r] = acc * s_f;
      }
      __syncthreads();
      for (int e = tid; e < nloc * m; e += blockDim.x) {   // T[:, c] -= u conj(v_c)
        const int lc = e / m, r = e % m;
        const int cc = rank + lc * ECL - mcol0;
        if (cc > j && cc < m) cols[lc * MMAX + r] -= uvec[r] * conjg(lv[cc - j - 1]);
      }
      __syncthreads();
    }
  }
  // ---- H and R^{-1} to the work buffer, then CTA 0 alone
  for (int e = tid; e < nloc * m; e += blockDim.x) {
    const int lc = e / m, r = e % m, g = rank + lc * ECL;
    if (g >= mcol0 && g < mcol0 + m) work[W_H + r + (g - mcol0) * MMAX] = to_zd(cols[lc * MMAX + r]);
    else if (has_R && g >= 2 * m) work[W_RI + r + (g - 2 * m) * MMAX] = to_zd(cols[lc * MMAX + r]);
  }
  __threadfence();
  cl.sync();   // every CTA's writes are visible; no shared memory of another CTA is read after this
  if (rank != 0) {
    // CTAs 1 .. ECL-1, while CTA 0 runs the QR: Q = P_0 P_1 ... P_{m-3} explicitly, column c =
    // Q e_c with the reflectors applied last to first (P_j leaves e_c alone for j >= c), one
    // warp per column in shared memory.  k_eig_h then back-transforms with one dense product
    // instead of m - 2 dependent reflector applications.
    if (failed) return;
    const zd* QVg = work + W_QV;
    const zd* QFg = work + W_QF;
    zd* Qg = work + W_Q;
    zd* yv = reinterpret_cast<zd*>(smraw) + warp * MMAX;   // the local columns are done with
    for (int c = (rank - 1) * nwarp + warp; c < m; c += (ECL - 1) * nwarp) {
      for (int i = lane; i < m; i += 32) yv[i] = i == c ? zd(1.0) : zd();
      __syncwarp();
      for (int j = min(m - 3, c - 1); j >= 0; --j) {
        const zd fj = QFg[j];
        if (fj.re == 0.0 && fj.im == 0.0) continue;
        const int len = m - j - 1;
        zd w = zd();
        for (int i = lane; i < len; i += 32) w += cmul(QVg[i + j * MMAX], yv[j + 1 + i]);
        w = bcast0(warp_sum(w)) * fj;
        for (int i = lane; i < len; i += 32) yv[j + 1 + i] -= QVg[i + j * MMAX] * w;
        __syncwarp();
      }
      for (int i = lane; i < m; i += 32) Qg[i + c * MMAX] = yv[i];
      __syncwarp();
    }
    return;
  }
  if (failed) {
    if (tid == 0) { st->eig_status = 1; st->kk = 0; *ei.ncand = 0; }
    return;
  }
  const zd* Hg = work + W_H;
  const int ld = m | 1;
  zf* H = reinterpret_cast<zf*>(smraw);   // FP32 copy scaled to entries of order one
  double amax = 0.0;
  for (int e = tid; e < m * m; e += blockDim.x) amax = fmax(amax, cabs1_(Hg[(e % m) + (e / m) * MMAX]));
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if (lane == 0) s_red[warp] = amax;
  __syncthreads();
  amax = 0.0;
  for (int w = 0; w < nwarp; ++w) amax = fmax(amax, s_red[w]);
  if (!(amax > 0.0) || !isfinite(amax)) {
    if (tid == 0) { st->eig_status = 1; st->kk = 0; *ei.ncand = 0; }
    return;
  }
  const double inv = 1.0 / amax;
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int r = e % m, c = e / m;
    const zd h = Hg[r + c * MMAX];
    H[r + c * ld] = zf((float)(h.re * inv), (float)(h.im * inv));
  }
  __shared__ int s_ok;
  if (tid == 0) s_ok = 1;
  __syncthreads();
  {
    const bool ok = qr_eigs_block_f32(H, m, ld, st->dbg);
    if (tid == 0 && !ok) s_ok = 0;
  }
  __syncthreads();
  if (!s_ok) { if (tid == 0) { st->eig_status = 2; st->kk = 0; *ei.ncand = 0; } return; }
  if (tid == 0) {
    // candidates: the k + NCAND_EXTRA finite FP32 eigenvalues closest to the origin; real /
    // complex classification and the final selection wait for the FP64 refinement
    int order[MMAX];
    float mag[MMAX];
    int cnt = 0;
    for (int i = 0; i < m; ++i) {
      const zf h = H[i + i * ld];
      mag[i] = abs2(h);
      if (isfinite(h.re) && isfinite(h.im)) order[cnt++] = i;
    }
    for (int a = 1; a < cnt; ++a) {
      const int vv = order[a];
      const float av = mag[vv];
      int b = a - 1;
      while (b >= 0 && mag[order[b]] > av) { order[b + 1] = order[b]; --b; }
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

// Leading dimension of the shared copy of H - sigma I in k_eig_h: MMAX + 1 makes a row of 16-byte
// entries fall on distinct bank groups (with MMAX every lane of a row access hit the same banks).
constexpr int LDH = MMAX + 1;

// One warp: LU with partial pivoting of the upper Hessenberg A = H - sigma I (ld LDH) in place.
// Step k exchanges rows k and k+1 when that gives the larger pivot (sw[k]) and stores the
// multiplier at A[k+1, k]; dinv[k] receives 1 / U[k, k] (a zero pivot is replaced by a tiny one:
// sigma is then an eigenvalue to working precision, which inverse iteration tolerates).
__device__ void hess_lu_warp(zd* A, int m, int* sw, zd* dinv, double tiny) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k + 1 < m; ++k) {
    const bool swp = cabs1_(A[k + 1 + k * LDH]) > cabs1_(A[k + k * LDH]);
    if (swp)
      for (int c = k + lane; c < m; c += 32) {
        const zd t = A[k + c * LDH]; A[k + c * LDH] = A[k + 1 + c * LDH]; A[k + 1 + c * LDH] = t;
      }
    __syncwarp();
    zd piv = A[k + k * LDH];
    if (cabs1_(piv) == 0.0) piv = zd(tiny);
    const zd rp = crcp(piv);
    const zd l = A[k + 1 + k * LDH] * rp;
    __syncwarp();
    for (int c = k + 1 + lane; c < m; c += 32) A[k + 1 + c * LDH] -= l * A[k + c * LDH];
    if (lane == 0) { A[k + k * LDH] = piv; A[k + 1 + k * LDH] = l; sw[k] = swp; dinv[k] = rp; }
    __syncwarp();
  }
  if (lane == 0) {
    zd& d = A[(m - 1) + (m - 1) * LDH];
    if (cabs1_(d) == 0.0) d = zd(tiny);
    dinv[m - 1] = crcp(d);
  }
  __syncwarp();
}

// One warp: y <- A^{-1} y for the factorisation of hess_lu_warp.
__device__ void hess_solve_warp(const zd* A, int m, const int* sw, const zd* dinv, zd* y) {
  const int lane = threadIdx.x & 31;
  if (lane == 0)
    for (int k = 0; k + 1 < m; ++k) {
      if (sw[k]) { const zd t = y[k]; y[k] = y[k + 1]; y[k + 1] = t; }
      y[k + 1] -= A[k + 1 + k * LDH] * y[k];
    }
  __syncwarp();
  for (int c = m - 1; c >= 0; --c) {   // U x = y, column oriented
    const zd yc = y[c] * dinv[c];
    __syncwarp();
    if (lane == 0) y[c] = yc;
    for (int r = lane; r < c; r += 32) y[r] -= A[r + c * LDH] * yc;
    __syncwarp();
  }
}

// One warp: y <- A^{-H} y.  A = P_0 E_0^{-1} ... P_{m-2} E_{m-2}^{-1} U, so A^H w = y is
// U^H w' = y followed by w = P_0 E_0^H ... P_{m-2} E_{m-2}^H w'.
__device__ void hess_solve_adj_warp(const zd* A, int m, const int* sw, const zd* dinv, zd* y) {
  const int lane = threadIdx.x & 31;
  for (int c = 0; c < m; ++c) {   // U^H lower triangular: column c holds conj(U[c, r]), r > c
    const zd yc = y[c] * conjg(dinv[c]);
    __syncwarp();
    if (lane == 0) y[c] = yc;
    for (int r = c + 1 + lane; r < m; r += 32) y[r] -= conjg(A[c + r * LDH]) * yc;
    __syncwarp();
  }
  if (lane == 0)
    for (int k = m - 2; k >= 0; --k) {
      y[k] -= conjg(A[k + 1 + k * LDH]) * y[k + 1];
      if (sw[k]) { const zd t = y[k]; y[k] = y[k + 1]; y[k + 1] = t; }
    }
  __syncwarp();
}

// One warp: largest |re| + |im| scaled to 1 (t -> y)
__device__ void normalise_warp(const zd* t, zd* y, int m) {
  const int lane = threadIdx.x & 31;
  double big = 0.0;
  for (int i = lane; i < m; i += 32) big = fmax(big, cabs1_(t[i]));
  for (int o = 16; o > 0; o >>= 1) big = fmax(big, __shfl_xor_sync(0xffffffffu, big, o));
  const double sc = big > 0.0 ? 1.0 / big : 1.0;
  for (int i = lane; i < m; i += 32) y[i] = t[i] * sc;
  __syncwarp();
}

// sum of f(c) over c in [c0, c1) as four interleaved partial sums added in a fixed order: four
// independent FP64 dependency chains instead of one (a dependent FP64 operation costs about 60
// cycles on this part)
template <class F>
__device__ __forceinline__ zd dot4(int c0, int c1, F f) {
  zd s0 = zd(), s1 = zd(), s2 = zd(), s3 = zd();
  int c = c0;
  for (; c + 3 < c1; c += 4) { s0 += f(c); s1 += f(c + 1); s2 += f(c + 2); s3 += f(c + 3); }
  for (; c < c1; ++c) s0 += f(c);
  return (s0 + s1) + (s2 + s3);
}

__global__ void __launch_bounds__(64) k_eig_h(zd* work, int m, int has_R) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const EigInts ei = eig_ints(work);
  const int cand = blockIdx.x;
  if (cand >= *ei.ncand) return;
  zd* A = reinterpret_cast<zd*>(smraw);   // H - sigma I and its LU (ld LDH)
  zd* z = A + LDH * m;
  zd* zl = z + MMAX;
  zd* t = zl + MMAX;
  zd* tl = t + MMAX;
  zd* dinv = tl + MMAX;
  __shared__ int sw[MMAX];
  __shared__ zd s_num, s_den;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const zd* Hg = work + W_H;
  double hn = 0.0;   // scale of H for the zero-pivot replacement
  for (int e = lane; e < m * m; e += 32) hn = fmax(hn, cabs1_(Hg[(e % m) + (e / m) * MMAX]));
  for (int o = 16; o > 0; o >>= 1) hn = fmax(hn, __shfl_xor_sync(0xffffffffu, hn, o));
  const double tiny = 1e-15 * (hn > 0.0 ? hn : 1.0);
  zd sigma = work[W_LAM + cand];
  for (int e = threadIdx.x; e < m; e += blockDim.x) {
    const double v = 1.0 + 0.5 * sin(1.7 * e + 0.3);   // fixed start: no zero entries, no structure
    z[e] = zd(v, 0.0);
    zl[e] = zd(v, 0.0);
  }
  for (int pass = 0; pass < 2; ++pass) {
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int r = e % m, c = e / m;
      A[r + c * LDH] = r == c ? Hg[r + c * MMAX] - sigma : Hg[r + c * MMAX];
    }
    __syncthreads();
    if (warp == 0) hess_lu_warp(A, m, sw, dinv, tiny);
    __syncthreads();
    const int steps = pass == 0 ? 3 : 2;
    for (int it = 0; it < steps; ++it) {
      if (warp == 0) {
        for (int i = lane; i < m; i += 32) t[i] = z[i];
        __syncwarp();
        hess_solve_warp(A, m, sw, dinv, t);
        normalise_warp(t, z, m);
      } else {
        for (int i = lane; i < m; i += 32) tl[i] = zl[i];
        __syncwarp();
        hess_solve_adj_warp(A, m, sw, dinv, tl);
        normalise_warp(tl, zl, m);
      }
    }
    __syncthreads();
    // Rayleigh quotient of H: zl^H H z / zl^H z
    if (warp == 0) {
      zd num = zd(), den = zd();
      for (int r = lane; r < m; r += 32) {
        const zd hz = dot4(r > 0 ? r - 1 : 0, m, [&](int c) { return Hg[r + c * MMAX] * z[c]; });
        num += cmul(zl[r], hz);
        den += cmul(zl[r], z[r]);
      }
      num = warp_sum(num);
      den = warp_sum(den);
      if (lane == 0) { s_num = num; s_den = den; }
    }
    __syncthreads();
    const zd lam = cabs1_(s_den) > 0.0 ? s_num / s_den : sigma;
    if (!(isfinite(lam.re) && isfinite(lam.im)) || cabs1_(lam - sigma) <= 1e-10 * cabs1_(lam)) break;
    sigma = lam;
    __syncthreads();
  }
  __syncthreads();
  // pencil vectors: y = Q z (warp 0); yl = R^{-H} Q zl (warp 1)
  {
    // y = Q z (warp 0), Q zl (warp 1): dense products with the Q that k_eig_cl formed
    zd* src = warp == 0 ? z : zl;
    zd* tmp = warp == 0 ? t : tl;
    const zd* Qg = work + W_Q;
    for (int r = lane; r < m; r += 32) tmp[r] = dot4(0, m, [&](int c) { return Qg[r + c * MMAX] * src[c]; });
    __syncwarp();
    for (int r = lane; r < m; r += 32) src[r] = tmp[r];
    __syncwarp();
  }
  if (warp == 1) {
    if (has_R) {
      const zd* RI = work + W_RI;
      for (int r = lane; r < m; r += 32) {
        tl[r] = dot4(0, m, [&](int c) { return cmul(RI[c + r * MMAX], zl[c]); });
      }
      __syncwarp();
      for (int r = lane; r < m; r += 32) zl[r] = tl[r];
    }
  }
  __syncthreads();
  zd* Y = work + W_Y + cand * MMAX;
  zd* YL = work + W_YL + cand * MMAX;
  for (int e = threadIdx.x; e < m; e += blockDim.x) { Y[e] = z[e]; YL[e] = zl[e]; }
  // eigenvalue from the pencil itself: yl^H L y / yl^H R y
  if (warp == 0) {
    const zd* Lm = work + W_L;
    const zd* Rm = work + W_R;
    zd num = zd(), den = zd();
    for (int r = lane; r < m; r += 32) {
      const zd ly = dot4(0, m, [&](int c) { return Lm[r + c * MMAX] * z[c]; });
      const zd ry = has_R ? dot4(0, m, [&](int c) { return Rm[r + c * MMAX] * z[c]; }) : z[r];
      num += cmul(zl[r], ly);
      den += cmul(zl[r], ry);
    }
    num = warp_sum(num);
    den = warp_sum(den);
    if (lane == 0) work[W_LAM2 + cand] = cabs1_(den) > 0.0 ? num / den : sigma;
  }
}

__global__ void __launch_bounds__(256) k_eig_c(RefreshInfo f, DevState* st, zd* work, zd* Wphi, zd* Wphit, int ldw,
                                               double* lam_out, int m, int raw) {
  const Layout Lay = make_layout(f);
  const EigInts ei = eig_ints(work);
  __shared__ int s_units;
  __shared__ zd s_raw[KMAX + NCAND_EXTRA], s_lam[KMAX + NCAND_EXTRA];
  const int nc = st->eig_status == 0 ? *ei.ncand : 0;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) s_raw[c] = work[W_LAM2 + c];
  __syncthreads();
  // a candidate that refined to the eigenvalue of an earlier one is dropped (candidate c is
  // compared with every earlier refined value; one thread per candidate)
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    zd lc = s_raw[c];
    for (int q = 0; q < c; ++q)
      if (cabs1_(lc - s_raw[q]) <= 1e-8 * cabs1_(lc)) { lc = zd(nan(""), 0.0); break; }
    s_lam[c] = lc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int units = 0, cols = 0;
    if (nc > 0) units = select_units(s_lam, nc, f.k, f.real_path, ei.sel, ei.pair, &cols);
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
  {   // unit norm, largest component real and positive: one warp per vector
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int vi = wp; vi < 2 * units; vi += nw) {
      const int u = vi % units;
      zd* w = (vi >= units ? Lv : Rv) + u * MMAX;
      double nrm = 0.0, big = -1.0;
      int bi = 0;
      for (int r = lane; r < m; r += 32) { const double a2 = abs2(w[r]); nrm += a2; if (a2 > big) { big = a2; bi = r; } }
      for (int o = 16; o > 0; o >>= 1) {   // sum (lane 0's order is broadcast) and first argmax
        nrm += __shfl_down_sync(0xffffffffu, nrm, o);
        const double ob = __shfl_xor_sync(0xffffffffu, big, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > big || (ob == big && oi < bi)) { big = ob; bi = oi; }
      }
      nrm = __shfl_sync(0xffffffffu, nrm, 0);
      const zd wb = w[bi];
      const zd ph = nrm > 0.0 && big > 0.0 ? conjg(wb) * rsqrt(abs2(wb) * nrm) : zd(1.0);
      __syncwarp();
      for (int r = lane; r < m; r += 32) w[r] = w[r] * ph;
    }
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
  const size_t smem_cl = std::max<size_t>((size_t)ECL_COLS * MMAX * sizeof(zd), (size_t)MMAX * (MMAX + 1) * sizeof(zf));
  const size_t smem_h = (size_t)(LDH * m + 5 * MMAX) * sizeof(zd);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_eig_cl<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cl);
    cudaFuncSetAttribute(k_eig_cl<zd>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cl);
    cudaFuncSetAttribute(k_eig_h, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)((LDH * MMAX + 5 * MMAX) * sizeof(zd)));
    attr_set = true;
  }
  if (info.real_path) k_eig_cl<double><<<ECL, 256, smem_cl, s>>>(info, st, work, has_R, m);
  else k_eig_cl<zd><<<ECL, 256, smem_cl, s>>>(info, st, work, has_R, m);
  k_eig_h<<<KMAX + NCAND_EXTRA, 64, smem_h, s>>>(work, m, has_R);
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
// Rotation of one-sided Jacobi for the column pair (a, b) with squared norms app, aqq and
// inner product apq = a^H b (|apq|^2 = g2 > 0): cosine cs, sine sn and phase e, so that
// [a, b] <- [cs a - sn conj(e) b, sn e a + cs b] makes the two columns orthogonal.
// FP32 version: everything in FP32.
template <class E>   // E: zf, or float for a real matrix
__device__ __forceinline__ bool jacobi_rot(float app, float aqq, E apq, float g2, float* cs, float* sn, E* e) {
  const float rg = rsqrtf(g2);
  const float zeta = (aqq - app) * 0.5f * rg, az = fabsf(zeta);
  const float t = az > 1e18f ? 0.5f / zeta : copysignf(1.f, zeta) / (az + sqrtf(1.f + zeta * zeta));
  if (t == 0.f) return false;
  *cs = rsqrtf(1.f + t * t);
  *sn = *cs * t;
  *e = apq * rg;
  return true;
}
// FP64 version: the angle in FP32 (an inexact angle only leaves a little of a^H b for the next
// sweep), cosine, sine and phase in FP64 so that the rotation is unitary to FP64 rounding.
template <class E>   // E: zd, or double for a real matrix
__device__ __forceinline__ bool jacobi_rot(double app, double aqq, E apq, double g2, double* cs, double* sn, E* e) {
  const double rg = rsqrt(g2);   // one reciprocal square root serves the angle and the phase
  const double zq = (aqq - app) * 0.5 * rg;
  const float zeta = (float)zq, az = fabsf(zeta);
  const float tf = az > 1e18f ? 0.5f / zeta : copysignf(1.f, zeta) / (az + sqrtf(1.f + zeta * zeta));
  if (tf == 0.f) return false;
  const double t = (double)tf;
  *cs = rsqrt(1.0 + t * t);
  *sn = *cs * t;
  *e = apq * rg;
  return true;
}

// Block-wide one-sided Jacobi sweeps on the k x k column-major A (V accumulates the right
// rotations), round-robin (circle) pair ordering, warp w handles pairs w, w + nwarps, ...  A pair is
// converged when |a^H b|^2 <= tol2 |a|^2 |b|^2.  Returns the sweeps run.
template <class C, class Rl>
__device__ int jacobi_sweeps(C* A, C* V, int k, int max_sweeps, Rl tol2, int* s_rot) {
  const int kk = (k + 1) & ~1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *s_rot = 0;
    __syncthreads();
    for (int round = 0; round < kk - 1; ++round) {
      for (int pr = warp; pr < kk / 2; pr += nw) {
        // circle method: position 0 fixed, positions 1..kk-1 rotate by `round`
        int a = pr == 0 ? 0 : 1 + (pr - 1 + round) % (kk - 1);
        const int pb = kk - 1 - pr;
        int b = 1 + (pb - 1 + round) % (kk - 1);
        if (a > b) { const int t = a; a = b; b = t; }
        if (b >= k || a == b) continue;
        Rl app = 0, aqq = 0;
        C apq = C(Rl(0));
        for (int r = lane; r < k; r += 32) {
          const C x = A[r + a * k], y = A[r + b * k];
          app += abs2(x); aqq += abs2(y); apq += cmul(x, y);
        }
        app = warp_sum(app); aqq = warp_sum(aqq); apq = warp_sum(apq);
        app = __shfl_sync(0xffffffffu, app, 0); aqq = __shfl_sync(0xffffffffu, aqq, 0);
        apq = bcast0(apq);
        const Rl g2 = abs2(apq);
        if (g2 <= tol2 * (app * aqq) || g2 == Rl(0)) continue;
        Rl cs, sn;
        C e;
        if (!jacobi_rot(app, aqq, apq, g2, &cs, &sn, &e)) continue;
        if (lane == 0) *s_rot = 1;
        __syncwarp();   // all lanes' reads of columns a, b precede the writes
        for (int r = lane; r < k; r += 32) {
          const C x = A[r + a * k], y = A[r + b * k];
          A[r + a * k] = cs * x - sn * (conjg(e) * y);
          A[r + b * k] = sn * (e * x) + cs * y;
          const C vx = V[r + a * k], vy = V[r + b * k];
          V[r + a * k] = cs * vx - sn * (conjg(e) * vy);
          V[r + b * k] = sn * (e * vx) + cs * vy;
        }
      }
      __syncthreads();
    }
    if (!*s_rot) break;
    __syncthreads();
  }
  __syncthreads();
  return sweep;
}

// C / Cf = zd / zf, or double / float for a real problem (its Ct^H C is real: real rotations, a
// quarter of the complex FP64 work).
template <class C, class Cf>
__global__ void __launch_bounds__(512) k_svd(const int* k_dev, int kmax, const zd* S2, double svd_tol,
                                             zd* Nmat, zd* Mmat, double* sigma, int* p_dev, double* Dc_dev,
                                             int* status) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C* A = reinterpret_cast<C*>(smraw);     // column-major k x k: A = S_norm, rotated to M Sigma
  C* V = A + KMAX * KMAX;                 // accumulated right rotations (N)
  C* A0 = V + KMAX * KMAX;                // S_norm (kept for the FP64 restart)
  Cf* Af = reinterpret_cast<Cf*>(A0 + KMAX * KMAX);
  Cf* Vf = Af + KMAX * KMAX;
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
    const C a = from_zd<C>(S2[r * ld2 + c] * (sr * scc));
    A0[r + c * k] = a;
    Af[r + c * k] = cvt<Cf>(a);   // entries <= 1 after the unit-norm scaling
    Vf[r + c * k] = r == c ? Cf(1.f) : Cf(0.f);
  }
  __syncthreads();
  // FP32 sweeps to about FP32 orthogonality, then A <- A0 Vf and V <- Vf in FP64 and FP64
  // sweeps from there (one or two: the convergence of cyclic Jacobi is quadratic).
  jacobi_sweeps<Cf, float>(Af, Vf, k, 30, (8e-8f * k) * (8e-8f * k), &s_rot);
  // Vf is unitary only to FP32 rounding: two Newton-Schulz steps in FP64, V <- V (3 I - V^H V) / 2,
  // make it unitary to FP64 rounding (the error squares at each step); G = V^H V goes in A.
  for (int e = threadIdx.x; e < k * k; e += blockDim.x)
    V[e] = cvt<C>(Vf[e]);
  __syncthreads();
  for (int ns = 0; ns < 2; ++ns) {
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
      const int r = e % k, c = e / k;
      C acc = C();
      for (int q = 0; q < k; ++q) acc += cmul(V[q + r * k], V[q + c * k]);
      A[r + c * k] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {   // A0's spare copy: Af/Vf area
      const int r = e % k, c = e / k;
      C acc = C();
      for (int q = 0; q < k; ++q) acc += V[r + q * k] * ((q == c ? C(3.0) : C()) - A[q + c * k]);
      reinterpret_cast<C*>(Af)[r + c * k] = acc * 0.5;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) V[e] = reinterpret_cast<C*>(Af)[e];
    __syncthreads();
  }
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {   // A = A0 V
    const int r = e % k, c = e / k;
    C acc = C();
    for (int q = 0; q < k; ++q) acc += A0[r + q * k] * V[q + c * k];
    A[r + c * k] = acc;
  }
  __syncthreads();
  // converged pair: |a^H b| at the rounding floor of a k-term FP64 inner product (about
  // k eps ||a|| ||b||); a threshold below it never lets the sweeps stop
  jacobi_sweeps<C, double>(A, V, k, 10, (4e-16 * k) * (4e-16 * k), &s_rot);
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
    C nv = C(), mv = C();
    if (a < k && c < p) {
      const int oc = ord[c];
      nv = V[a + oc * k] * (dn[a] > 0.0 ? 1.0 / dn[a] : 0.0);
      mv = A[a + oc * k] * ((dtn[a] > 0.0 ? 1.0 / dtn[a] : 0.0) / sg[oc]);
    }
    Nmat[e] = to_zd(nv);
    Mmat[e] = to_zd(mv);
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
  const size_t smem = 3 * KMAX * KMAX * sizeof(zd) + 2 * KMAX * KMAX * sizeof(zf);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_svd<zd, zf>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_svd<double, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  if (real_path)
    k_svd<double, float><<<1, 512, smem, s>>>(k_dev, kmax, S, svd_tol, Nmat, Mmat, sigma, p_dev, Dc_dev, status_dev);
  else
    k_svd<zd, zf><<<1, 512, smem, s>>>(k_dev, kmax, S, svd_tol, Nmat, Mmat, sigma, p_dev, Dc_dev, status_dev);
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
