// kernels_basis.cu -- tall-skinny products of the recycle-space refresh (Sections 4.1-4.3):
//   * Gram G = X^H Y over lists of columns (Psit^H [Psi Phi] for the pencil of eq.
//     (finalGenEigValue); [Ct C]^H [C Ct] for the SVD of eq. (equationSVD));
//   * basis combination out = [src columns] W  (U_j = Phi_j W_j N_j, eq. (equationForUC));
//   * SpMM C = Op U, Ct = Op^H Ut (C = A U, Section 3 / 4.3);
//   * in-place rotation B <- B N (U <- U N_p, C <- C N_p).
// Each kernel streams the n rows once; the small matrices live in shared memory.
#include <algorithm>

#include "internal.cuh"

namespace rb {

// compute type for the products: FP32 (setup_fp32) or the storage precision
template <class T, bool F32> struct comp_of { typedef T type; };
template <> struct comp_of<double, true> { typedef float type; };
template <> struct comp_of<cplx<double>, true> { typedef cplx<float> type; };

constexpr int GT = 32;        // Gram tile (columns of X and of Y per block)
constexpr int GROWS = 16;     // rows staged per step
constexpr int GFLUSH = 16;    // steps accumulated in the compute type before an FP64 flush

// Block: one GT x GT tile of G for a contiguous range of rows.  Warp w computes the 8 x 16
// sub-tile (rows 8 (w & 3) .., columns 16 (w >> 2) ..), each lane a 2 x 2 block of it.  A warp
// whose sub-tile lies beyond the last column of X or Y skips the products (warp-uniform), so the
// FP64 work follows the actual column counts (the pencil's Grams are 40..110 columns wide, far
// from multiples of a large tile); every entry is accumulated over the rows in the same order
// whichever warp holds it.
template <class T, class Cm>
__global__ void __launch_bounds__(256) k_gram(ColList<T> X, ColList<T> Y, int64_t n, int64_t rows_per_block,
                                              typename traits<T>::acc* part) {
  typedef typename traits<T>::acc A;
  __shared__ Cm xs[GROWS][GT];
  __shared__ Cm ys[GROWS][GT];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ra = 8 * (warp & 3) + 2 * (lane & 3);      // tile rows ra, ra + 1
  const int cb = 16 * (warp >> 2) + 2 * (lane >> 2);   // tile columns cb, cb + 1
  const int ax0 = blockIdx.y * GT, by0 = blockIdx.z * GT;
  const bool active = ax0 + 8 * (warp & 3) < X.m && by0 + 16 * (warp >> 2) < Y.m;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < n ? r0 + rows_per_block : n;
  A acc[2][2];
  Cm loc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) { acc[i][j] = A(0.0); loc[i][j] = Cm(0); }
  int step = 0;
  for (int64_t rb0 = r0; rb0 < r1; rb0 += GROWS) {
    __syncthreads();
    // stage GROWS rows x GT columns of X and Y (row fastest within a half-warp)
    for (int e = threadIdx.x; e < GROWS * GT; e += 256) {
      const int rr = e % GROWS, cc = e / GROWS;
      const int64_t row = rb0 + rr;
      Cm xv = Cm(0), yv = Cm(0);
      if (row < r1) {
        if (ax0 + cc < X.m) { const ColSrc<T> s = X.c[ax0 + cc]; xv = cvt<Cm>(s.p[row * s.ld]); }
        if (by0 + cc < Y.m) { const ColSrc<T> s = Y.c[by0 + cc]; yv = cvt<Cm>(s.p[row * s.ld]); }
      }
      xs[rr][cc] = xv;
      ys[rr][cc] = yv;
    }
    __syncthreads();
    if (active) {
#pragma unroll 4
      for (int rr = 0; rr < GROWS; ++rr) {
        const Cm xa[2] = {xs[rr][ra], xs[rr][ra + 1]};
        const Cm yb[2] = {ys[rr][cb], ys[rr][cb + 1]};
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) loc[i][j] += cmul(xa[i], yb[j]);
      }
    }
    if (++step == GFLUSH) {
      step = 0;
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) { acc[i][j] += cvt<A>(loc[i][j]); loc[i][j] = Cm(0); }
    }
  }
  const int ntile = gridDim.y * gridDim.z;
  const int tile = blockIdx.y * gridDim.z + blockIdx.z;
  A* out = part + ((int64_t)blockIdx.x * ntile + tile) * (GT * GT);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) out[(ra + i) * GT + (cb + j)] = acc[i][j] + cvt<A>(loc[i][j]);
}

// Small Grams (X and Y at most GT columns, at most 2 entries per thread; the Section 4.3 SVD input
// C~_j^H C_j is k x k): thread t owns entries t and t + 256 of the mx x my block, so no FP64
// multiply-add is spent on padding (the 8 x 16 warp sub-tiles of k_gram compute 24 x 32 entries
// for a 20 x 20 Gram).  Staging, row order and flushes are those of k_gram, so every entry is
// the same sum in the same order; the partial tile has k_gram's layout.
template <class T, class Cm>
__global__ void __launch_bounds__(256) k_gram_small(ColList<T> X, ColList<T> Y, int64_t n, int64_t rows_per_block,
                                                    typename traits<T>::acc* part) {
  typedef typename traits<T>::acc A;
  __shared__ Cm xs[GROWS][GT];
  __shared__ Cm ys[GROWS][GT];
  const int mx = X.m, my = Y.m, ne = mx * my;
  const int e0 = threadIdx.x, e1 = threadIdx.x + 256;
  const int a0 = e0 < ne ? e0 / my : 0, b0 = e0 < ne ? e0 % my : 0;
  const int a1 = e1 < ne ? e1 / my : 0, b1 = e1 < ne ? e1 % my : 0;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < n ? r0 + rows_per_block : n;
  A acc0 = A(0.0), acc1 = A(0.0);
  Cm loc0 = Cm(0), loc1 = Cm(0);
  int step = 0;
  for (int64_t rb0 = r0; rb0 < r1; rb0 += GROWS) {
    __syncthreads();
    for (int e = threadIdx.x; e < GROWS * GT; e += 256) {
      const int rr = e % GROWS, cc = e / GROWS;
      const int64_t row = rb0 + rr;
      Cm xv = Cm(0), yv = Cm(0);
      if (row < r1) {
        if (cc < mx) { const ColSrc<T> sx = X.c[cc]; xv = cvt<Cm>(sx.p[row * sx.ld]); }
        if (cc < my) { const ColSrc<T> sy = Y.c[cc]; yv = cvt<Cm>(sy.p[row * sy.ld]); }
      }
      xs[rr][cc] = xv;
      ys[rr][cc] = yv;
    }
    __syncthreads();
    if (e0 < ne) {
#pragma unroll 4
      for (int rr = 0; rr < GROWS; ++rr) {
        loc0 += cmul(xs[rr][a0], ys[rr][b0]);
        if (e1 < ne) loc1 += cmul(xs[rr][a1], ys[rr][b1]);
      }
    }
    if (++step == GFLUSH) {
      step = 0;
      acc0 += cvt<A>(loc0); loc0 = Cm(0);
      acc1 += cvt<A>(loc1); loc1 = Cm(0);
    }
  }
  A* out = part + (int64_t)blockIdx.x * (GT * GT);
  if (e0 < ne) out[a0 * GT + b0] = acc0 + cvt<A>(loc0);
  if (e1 < ne) out[a1 * GT + b1] = acc1 + cvt<A>(loc1);
}

// Warp-shuffle sum in a fixed order (xor 16, 8, 4, 2, 1): the same bits whatever the timing.
__device__ __forceinline__ double warp_sum_fixed(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ cplx<double> warp_sum_fixed(cplx<double> v) {
  return cplx<double>(warp_sum_fixed(v.re), warp_sum_fixed(v.im));
}

// G[e] = sum over the row chunks of the partial tiles: one warp per entry, lane l summing chunks
// l, l + 32, ... in order, then the fixed shuffle tree (the chain is nchunk / 32 long instead of
// nchunk: with several waves of Gram blocks there are hundreds of chunks)
template <class A>
__global__ void k_gram_reduce(const A* part, int nchunk, int ty, int tz, int mx, int my, A* G) {
  const int ntile = ty * tz;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < mx * my; e += gridDim.x * wpb) {
    const int a = e / my, b = e % my;
    const int tile = (a / GT) * tz + (b / GT);
    const int64_t off = (int64_t)tile * GT * GT + (a % GT) * GT + (b % GT);
    A s = A(0.0);
    for (int c = lane; c < nchunk; c += 32) s += part[(int64_t)c * ntile * GT * GT + off];
    s = warp_sum_fixed(s);
    if (lane == 0) G[e] = s;
  }
}

template <class T>
void launch_gram(const ColList<T>& X, const ColList<T>& Y, int64_t n, int fp32, void* part, int grid,
                 typename traits<T>::acc* G, cudaStream_t s) {
  typedef typename traits<T>::acc A;
  const int ty = (X.m + GT - 1) / GT, tz = (Y.m + GT - 1) / GT;
  int nchunk = std::max(1, grid / (ty * tz));
  int64_t rpb = (n + nchunk - 1) / nchunk;
  rpb = ((rpb + GROWS - 1) / GROWS) * GROWS;
  nchunk = (int)((n + rpb - 1) / rpb);
  dim3 g(nchunk, ty, tz);
  const bool small = X.m <= GT && Y.m <= GT && X.m * Y.m <= 512;
  if (small && fp32)
    k_gram_small<T, typename comp_of<T, true>::type><<<g, 256, 0, s>>>(X, Y, n, rpb, (A*)part);
  else if (small)
    k_gram_small<T, T><<<g, 256, 0, s>>>(X, Y, n, rpb, (A*)part);
  else if (fp32)
    k_gram<T, typename comp_of<T, true>::type><<<g, 256, 0, s>>>(X, Y, n, rpb, (A*)part);
  else
    k_gram<T, T><<<g, 256, 0, s>>>(X, Y, n, rpb, (A*)part);
  k_gram_reduce<A><<<std::max(1, std::min(1024, (X.m * Y.m + 7) / 8)), 256, 0, s>>>((const A*)part, nchunk, ty, tz,
                                                                                   X.m, Y.m, G);
}

// ------------------------------------------------------------------------------------
// Input of the Section 4.3 SVD: S = Ct^H C (k x k) and the column norms of C and Ct, packed
// where the SVD kernel reads them in a 2 kmax x 2 kmax row-major array (S top-left, ||C e_c||^2
// on the diagonal of the bottom-left block, ||Ct e_c||^2 on that of the top-right block).  The
// norms are column sums of squares of the row-major n x ld blocks: thread (t % 64) holds one
// column (C's k, then Ct's k), thread t / 64 one of four row lanes; blocks write per-column
// partials, one block adds them in block order.
// ------------------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_colnorms(const T* __restrict__ C, const T* __restrict__ Ct, int ld, int k,
                                                  int64_t n, int64_t rows_per_block, double* part) {
  __shared__ double red[4][64];
  const int c = threadIdx.x & 63, lanes = 4, l = threadIdx.x >> 6;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < n ? r0 + rows_per_block : n;
  double acc = 0.0;
  if (c < 2 * k) {
    const T* B = c < k ? C : Ct;
    const int cc = c < k ? c : c - k;
    for (int64_t row = r0 + l; row < r1; row += lanes) acc += (double)abs2(B[row * ld + cc]);
  }
  red[l][c] = acc;
  __syncthreads();
  if (threadIdx.x < 64) part[(int64_t)blockIdx.x * 64 + c] = red[0][c] + red[1][c] + red[2][c] + red[3][c];
}

template <class A>
__global__ void k_svd_pack(const double* part, int nblk, const A* G, int k, int kmax, zd* S2) {
  const int ld2 = 2 * kmax;
  for (int e = threadIdx.x; e < ld2 * ld2; e += blockDim.x) S2[e] = zd(0.0);
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) S2[(e / k) * ld2 + e % k] = to_zd(G[e]);
  // column sums of the blocks' partials: one warp per column, fixed order (see k_gram_reduce)
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int c = threadIdx.x >> 5; c < 2 * k; c += wpb) {
    double sacc = 0.0;
    for (int b = lane; b < nblk; b += 32) sacc += part[(int64_t)b * 64 + c];
    sacc = warp_sum_fixed(sacc);
    if (lane == 0) {
      if (c < k) S2[(kmax + c) * ld2 + c] = zd(sacc);              // ||C e_c||^2
      else S2[(c - k) * ld2 + kmax + (c - k)] = zd(sacc);            // ||Ct e_c||^2
    }
  }
}

template <class T>
void launch_svd_input(const T* C, const T* Ct, int ld, int k, int kmax, int64_t n, void* part, int grid,
                      typename traits<T>::acc* G, zd* S2, cudaStream_t s) {
  typedef typename traits<T>::acc A;
  ColList<T> X{}, Y{};
  for (int c = 0; c < k; ++c) { X.c[c].p = Ct + c; X.c[c].ld = ld; Y.c[c].p = C + c; Y.c[c].ld = ld; }
  X.m = Y.m = k;
  launch_gram<T>(X, Y, n, 0, part, grid, G, s);
  // the norms' partials go after the Gram's (the Gram uses at most grid x GT^2 entries)
  double* np = reinterpret_cast<double*>(reinterpret_cast<A*>(part) + (size_t)grid * GT * GT);
  const int nb = std::max(1, std::min(grid, (int)((n + 255) / 256)));
  const int64_t rpb = (n + nb - 1) / nb;
  k_colnorms<T><<<nb, 256, 0, s>>>(C, Ct, ld, k, n, rpb, np);
  k_svd_pack<A><<<1, 256, 0, s>>>(np, nb, G, k, kmax, S2);
}

// out[row, c] = sum_a src_a[row] * W[a, c]   (c < ncols, read on the device)
// KC: accumulators per row, one of 8, 12, 16, 20, 24, 32, >= ncols_max (the recycle dimension)
template <class T, class Cm, int KC>
__global__ void __launch_bounds__(256) k_combine(ColList<T> src, const zd* W, int ldw, const int* ncols_dev,
                                                 int ncols_max, T* out, int ldo, int64_t n) {
  extern __shared__ unsigned char smraw[];
  Cm* Ws = reinterpret_cast<Cm*>(smraw);   // src.m x KC
  const int nc = min(*ncols_dev, ncols_max);
  for (int e = threadIdx.x; e < src.m * KC; e += blockDim.x) {
    const int a = e / KC, c = e % KC;
    Ws[e] = c < nc ? from_zd<Cm>(W[a * ldw + c]) : Cm(0);
  }
  __syncthreads();
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x) {
    Cm acc[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) acc[c] = Cm(0);
#pragma unroll 4
    for (int a = 0; a < src.m; ++a) {
      const ColSrc<T> sc = src.c[a];
      const Cm xv = cvt<Cm>(sc.p[row * sc.ld]);
      const Cm* w = Ws + a * KC;
#pragma unroll
      for (int c = 0; c < KC; ++c) acc[c] += xv * w[c];
    }
    T* o = out + row * ldo;
#pragma unroll
    for (int c = 0; c < KC; ++c)   // constant indices keep acc in registers (ldo <= KC)
      if (c < ldo) o[c] = c < nc ? cvt<T>(acc[c]) : T(0);
  }
}

template <class T>
void launch_combine(const ColList<T>& src, const zd* W, int ldw, const int* ncols_dev, int ncols_max, T* out,
                    int ldo, int64_t n, int fp32, cudaStream_t s) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
  // src.m <= MMAX + 2 columns; complex FP64 coefficients can exceed the 48 KB default
  const int maxsm = (MMAX + 2) * KMAX * (int)sizeof(T);
#define RB_COMB(KC)                                                                                           \
  if (fp32) {                                                                                                 \
    typedef typename comp_of<T, true>::type Cm;                                                               \
    cudaFuncSetAttribute(k_combine<T, Cm, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm);           \
    k_combine<T, Cm, KC><<<grid, 256, src.m * KC * sizeof(Cm), s>>>(src, W, ldw, ncols_dev, ncols_max, out, ldo, n); \
  } else {                                                                                                    \
    cudaFuncSetAttribute(k_combine<T, T, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm);            \
    k_combine<T, T, KC><<<grid, 256, src.m * KC * sizeof(T), s>>>(src, W, ldw, ncols_dev, ncols_max, out, ldo, n); \
  }
  // accumulators per row: the recycle dimension rounded up to 4 (k = 10, 16, 20 are common), so
  // the FP64 products follow k instead of a coarser multiple
  if (ncols_max <= 8) { RB_COMB(8) }
  else if (ncols_max <= 12) { RB_COMB(12) }
  else if (ncols_max <= 16) { RB_COMB(16) }
  else if (ncols_max <= 20) { RB_COMB(20) }
  else if (ncols_max <= 24) { RB_COMB(24) }
  else { RB_COMB(32) }
#undef RB_COMB
}

// in-place B[row, 0..kout) <- sum_{a < kin} B[row, a] N[a, c]
template <class T, class Cm, int KC>
__global__ void __launch_bounds__(256) k_rotate(T* B, int ld, const zd* Nmat, const int* kin_dev, const int* kout_dev,
                                                int kmax, int64_t n) {
  __shared__ Cm Ns[KC * KC];
  const int kin = min(*kin_dev, kmax), kout = min(*kout_dev, kmax);
  for (int e = threadIdx.x; e < KC * KC; e += blockDim.x) {
    const int a = e / KC, c = e % KC;
    Ns[e] = (a < kin && c < kout) ? from_zd<Cm>(Nmat[a * KMAX + c]) : Cm(0);
  }
  __syncthreads();
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x) {
    T* b = B + row * ld;
    Cm acc[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) acc[c] = Cm(0);
    for (int a = 0; a < kin; ++a) {
      const Cm xv = cvt<Cm>(b[a]);
#pragma unroll
      for (int c = 0; c < KC; ++c) acc[c] += xv * Ns[a * KC + c];
    }
#pragma unroll
    for (int c = 0; c < KC; ++c)   // constant indices keep acc in registers (ld <= KC)
      if (c < ld) b[c] = c < kout ? cvt<T>(acc[c]) : T(0);
  }
}

template <class T>
void launch_rotate(T* B, int ld, const zd* Nmat, const int* kin_dev, const int* kout_dev, int kmax, int64_t n,
                   int fp32, cudaStream_t s) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
#define RB_ROT(KC)                                                                                         \
  if (fp32)                                                                                                \
    k_rotate<T, typename comp_of<T, true>::type, KC><<<grid, 256, 0, s>>>(B, ld, Nmat, kin_dev, kout_dev, kmax, n); \
  else                                                                                                     \
    k_rotate<T, T, KC><<<grid, 256, 0, s>>>(B, ld, Nmat, kin_dev, kout_dev, kmax, n);
  if (kmax <= 8) { RB_ROT(8) }
  else if (kmax <= 12) { RB_ROT(12) }
  else if (kmax <= 16) { RB_ROT(16) }
  else if (kmax <= 20) { RB_ROT(20) }
  else if (kmax <= 24) { RB_ROT(24) }
  else { RB_ROT(32) }
#undef RB_ROT
}

// out[row, c] = (Op U)[row, c]  for c < ncols; Op = A (adjoint = 0) or Op^H (adjoint = 1)
template <class V, class T, class Cm, int KC>
__global__ void __launch_bounds__(256) k_spmm(OpArgs<V> op, int adjoint, const T* U, int ldu, const int* ncols_dev,
                                              int ncols_max, T* out) {
  const int nc = min(*ncols_dev, ncols_max);
  const int* rp = adjoint ? op.trp : op.rp;
  const int* ci = adjoint ? op.tci : op.ci;
  const V* va = adjoint ? op.tva : op.va;
  Cm sh = from_zd<Cm>(zd(op.sh_re, adjoint ? -op.sh_im : op.sh_im));
  typedef typename val_of<V, Cm>::type Va;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < op.n; row += gridDim.x * blockDim.x) {
    SpAcc<Cm> acc[KC];   // compensated for FP32 compute types (see SpAcc)
    for (int e = rp[row]; e < rp[row + 1]; ++e) {
      const Va a = cvt<Va>(va[e]);
      const T* u = U + (int64_t)ci[e] * ldu;
#pragma unroll
      for (int c = 0; c < KC; ++c)
        if (c < nc) acc[c].add(a, cvt<Cm>(u[c]));
    }
    T* o = out + (int64_t)row * ldu;
    const T* ur = U + (int64_t)row * ldu;
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      if (c >= ldu) break;
      const Cm v = op.has_shift ? acc[c].shifted(sh, cvt<Cm>(ur[c])) : acc[c].value();
      o[c] = c < nc ? cvt<T>(v) : T(0);
    }
  }
}

template <class V, class T>
void launch_spmm(const OpArgs<V>& op, int adjoint, const T* U, int ldu, const int* ncols_dev, int ncols_max, T* out,
                 int fp32, cudaStream_t s) {
  const int grid = std::max(1, std::min((op.n + 255) / 256, 152 * 8));
  // fp32: per-cycle C_j = A U_j in FP32 arithmetic (it feeds only the FP32 Grams and SVD of
  // the refreshes; the system start forms C = A U in FP64)
#define RB_SPMM(KC)                                                                                          \
  if (fp32)                                                                                                  \
    k_spmm<V, T, typename comp_of<T, true>::type, KC><<<grid, 256, 0, s>>>(op, adjoint, U, ldu, ncols_dev, ncols_max, out); \
  else                                                                                                       \
    k_spmm<V, T, T, KC><<<grid, 256, 0, s>>>(op, adjoint, U, ldu, ncols_dev, ncols_max, out);
  if (ldu <= 8) { RB_SPMM(8) }
  else if (ldu <= 16) { RB_SPMM(16) }
  else if (ldu <= 24) { RB_SPMM(24) }
  else { RB_SPMM(32) }
#undef RB_SPMM
}

template <class Tfrom, class Tto>
__global__ void k_convert(const Tfrom* a, Tto* b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = cvt<Tto>(a[i]);
}
template <class Tfrom, class Tto>
void launch_convert(const Tfrom* a, Tto* b, int64_t n, cudaStream_t s) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
  k_convert<Tfrom, Tto><<<grid, 256, 0, s>>>(a, b, n);
}

template <class T>
__global__ void k_axpy_inplace(T* y, const T* x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = y[i] + x[i];
}
template <class T>
void launch_axpy_inplace(T* y, const T* x, int64_t n, cudaStream_t s) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
  k_axpy_inplace<T><<<grid, 256, 0, s>>>(y, x, n);
}

// ---------------------------------------------------------------- instantiations
#define RB_INST_T(T)                                                                                          \
  template void launch_gram<T>(const ColList<T>&, const ColList<T>&, int64_t, int, void*, int,                \
                               typename traits<T>::acc*, cudaStream_t);                                      \
  template void launch_combine<T>(const ColList<T>&, const zd*, int, const int*, int, T*, int, int64_t, int,  \
                                  cudaStream_t);                                                             \
  template void launch_rotate<T>(T*, int, const zd*, const int*, const int*, int, int64_t, int, cudaStream_t); \
  template void launch_axpy_inplace<T>(T*, const T*, int64_t, cudaStream_t);                                 \
  template void launch_svd_input<T>(const T*, const T*, int, int, int, int64_t, void*, int,                   \
                                    typename traits<T>::acc*, zd*, cudaStream_t);

RB_INST_T(double)
RB_INST_T(float)
RB_INST_T(cplx<double>)
RB_INST_T(cplx<float>)

template void launch_spmm<double, double>(const OpArgs<double>&, int, const double*, int, const int*, int, double*,
                                          int, cudaStream_t);
template void launch_spmm<float, float>(const OpArgs<float>&, int, const float*, int, const int*, int, float*, int,
                                        cudaStream_t);
template void launch_spmm<double, cplx<double>>(const OpArgs<double>&, int, const cplx<double>*, int, const int*,
                                                int, cplx<double>*, int, cudaStream_t);
template void launch_spmm<cplx<double>, cplx<double>>(const OpArgs<cplx<double>>&, int, const cplx<double>*, int,
                                                      const int*, int, cplx<double>*, int, cudaStream_t);
template void launch_spmm<float, cplx<float>>(const OpArgs<float>&, int, const cplx<float>*, int, const int*, int,
                                              cplx<float>*, int, cudaStream_t);
template void launch_spmm<cplx<float>, cplx<float>>(const OpArgs<cplx<float>>&, int, const cplx<float>*, int,
                                                    const int*, int, cplx<float>*, int, cudaStream_t);

template void launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template void launch_convert<cplx<double>, cplx<float>>(const cplx<double>*, cplx<float>*, int64_t, cudaStream_t);
template void launch_convert<cplx<float>, cplx<double>>(const cplx<float>*, cplx<double>*, int64_t, cudaStream_t);

}  // namespace rb
