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

constexpr int GT = 64;        // Gram tile (columns of X and of Y per block)
constexpr int GROWS = 16;     // rows staged per step
constexpr int GFLUSH = 16;    // steps accumulated in the compute type before an FP64 flush

template <class T, class Cm>
__global__ void __launch_bounds__(256) k_gram(ColList<T> X, ColList<T> Y, int64_t n, int64_t rows_per_block,
                                              typename traits<T>::acc* part) {
  typedef typename traits<T>::acc A;
  __shared__ Cm xs[GROWS][GT];
  __shared__ Cm ys[GROWS][GT];
  const int ta = threadIdx.x & 15, tb = threadIdx.x >> 4;
  const int ax0 = blockIdx.y * GT, by0 = blockIdx.z * GT;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < n ? r0 + rows_per_block : n;
  A acc[4][4];
  Cm loc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { acc[i][j] = A(0.0); loc[i][j] = Cm(0); }
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
#pragma unroll 4
    for (int rr = 0; rr < GROWS; ++rr) {
      Cm xa[4], yb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { xa[i] = xs[rr][ta + 16 * i]; yb[i] = ys[rr][tb + 16 * i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) loc[i][j] += cmul(xa[i], yb[j]);
    }
    if (++step == GFLUSH) {
      step = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { acc[i][j] += cvt<A>(loc[i][j]); loc[i][j] = Cm(0); }
    }
  }
  const int ntile = gridDim.y * gridDim.z;
  const int tile = blockIdx.y * gridDim.z + blockIdx.z;
  A* out = part + ((int64_t)blockIdx.x * ntile + tile) * (GT * GT);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(ta + 16 * i) * GT + (tb + 16 * j)] = acc[i][j] + cvt<A>(loc[i][j]);
}

template <class A>
__global__ void k_gram_reduce(const A* part, int nchunk, int ty, int tz, int mx, int my, A* G) {
  const int ntile = ty * tz;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < mx * my; e += gridDim.x * blockDim.x) {
    const int a = e / my, b = e % my;
    const int tile = (a / GT) * tz + (b / GT);
    const int64_t off = (int64_t)tile * GT * GT + (a % GT) * GT + (b % GT);
    A s = A(0.0);
    for (int c = 0; c < nchunk; ++c) s += part[(int64_t)c * ntile * GT * GT + off];
    G[e] = s;
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
  if (fp32)
    k_gram<T, typename comp_of<T, true>::type><<<g, 256, 0, s>>>(X, Y, n, rpb, (A*)part);
  else
    k_gram<T, T><<<g, 256, 0, s>>>(X, Y, n, rpb, (A*)part);
  k_gram_reduce<A><<<std::max(1, std::min(64, (X.m * Y.m + 255) / 256)), 256, 0, s>>>((const A*)part, nchunk, ty,
                                                                                     tz, X.m, Y.m, G);
}

// out[row, c] = sum_a src_a[row] * W[a, c]   (c < ncols, read on the device)
// KC: accumulators per row, a multiple of 8 >= ncols_max (the recycle dimension)
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
  if (ncols_max <= 8) { RB_COMB(8) }
  else if (ncols_max <= 16) { RB_COMB(16) }
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
  else if (kmax <= 16) { RB_ROT(16) }
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
  template void launch_axpy_inplace<T>(T*, const T*, int64_t, cudaStream_t);

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
