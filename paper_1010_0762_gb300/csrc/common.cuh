// common.cuh -- scalar types, traits and deterministic reductions shared by the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#define RB_HD __host__ __device__ __forceinline__

namespace rb {

// ------------------------------------------------------------------------------------
// Complex numbers (interleaved re, im; layout-compatible with C99 / numpy complex).
// ------------------------------------------------------------------------------------
// A product rounded on its own (never fused into a neighbouring add), and a fused
// multiply-add.  The complex products below say which of their two products is fused and which
// is rounded, so that every kernel that inlines them -- a solve's kernel and its batched twin
// among them -- computes the same bits.
RB_HD double mul_rn(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  return a * b;
#endif
}
RB_HD float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
RB_HD double fmar(double a, double b, double c) { return fma(a, b, c); }
RB_HD float fmar(float a, float b, float c) { return fmaf(a, b, c); }

template <class R>
struct alignas(2 * sizeof(R)) cplx {
  R re, im;
  cplx() = default;
  RB_HD cplx(R r) : re(r), im(0) {}
  RB_HD cplx(R r, R i) : re(r), im(i) {}
  template <class S>
  RB_HD explicit cplx(const cplx<S>& o) : re(R(o.re)), im(R(o.im)) {}
};
template <class R> RB_HD cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> RB_HD cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> RB_HD cplx<R> operator-(cplx<R> a) { return {-a.re, -a.im}; }
template <class R> RB_HD cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return {fmar(a.re, b.re, -mul_rn(a.im, b.im)), fmar(a.re, b.im, mul_rn(a.im, b.re))};
}
template <class R> RB_HD cplx<R> operator*(R a, cplx<R> b) { return {a * b.re, a * b.im}; }
template <class R> RB_HD cplx<R> operator*(cplx<R> b, R a) { return {a * b.re, a * b.im}; }
template <class R> RB_HD cplx<R>& operator+=(cplx<R>& a, cplx<R> b) { a.re += b.re; a.im += b.im; return a; }
template <class R> RB_HD cplx<R>& operator-=(cplx<R>& a, cplx<R> b) { a.re -= b.re; a.im -= b.im; return a; }
template <class R> RB_HD cplx<R> operator/(cplx<R> a, cplx<R> b) {
  // scaled division (Smith's method) to avoid overflow in |b|^2
  if (fabs(b.re) >= fabs(b.im)) {
    R t = b.im / b.re, d = b.re + b.im * t;
    return {(a.re + a.im * t) / d, (a.im - a.re * t) / d};
  } else {
    R t = b.re / b.im, d = b.re * t + b.im;
    return {(a.re * t + a.im) / d, (a.im * t - a.re) / d};
  }
}
template <class R> RB_HD cplx<R> operator/(cplx<R> a, R b) { return {a.re / b, a.im / b}; }

// ------------------------------------------------------------------------------------
// Uniform helpers over real and complex scalars.
// ------------------------------------------------------------------------------------
RB_HD double conjg(double a) { return a; }
RB_HD float conjg(float a) { return a; }
template <class R> RB_HD cplx<R> conjg(cplx<R> a) { return {a.re, -a.im}; }

RB_HD double abs2(double a) { return a * a; }
RB_HD float abs2(float a) { return a * a; }
template <class R> RB_HD R abs2(cplx<R> a) { return fmar(a.re, a.re, mul_rn(a.im, a.im)); }

RB_HD double absval(double a) { return fabs(a); }
template <class R> RB_HD R absval(cplx<R> a) { return hypot(a.re, a.im); }

RB_HD double real_of(double a) { return a; }
RB_HD float real_of(float a) { return a; }
template <class R> RB_HD R real_of(cplx<R> a) { return a.re; }
RB_HD double imag_of(double) { return 0.0; }
RB_HD float imag_of(float) { return 0.0f; }
template <class R> RB_HD R imag_of(cplx<R> a) { return a.im; }

// conj(a) * b
RB_HD double cmul(double a, double b) { return a * b; }
RB_HD float cmul(float a, float b) { return a * b; }
template <class R> RB_HD cplx<R> cmul(cplx<R> a, cplx<R> b) {
  return {fmar(a.re, b.re, mul_rn(a.im, b.im)), fmar(a.re, b.im, -mul_rn(a.im, b.re))};
}

// 1 / z as conj(z) / |z|^2: one real division.  A dependent FP64 operation costs about 60
// cycles on this part, a division about 570 and the scaled (Smith) complex quotient about
// 2000, so the quotients on critical paths (pivots, reflector factors, the iteration scalars
// alpha and beta) use this form; |z|^2 falls back to the scaled quotient when it would over- or
// underflow.
__device__ __forceinline__ cplx<double> crcp(cplx<double> z) {
  const double n2 = fma(z.re, z.re, z.im * z.im);
  if (!(n2 > 1e-290 && n2 < 1e290)) return cplx<double>(1.0) / z;
  const double d = 1.0 / n2;
  return cplx<double>(z.re * d, -z.im * d);
}

RB_HD bool finite_of(double a) { return isfinite(a); }
template <class R> RB_HD bool finite_of(cplx<R> a) { return isfinite(a.re) && isfinite(a.im); }

// Scalar traits: real type, FP64 accumulation type, complex flag.
template <class T> struct traits;
template <> struct traits<double> { typedef double real; typedef double acc; static const bool cx = false; };
template <> struct traits<float> { typedef float real; typedef double acc; static const bool cx = false; };
template <> struct traits<cplx<double>> { typedef double real; typedef cplx<double> acc; static const bool cx = true; };
template <> struct traits<cplx<float>> { typedef float real; typedef cplx<double> acc; static const bool cx = true; };

// Conversions between storage, compute and accumulation types.
template <class To, class From> struct conv;
template <class From> struct conv<double, From> { static RB_HD double f(From a) { return (double)a; } };
template <class From> struct conv<float, From> { static RB_HD float f(From a) { return (float)a; } };
template <class R, class S> struct conv<cplx<R>, cplx<S>> { static RB_HD cplx<R> f(cplx<S> a) { return cplx<R>((R)a.re, (R)a.im); } };
template <class R> struct conv<cplx<R>, double> { static RB_HD cplx<R> f(double a) { return cplx<R>((R)a, (R)0); } };
template <class R> struct conv<cplx<R>, float> { static RB_HD cplx<R> f(float a) { return cplx<R>((R)a, (R)0); } };
template <class To, class From> RB_HD To cvt(From a) { return conv<To, From>::f(a); }

// Value * vector-type product where the value may be real and the vector complex.
RB_HD double vmul(double v, double x) { return v * x; }
RB_HD float vmul(float v, float x) { return v * x; }
template <class R> RB_HD cplx<R> vmul(R v, cplx<R> x) { return {v * x.re, v * x.im}; }
template <class R> RB_HD cplx<R> vmul(cplx<R> v, cplx<R> x) { return v * x; }
// conj(value) * x
RB_HD double vcmul(double v, double x) { return v * x; }
RB_HD float vcmul(float v, float x) { return v * x; }
template <class R> RB_HD cplx<R> vcmul(R v, cplx<R> x) { return {v * x.re, v * x.im}; }
template <class R> RB_HD cplx<R> vcmul(cplx<R> v, cplx<R> x) { return cmul(v, x); }

// ------------------------------------------------------------------------------------
// Warp / block reductions with a fixed order (deterministic for a given launch shape).
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ cplx<double> shfl_down(cplx<double> v, int o) {
  return {__shfl_down_sync(0xffffffffu, v.re, o), __shfl_down_sync(0xffffffffu, v.im, o)};
}
__device__ __forceinline__ float shfl_down(float v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ cplx<float> shfl_down(cplx<float> v, int o) {
  return {__shfl_down_sync(0xffffffffu, v.re, o), __shfl_down_sync(0xffffffffu, v.im, o)};
}
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ cplx<double> shfl_xor(cplx<double> v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.re, o), __shfl_xor_sync(0xffffffffu, v.im, o)};
}
template <class A>
__device__ __forceinline__ A warp_sum(A v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += shfl_down(v, o);
  return v;
}

// Sum `cnt` values per thread over the block; result valid in thread 0's out[] (and
// written to smem red[cnt]).  smem must hold (blockDim/32) * cnt values of A.
template <class A>
__device__ void block_sum_vec(A* vals, int cnt, A* smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = 0; c < cnt; ++c) {
    A v = warp_sum(vals[c]);
    if (lane == 0) smem[warp * cnt + c] = v;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    A s = smem[threadIdx.x];
    for (int w = 1; w < nw; ++w) s += smem[w * cnt + threadIdx.x];
    smem[threadIdx.x] = s;  // row 0 now holds the block totals
  }
  __syncthreads();
}

}  // namespace rb
