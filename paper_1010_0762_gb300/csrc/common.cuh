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
// Sparse row sums sum_e a_e x_e.  In FP32 the 5-/7-point stencil rows cancel almost completely
// on the smooth vectors that decide BiCG's convergence (the diagonal and the neighbour sum agree
// to about log10(cond) digits), and a plain FP32 sum keeps only the few digits left: FP32 BiCG
// then stalls near ||r|| ~ ||b|| on a 128 x 128 grid, while the same recurrences with the row
// sums exact to FP32 rounding converge like FP64 BiCG.  So the FP32 types accumulate with a
// compensated dot product (Ogita, Rump and Oishi, "Accurate sum and dot product", 2005): each
// product is split into its rounded value and its exact error by a fused multiply-add, each
// running-sum addition into its rounded value and its exact error by Knuth's two-sum, and the
// errors are summed in a second FP32 accumulator; the result is as accurate as a sum in twice
// the working precision, rounded once.  The FP64 types keep a plain sum.
// ------------------------------------------------------------------------------------
struct Dot2f {
  float s, c;
  RB_HD Dot2f() : s(0.f), c(0.f) {}
  RB_HD void two_sum_into(float p) {
#ifdef __CUDA_ARCH__
    const float t = __fadd_rn(s, p);
    const float bb = __fadd_rn(t, -s);
    const float err = __fadd_rn(__fadd_rn(s, -__fadd_rn(t, -bb)), __fadd_rn(p, -bb));
#else
    const float t = s + p, bb = t - s, err = (s - (t - bb)) + (p - bb);
#endif
    s = t;
    c += err;
  }
  RB_HD void add_prod(float a, float x) {
#ifdef __CUDA_ARCH__
    const float p = __fmul_rn(a, x);
#else
    const float p = a * x;
#endif
    const float e = fmaf(a, x, -p);
    two_sum_into(p);
    c += e;
  }
  RB_HD float value() const { return s + c; }
};

// Type of an operator value in a sum over vectors of compute type Cm: real operators stay real
// (a real-by-complex product is two real products), complex ones take Cm.
template <class V, class Cm> struct val_of { typedef Cm type; };
template <class Cm> struct val_of<double, Cm> { typedef typename traits<Cm>::real type; };
template <class Cm> struct val_of<float, Cm> { typedef typename traits<Cm>::real type; };

template <class T> struct SpAcc;
// FP64: a plain sum, so that the FP64 kernels keep their arithmetic
template <> struct SpAcc<double> {
  double acc = 0.0;
  RB_HD void add(double a, double x) { acc += a * x; }
  RB_HD double value() const { return acc; }
  RB_HD double shifted(double sh, double prow) const { return sh * prow - acc; }
};
template <> struct SpAcc<cplx<double>> {
  cplx<double> acc = cplx<double>(0.0);
  RB_HD void add(double a, cplx<double> x) { acc += vmul(a, x); }
  RB_HD void add(cplx<double> a, cplx<double> x) { acc += vmul(a, x); }
  RB_HD cplx<double> value() const { return acc; }
  RB_HD cplx<double> shifted(cplx<double> sh, cplx<double> prow) const { return sh * prow - acc; }
};
// FP32: compensated
template <> struct SpAcc<float> {
  Dot2f d;
  RB_HD void add(float a, float x) { d.add_prod(a, x); }
  RB_HD float value() const { return d.value(); }
  RB_HD float shifted(float sh, float prow) const {   // sh prow - sum, one compensated sum
    Dot2f q;
    q.add_prod(sh, prow);
    q.two_sum_into(-d.s);
    q.c -= d.c;
    return q.value();
  }
};
template <> struct SpAcc<cplx<float>> {
  Dot2f re, im;
  RB_HD void add(float a, cplx<float> x) { re.add_prod(a, x.re); im.add_prod(a, x.im); }
  RB_HD void add(cplx<float> a, cplx<float> x) {
    re.add_prod(a.re, x.re); re.add_prod(-a.im, x.im);
    im.add_prod(a.re, x.im); im.add_prod(a.im, x.re);
  }
  RB_HD cplx<float> value() const { return cplx<float>(re.value(), im.value()); }
  RB_HD cplx<float> shifted(cplx<float> sh, cplx<float> prow) const {
    Dot2f qr, qi;
    qr.add_prod(sh.re, prow.re); qr.add_prod(-sh.im, prow.im);
    qi.add_prod(sh.re, prow.im); qi.add_prod(sh.im, prow.re);
    qr.two_sum_into(-re.s); qr.c -= re.c;
    qi.two_sum_into(-im.s); qi.c -= im.c;
    return cplx<float>(qr.value(), qi.value());
  }
};

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
