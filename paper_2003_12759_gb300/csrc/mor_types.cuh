// Scalar types and small device helpers shared by the kernels of the
// shifted-solve library.  Scalars are real (float/double) or complex
// (cfloat/cdouble, interleaved re/im); kernels are templated on them so that
// one source serves the FP64 path and the FP32/complex64 inner path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#define MOR_HD __host__ __device__ __forceinline__

template <typename R>
struct cplx {
  R re, im;
  MOR_HD cplx() {}
  MOR_HD cplx(R r) : re(r), im(R(0)) {}
  MOR_HD cplx(R r, R i) : re(r), im(i) {}
};
typedef cplx<float> cfloat;
typedef cplx<double> cdouble;

// ---- type traits ----------------------------------------------------------
template <typename S> struct real_of { typedef S type; };
template <typename R> struct real_of<cplx<R>> { typedef R type; };
template <typename S> struct is_cplx { static const bool value = false; };
template <typename R> struct is_cplx<cplx<R>> { static const bool value = true; };

// ---- arithmetic -----------------------------------------------------------
template <typename R> MOR_HD cplx<R> operator+(cplx<R> a, cplx<R> b) { return cplx<R>(a.re + b.re, a.im + b.im); }
template <typename R> MOR_HD cplx<R> operator-(cplx<R> a, cplx<R> b) { return cplx<R>(a.re - b.re, a.im - b.im); }
template <typename R> MOR_HD cplx<R> operator-(cplx<R> a) { return cplx<R>(-a.re, -a.im); }
template <typename R> MOR_HD cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return cplx<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R> MOR_HD cplx<R> operator*(R a, cplx<R> b) { return cplx<R>(a * b.re, a * b.im); }
template <typename R> MOR_HD cplx<R> operator*(cplx<R> b, R a) { return cplx<R>(a * b.re, a * b.im); }
template <typename R> MOR_HD cplx<R>& operator+=(cplx<R>& a, cplx<R> b) { a.re += b.re; a.im += b.im; return a; }
template <typename R> MOR_HD cplx<R>& operator-=(cplx<R>& a, cplx<R> b) { a.re -= b.re; a.im -= b.im; return a; }

MOR_HD float conj_(float a) { return a; }
MOR_HD double conj_(double a) { return a; }
template <typename R> MOR_HD cplx<R> conj_(cplx<R> a) { return cplx<R>(a.re, -a.im); }

MOR_HD float abs2_(float a) { return a * a; }
MOR_HD double abs2_(double a) { return a * a; }
template <typename R> MOR_HD R abs2_(cplx<R> a) { return a.re * a.re + a.im * a.im; }

MOR_HD float real_(float a) { return a; }
MOR_HD double real_(double a) { return a; }
template <typename R> MOR_HD R real_(cplx<R> a) { return a.re; }
MOR_HD float imag_(float) { return 0.f; }
MOR_HD double imag_(double) { return 0.0; }
template <typename R> MOR_HD R imag_(cplx<R> a) { return a.im; }

// a * b with b real (matrix value times vector entry)
template <typename S, typename R> MOR_HD S scale_(R a, S b) { return a * b; }

// fused multiply-add acc += a * b for real a (matrix value), scalar b
MOR_HD void fma_r(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
MOR_HD void fma_r(double& acc, double a, double b) { acc = fma(a, b, acc); }
template <typename R> MOR_HD void fma_r(cplx<R>& acc, R a, cplx<R> b) {
  acc.re = fma(a, b.re, acc.re);
  acc.im = fma(a, b.im, acc.im);
}
// acc += a * b for scalars of the same type
MOR_HD void fma_s(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
MOR_HD void fma_s(double& acc, double a, double b) { acc = fma(a, b, acc); }
template <typename R> MOR_HD void fma_s(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}

// conversions between precisions / real-complex
template <typename D, typename S> struct cvt_ { static MOR_HD D f(S s) { return D(s); } };
template <typename R1, typename R2> struct cvt_<cplx<R1>, cplx<R2>> {
  static MOR_HD cplx<R1> f(cplx<R2> s) { return cplx<R1>(R1(s.re), R1(s.im)); }
};
template <typename R1, typename R2> struct cvt_<cplx<R1>, R2> {
  static MOR_HD cplx<R1> f(R2 s) { return cplx<R1>(R1(s), R1(0)); }
};
template <typename R1, typename R2> struct cvt_<R1, cplx<R2>> {
  static MOR_HD R1 f(cplx<R2> s) { return R1(s.re); }   // drops the imaginary part
};
template <typename D, typename S> MOR_HD D cvt(S s) { return cvt_<D, S>::f(s); }

// complex division (scaled to avoid overflow; FP64 scalar work only)
MOR_HD cdouble cdiv(cdouble a, cdouble b) {
  double s = fabs(b.re) + fabs(b.im);
  double br = b.re / s, bi = b.im / s;
  double ar = a.re / s, ai = a.im / s;
  double d = br * br + bi * bi;
  return cdouble((ar * br + ai * bi) / d, (ai * br - ar * bi) / d);
}
MOR_HD double cabs_(cdouble a) { return hypot(a.re, a.im); }

// ---- warp reductions ------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename R> __device__ __forceinline__ cplx<R> warp_sum(cplx<R> v) {
  return cplx<R>(warp_sum(v.re), warp_sum(v.im));
}
