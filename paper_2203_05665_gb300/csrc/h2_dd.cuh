// Double-float arithmetic ("dd"): a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  On
// GB300 the FP64 pipe runs at 1/58 of the FP32 rate, so FP64-accurate
// products are computed in this representation on the FP32 pipe.
//
// The operations are the classical error-free transformations: TwoSum
// (Knuth), TwoProduct through a fused multiply-add, and the double-length
// addition and multiplication built from them (Dekker 1971; the same
// construction as Hida, Li and Bailey's double-double library, here with
// single-precision components).  Relative error per operation < 2^-44.
#pragma once

namespace h2 {

struct __align__(8) dd {
  float hi, lo;
};

__host__ __device__ __forceinline__ dd dd_from_double(double v) {
  float h = (float)v;
  return dd{h, (float)(v - (double)h)};
}

__host__ __device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly (no magnitude condition)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// renormalise (s, e) with |e| small against |s|
__device__ __forceinline__ dd quick_norm(float s, float e) {
  float h = s + e;
  return dd{h, e - (h - s)};
}

__device__ __forceinline__ dd operator+(dd a, dd b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  return quick_norm(s, e);
}

__device__ __forceinline__ dd operator*(dd a, dd b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return quick_norm(p, e);
}

__device__ __forceinline__ dd &operator+=(dd &a, dd b) {
  a = a + b;
  return a;
}

// c + a b: fused multiply-add of each arithmetic (dd: one renormalisation)
__device__ __forceinline__ float madd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double madd(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ dd madd(dd a, dd b, dd c) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s, t;
  two_sum(c.hi, p, s, t);
  t += c.lo + e;
  return quick_norm(s, t);
}

// Accumulation inside one block of a contraction: acc += a b without the
// final renormalisation (12 FP32 instructions for dd; the low word collects
// the exact rounding errors of the high sums and the product errors); call
// acc_norm once the block is done.
__device__ __forceinline__ void acc_fma(float &acc, float a, float b) { acc = fmaf(a, b, acc); }
__device__ __forceinline__ void acc_fma(double &acc, double a, double b) { acc = ::fma(a, b, acc); }
__device__ __forceinline__ void acc_fma(dd &acc, dd a, dd b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s, t;
  two_sum(acc.hi, p, s, t);
  acc.hi = s;
  acc.lo += t + e;
}
__device__ __forceinline__ void acc_norm(float &) {}
__device__ __forceinline__ void acc_norm(double &) {}
__device__ __forceinline__ void acc_norm(dd &a) {
  float s, e;
  two_sum(a.hi, a.lo, s, e);
  a = dd{s, e};
}

// conversions used by the templated kernels
template <class T>
__host__ __device__ __forceinline__ T from_double(double v) {
  return (T)v;
}
template <>
__host__ __device__ __forceinline__ dd from_double<dd>(double v) {
  return dd_from_double(v);
}

template <class To, class From>
__device__ __forceinline__ To convert(From v) {
  return (To)v;
}
template <>
__device__ __forceinline__ dd convert<dd, double>(double v) {
  return dd_from_double(v);
}
template <>
__device__ __forceinline__ double convert<double, dd>(dd v) {
  return dd_to_double(v);
}
template <>
__device__ __forceinline__ dd convert<dd, dd>(dd v) {
  return v;
}

template <class T>
__host__ __device__ __forceinline__ T zero_of() {
  return (T)0;
}
template <>
__host__ __device__ __forceinline__ dd zero_of<dd>() {
  return dd{0.0f, 0.0f};
}

}  // namespace h2
