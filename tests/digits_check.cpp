// Host check of the digit decomposition used by the tensor-core phases
// (paper_2203_05665_gb300/csrc/h2_digits.hpp): every digit within [-16, 16],
// the digits reconstruct X exactly, each digit is an exact FP8 E4M3 value,
// and the digit-pair products kept by the kernels (levels i + k <= ND, digits
// counted from 0) reproduce X * Y to within the bound quoted there
// (2^52 of 2^98 for ten digits, 2^31 of 2^58 for six).  Exit status 0 on
// success.
#include <cuda_fp8.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <random>

#include "h2_digits.hpp"

template <int ND>
static int check(long long lim, int samples, long long bound) {
  std::mt19937_64 g(20260 + ND);
  int bad = 0;
  auto one = [&](long long X, long long Y) {
    int s[ND], t[ND];
    h2::split_digits<ND>(X, s);
    h2::split_digits<ND>(Y, t);
    long long rx = 0, ry = 0;
    for (int i = 0; i < ND; ++i) {
      if (s[i] < -16 || s[i] > 16 || t[i] < -16 || t[i] > 16) ++bad;
      rx = rx * 32 + s[i];
      ry = ry * 32 + t[i];
    }
    if (rx != X || ry != Y) ++bad;
    __int128 kept = 0;
    for (int i = 0; i < ND; ++i)
      for (int k = 0; k < ND; ++k)
        if (i + k <= ND - 1)
          kept += (__int128)(s[i] * t[k]) << (5 * (ND - 1 - i) + 5 * (ND - 1 - k));
    __int128 err = (__int128)X * Y - kept;
    if (err < 0) err = -err;
    if (err > (__int128)bound) ++bad;
  };
  const long long edge[] = {0, 1, -1, 15, 16, 17, -16, -17, 31, 32, lim, -lim, lim - 1, -lim + 1};
  for (long long a : edge)
    for (long long b : edge) one(a, b);
  for (int e = 0; (1LL << e) <= lim; ++e)
    for (long long d = -3; d <= 3; ++d) {
      const long long a = (1LL << e) + d, b = -(1LL << e) + d;
      if (a <= lim && a >= -lim) one(a, lim - 7);
      if (b <= lim && b >= -lim) one(b, -lim + 3);
    }
  std::uniform_int_distribution<long long> u(-lim, lim);
  for (int n = 0; n < samples; ++n) one(u(g), u(g));
  return bad;
}

// split_digits_f (32-bit operations, float digits) against split_digits of
// the 64-bit integer rint(hs) + rint(ls), for double-float pairs (hi, lo) and
// FP32 values scaled as the kernels scale them (|hs| < 2^(5 ND - 2)), on
// boundary values and random samples
template <int ND>
static int check_f(int samples) {
  std::mt19937_64 g(4242 + ND);
  int bad = 0;
  auto one = [&](float hs, float ls) {
    float f[ND];
    int s[ND];
    h2::split_digits_f<ND>(hs, ls, f);
    h2::split_digits<ND>(llrintf(hs) + llrintf(ls), s);
    for (int i = 0; i < ND; ++i)
      if (f[i] != (float)s[i]) ++bad;
  };
  const float top = std::ldexp(1.0f, 5 * ND - 2);
  const float edge[] = {0.0f, 0.5f, 1.5f, 2.5f, 15.5f, 16.5f, 8388607.5f, 16777216.0f, 33554431.0f,
                        33554432.0f, 50331648.0f, std::nextafter(top, 0.0f), top / 3};
  for (float a : edge)
    for (float b : {0.0f, 0.5f, -0.5f, 1.5f, -2.5f, 16777216.0f, -33554430.0f}) {
      if (ND == 6) b = 0.0f;
      one(a, b);
      one(-a, -b);
      one(a, -b);
    }
  std::uniform_real_distribution<float> u(-1.0f, 1.0f);
  std::uniform_int_distribution<int> ex(-30, 5 * ND - 3);
  for (int n = 0; n < samples; ++n) {
    const float hi = std::ldexp(u(g), ex(g));   // |hi| < 2^(5 ND - 2)
    float lo = 0.0f;
    if (ND == 10) {
      const float ul = std::nextafter(std::fabs(hi), INFINITY) - std::fabs(hi);
      lo = u(g) * ul * 0.5f;
    }
    one(hi, lo);
  }
  // the packed conversion: the first element in the low byte
  for (int a = -16; a <= 16; ++a)
    for (int b = -16; b <= 16; ++b) {
      const __nv_fp8x2_storage_t p = __nv_cvt_float2_to_fp8x2(float2{(float)a, (float)b}, __NV_SATFINITE, __NV_E4M3);
      const unsigned lo8 = __nv_cvt_float_to_fp8((float)a, __NV_SATFINITE, __NV_E4M3);
      const unsigned hi8 = __nv_cvt_float_to_fp8((float)b, __NV_SATFINITE, __NV_E4M3);
      if (p != (__nv_fp8x2_storage_t)(lo8 | (hi8 << 8))) ++bad;
    }
  return bad;
}

int main() {
  int bad = 0;
  for (int s = -16; s <= 16; ++s) {
    const __nv_fp8_storage_t b = __nv_cvt_float_to_fp8((float)s, __NV_SATFINITE, __NV_E4M3);
    const __half_raw h = __nv_cvt_fp8_to_halfraw(b, __NV_E4M3);
    if (__half2float(__half(h)) != (float)s) ++bad;
  }
  const int b10 = check<10>(1LL << 49, 2000000, 1LL << 52);
  const int b6 = check<6>(1LL << 29, 2000000, 1LL << 31);
  const int f10 = check_f<10>(2000000);
  const int f6 = check_f<6>(2000000);
  std::printf("e4m3 %d, ten digits %d, six digits %d, 32-bit cut %d / %d\n", bad, b10, b6, f10, f6);
  return bad + b10 + b6 + f10 + f6 != 0;
}
