// Signed 5-bit digits of the fixed-point integers of the tensor-core
// phases (h2_tc.cu), host and device: X = sum_i s_i 2^(5 (ND - 1 - i)),
// |s_i| <= 16, so that every digit is an exact FP8 E4M3 value.  A header of
// its own so that the decomposition can be checked on the host.
#pragma once

#ifndef __CUDACC__
#ifndef __host__
#define __host__
#endif
#ifndef __device__
#define __device__
#endif
#ifndef __forceinline__
#define __forceinline__ inline
#endif
#endif

#include <cstdint>
#ifndef __CUDA_ARCH__
#include <cmath>
#include <cstring>
#endif

namespace h2 {

// split X (|X| <= 2^49) into ten signed 5-bit digits, most significant
// first: X = sum_i s_i 2^(45 - 5i), |s_i| <= 16.  X = A 2^25 + B with B in
// [-2^24, 2^24) gives two 32-bit halves; digits are taken from the low end,
// d = ((v + 16) mod 32) - 16 in [-16, 15] and v = (v - d) / 32 exactly, B's
// remainder (0 or 1) carries into A, and A's remainder after four digits is
// the top digit, within [-16, 16] because |A| <= 2^24 + 2.
// The same for six digits of |X| <= 2^29 (one 32-bit value; the top digit
// stays within [-16, 16] by the same bound).
template <int ND>
__host__ __device__ __forceinline__ void split_digits(long long X, int (&s)[ND]) {
  static_assert(ND == 10 || ND == 6, "digit counts");
  if (ND == 10) {
    int b = (int)(((X + (1LL << 24)) & ((1LL << 25) - 1)) - (1LL << 24));
    int a = (int)((X - b) >> 25);
#pragma unroll
    for (int i = ND - 1; i >= ND / 2; --i) {
      const int d = ((b + 16) & 31) - 16;
      s[i] = d;
      b = (b - d) >> 5;
    }
    a += b;
#pragma unroll
    for (int i = ND / 2 - 1; i >= 1; --i) {
      const int d = ((a + 16) & 31) - 16;
      s[i] = d;
      a = (a - d) >> 5;
    }
    s[0] = a;
  } else {
    int a = (int)X;
#pragma unroll
    for (int i = ND - 1; i >= 1; --i) {
      const int d = ((a + 16) & 31) - 16;
      s[i] = d;
      a = (a - d) >> 5;
    }
    s[0] = a;
  }
}

// The same digits, as exact FP32 values, of X = rint(hs) + rint(ls) (hs, ls
// the two words of a double-float value, or an FP32 value and 0, already
// scaled by 2^sc: power-of-two products, exact), formed with 32-bit
// operations only.  For ten digits: H = rint(hs) is an integer-valued float,
// A = rint(H 2^-25) and B = H - A 2^25 (|B| <= 2^24, an exact float
// difference) split it, and L = rint(ls) fits in 32 bits, so X = A 2^25 + bt
// with bt = B + L, whose low 25 bits are those of X: the halves (a, b) of
// split_digits follow from (A, bt) with 32-bit integer arithmetic.  A digit
// d = (w & 31) - 16 (w = v + 16) becomes a float by placing w & 31 in the
// significand of 2^23 and subtracting 2^23 + 16; the next v is w >> 5.
__host__ __device__ __forceinline__ float bits_float(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}

__host__ __device__ __forceinline__ float digit_f(int &v) {
  const int w = v + 16;
  v = w >> 5;
  return bits_float(0x4B000000u | (uint32_t)(w & 31)) - 8388624.0f;
}

template <int ND>
__host__ __device__ __forceinline__ void split_digits_f(float hs, float ls, float (&f)[ND]) {
  static_assert(ND == 10 || ND == 6, "digit counts");
  if (ND == 10) {
    const float H = rintf(hs);
    const float A = rintf(H * 0x1p-25f);
    const float B = fmaf(-A, 0x1p25f, H);
    const int bt = (int)B + (int)rintf(ls);
    int b = ((bt + (1 << 24)) & ((1 << 25) - 1)) - (1 << 24);
    int a = (int)A + ((bt - b) >> 25);
#pragma unroll
    for (int i = ND - 1; i >= ND / 2; --i) f[i] = digit_f(b);
    a += b;
#pragma unroll
    for (int i = ND / 2 - 1; i >= 1; --i) f[i] = digit_f(a);
    f[0] = (float)a;
  } else {
    int a = (int)rintf(hs) + (int)rintf(ls);
#pragma unroll
    for (int i = ND - 1; i >= 1; --i) f[i] = digit_f(a);
    f[0] = (float)a;
  }
}

}  // namespace h2
