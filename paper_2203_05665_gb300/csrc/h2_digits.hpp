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

}  // namespace h2
