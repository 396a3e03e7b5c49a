// Transfer steps of the H^2 product (Algorithms 1 and 2) with the factored
// transfer matrices E = Ex (x) Ey (x) Ez of tensor Chebyshev interpolation
// (Eq. (9)): three m x m mode products per child instead of one k x k
// product.  Shared by the single-matrix and the batched products.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "h2_dd.cuh"

namespace h2 {
namespace {

// One mode product of the factored transfer on a [k][rp] coefficient tensor
// (nu = jx + m jy + m^2 jz): every thread owns one fibre along axis d for one
// column, reads its m entries once and writes m results.
//   trans: out[.., j, ..] = sum_{j'} F[j'][j] in[.., j', ..]   (E^T, upward)
//   plain: out[.., j', ..] = sum_{j} F[j'][j] in[.., j, ..]    (E, downward)
constexpr int kMaxM = 5;

template <class T>
__device__ __forceinline__ void mode_fibres(const T *F, const T *in, T *out, int m, int k, int rp, int d, bool trans,
                                            int tid, int nthr) {
  const int stride = d == 0 ? 1 : (d == 1 ? m : m * m);
  const int items = (k / m) * rp;
  for (int it = tid; it < items; it += nthr) {
    const int c = it % rp, f = it / rp;
    const int lo = f % stride, hi = f / stride;
    const int base = lo + hi * stride * m;
    T v[kMaxM];
#pragma unroll
    for (int i = 0; i < kMaxM; ++i)
      if (i < m) v[i] = in[(base + i * stride) * rp + c];
#pragma unroll
    for (int j = 0; j < kMaxM; ++j) {
      if (j >= m) break;
      // double-float: the low word collects the exact errors of the m terms,
      // one renormalisation per output
      T acc = zero_of<T>();
#pragma unroll
      for (int i = 0; i < kMaxM; ++i)
        if (i < m) acc_fma(acc, trans ? F[i * m + j] : F[j * m + i], v[i]);
      acc_norm(acc);
      out[(base + j * stride) * rp + c] = acc;
    }
  }
}

// storage -> compute conversion of a transfer factor
template <class TC, class TS>
__device__ __forceinline__ TC to_compute(TS v) {
  return convert<TC, TS>(v);
}
template <>
__device__ __forceinline__ float to_compute<float, __nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <>
__device__ __forceinline__ float to_compute<float, __half>(__half v) {
  return __half2float(v);
}

// upward step for one parent (Algorithm 1): x^_p = sum over both children c of E_c^T x^_c;
// smem holds 3 k rp + 6 m^2 values of T
template <class TS, class T>
__device__ __forceinline__ void upward_parent(const TS *__restrict__ Ef, int m, int k, int rp, int64_t par,
                                              T *__restrict__ xhat, unsigned char *smem_raw) {
  const int kr = k * rp, mm = m * m;
  T *a = reinterpret_cast<T *>(smem_raw);
  T *b = a + kr;
  T *acc = b + kr;
  T *F = acc + kr;   // 2 children x 3 axes x m x m
  for (int i = threadIdx.x; i < 6 * mm; i += blockDim.x) F[i] = to_compute<T>(Ef[(2 * par + 1) * 3 * mm + i]);
  for (int i = threadIdx.x; i < kr; i += blockDim.x) acc[i] = zero_of<T>();
  for (int ch = 0; ch < 2; ++ch) {
    const int64_t c = 2 * par + 1 + ch;
    for (int i = threadIdx.x; i < kr; i += blockDim.x) a[i] = xhat[c * kr + i];
    __syncthreads();
    const T *Fc = F + ch * 3 * mm;
    mode_fibres(Fc, a, b, m, k, rp, 0, true, threadIdx.x, blockDim.x);
    __syncthreads();
    mode_fibres(Fc + mm, b, a, m, k, rp, 1, true, threadIdx.x, blockDim.x);
    __syncthreads();
    mode_fibres(Fc + 2 * mm, a, b, m, k, rp, 2, true, threadIdx.x, blockDim.x);
    __syncthreads();
    for (int i = threadIdx.x; i < kr; i += blockDim.x) acc[i] = acc[i] + b[i];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kr; i += blockDim.x) xhat[par * kr + i] = acc[i];
}

// downward step below one parent (Algorithm 2): y^_c += E_c y^_parent for both children
template <class TS, class T>
__device__ __forceinline__ void downward_parent(const TS *__restrict__ Ef, int m, int k, int rp, int64_t par,
                                                T *__restrict__ yhat, unsigned char *smem_raw) {
  const int kr = k * rp, mm = m * m;
  T *p = reinterpret_cast<T *>(smem_raw);
  T *a = p + kr;
  T *b = a + kr;
  T *F = b + kr;
  for (int i = threadIdx.x; i < 6 * mm; i += blockDim.x) F[i] = to_compute<T>(Ef[(2 * par + 1) * 3 * mm + i]);
  for (int i = threadIdx.x; i < kr; i += blockDim.x) p[i] = yhat[par * kr + i];
  __syncthreads();
  for (int ch = 0; ch < 2; ++ch) {
    const int64_t c = 2 * par + 1 + ch;
    const T *Fc = F + ch * 3 * mm;
    mode_fibres(Fc, p, a, m, k, rp, 0, false, threadIdx.x, blockDim.x);
    __syncthreads();
    mode_fibres(Fc + mm, a, b, m, k, rp, 1, false, threadIdx.x, blockDim.x);
    __syncthreads();
    mode_fibres(Fc + 2 * mm, b, a, m, k, rp, 2, false, threadIdx.x, blockDim.x);
    __syncthreads();
    for (int i = threadIdx.x; i < kr; i += blockDim.x) yhat[c * kr + i] = yhat[c * kr + i] + a[i];
    __syncthreads();
  }
}

// Warp-level variants: one warp per parent, the warp's own shared memory
// (3 k rp + 6 m^2 values of T), warp synchronisation only.  For the small
// per-parent tensors of low orders and few right-hand sides a whole CTA per
// parent leaves most threads idle.
template <class TS, class T>
__device__ __forceinline__ void upward_parent_warp(const TS *__restrict__ Ef, int m, int k, int rp, int64_t par,
                                                   T *__restrict__ xhat, T *ws, int lane) {
  const int kr = k * rp, mm = m * m;
  T *a = ws;
  T *b = a + kr;
  T *acc = b + kr;
  T *F = acc + kr;
  for (int i = lane; i < 6 * mm; i += 32) F[i] = to_compute<T>(Ef[(2 * par + 1) * 3 * mm + i]);
  for (int ch = 0; ch < 2; ++ch) {
    const int64_t c = 2 * par + 1 + ch;
    for (int i = lane; i < kr; i += 32) a[i] = xhat[c * kr + i];
    __syncwarp();
    const T *Fc = F + ch * 3 * mm;
    mode_fibres(Fc, a, b, m, k, rp, 0, true, lane, 32);
    __syncwarp();
    mode_fibres(Fc + mm, b, a, m, k, rp, 1, true, lane, 32);
    __syncwarp();
    mode_fibres(Fc + 2 * mm, a, b, m, k, rp, 2, true, lane, 32);
    __syncwarp();
    for (int i = lane; i < kr; i += 32) acc[i] = ch == 0 ? b[i] : acc[i] + b[i];
    __syncwarp();
  }
  for (int i = lane; i < kr; i += 32) xhat[par * kr + i] = acc[i];
  __syncwarp();
}

template <class TS, class T>
__device__ __forceinline__ void downward_parent_warp(const TS *__restrict__ Ef, int m, int k, int rp, int64_t par,
                                                     T *__restrict__ yhat, T *ws, int lane) {
  const int kr = k * rp, mm = m * m;
  T *p = ws;
  T *a = p + kr;
  T *b = a + kr;
  T *F = b + kr;
  for (int i = lane; i < 6 * mm; i += 32) F[i] = to_compute<T>(Ef[(2 * par + 1) * 3 * mm + i]);
  for (int i = lane; i < kr; i += 32) p[i] = yhat[par * kr + i];
  __syncwarp();
  for (int ch = 0; ch < 2; ++ch) {
    const int64_t c = 2 * par + 1 + ch;
    const T *Fc = F + ch * 3 * mm;
    mode_fibres(Fc, p, a, m, k, rp, 0, false, lane, 32);
    __syncwarp();
    mode_fibres(Fc + mm, a, b, m, k, rp, 1, false, lane, 32);
    __syncwarp();
    mode_fibres(Fc + 2 * mm, b, a, m, k, rp, 2, false, lane, 32);
    __syncwarp();
    for (int i = lane; i < kr; i += 32) yhat[c * kr + i] = yhat[c * kr + i] + a[i];
    __syncwarp();
  }
}

}  // namespace
}  // namespace h2
