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


// ---------------------------------------------------------------------------
// Register transfer kernels for m = 3 and m = 4 (k = m^3): 64 threads per
// parent and 16 columns (grid.y runs over groups of 16 columns), thread
// (j, jz) = (column, z index; jz < m, the fourth lane of a column idles for
// m = 3) holds the m x m slab nu = jx + m jy + m^2 jz of one column in
// registers.  The x and y mode products run in registers, the z mode product
// takes the slab entries of the threads of the column (adjacent lanes) by
// warp shuffles.  Every output is formed exactly as in mode_fibres (m
// multiply-adds, one renormalisation), in the same axis order, so the
// results equal those of the shared-memory kernels above; the gain is that
// no CTA-wide barrier separates the three mode products.
constexpr int kRegParents = 4;   // parents per 256-thread CTA

__device__ __forceinline__ float shfl_t(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double shfl_t(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ dd shfl_t(dd v, int src) {
  return dd{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

// out[a] = sum_b F[a][b] in[b] (plain, E) or sum_b F[b][a] in[b] (trans, E^T)
template <class T, bool TRANS, int M>
__device__ __forceinline__ T modem_out(const T *F, const T (&in)[M], int a) {
  T acc = zero_of<T>();
#pragma unroll
  for (int b = 0; b < M; ++b) acc_fma(acc, TRANS ? F[b * M + a] : F[a * M + b], in[b]);
  acc_norm(acc);
  return acc;
}

// the transfer factors of the children of this CTA's parents: F[q][ch][axis][M x M]
template <class TS, class T, int M, int P = kRegParents>
__device__ __forceinline__ void load_factors(const TS *__restrict__ Ef, int64_t par0, int64_t npar,
                                             T (*F)[2][3][M * M]) {
  constexpr int kPer = 6 * M * M, kChild = 3 * M * M;
  for (int i = threadIdx.x; i < P * kPer; i += blockDim.x) {
    const int q = i / kPer, o = i % kPer;
    const int64_t pi = (int64_t)blockIdx.x * P + q;
    const int64_t pp = par0 + pi;
    F[q][o / kChild][(o % kChild) / (M * M)][o % (M * M)] =
        pi < npar ? to_compute<T>(Ef[(2 * pp + 1) * kChild + o]) : zero_of<T>();
  }
  __syncthreads();
}

// Upward (Algorithm 1): x^_parent = sum over both children of E_c^T x^_c.
// With xmax, also the largest |x^_parent| (|hi| for double-float) of every
// column over the launch, as float bits (atomicMax).
__device__ __forceinline__ float mag_of(float v) { return fabsf(v); }
__device__ __forceinline__ float mag_of(double v) { return (float)fabs(v); }
__device__ __forceinline__ float mag_of(dd v) { return fabsf(v.hi); }

template <class TS, class T, int M>
__global__ void __launch_bounds__(256, 2) k_up_reg(const TS *__restrict__ Ef, int rp, int64_t par0, int64_t npar,
                                                   T *__restrict__ xhat, unsigned *__restrict__ xmax) {
  constexpr int K = M * M * M;
  __shared__ T F[kRegParents][2][3][M * M];
  __shared__ unsigned loc[16];
  if (threadIdx.x < 16) loc[threadIdx.x] = 0u;
  load_factors<TS, T, M>(Ef, par0, npar, F);
  const int pl = threadIdx.x >> 6, t = threadIdx.x & 63, j = (t >> 2) + 16 * blockIdx.y, jz = t & 3;
  const int64_t pi = (int64_t)blockIdx.x * kRegParents + pl, par = par0 + pi;
  const bool act = pi < npar && j < rp && jz < M;
  const int base = (threadIdx.x & 31) & ~3;
  const int zq = jz < M ? jz : 0;
  T out[M][M];
#pragma unroll 1
  for (int ch = 0; ch < 2; ++ch) {
    const int64_t c = 2 * par + 1 + ch;
    const T *Fx = F[pl][ch][0], *Fy = F[pl][ch][1], *Fz = F[pl][ch][2];
    T v[M][M], a[M][M], b[M][M];
#pragma unroll
    for (int jy = 0; jy < M; ++jy)
#pragma unroll
      for (int jx = 0; jx < M; ++jx)
        v[jy][jx] = act ? xhat[(c * K + jx + M * jy + M * M * jz) * rp + j] : zero_of<T>();
#pragma unroll
    for (int jy = 0; jy < M; ++jy)
#pragma unroll
      for (int jx = 0; jx < M; ++jx) a[jy][jx] = modem_out<T, true, M>(Fx, v[jy], jx);
#pragma unroll
    for (int jx = 0; jx < M; ++jx) {
      T col[M];
#pragma unroll
      for (int jy = 0; jy < M; ++jy) col[jy] = a[jy][jx];
#pragma unroll
      for (int jy = 0; jy < M; ++jy) b[jy][jx] = modem_out<T, true, M>(Fy, col, jy);
    }
#pragma unroll
    for (int jy = 0; jy < M; ++jy)
#pragma unroll
      for (int jx = 0; jx < M; ++jx) {
        T in[M];
#pragma unroll
        for (int q = 0; q < M; ++q) in[q] = shfl_t(b[jy][jx], base + q);
        const T r = modem_out<T, true, M>(Fz, in, zq);
        out[jy][jx] = ch == 0 ? zero_of<T>() + r : out[jy][jx] + r;
      }
  }
  float mx = 0.0f;
#pragma unroll
  for (int jy = 0; jy < M; ++jy)
#pragma unroll
    for (int jx = 0; jx < M; ++jx) {
      if (act) xhat[(par * K + jx + M * jy + M * M * jz) * rp + j] = out[jy][jx];
      if (act) mx = fmaxf(mx, mag_of(out[jy][jx]));
    }
  if (xmax) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
    if (act && jz == 0 && mx > 0.0f) atomicMax(&loc[j & 15], __float_as_uint(mx));
    __syncthreads();
    if (threadIdx.x < 16 && loc[threadIdx.x]) atomicMax(&xmax[threadIdx.x], loc[threadIdx.x]);
  }
}

// Child-split variants: 128 threads per parent, the two 64-thread halves
// taking one child each (two parents per 256-thread CTA), so every thread
// forms half the mode products.  On levels with few parents a CTA's time is
// the latency of one thread's chain of double-float operations, which this
// halves.  The upward step adds the second child's part to the first through
// shared memory in the order of k_up_reg (same bits).
//
// Downward (Algorithm 2): y^_c += E_c y^_parent for both children of parents
// par0 .. par0 + npar - 1, the children independent.
constexpr int kSplitParents = 2;   // parents per 256-thread CTA
// upward levels of at most this many parents take the split kernel (the
// downward pass takes it at every level; both measured at level 7, 16 RHS)
constexpr int64_t kUpSplitMax = 4096;

template <class TS, class T, int M>
__global__ void __launch_bounds__(256, 2) k_down_split(const TS *__restrict__ Ef, int rp, int64_t par0, int64_t npar,
                                                       T *__restrict__ yhat) {
  constexpr int K = M * M * M;
  __shared__ T F[kSplitParents][2][3][M * M];
  load_factors<TS, T, M, kSplitParents>(Ef, par0, npar, F);
  const int pl = threadIdx.x >> 7, ch = (threadIdx.x >> 6) & 1, t = threadIdx.x & 63;
  const int j = (t >> 2) + 16 * blockIdx.y, jz = t & 3;
  const int64_t pi = (int64_t)blockIdx.x * kSplitParents + pl, par = par0 + pi;
  const bool act = pi < npar && j < rp && jz < M;
  const int base = (threadIdx.x & 31) & ~3;
  const int zq = jz < M ? jz : 0;
  const T *Fx = F[pl][ch][0], *Fy = F[pl][ch][1], *Fz = F[pl][ch][2];
  const int64_t c = 2 * par + 1 + ch;
  T v[M][M], yc[M][M];
#pragma unroll
  for (int jy = 0; jy < M; ++jy)
#pragma unroll
    for (int jx = 0; jx < M; ++jx) {
      const int64_t nu = jx + M * jy + M * M * jz;
      v[jy][jx] = act ? yhat[(par * K + nu) * rp + j] : zero_of<T>();
      yc[jy][jx] = act ? yhat[(c * K + nu) * rp + j] : zero_of<T>();
    }
  T a[M][M], b[M][M];
#pragma unroll
  for (int jy = 0; jy < M; ++jy)
#pragma unroll
    for (int jx = 0; jx < M; ++jx) a[jy][jx] = modem_out<T, false, M>(Fx, v[jy], jx);
#pragma unroll
  for (int jx = 0; jx < M; ++jx) {
    T col[M];
#pragma unroll
    for (int jy = 0; jy < M; ++jy) col[jy] = a[jy][jx];
#pragma unroll
    for (int jy = 0; jy < M; ++jy) b[jy][jx] = modem_out<T, false, M>(Fy, col, jy);
  }
#pragma unroll
  for (int jy = 0; jy < M; ++jy)
#pragma unroll
    for (int jx = 0; jx < M; ++jx) {
      T in[M];
#pragma unroll
      for (int q = 0; q < M; ++q) in[q] = shfl_t(b[jy][jx], base + q);
      const T r = modem_out<T, false, M>(Fz, in, zq);
      if (act) yhat[(c * K + jx + M * jy + M * M * jz) * rp + j] = yc[jy][jx] + r;
    }
}

template <class TS, class T, int M>
__global__ void __launch_bounds__(256, 2) k_up_split(const TS *__restrict__ Ef, int rp, int64_t par0, int64_t npar,
                                                     T *__restrict__ xhat, unsigned *__restrict__ xmax) {
  constexpr int K = M * M * M;
  __shared__ T F[kSplitParents][2][3][M * M];
  __shared__ T R[kSplitParents][M * M][64];   // the second child's part
  __shared__ unsigned loc[16];
  if (threadIdx.x < 16) loc[threadIdx.x] = 0u;
  load_factors<TS, T, M, kSplitParents>(Ef, par0, npar, F);
  const int pl = threadIdx.x >> 7, ch = (threadIdx.x >> 6) & 1, t = threadIdx.x & 63;
  const int j = (t >> 2) + 16 * blockIdx.y, jz = t & 3;
  const int64_t pi = (int64_t)blockIdx.x * kSplitParents + pl, par = par0 + pi;
  const bool act = pi < npar && j < rp && jz < M;
  const int base = (threadIdx.x & 31) & ~3;
  const int zq = jz < M ? jz : 0;
  const int64_t c = 2 * par + 1 + ch;
  const T *Fx = F[pl][ch][0], *Fy = F[pl][ch][1], *Fz = F[pl][ch][2];
  T v[M][M], a[M][M], b[M][M];
#pragma unroll
  for (int jy = 0; jy < M; ++jy)
#pragma unroll
    for (int jx = 0; jx < M; ++jx)
      v[jy][jx] = act ? xhat[(c * K + jx + M * jy + M * M * jz) * rp + j] : zero_of<T>();
#pragma unroll
  for (int jy = 0; jy < M; ++jy)
#pragma unroll
    for (int jx = 0; jx < M; ++jx) a[jy][jx] = modem_out<T, true, M>(Fx, v[jy], jx);
#pragma unroll
  for (int jx = 0; jx < M; ++jx) {
    T col[M];
#pragma unroll
    for (int jy = 0; jy < M; ++jy) col[jy] = a[jy][jx];
#pragma unroll
    for (int jy = 0; jy < M; ++jy) b[jy][jx] = modem_out<T, true, M>(Fy, col, jy);
  }
  // the z mode product into a (the slab is free again)
#pragma unroll
  for (int jy = 0; jy < M; ++jy)
#pragma unroll
    for (int jx = 0; jx < M; ++jx) {
      T in[M];
#pragma unroll
      for (int q = 0; q < M; ++q) in[q] = shfl_t(b[jy][jx], base + q);
      a[jy][jx] = modem_out<T, true, M>(Fz, in, zq);
    }
  if (ch == 1)
#pragma unroll
    for (int jy = 0; jy < M; ++jy)
#pragma unroll
      for (int jx = 0; jx < M; ++jx) R[pl][jx + M * jy][t] = a[jy][jx];
  __syncthreads();
  float mx = 0.0f;
  if (ch == 0)
#pragma unroll
    for (int jy = 0; jy < M; ++jy)
#pragma unroll
      for (int jx = 0; jx < M; ++jx) {
        const T o = (zero_of<T>() + a[jy][jx]) + R[pl][jx + M * jy][t];
        if (act) xhat[(par * K + jx + M * jy + M * M * jz) * rp + j] = o;
        if (act) mx = fmaxf(mx, mag_of(o));
      }
  if (xmax) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
    if (ch == 0 && act && jz == 0 && mx > 0.0f) atomicMax(&loc[j & 15], __float_as_uint(mx));
    __syncthreads();
    if (threadIdx.x < 16 && loc[threadIdx.x]) atomicMax(&xmax[threadIdx.x], loc[threadIdx.x]);
  }
}

}  // namespace
}  // namespace h2
