// The H^2 matrix-vector product y = G~ x on the device (Boerm, Section 2,
// Algorithms 1-3), level-synchronous:
//   permute in      x (caller order, column-major) -> xpad (leaf-padded, RHS-contiguous)
//   leaf forward    x^_s = V_s^T x|s for every leaf               (Algorithm 1, leaves)
//   upward          x^_s = sum_{s'} E_{s'}^T x^_{s'}, level by level   (Algorithm 1)
//   coupling        y^_t = sum_{(t,s) admissible} S_ts x^_s        (Algorithm 3)
//   downward        y^_{t'} += E_{t'} y^_t, level by level         (Algorithm 2)
//   leaf + near     y|t = V_t y^_t + sum_{(t,s) inadmissible} G|ts x|s   (Algorithms 2, 3)
//   permute out     ypad -> y (caller order)
// Transfer matrices are applied in factored form E = Ex (x) Ey (x) Ez
// (Eq. (9) with tensor Chebyshev points): three m x m mode products.
// Coefficient layout: x^[cluster][nu][rhs], nu = jx + m jy + m^2 jz.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "h2_dd.cuh"
#include "h2_internal.hpp"
#include "h2_ptx.cuh"
#include "h2_transfer.cuh"

namespace h2 {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxOut = 16;   // outputs per thread in the block-row kernels

// Range guard of the double-float arithmetic (H2_F64 handles): a double-float
// value has the exponent range of FP32, so a column of x whose largest entry
// lies outside [2^-40, 2^40] is multiplied by the power of two that brings
// that entry to [1, 2) on the way in and divided by it on the way out (exact;
// columns inside the range are not touched).  colmax[c] holds the bits of
// max |x[:, c]| as a double (non-negative doubles order like their bits).
template <class Tin>
__global__ void k_colmax(const Tin *__restrict__ x, int64_t n, unsigned long long *__restrict__ colmax) {
  __shared__ double wmax[32];
  const Tin *xc = x + (int64_t)blockIdx.y * n;
  // four independent maxima per thread keep several loads in flight
  double m4[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride)
#pragma unroll
    for (int u = 0; u < 4; ++u) m4[u] = fmax(m4[u], fabs((double)xc[i + u * stride]));
  for (; i < n; i += stride) m4[0] = fmax(m4[0], fabs((double)xc[i]));
  double mx = fmax(fmax(m4[0], m4[1]), fmax(m4[2], m4[3]));
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, wmax[w]);
    if (mx > 0.0) atomicMax(&colmax[blockIdx.y], (unsigned long long)__double_as_longlong(mx));
  }
}

// 2^e as a double for -1022 <= e <= 1023
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }
// v 2^e, exact unless the result leaves the normal range: two factors that
// are normal doubles for |e| <= 2044
__device__ __forceinline__ double scale_pow2(double v, int e) {
  const int h = e / 2;
  return v * pow2d(h) * pow2d(e - h);
}

// the power of two by which column c is scaled (0: untouched; zero, infinite
// and NaN columns are not scaled)
__host__ __device__ inline int range_shift(unsigned long long bits) {
  const int ex = (int)((bits >> 52) & 0x7ff);
  if (bits == 0 || ex == 0x7ff) return 0;
  const int e = ex == 0 ? -1022 : ex - 1023;
  return (e < -40 || e > 40) ? -e : 0;
}

// Permutations between the caller's order (column-major n x nrhs) and the
// leaf-padded cluster order (xpad[p][c], rp columns): a CTA takes a tile of
// kPermRows padded DoFs and stages it in shared memory, so that the caller's
// side is walked column by column (neighbouring DoFs of a cluster are
// neighbouring triangles of the mesh, so the gathered addresses are close)
// and the padded side row by row (contiguous).  Rows of the tile are padded
// by one value against bank conflicts.
constexpr int kPermRows = 64;

// xpad[p][c] (zero beyond nrhs and for padding rows) from x[src][c], scaled by
// the column's range-guard power of two; with xmax also the largest |xpad|
// (|hi| for double-float) of every column, as float bits (atomicMax), the
// maxima the nearfield's input digits are cut with
template <class Tin, class Tout>
__global__ void __launch_bounds__(256) k_permute_in(const Tin *__restrict__ x, int64_t n, int nrhs, int rp,
                                                    const int32_t *__restrict__ pad_src, int64_t npad,
                                                    const unsigned long long *__restrict__ colmax,
                                                    Tout *__restrict__ xpad, unsigned *__restrict__ xmax = nullptr) {
  extern __shared__ __align__(16) unsigned char perm_smem[];
  Tout *tile = reinterpret_cast<Tout *>(perm_smem);
  __shared__ int shift[64];
  __shared__ unsigned smax[64];
  __shared__ int32_t src[kPermRows];
  if (threadIdx.x < 64) smax[threadIdx.x] = 0u;
  const int w = rp + 1;
  const int64_t p0 = (int64_t)blockIdx.x * kPermRows;
  if (threadIdx.x < kPermRows) src[threadIdx.x] = p0 + threadIdx.x < npad ? pad_src[p0 + threadIdx.x] : -1;
  if (threadIdx.x < 64) shift[threadIdx.x] = (colmax && (int)threadIdx.x < nrhs) ? range_shift(colmax[threadIdx.x]) : 0;
  __syncthreads();
  // the gathered loads of four passes are issued before any of them is used
  for (int i0 = 0; i0 < kPermRows * rp; i0 += 4 * (int)blockDim.x) {
    Tin u[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = i0 + a * (int)blockDim.x + (int)threadIdx.x;
      const int c = i / kPermRows, q = i - c * kPermRows;
      const int32_t sp = i < kPermRows * rp ? src[q] : -1;
      u[a] = (sp >= 0 && c < nrhs) ? x[sp + (int64_t)c * n] : (Tin)0;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = i0 + a * (int)blockDim.x + (int)threadIdx.x;
      if (i >= kPermRows * rp) break;
      const int c = i / kPermRows, q = i - c * kPermRows;
      Tin v = u[a];
      if (c < nrhs && shift[c]) v = (Tin)scale_pow2((double)v, shift[c]);
      tile[q * w + c] = (src[q] >= 0 && c < nrhs) ? convert<Tout, Tin>(v) : zero_of<Tout>();
    }
  }
  __syncthreads();
  const int64_t rows = npad - p0 < kPermRows ? npad - p0 : kPermRows;
  for (int i = threadIdx.x; i < rows * rp; i += blockDim.x) {
    const int q = i / rp, c = i - q * rp;
    const Tout v = tile[q * w + c];
    xpad[(p0 + q) * rp + c] = v;
    if (xmax) {
      const float m = mag_of(v);
      if (m > 0.0f) atomicMax(&smax[c], __float_as_uint(m));
    }
  }
  if (xmax) {
    __syncthreads();
    if ((int)threadIdx.x < rp && smax[threadIdx.x]) atomicMax(&xmax[threadIdx.x], smax[threadIdx.x]);
  }
}

// y[src][c] (caller order) from ypad[p][c], divided by the column's range-guard
// power of two; with acc the value is added to what y holds (y <- y + G~ x)
template <class Tin, class Tout>
__global__ void __launch_bounds__(256) k_permute_out(const Tin *__restrict__ ypad, int64_t n, int nrhs, int rp,
                                                     const int32_t *__restrict__ pad_src, int64_t npad,
                                                     const unsigned long long *__restrict__ colmax, int acc,
                                                     Tout *__restrict__ y) {
  extern __shared__ __align__(16) unsigned char perm_smem[];
  Tin *tile = reinterpret_cast<Tin *>(perm_smem);
  __shared__ int shift[64];
  __shared__ int32_t src[kPermRows];
  const int w = rp + 1;
  const int64_t p0 = (int64_t)blockIdx.x * kPermRows;
  if (threadIdx.x < kPermRows) src[threadIdx.x] = p0 + threadIdx.x < npad ? pad_src[p0 + threadIdx.x] : -1;
  if (threadIdx.x < 64) shift[threadIdx.x] = (colmax && (int)threadIdx.x < nrhs) ? range_shift(colmax[threadIdx.x]) : 0;
  const int64_t rows = npad - p0 < kPermRows ? npad - p0 : kPermRows;
  for (int i = threadIdx.x; i < rows * rp; i += blockDim.x) {
    const int q = i / rp, c = i - q * rp;
    tile[q * w + c] = ypad[(p0 + q) * rp + c];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kPermRows * nrhs; i += blockDim.x) {
    const int c = i / kPermRows, q = i - c * kPermRows;
    const int32_t sp = src[q];
    if (sp < 0) continue;
    Tout v = convert<Tout, Tin>(tile[q * w + c]);
    if (shift[c]) v = (Tout)scale_pow2((double)v, -shift[c]);
    Tout *dst = y + sp + (int64_t)c * n;
    *dst = acc ? *dst + v : v;
  }
}

// upward step for the parents of level l (Algorithm 1), one CTA per parent
template <class TS, class T>
__global__ void k_upward(const TS *__restrict__ Ef, int m, int k, int rp, int64_t par0, T *__restrict__ xhat) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  upward_parent<TS, T>(Ef, m, k, rp, par0 + blockIdx.x, xhat, smem_raw);
}

// downward step for the children of level l+1 (Algorithm 2), one CTA per parent of level l
template <class TS, class T>
__global__ void k_downward(const TS *__restrict__ Ef, int m, int k, int rp, int64_t par0, T *__restrict__ yhat) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  downward_parent<TS, T>(Ef, m, k, rp, par0 + blockIdx.x, yhat, smem_raw);
}

template <class T>
struct Vec16;
template <>
struct Vec16<float> {
  using V = float4;
  static constexpr int N = 4;
};
template <>
struct Vec16<double> {
  using V = double2;
  static constexpr int N = 2;
};
template <>
struct Vec16<dd> {
  using V = float4;
  static constexpr int N = 2;
};

// the value of lane q (< N) of a 16-byte vector
template <class T>
__device__ __forceinline__ T lane(const typename Vec16<T>::V &v, int q);
template <>
__device__ __forceinline__ float lane<float>(const float4 &v, int q) {
  return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}
template <>
__device__ __forceinline__ double lane<double>(const double2 &v, int q) {
  return q == 0 ? v.x : v.y;
}
template <>
__device__ __forceinline__ dd lane<dd>(const float4 &v, int q) {
  return q == 0 ? dd{v.x, v.y} : dd{v.z, v.w};
}

// four consecutive stored values (aligned to four elements) as compute values
template <class TS, class TC>
__device__ __forceinline__ void load4(const TS *p, TC *out);
template <>
__device__ __forceinline__ void load4<float, float>(const float *p, float *out) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}
template <>
__device__ __forceinline__ void load4<double, double>(const double *p, double *out) {
  const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
  out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}
template <>
__device__ __forceinline__ void load4<dd, dd>(const dd *p, dd *out) {
  const float4 a = reinterpret_cast<const float4 *>(p)[0], b = reinterpret_cast<const float4 *>(p)[1];
  out[0] = dd{a.x, a.y}; out[1] = dd{a.z, a.w}; out[2] = dd{b.x, b.y}; out[3] = dd{b.z, b.w};
}
template <>
__device__ __forceinline__ void load4<__nv_bfloat16, float>(const __nv_bfloat16 *p, float *out) {
  const uint2 v = *reinterpret_cast<const uint2 *>(p);
  out[0] = __uint_as_float(v.x << 16); out[1] = __uint_as_float(v.x & 0xffff0000u);
  out[2] = __uint_as_float(v.y << 16); out[3] = __uint_as_float(v.y & 0xffff0000u);
}
template <>
__device__ __forceinline__ void load4<__half, float>(const __half *p, float *out) {
  const uint2 v = *reinterpret_cast<const uint2 *>(p);
  const __half2 a = *reinterpret_cast<const __half2 *>(&v.x), b = *reinterpret_cast<const __half2 *>(&v.y);
  const float2 fa = __half22float2(a), fb = __half22float2(b);
  out[0] = fa.x; out[1] = fa.y; out[2] = fb.x; out[3] = fb.y;
}

// scale of a term (per-block power of two of FP16 storage); only FP32 compute is scaled
__device__ __forceinline__ void scale_by(float &v, float s) { v *= s; }
__device__ __forceinline__ void scale_by(double &, float) {}
__device__ __forceinline__ void scale_by(dd &, float) {}

constexpr float kInv4PiF = 0.0795774715459476679f;
constexpr uint32_t kMetaBytes = 32;   // per-term values at the end of every stage

// Launch geometry of the block-row kernel (computed on the host).
struct RowCfg {
  int M, Mp, rp;             // rows of an output tile, rows padded to 4, columns (padded to 16 bytes)
  int nvg, ncg, tiles;       // row groups (4 R rows), 16-byte column groups, register tiles of 4 R x (16 bytes)
  int ksplit;                // the contraction range of every term is split in ksplit slices
  int nst;                   // pipeline stages
  uint32_t a_bytes, stage_bytes, bar_off;   // A region of a stage, stage size, mbarrier offset
};

// One term A X of an output row: A stored [K][Mp] (contraction index major), X stored [K][rp].
template <class TS, class TC>
struct Term {
  const TS *A;
  const TC *X;
  int K;
};

// Row sources of the block-row kernel.  Every row has count(r) terms; the
// terms of all rows form one flat sequence (first(r) = flat index of row r's
// first term, first(nrows) = total), term(e) gives the tiles of flat term e,
// kdim(e) its contraction length and meta(e) a few values the producer puts
// beside the tiles: [0] the power of two the stored A tile was divided by
// (FP16 storage; 1 otherwise), [1..6] the box data of generated A tiles.
// kGen rows compute their A tiles in the consumer threads instead of loading
// them.

// Coupling (Algorithm 3, admissible blocks): row r = cluster row0 + r, terms
// S_b x^_{s_b} for the admissible blocks b of that row (S_b stored [mu][nu]).
template <class TS, class TC>
struct CouplingRows {
  static constexpr bool kGen = false;
  const TS *S;
  const int64_t *ptr;
  const int32_t *col;
  const TC *xhat;
  int k, kp, rp;
  int64_t row0;
  __device__ int kdim(int64_t) const { return k; }
  __device__ void meta(int64_t, float *mt) const { mt[0] = 1.0f; }
  __device__ int64_t first(int64_t r) const { return ptr[row0 + r] - ptr[row0]; }
  __device__ Term<TS, TC> term(int64_t e) const {
    const int64_t b = ptr[row0] + e;
    return Term<TS, TC>{S + b * (int64_t)k * kp, xhat + (int64_t)col[b] * k * rp, k};
  }
};

// Coupling with S_b regenerated on the fly in FP32 (Eq. (6c)): s_{nu mu} =
// 1/(4 pi |xi_{t,nu} - xi_{s,mu}|) from the clusters' interpolation boxes
// (centre c, half width h, Chebyshev nodes c + h t_j); the difference of the
// centres is formed in FP64 before rounding, so the distance keeps FP32
// relative accuracy for well-separated small clusters.
struct CouplingGenRows {
  static constexpr bool kGen = true;
  const int64_t *ptr;
  const int32_t *col;
  const float *xhat;
  const float4 *dc;     // [admissible blocks]: centre of t minus centre of s, formed in FP64
  const float *half;    // [clusters][3]
  float t[kMaxM];       // reference Chebyshev nodes cos((2j+1) pi / (2m))
  int m, k, kp, rp;
  int64_t row0;
  __device__ int kdim(int64_t) const { return k; }
  // scale, centre gap (3), half widths of the column cluster (3)
  __device__ void meta(int64_t e, float *mt) const {
    const int64_t b = ptr[row0] + e;
    const int64_t sg = col[b];
    const float4 g = dc[b];
    mt[0] = 1.0f;
    mt[1] = g.x;
    mt[2] = g.y;
    mt[3] = g.z;
    mt[4] = half[3 * sg];
    mt[5] = half[3 * sg + 1];
    mt[6] = half[3 * sg + 2];
  }
  __device__ int64_t first(int64_t r) const { return ptr[row0 + r] - ptr[row0]; }
  __device__ Term<float, float> term(int64_t e) const {
    const int64_t b = ptr[row0] + e;
    return Term<float, float>{nullptr, xhat + (int64_t)col[b] * k * rp, k};
  }
};

// Leaf forward step (Algorithm 1 on the leaves): row j = leaf j, one term
// V_j^T x|j (V_j stored [t][nu], padded to kp).
template <class TS, class TC>
struct LeafForwardRows {
  static constexpr bool kGen = false;
  const TS *V;
  const TC *xpad;
  const float *vscale;   // per leaf, or NULL
  int L, kp, rp;
  __device__ int kdim(int64_t) const { return L; }
  __device__ void meta(int64_t e, float *mt) const { mt[0] = vscale ? vscale[e] : 1.0f; }
  __device__ int64_t first(int64_t r) const { return r; }
  __device__ Term<TS, TC> term(int64_t e) const {
    return Term<TS, TC>{V + e * (int64_t)L * kp, xpad + e * (int64_t)L * rp, L};
  }
};

// Leaf backward step (Algorithm 2 on the leaves): row j = leaf j, one term
// V_j y^_j (V_j stored transposed [nu][t], padded to Lp).
template <class TS, class TC>
struct LeafBackwardRows {
  static constexpr bool kGen = false;
  const TS *Vt;
  const TC *yhat;
  const float *vscale;
  int k, Lp, rp;
  int64_t leaf0;
  __device__ int kdim(int64_t) const { return k; }
  __device__ void meta(int64_t e, float *mt) const { mt[0] = vscale ? vscale[e] : 1.0f; }
  __device__ int64_t first(int64_t r) const { return r; }
  __device__ Term<TS, TC> term(int64_t e) const {
    return Term<TS, TC>{Vt + e * (int64_t)k * Lp, yhat + (leaf0 + e) * (int64_t)k * rp, k};
  }
};

// Nearfield (Algorithm 3, inadmissible blocks): row j = leaf j, terms G_b x|s_b
// for the inadmissible blocks b of row j (G_b stored transposed [c][t]).  With
// blk the e-th term of the CSR uses stored block blk[e] (a CSR over a subset
// of the blocks), else block e.
template <class TS, class TC>
struct NearRows {
  static constexpr bool kGen = false;
  const TS *near;
  const int64_t *ptr;
  const int32_t *col;
  const TC *xpad;
  const float *nscale;   // per stored block, or NULL
  int L, Lp, rp;
  const int32_t *blk;    // stored block of every term, or NULL
  __device__ int64_t block(int64_t e) const { return blk ? (int64_t)blk[e] : e; }
  __device__ int kdim(int64_t) const { return L; }
  __device__ void meta(int64_t e, float *mt) const { mt[0] = nscale ? nscale[block(e)] : 1.0f; }
  __device__ int64_t first(int64_t r) const { return ptr[r]; }
  __device__ Term<TS, TC> term(int64_t e) const {
    return Term<TS, TC>{near + block(e) * (int64_t)L * Lp, xpad + (int64_t)col[e] * L * rp, L};
  }
};

// GCA-H^2 coupling at one tree level (Algorithm 3 with the pivot bases):
// row r = cluster c0 + r, terms S_b x^_s over the admissible blocks b of
// the row; the level's coupling matrices are stored consecutively from its
// first block ([K][K], S_b transposed) and its coefficients from its first
// cluster ([c - c0][K][rp]).
template <class TS, class TC>
struct GcaCouplingRows {
  static constexpr bool kGen = false;
  const TS *S;
  const int64_t *ptr;
  const int32_t *col;
  const TC *xhat;
  int K, rp;
  int64_t c0;
  __device__ int kdim(int64_t) const { return K; }
  __device__ void meta(int64_t, float *mt) const { mt[0] = 1.0f; }
  __device__ int64_t first(int64_t r) const { return ptr[c0 + r] - ptr[c0]; }
  __device__ Term<TS, TC> term(int64_t e) const {
    const int64_t b = ptr[c0] + e;
    return Term<TS, TC>{S + e * (int64_t)K * K, xhat + (int64_t)(col[b] - c0) * K * rp, K};
  }
};

// GCA-H^2 upward step (Algorithm 1): row r = parent r of level l - 1, terms
// E_s^T x^_s over its two sons s (sons 2r, 2r + 1 of level l, E_s stored
// [Kc][Kp]: the son's index is the contraction index).
template <class TS, class TC>
struct GcaUpRows {
  static constexpr bool kGen = false;
  const TS *E;
  const TC *xs;
  int Kc, Kp, rp;
  __device__ int kdim(int64_t) const { return Kc; }
  __device__ void meta(int64_t, float *mt) const { mt[0] = 1.0f; }
  __device__ int64_t first(int64_t r) const { return 2 * r; }
  __device__ Term<TS, TC> term(int64_t e) const {
    return Term<TS, TC>{E + e * (int64_t)Kc * Kp, xs + e * (int64_t)Kc * rp, Kc};
  }
};

// GCA-H^2 downward step (Algorithm 2): row r = son r of level l, one term
// E_r y^_parent (E_r stored transposed [Kp][Kc]); added to the son's y^.
template <class TS, class TC>
struct GcaDownRows {
  static constexpr bool kGen = false;
  const TS *Et;
  const TC *yp;
  int Kc, Kp, rp;
  __device__ int kdim(int64_t) const { return Kp; }
  __device__ void meta(int64_t, float *mt) const { mt[0] = 1.0f; }
  __device__ int64_t first(int64_t r) const { return r; }
  __device__ Term<TS, TC> term(int64_t e) const {
    return Term<TS, TC>{Et + e * (int64_t)Kp * Kc, yp + (e >> 1) * (int64_t)Kp * rp, Kp};
  }
};

// Block rows with small tiles (the GCA-H^2 coupling and transfer steps): one
// warp per row, out_r (M x rp) = sum over the row's terms of A X (A stored
// [K][Mp], rows padded to Mp, X [K][rp]).  The warp stages the tiles of a
// term in its own two shared-memory buffers with 16-byte asynchronous
// copies, the next term's copies in flight while it multiplies the current
// one.  A lane owns up to TPL register tiles of 4 rows x one 16-byte group
// of columns (tile q of the row: rows 4 (q mod Mp/4) .., column group
// q div (Mp/4)); every output is summed by one lane in a fixed order, so
// results are reproducible.  No waits on other threads beyond the warp's
// own copies.
template <class TS, class TC, int TPL, class Rows>
__global__ void __launch_bounds__(128) k_rows_warp(Rows rows, int M, int Mp, int rp, int Kmax, int64_t nrows,
                                                   int accumulate, TC *__restrict__ out) {
  using XV = typename Vec16<TC>::V;
  constexpr int VN = Vec16<TC>::N;
  extern __shared__ __align__(16) unsigned char rwsm[];
  const int ln = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint32_t abytes = (uint32_t)((sizeof(TS) * Kmax * Mp + 15) / 16 * 16);
  const uint32_t xbytes = (uint32_t)((sizeof(TC) * Kmax * rp + 15) / 16 * 16);
  unsigned char *buf = rwsm + (size_t)wib * 2 * (abytes + xbytes);
  const int nvg = Mp / 4, tiles = nvg * (rp / VN);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + wib; r < nrows; r += nw) {
    TC acc[TPL][4][VN];
#pragma unroll
    for (int t = 0; t < TPL; ++t)
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < VN; ++c) acc[t][a][c] = zero_of<TC>();
    const int64_t e0 = rows.first(r), e1 = rows.first(r + 1);
    auto issue = [&](int64_t e) {
      unsigned char *st = buf + (size_t)((e - e0) & 1) * (abytes + xbytes);
      const Term<TS, TC> tm = rows.term(e);
      const uint32_t ab = (uint32_t)(sizeof(TS) * tm.K * Mp), xb = (uint32_t)(sizeof(TC) * tm.K * rp);
      const unsigned char *sa = reinterpret_cast<const unsigned char *>(tm.A);
      const unsigned char *sx = reinterpret_cast<const unsigned char *>(tm.X);
      for (uint32_t o = 16 * ln; o < ab; o += 16 * 32) cp_async16(st + o, sa + o);
      for (uint32_t o = 16 * ln; o < xb; o += 16 * 32) cp_async16(st + abytes + o, sx + o);
      cp_async_commit();
    };
    if (e0 < e1) issue(e0);
    for (int64_t e = e0; e < e1; ++e) {
      if (e + 1 < e1) {
        issue(e + 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
      const unsigned char *st = buf + (size_t)((e - e0) & 1) * (abytes + xbytes);
      const TS *sA = reinterpret_cast<const TS *>(st);
      const TC *sX = reinterpret_cast<const TC *>(st + abytes);
      const int K = rows.kdim(e);
#pragma unroll
      for (int t = 0; t < TPL; ++t) {
        const int q = ln + 32 * t;
        if (q < tiles) {
          const int g = q % nvg, cg = q / nvg;
          for (int mu = 0; mu < K; ++mu) {
            TC av[4];
            load4<TS, TC>(sA + mu * Mp + 4 * g, av);
            const XV xv = *reinterpret_cast<const XV *>(sX + mu * rp + VN * cg);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int c = 0; c < VN; ++c) acc_fma(acc[t][a][c], av[a], lane<TC>(xv, c));
          }
        }
      }
      __syncwarp();
    }
    TC *o = out + r * (int64_t)M * rp;
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
      const int q = ln + 32 * t;
      if (q < tiles) {
        const int g = q % nvg, cg = q / nvg;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < VN; ++c) {
            acc_norm(acc[t][a][c]);
            if (4 * g + a < M) {
              TC *dst = o + (int64_t)(4 * g + a) * rp + VN * cg + c;
              *dst = accumulate ? *dst + acc[t][a][c] : acc[t][a][c];
            }
          }
      }
    }
  }
}

// Block-row product, persistent and warp-specialised: output tile out_r
// (M x rp) = sum over the terms of row r of A X.  Each CTA takes a contiguous
// range of rows holding about 1/gridDim of all terms.  The last warp is the
// producer: one lane streams the A and X tiles of the CTA's terms through an
// nst-stage shared-memory ring with bulk copies (TMA engine), each stage
// completing on its "full" mbarrier, and refills a stage once every consumer
// warp has released it on its "empty" mbarrier.  The other warps consume:
// a thread's register tile holds R groups of 4 rows (rows g Mp/R + 4 vg + a,
// so that the lanes of a warp read contiguous 16-byte pieces of one A row)
// times one 16-byte group of columns, for one slice of the contraction
// index; at the end of a row the slices are summed in a fixed order (no
// atomics: results are bit-reproducible).  With accumulate the row is added
// to out instead of overwriting it.  Every wait is bounded; a timeout raises
// the device error word and all warps leave after the copies in flight have
// landed.  Used for the coupling (rows = clusters), the leaf forward and
// backward steps and the nearfield (rows = leaves).
template <class TS, class TC, int R, class Rows>
__global__ void __launch_bounds__(kThreads + 32, 2)
    k_blockrow(Rows rows, RowCfg cfg, int64_t nrows, int accumulate, TC *__restrict__ out) {
  using XV = typename Vec16<TC>::V;
  constexpr int VN = Vec16<TC>::N;
  extern __shared__ __align__(128) unsigned char smem[];
  TC *red = reinterpret_cast<TC *>(smem + (size_t)cfg.nst * cfg.stage_bytes);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + cfg.bar_off);
  uint64_t *empty = full + cfg.nst;
  volatile int *abort = reinterpret_cast<volatile int *>(empty + cfg.nst);
  const int tid = threadIdx.x;
  const int ncons = blockDim.x - 32, nwc = ncons / 32;
  const int Mp = cfg.Mp, rp = cfg.rp;

  // rows of this CTA: from the first row whose terms start at or after its share
  const int64_t total = rows.first(nrows);
  auto row_at = [&](int64_t w) -> int64_t {
    if (w >= (int64_t)gridDim.x) return nrows;
    const int64_t target = total * w / gridDim.x;
    int64_t lo = 0, hi = nrows;  // smallest r with first(r) >= target
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if (rows.first(mid) >= target) hi = mid;
      else lo = mid + 1;
    }
    return lo;
  };
  const int64_t r_begin = blockIdx.x == 0 ? 0 : row_at(blockIdx.x);
  const int64_t r_end = row_at(blockIdx.x + 1);
  const int64_t e_begin = rows.first(r_begin), e_end = rows.first(r_end);

  if (tid == 0) {
    for (int s = 0; s < cfg.nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], nwc);
    }
    *abort = 0;
    mbar_fence_init();
  }
  __syncthreads();

  if (tid >= ncons) {
    // ---------------- producer warp ----------------
    if (tid == ncons) {
      int64_t e = e_begin;
      for (; e < e_end; ++e) {
        const int64_t i = e - e_begin;
        const int s = (int)(i % cfg.nst);
        if (i >= cfg.nst && !mbar_wait_or_abort(&empty[s], (uint32_t)((i / cfg.nst - 1) & 1), abort)) break;
        unsigned char *st = smem + (size_t)s * cfg.stage_bytes;
        const Term<TS, TC> tm = rows.term(e);
        const uint32_t ab = Rows::kGen ? 0u : (uint32_t)(sizeof(TS) * tm.K * Mp);
        const uint32_t xb = (uint32_t)(sizeof(TC) * tm.K * rp);
        // the term's metadata goes beside the tiles; the arrival below releases it
        rows.meta(e, reinterpret_cast<float *>(st + cfg.stage_bytes - kMetaBytes));
        mbar_expect_tx(&full[s], ab + xb);
        if (!Rows::kGen) bulk_g2s(st, tm.A, ab, &full[s]);
        bulk_g2s(st + cfg.a_bytes, tm.X, xb, &full[s]);
      }
      if (*abort) {
        // let the copies in flight land before the CTA leaves (bounded)
        const int64_t j0 = e - cfg.nst > e_begin ? e - cfg.nst : e_begin;
        for (int64_t j = j0; j < e; ++j) {
          const int64_t ij = j - e_begin;
          mbar_wait_bounded(&full[ij % cfg.nst], (uint32_t)((ij / cfg.nst) & 1));
        }
      }
    }
    return;
  }

  // ---------------- consumer warps ----------------
  const int tile = tid % cfg.tiles, ks = tid / cfg.tiles;
  const bool active = ks < cfg.ksplit;
  const int vg = tile % cfg.nvg, cg = tile / cfg.nvg;
  const int gstride = Mp / R;
  const int lane_id = tid & 31;
  int64_t e = e_begin;
  for (int64_t r = r_begin; r < r_end; ++r) {
    TC acc[4 * R][VN];
#pragma unroll
    for (int a = 0; a < 4 * R; ++a)
#pragma unroll
      for (int c = 0; c < VN; ++c) acc[a][c] = zero_of<TC>();
    // generated coupling: node offsets of this thread's rows in the row cluster
    float gnode[Rows::kGen ? 4 * R : 1][3];
    bool gvalid[Rows::kGen ? 4 * R : 1];
    if constexpr (Rows::kGen) {
      const int64_t grow = rows.row0 + r;
      const int m = rows.m;
#pragma unroll
      for (int a = 0; a < 4 * R; ++a) {
        const int nu = (a / 4) * gstride + 4 * vg + (a % 4);
        gvalid[a] = nu < rows.k;
        const int jj[3] = {nu % m, (nu / m) % m, min(nu / (m * m), m - 1)};
#pragma unroll
        for (int d = 0; d < 3; ++d) gnode[a][d] = rows.half[3 * grow + d] * rows.t[jj[d]];
      }
    }
    const int64_t e_row_end = rows.first(r + 1);
    for (; e < e_row_end; ++e) {
      const int64_t i = e - e_begin;
      const int s = (int)(i % cfg.nst);
      // every consumer thread waits (also idle ones), so that no warp releases a
      // stage it has not seen filled
      const bool ready = !*abort && mbar_wait_or_abort(&full[s], (uint32_t)((i / cfg.nst) & 1), abort);
      if (ready && active) {
        const TS *sA = reinterpret_cast<const TS *>(smem + (size_t)s * cfg.stage_bytes);
        const TC *sX = reinterpret_cast<const TC *>(smem + (size_t)s * cfg.stage_bytes + cfg.a_bytes);
        const float *mt = reinterpret_cast<const float *>(smem + (size_t)(s + 1) * cfg.stage_bytes - kMetaBytes);
        const int K = rows.kdim(e);
        const int kc = (K + cfg.ksplit - 1) / cfg.ksplit;
        const int mu0 = ks * kc, mu1 = min(K, mu0 + kc);
        const float sc = mt[0];
        float hs[3] = {0.f, 0.f, 0.f};
        float gbase[Rows::kGen ? 4 * R : 1][3];
        if constexpr (Rows::kGen) {
#pragma unroll
          for (int a = 0; a < 4 * R; ++a) {
            gbase[a][0] = mt[1] + gnode[a][0];
            gbase[a][1] = mt[2] + gnode[a][1];
            gbase[a][2] = mt[3] + gnode[a][2];
          }
          hs[0] = mt[4];
          hs[1] = mt[5];
          hs[2] = mt[6];
        }
#pragma unroll 2
        for (int mu = mu0; mu < mu1; ++mu) {
          TC av[4 * R];
          if constexpr (Rows::kGen) {
            const int m = rows.m;
            const float ox = hs[0] * rows.t[mu % m], oy = hs[1] * rows.t[(mu / m) % m], oz = hs[2] * rows.t[mu / (m * m)];
#pragma unroll
            for (int a = 0; a < 4 * R; ++a) {
              const float dx = gbase[a][0] - ox, dy = gbase[a][1] - oy, dz = gbase[a][2] - oz;
              const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
              av[a] = gvalid[a] ? kInv4PiF * rsqrtf(r2) : 0.0f;
            }
          } else {
#pragma unroll
            for (int g = 0; g < R; ++g) load4<TS, TC>(sA + mu * Mp + g * gstride + 4 * vg, av + 4 * g);
          }
          const XV xv = *reinterpret_cast<const XV *>(sX + mu * rp + VN * cg);
          TC xs[VN];
#pragma unroll
          for (int l = 0; l < VN; ++l) {
            xs[l] = lane<TC>(xv, l);
            scale_by(xs[l], sc);
          }
#pragma unroll
          for (int a = 0; a < 4 * R; ++a)
#pragma unroll
            for (int c = 0; c < VN; ++c) acc_fma(acc[a][c], av[a], xs[c]);
        }
#pragma unroll
        for (int a = 0; a < 4 * R; ++a)
#pragma unroll
          for (int c = 0; c < VN; ++c) acc_norm(acc[a][c]);
      }
      __syncwarp();
      if (lane_id == 0) mbar_arrive(&empty[s]);
    }
    // end of row r: agree on abort, then sum the slices in a fixed order
    if (named_sync_or(ncons, *abort)) return;
    if (active) {
#pragma unroll
      for (int a = 0; a < 4 * R; ++a)
#pragma unroll
        for (int c = 0; c < VN; ++c)
          red[((int64_t)ks * Mp + (a / 4) * gstride + 4 * vg + (a % 4)) * rp + VN * cg + c] = acc[a][c];
    }
    named_sync(ncons);
    TC *o = out + r * (int64_t)cfg.M * rp;
    for (int q = tid; q < cfg.M * rp; q += ncons) {
      const int nu = q / rp, c = q - nu * rp;
      TC sum = accumulate ? o[q] : zero_of<TC>();
      for (int z = 0; z < cfg.ksplit; ++z) sum = sum + red[((int64_t)z * Mp + nu) * rp + c];
      o[q] = sum;
    }
    named_sync(ncons);
  }
}

// Coupling regenerated in FP32, warp per row cluster (for up to 64 rows and
// 16 columns): lane l owns rows nu = l + 32 q of y^_t for all columns and
// loops over the admissible blocks of the row; per block the warp stages
// x^_s and the column cluster's node offsets in its own shared memory and
// evaluates s_{nu mu} = 1/(4 pi |xi_{t,nu} - xi_{s,mu}|) in registers (the
// centre gap comes precomputed from FP64).  No cross-warp reduction: each
// output is summed by one lane in a fixed order.
constexpr int kRegenWarps = 4;

template <int QR, int CP>
__global__ void __launch_bounds__(32 * kRegenWarps)
    k_coupling_regen_warp(const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                          const float4 *__restrict__ dc, const float *__restrict__ half,
                          const float *__restrict__ xhat, CouplingGenRows g, int64_t nrows, float *__restrict__ yhat) {
  extern __shared__ __align__(16) float wsm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int k = g.k, m = g.m, rp = g.rp;
  float *tn = wsm;                                          // reference nodes
  float *xs = wsm + 16 + (size_t)w * (64 * CP + 3 * 64);   // [k][rp] then offsets [3][k]
  float *offs = xs + 64 * CP;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < kMaxM; ++j) tn[j] = g.t[j];   // constant indices: no local copy of the parameters
  }
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * kRegenWarps + w;
  if (r >= nrows) return;
  const int64_t t = g.row0 + r;
  float node[QR][3];
  bool valid[QR];
#pragma unroll
  for (int q = 0; q < QR; ++q) {
    const int nu = lane + 32 * q;
    valid[q] = nu < k;
    const int j[3] = {nu % m, (nu / m) % m, min(nu / (m * m), m - 1)};
#pragma unroll
    for (int d = 0; d < 3; ++d) node[q][d] = half[3 * t + d] * tn[j[d]];
  }
  float acc[QR][CP];
#pragma unroll
  for (int q = 0; q < QR; ++q)
#pragma unroll
    for (int c = 0; c < CP; ++c) acc[q][c] = 0.0f;
  const int64_t b0 = ptr[t], b1 = ptr[t + 1];
  for (int64_t b = b0; b < b1; ++b) {
    const int64_t sg = col[b];
    const float4 gap = dc[b];
    __syncwarp();
    const float *xsrc = xhat + sg * (int64_t)k * rp;
    for (int i = lane; i < k * rp; i += 32) xs[i] = xsrc[i];
    for (int i = lane; i < k; i += 32) {
      offs[i] = half[3 * sg] * tn[i % m];
      offs[64 + i] = half[3 * sg + 1] * tn[(i / m) % m];
      offs[128 + i] = half[3 * sg + 2] * tn[i / (m * m)];
    }
    __syncwarp();
    float base[QR][3];
#pragma unroll
    for (int q = 0; q < QR; ++q) {
      base[q][0] = gap.x + node[q][0];
      base[q][1] = gap.y + node[q][1];
      base[q][2] = gap.z + node[q][2];
    }
#pragma unroll 3
    for (int mu = 0; mu < k; ++mu) {
      const float ox = offs[mu], oy = offs[64 + mu], oz = offs[128 + mu];
      float xv[CP];
#pragma unroll
      for (int c = 0; c < CP; c += 4) {
        const float4 v = *reinterpret_cast<const float4 *>(xs + mu * rp + c);
        xv[c] = v.x; xv[c + 1] = v.y; xv[c + 2] = v.z; xv[c + 3] = v.w;
      }
#pragma unroll
      for (int q = 0; q < QR; ++q) {
        const float dx = base[q][0] - ox, dy = base[q][1] - oy, dz = base[q][2] - oz;
        const float sv = valid[q] ? kInv4PiF * rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) : 0.0f;
#pragma unroll
        for (int c = 0; c < CP; ++c)
          if (c < rp) acc[q][c] = fmaf(sv, xv[c], acc[q][c]);
      }
    }
  }
  float *out = yhat + t * (int64_t)k * rp;
#pragma unroll
  for (int q = 0; q < QR; ++q)
    if (valid[q])
#pragma unroll
      for (int c = 0; c < CP; ++c)
        if (c < rp) out[(lane + 32 * q) * rp + c] = acc[q][c];
}

template <int QR, int CP>
int launch_regen_warp(const CouplingGenRows &g, int64_t nrows, float *yhat, cudaStream_t st) {
  const size_t sm = (16 + (size_t)kRegenWarps * (64 * CP + 3 * 64)) * sizeof(float);
  const unsigned grid = (unsigned)((nrows + kRegenWarps - 1) / kRegenWarps);
  k_coupling_regen_warp<QR, CP><<<grid, 32 * kRegenWarps, sm, st>>>(g.ptr, g.col, g.dc, g.half, g.xhat, g, nrows,
                                                                     yhat);
  return H2_OK;
}

// warp-per-row regenerated coupling when k <= 64 and rp <= 16, else -1;
// yhat is the base of [clusters][k][rp] (rows g.row0 .. g.row0 + nrows - 1 are written)
int regen_warp(const CouplingGenRows &g, int64_t nrows, float *yhat, cudaStream_t st) {
  if (g.k > 64 || g.rp > 16 || nrows <= 0) return -1;
  const int QR = g.k > 32 ? 2 : 1, CP = g.rp <= 4 ? 4 : (g.rp <= 8 ? 8 : 16);
  if (QR == 1) return CP == 4 ? launch_regen_warp<1, 4>(g, nrows, yhat, st)
                              : CP == 8 ? launch_regen_warp<1, 8>(g, nrows, yhat, st)
                                        : launch_regen_warp<1, 16>(g, nrows, yhat, st);
  return CP == 4 ? launch_regen_warp<2, 4>(g, nrows, yhat, st)
                 : CP == 8 ? launch_regen_warp<2, 8>(g, nrows, yhat, st) : launch_regen_warp<2, 16>(g, nrows, yhat, st);
}

constexpr size_t kSmemMax = 227 * 1024;

// geometry for output tiles M x rp and contraction lengths up to Kmax;
// threads: the number of threads the kernel is launched with
template <class TS, class T>
int row_cfg(int M, int Mp, int rp, int Kmax, int threads, int R, bool gen, RowCfg &cfg) {
  constexpr int VN = Vec16<T>::N;
  cfg.M = M;
  cfg.Mp = Mp;
  cfg.rp = rp;
  cfg.nvg = Mp / (4 * R);
  cfg.ncg = rp / VN;
  cfg.tiles = cfg.nvg * cfg.ncg;
  if (cfg.tiles > threads) return fail(H2_EINVAL, "tile rows x right-hand sides too large for one CTA");
  cfg.ksplit = std::max(1, std::min(threads / cfg.tiles, Kmax));
  cfg.a_bytes = gen ? 0u : (uint32_t)((sizeof(TS) * Kmax * Mp + 15) / 16 * 16);
  cfg.stage_bytes = cfg.a_bytes + (uint32_t)((sizeof(T) * Kmax * rp + 15) / 16 * 16) + kMetaBytes;
  const size_t red = sizeof(T) * (size_t)cfg.ksplit * Mp * rp;   // slice sums, after the ring
  // stages: up to 8, sized so that 512 consumer threads per SM stay resident when possible
  const size_t budget = kSmemMax / (512 / threads);
  int nst = 8;
  while (nst > 2 && (size_t)nst * cfg.stage_bytes + red + 128 > budget) --nst;
  while (nst > 1 && (size_t)nst * cfg.stage_bytes + red + 128 > kSmemMax) --nst;
  cfg.nst = nst;
  const size_t body = (size_t)nst * cfg.stage_bytes + red;
  cfg.bar_off = (uint32_t)((body + 15) / 16 * 16);
  if (cfg.bar_off + 16 * nst + 16 > kSmemMax) return fail(H2_EINVAL, "block-row tile does not fit in shared memory");
  return H2_OK;
}

// row groups per register tile: two for FP32 compute when the rows split evenly
template <class T>
inline int row_groups(int Mp) {
  return (sizeof(T) == 4 && Mp % 8 == 0) ? 2 : 1;
}

// consumer threads per CTA: enough slices of the contraction for about 4 to 8 steps each
inline int row_threads(int Mp, int rp, int Kmax, size_t esize, int R) {
  const int tiles = (Mp / (4 * R)) * (rp / (int)(16 / esize));
  const int want = tiles * std::max(1, Kmax / 8);
  for (int t : {32, 64, 128})
    if (want <= t && tiles <= t) return t;
  return 256;
}

int grid_for(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

// Allow the kernel the largest dynamic shared memory once it needs more than
// the default 48 KB.  Always the same value: products of different handles
// run concurrently from several threads (serving), and a smaller limit set
// by one of them must never undercut another's launch.
template <class T>
int set_smem(const void *fn, size_t bytes) {
  if (bytes > kSmemMax) return fail(H2_EINVAL, "tile does not fit in shared memory");
  if (bytes > 48 * 1024)
    H2_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
  return H2_OK;
}

// per-phase event marks of one product (only while profiling)
struct Marks {
  Ctx &c;
  cudaEvent_t ev[H2_NPHASE + 1] = {};
  int64_t launches[H2_NPHASE] = {0};
  explicit Marks(Ctx &cc) : c(cc) {
    if (!c.prof.on) return;
    for (auto &e : ev) cudaEventCreate(&e);
  }
  void mark(int ph) {
    if (c.prof.on) cudaEventRecord(ev[ph], c.stream);
  }
  void count(int ph, int64_t n = 1) { launches[ph] += n; }
  void finish() {
    if (!c.prof.on) return;
    c.prof.ev.insert(c.prof.ev.end(), ev, ev + H2_NPHASE + 1);
    if (c.prof.launches.size() < H2_NPHASE) c.prof.launches.assign(H2_NPHASE, 0);
    for (int i = 0; i < H2_NPHASE; ++i) c.prof.launches[i] += launches[i];
    c.prof.products++;
  }
};

// persistent launch: as many CTAs as stay resident, at most one per row
template <class TS, class TC, int R, class Rows>
int launch_rows_r(const Rows &rows, const RowCfg &cfg, int threads, int64_t nrows, int accumulate, TC *out,
                  cudaStream_t st) {
  const void *fn = (const void *)k_blockrow<TS, TC, R, Rows>;
  const size_t sm = cfg.bar_off + 16 * cfg.nst + 16;
  threads += 32;   // the producer warp
  int rc;
  if ((rc = set_smem<TC>(fn, sm))) return rc;
  int per_sm = 0, dev = 0, sms = 0;
  H2_CUDA_TRY(cudaGetDevice(&dev));
  H2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  H2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, sm));
  if (per_sm < 1) return fail(H2_EINVAL, "block-row kernel cannot be resident");
  const int64_t grid = std::min<int64_t>(nrows, (int64_t)per_sm * sms);
  k_blockrow<TS, TC, R, Rows><<<(unsigned)grid, threads, sm, st>>>(rows, cfg, nrows, accumulate, out);
  return H2_OK;
}

template <class TS, class TC, class Rows>
int launch_rows(const Rows &rows, const RowCfg &cfg, int threads, int R, int64_t nrows, int accumulate, TC *out,
                cudaStream_t st) {
  if (nrows <= 0) return H2_OK;
  if (R == 2) return launch_rows_r<TS, TC, 2>(rows, cfg, threads, nrows, accumulate, out, st);
  return launch_rows_r<TS, TC, 1>(rows, cfg, threads, nrows, accumulate, out, st);
}


// Leaf steps (Algorithm 1 at the leaves, x^_t = V_t^T x|t; Algorithm 2 at the
// leaves, y|t = V_t y^_t) for leaves of at most 32 triangles, k <= 64 and
// rp <= 16: one CTA per leaf stages V_t (converted to the arithmetic type)
// and the leaf's vector block in shared memory; in the forward step thread
// (nu, jq) forms x^[nu][jq + 4u], in the backward step thread (r, jo) forms
// y[r][jo + 8u], each as one contraction with a single renormalisation, then
// multiplied by the leaf's power-of-two scale (16-bit storage) if there is
// one.  The generic block-row kernel pipelines many terms per row; a leaf
// row has one.
template <class TS, class T>
__global__ void __launch_bounds__(256) k_leaf_fwd_reg(const TS *__restrict__ V, const T *__restrict__ xpad,
                                                      const float *__restrict__ vscale, int L, int kp, int k, int rp,
                                                      T *__restrict__ xleaf) {
  extern __shared__ __align__(16) unsigned char lsm[];
  T *Vs = reinterpret_cast<T *>(lsm);   // [L][kp]
  T *xs = Vs + L * kp;                   // [L][rp]
  const int64_t t = blockIdx.x;
  const TS *vt = V + t * (int64_t)L * kp;
  const T *xt = xpad + t * (int64_t)L * rp;
  for (int i = threadIdx.x; i < L * kp; i += blockDim.x) Vs[i] = to_compute<T>(vt[i]);
  for (int i = threadIdx.x; i < L * rp; i += blockDim.x) xs[i] = xt[i];
  __syncthreads();
  const int nu = threadIdx.x >> 2, jq = threadIdx.x & 3;
  if (nu >= k) return;
  T acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = zero_of<T>();
  for (int r = 0; r < L; ++r) {
    const T v = Vs[r * kp + nu];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (jq + 4 * u < rp) acc_fma(acc[u], v, xs[r * rp + jq + 4 * u]);
  }
  const float sc = vscale ? vscale[t] : 1.0f;
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (jq + 4 * u < rp) {
      acc_norm(acc[u]);
      xleaf[(t * k + nu) * rp + jq + 4 * u] = vscale ? acc[u] * from_double<T>(sc) : acc[u];
    }
}

// With gself (FP32 self blocks of bfloat16 handles, [leaf][c][Lp]) the
// leaf's self block joins the contraction: y|t = V_t y^_t + G_tt x|t.
template <class TS, class T>
__global__ void __launch_bounds__(256) k_leaf_bwd_reg(const TS *__restrict__ Vt, const T *__restrict__ yleaf,
                                                      const float *__restrict__ vscale, int L, int Lp, int k, int rp,
                                                      const float *__restrict__ gself, const T *__restrict__ xpad,
                                                      T *__restrict__ ypad) {
  extern __shared__ __align__(16) unsigned char lsm[];
  T *Vs = reinterpret_cast<T *>(lsm);   // [k][Lp]
  T *ys = Vs + k * Lp;                   // [k][rp]
  T *Gs = ys + k * rp;                   // [L][Lp] (with gself)
  T *xs = Gs + L * Lp;                   // [L][rp] (with gself)
  const int64_t t = blockIdx.x;
  const TS *vt = Vt + t * (int64_t)k * Lp;
  const T *yt = yleaf + t * (int64_t)k * rp;
  for (int i = threadIdx.x; i < k * Lp; i += blockDim.x) Vs[i] = to_compute<T>(vt[i]);
  for (int i = threadIdx.x; i < k * rp; i += blockDim.x) ys[i] = yt[i];
  if (gself) {
    for (int i = threadIdx.x; i < L * Lp; i += blockDim.x) Gs[i] = from_double<T>(gself[t * (int64_t)L * Lp + i]);
    for (int i = threadIdx.x; i < L * rp; i += blockDim.x) xs[i] = xpad[t * (int64_t)L * rp + i];
  }
  __syncthreads();
  const int r = threadIdx.x >> 3, jo = threadIdx.x & 7;
  if (r >= L) return;
  T acc[2] = {zero_of<T>(), zero_of<T>()};
  for (int nu = 0; nu < k; ++nu) {
    const T w = Vs[nu * Lp + r];
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (jo + 8 * u < rp) acc_fma(acc[u], w, ys[nu * rp + jo + 8 * u]);
  }
  if (gself)
    for (int c = 0; c < L; ++c) {
      const T w = Gs[c * Lp + r];
#pragma unroll
      for (int u = 0; u < 2; ++u)
        if (jo + 8 * u < rp) acc_fma(acc[u], w, xs[c * rp + jo + 8 * u]);
    }
  const float sc = vscale ? vscale[t] : 1.0f;
#pragma unroll
  for (int u = 0; u < 2; ++u)
    if (jo + 8 * u < rp) {
      acc_norm(acc[u]);
      ypad[(t * L + r) * rp + jo + 8 * u] = vscale ? acc[u] * from_double<T>(sc) : acc[u];
    }
}

// TS: storage type of S and the nearfield; TV: of the leaf bases V; TE: of
// the transfer factors; T: arithmetic and vector type; Tio: type of the
// caller's x and y.  acc: y += G~ x.
template <class TS, class TV, class TE, class T, class Tio>
int matvec_typed(Ctx &c, const Tio *x, Tio *y, int nrhs, bool acc) {
  Dev &d = c.d;
  cudaStream_t st = c.stream;
  const int k = d.k, kp = d.kp, m = d.m, L = (int)d.lmax, Lp = (int)d.lp, D = d.depth, lmin = d.first_adm_level;
  const int rp = padded_rhs(nrhs, sizeof(T));   // every kernel below works on rp columns
  const int64_t leaf0 = d.nleaf - 1;
  T *xpad = (T *)d.xpad, *ypad = (T *)d.ypad, *xhat = (T *)d.xhat, *yhat = (T *)d.yhat;
  const bool far = lmin <= D, gen = d.coupling == 1;
  int rc;
  RowCfg cf_fwd{}, cf_cpl{}, cf_back{}, cf_near{};
  const int Rk = row_groups<T>(kp), RL = row_groups<T>(Lp);
  const int t_fwd = row_threads(kp, rp, L, sizeof(T), Rk), t_cpl = row_threads(kp, rp, k, sizeof(T), Rk);
  const int t_back = row_threads(Lp, rp, k, sizeof(T), RL), t_near = row_threads(Lp, rp, L, sizeof(T), RL);
  if (far) {
    if ((rc = row_cfg<TV, T>(k, kp, rp, L, t_fwd, Rk, false, cf_fwd))) return rc;
    if ((rc = row_cfg<TS, T>(k, kp, rp, k, t_cpl, Rk, gen, cf_cpl))) return rc;
    if ((rc = row_cfg<TV, T>(L, Lp, rp, k, t_back, RL, false, cf_back))) return rc;
  }
  if ((rc = row_cfg<TS, T>(L, Lp, rp, L, t_near, RL, false, cf_near))) return rc;
  const float *vscale = (const float *)d.vscale, *nscale = (const float *)d.nscale;
  Marks mk(c);

  mk.mark(H2_PH_PERMUTE_IN);
  // double-float handles: column maxima of x for the range guard
  const unsigned long long *cmx = std::is_same<T, dd>::value ? d.colmax : nullptr;
  if (cmx) {
    H2_CUDA_TRY(cudaMemsetAsync(d.colmax, 0, sizeof(unsigned long long) * nrhs, st));
    const int64_t nb = std::min<int64_t>((d.n + 8 * kThreads - 1) / (8 * kThreads), 64);
    k_colmax<Tio><<<dim3((unsigned)std::max<int64_t>(nb, 1), nrhs), kThreads, 0, st>>>(x, d.n, d.colmax);
    mk.count(H2_PH_PERMUTE_IN);
  }
  const unsigned perm_grid = (unsigned)((d.npad + kPermRows - 1) / kPermRows);
  // FP64-accurate with the tensor-core nearfield and coupling: the leaf
  // forward step from the input digits the nearfield reads anyway; the
  // permutation takes the input's column maxima on the way
  const bool leaf_tc = std::is_same<T, dd>::value && far && d.ntc && d.Vtc && rp <= 16;
  if (leaf_tc) H2_CUDA_TRY(cudaMemsetAsync(d.ntc_xmax, 0, sizeof(unsigned) * 16, st));
  k_permute_in<Tio, T><<<perm_grid, 256, (size_t)kPermRows * (rp + 1) * sizeof(T), st>>>(
      x, d.n, nrhs, rp, d.pad_src, d.npad, cmx, xpad, leaf_tc ? d.ntc_xmax : nullptr);
  mk.count(H2_PH_PERMUTE_IN);
  mk.mark(H2_PH_LEAF_FORWARD);
  // leaf steps with one CTA per leaf when the stored values are in the arithmetic type
  const bool leaf_reg = L <= 32 && k <= 64 && rp <= 16;
  if (leaf_tc) {
    int64_t nl = 0;
    if ((rc = ntc_input(c, xpad, rp, &nl, true))) return rc;
    if ((rc = tc_leaf_forward(c, xhat, rp))) return rc;
    mk.count(H2_PH_LEAF_FORWARD, nl + 1);
  } else if (far && leaf_reg) {
    const size_t sm = (size_t)L * (kp + rp) * sizeof(T);
    k_leaf_fwd_reg<TV, T><<<(unsigned)d.nleaf, 256, sm, st>>>((const TV *)d.V, xpad, vscale, L, kp, k, rp,
                                                             xhat + leaf0 * (int64_t)k * rp);
    mk.count(H2_PH_LEAF_FORWARD);
  } else if (far) {
    LeafForwardRows<TV, T> rows{(const TV *)d.V, xpad, vscale, L, kp, rp};
    if ((rc = launch_rows<TV, T>(rows, cf_fwd, t_fwd, Rk, d.nleaf, 0, xhat + leaf0 * (int64_t)k * rp, st))) return rc;
    mk.count(H2_PH_LEAF_FORWARD);
  }
  mk.mark(H2_PH_UPWARD);
  const bool tcpath = d.tc && rp <= 16 &&
                      ((std::is_same<T, dd>::value && d.tc_nd == 10) ||
                       (std::is_same<T, float>::value && std::is_same<TS, float>::value && d.tc_nd == 6));
  if (far && tcpath) {
    // with the column maxima and coefficient slices of the tensor-core coupling
    int64_t nl = 0;
    if ((rc = tc_upward(c, xhat, rp, &nl, leaf_tc))) return rc;
    mk.count(H2_PH_UPWARD, nl);
  } else if (far && (m == 3 || m == 4)) {
    // orders 3 and 4: register kernels (the z mode product by warp shuffles)
    for (int l = D - 1; l >= lmin; --l) {
      const int64_t np = (int64_t)1 << l;
      const dim3 grid((unsigned)((np + kRegParents - 1) / kRegParents), (rp + 15) / 16);
      const dim3 grid2((unsigned)((np + kSplitParents - 1) / kSplitParents), (rp + 15) / 16);
      if (np <= kUpSplitMax) {
        if (m == 4) k_up_split<TE, T, 4><<<grid2, 256, 0, st>>>((const TE *)d.Ef, rp, np - 1, np, xhat, nullptr);
        else k_up_split<TE, T, 3><<<grid2, 256, 0, st>>>((const TE *)d.Ef, rp, np - 1, np, xhat, nullptr);
      } else if (m == 4) k_up_reg<TE, T, 4><<<grid, 256, 0, st>>>((const TE *)d.Ef, rp, np - 1, np, xhat, nullptr);
      else k_up_reg<TE, T, 3><<<grid, 256, 0, st>>>((const TE *)d.Ef, rp, np - 1, np, xhat, nullptr);
      mk.count(H2_PH_UPWARD);
    }
  } else if (far) {
    size_t sm = ((size_t)3 * k * rp + 6 * m * m) * sizeof(T);
    if ((rc = set_smem<T>((const void *)k_upward<TE, T>, sm))) return rc;
    for (int l = D - 1; l >= lmin; --l) {
      int64_t par0 = ((int64_t)1 << l) - 1;
      k_upward<TE, T><<<(unsigned)((int64_t)1 << l), transfer_threads(l), sm, st>>>((const TE *)d.Ef, m, k, rp, par0,
                                                                                   xhat);
      mk.count(H2_PH_UPWARD);
    }
  }
  mk.mark(H2_PH_COUPLING);
  if (far) {
    int64_t row0 = ((int64_t)1 << lmin) - 1;
    T *out = yhat + row0 * (int64_t)k * rp;
    if (gen) {
      if constexpr (std::is_same<T, float>::value) {
        CouplingGenRows rows{};
        rows.ptr = d.adm_ptr;
        rows.col = d.adm_col;
        rows.xhat = xhat;
        rows.dc = (const float4 *)d.adm_dc;
        rows.half = d.ihalf;
        for (int j = 0; j < kMaxM; ++j) rows.t[j] = j < m ? (float)std::cos((2 * j + 1) * 3.14159265358979323846 / (2.0 * m)) : 0.f;
        rows.m = m;
        rows.k = k;
        rows.kp = kp;
        rows.rp = rp;
        rows.row0 = row0;
        // the warp kernel indexes y^ by absolute cluster number: give it the base
        const int wr = regen_warp(rows, d.nclu - row0, yhat, st);
        if (wr < 0 && (rc = launch_rows<float, T>(rows, cf_cpl, t_cpl, Rk, d.nclu - row0, 0, out, st))) return rc;
      } else {
        return fail(H2_EINVAL, "the regenerated coupling runs in FP32 arithmetic only");
      }
    } else if (tcpath) {
      // FP64-accurate: integer slices on the tensor cores
      if ((rc = tc_coupling(c, xhat, yhat, rp))) return rc;
    } else {
      CouplingRows<TS, T> rows{(const TS *)d.S, d.adm_ptr, d.adm_col, xhat, k, kp, rp, row0};
      if ((rc = launch_rows<TS, T>(rows, cf_cpl, t_cpl, Rk, d.nclu - row0, 0, out, st))) return rc;
    }
    mk.count(H2_PH_COUPLING);
  }
  mk.mark(H2_PH_DOWNWARD);
  if (far && (m == 3 || m == 4)) {
    for (int l = lmin; l < D; ++l) {
      const int64_t np = (int64_t)1 << l;
      const dim3 grid((unsigned)((np + kSplitParents - 1) / kSplitParents), (rp + 15) / 16);
      if (m == 4) k_down_split<TE, T, 4><<<grid, 256, 0, st>>>((const TE *)d.Ef, rp, np - 1, np, yhat);
      else k_down_split<TE, T, 3><<<grid, 256, 0, st>>>((const TE *)d.Ef, rp, np - 1, np, yhat);
      mk.count(H2_PH_DOWNWARD);
    }
  } else if (far) {
    size_t sm = ((size_t)3 * k * rp + 6 * m * m) * sizeof(T);
    if ((rc = set_smem<T>((const void *)k_downward<TE, T>, sm))) return rc;
    for (int l = lmin; l < D; ++l) {
      int64_t par0 = ((int64_t)1 << l) - 1;
      k_downward<TE, T><<<(unsigned)((int64_t)1 << l), transfer_threads(l), sm, st>>>((const TE *)d.Ef, m, k, rp,
                                                                                     par0, yhat);
      mk.count(H2_PH_DOWNWARD);
    }
  }
  mk.mark(H2_PH_LEAF_NEAR);
  // bfloat16 handles: the FP32 self blocks join the leaf backward step when it runs per leaf
  const bool self_fused = far && leaf_reg && d.nself && std::is_same<T, float>::value;
  if (far && leaf_reg) {
    const size_t sm = ((size_t)k * (Lp + rp) + (self_fused ? (size_t)L * (Lp + rp) : 0)) * sizeof(T);
    k_leaf_bwd_reg<TV, T><<<(unsigned)d.nleaf, 256, sm, st>>>((const TV *)d.Vt, yhat + leaf0 * (int64_t)k * rp,
                                                             vscale, L, Lp, k, rp, self_fused ? d.nself : nullptr,
                                                             xpad, ypad);
    mk.count(H2_PH_LEAF_NEAR);
  } else if (far) {
    LeafBackwardRows<TV, T> rows{(const TV *)d.Vt, yhat, vscale, k, Lp, rp, leaf0};
    if ((rc = launch_rows<TV, T>(rows, cf_back, t_back, RL, d.nleaf, 0, ypad, st))) return rc;
    mk.count(H2_PH_LEAF_NEAR);
  }
  if (std::is_same<T, dd>::value && d.ntc && rp <= 16) {
    // FP64-accurate: integer digits on the tensor cores
    int64_t nl = 0;
    if ((rc = ntc_near(c, xpad, ypad, rp, far ? 1 : 0, &nl, leaf_tc))) return rc;
    mk.count(H2_PH_LEAF_NEAR, nl);
  } else if (d.nself) {
    // bfloat16: the blocks of other leaves, then the self blocks G_jj in FP32
    NearRows<TS, T> rows{(const TS *)d.near, d.near_ptr2, d.near_col2, xpad, nscale, L, Lp, rp, d.near_blk2};
    if ((rc = launch_rows<TS, T>(rows, cf_near, t_near, RL, d.nleaf, far ? 1 : 0, ypad, st))) return rc;
    mk.count(H2_PH_LEAF_NEAR);
    if constexpr (std::is_same<T, float>::value) {
      if (!self_fused) {
      RowCfg cf_self{};
      if ((rc = row_cfg<float, T>(L, Lp, rp, L, t_near, RL, false, cf_self))) return rc;
      NearRows<float, T> self{d.nself, d.self_ptr, d.self_col, xpad, nullptr, L, Lp, rp, nullptr};
      if ((rc = launch_rows<float, T>(self, cf_self, t_near, RL, d.nleaf, 1, ypad, st))) return rc;
      mk.count(H2_PH_LEAF_NEAR);
      }
    }
  } else {
    NearRows<TS, T> rows{(const TS *)d.near, d.near_ptr, d.near_col, xpad, nscale, L, Lp, rp, nullptr};
    if ((rc = launch_rows<TS, T>(rows, cf_near, t_near, RL, d.nleaf, far ? 1 : 0, ypad, st))) return rc;
    mk.count(H2_PH_LEAF_NEAR);
  }
  mk.mark(H2_PH_PERMUTE_OUT);
  k_permute_out<T, Tio><<<perm_grid, 256, (size_t)kPermRows * (rp + 1) * sizeof(T), st>>>(
      ypad, d.n, nrhs, rp, d.pad_src, d.npad, cmx, acc ? 1 : 0, y);
  mk.count(H2_PH_PERMUTE_OUT);
  mk.mark(H2_NPHASE);
  mk.finish();
  H2_CUDA_TRY(cudaGetLastError());
  d.last_nrhs = nrhs;
  d.last_rp = rp;
  return H2_OK;
}

// One block-row launch over nrows rows with output tiles of M rows (A rows
// padded to Mp) whose terms contract over at most Kmax: the warp-per-row
// kernel when warp is set, its lane tiles fit the registers and two buffers
// of four warps fit shared memory, else the pipelined block-row kernel.
template <class TS, class T, class Rows>
int gca_rows_launch(const Rows &rows, int M, int Mp, int Kmax, int rp, int64_t nrows, int accumulate, T *out,
                    cudaStream_t st, bool warp, int tmax = 256) {
  if (nrows <= 0) return H2_OK;
  if (warp) {
    constexpr int VN = Vec16<T>::N;
    const int tiles = (Mp / 4) * (rp / VN);
    const size_t per_warp = 2 * ((sizeof(TS) * Kmax * Mp + 15) / 16 * 16 + (sizeof(T) * Kmax * rp + 15) / 16 * 16);
    if (Mp % 4 == 0 && tiles <= 32 * 4 && 4 * per_warp <= kSmemMax) {
      const size_t sm = 4 * per_warp;
      int dev = 0, sms = 0, per_sm = 0;
      H2_CUDA_TRY(cudaGetDevice(&dev));
      H2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      auto go = [&](auto kern) -> int {
        if (sm > 48 * 1024)
          H2_CUDA_TRY(cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kSmemMax));
        H2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, sm));
        if (per_sm < 1) return fail(H2_EINVAL, "warp block-row kernel cannot be resident");
        const int64_t grid = std::min<int64_t>((nrows + 3) / 4, (int64_t)per_sm * sms);
        kern<<<(unsigned)grid, 128, sm, st>>>(rows, M, Mp, rp, Kmax, nrows, accumulate, out);
        return H2_OK;
      };
      if (tiles <= 32) return go(k_rows_warp<TS, T, 1, Rows>);
      if (tiles <= 64) return go(k_rows_warp<TS, T, 2, Rows>);
      return go(k_rows_warp<TS, T, 4, Rows>);
    }
  }
  const int R = row_groups<T>(Mp);
  int threads = row_threads(Mp, rp, Kmax, sizeof(T), R);
  {
    // at most tmax consumer threads (a smaller contraction split), as long as every tile keeps a thread
    constexpr int VN = Vec16<T>::N;
    const int tiles = (Mp / (4 * R)) * (rp / VN);
    while (threads > tmax && threads / 2 >= tiles) threads /= 2;
  }
  RowCfg cfg{};
  int rc;
  if ((rc = row_cfg<TS, T>(M, Mp, rp, Kmax, threads, R, false, cfg))) return rc;
  return launch_rows<TS, T>(rows, cfg, threads, R, nrows, accumulate, out, st);
}

// y = G~ x with a GCA-H^2 matrix (Algorithms 1-3 with the pivot bases):
// the same permutations, leaf steps and nearfield as the interpolation
// product, the transfer and coupling steps level by level with the level's
// padded rank.  Coefficients of level l start at gX[l] * rp.
template <class TS, class T, class Tio>
int matvec_gca(Ctx &c, const Tio *x, Tio *y, int nrhs, bool acc) {
  Dev &d = c.d;
  cudaStream_t st = c.stream;
  const int L = (int)d.lmax, Lp = (int)d.lp, D = d.depth, lmin = d.first_adm_level;
  const int rp = padded_rhs(nrhs, sizeof(T));
  // every output tile (the largest padded rank or leaf x the padded columns)
  // must fit the threads of one block-row CTA: refuse before any launch
  if ((int64_t)(std::max<int64_t>(d.k, Lp) / 4) * (rp / Vec16<T>::N) > kThreads)
    return fail(H2_EINVAL, "GCA-H^2 product: rank " + std::to_string(d.k) + " with " + std::to_string(nrhs) +
                               " right-hand sides exceeds one tile; use fewer right-hand sides per call");
  T *xpad = (T *)d.xpad, *ypad = (T *)d.ypad, *xhat = (T *)d.xhat, *yhat = (T *)d.yhat;
  const bool far = lmin <= D;
  int rc;
  Marks mk(c);
  mk.mark(H2_PH_PERMUTE_IN);
  const unsigned long long *cmx = std::is_same<T, dd>::value ? d.colmax : nullptr;
  if (cmx) {
    H2_CUDA_TRY(cudaMemsetAsync(d.colmax, 0, sizeof(unsigned long long) * nrhs, st));
    const int64_t nb = std::min<int64_t>((d.n + 8 * kThreads - 1) / (8 * kThreads), 64);
    k_colmax<Tio><<<dim3((unsigned)std::max<int64_t>(nb, 1), nrhs), kThreads, 0, st>>>(x, d.n, d.colmax);
    mk.count(H2_PH_PERMUTE_IN);
  }
  const unsigned perm_grid = (unsigned)((d.npad + kPermRows - 1) / kPermRows);
  k_permute_in<Tio, T><<<perm_grid, 256, (size_t)kPermRows * (rp + 1) * sizeof(T), st>>>(x, d.n, nrhs, rp, d.pad_src,
                                                                                        d.npad, cmx, xpad);
  mk.count(H2_PH_PERMUTE_IN);
  auto X = [&](T *base, int l) { return base + d.gX[l] * rp; };
  // FP32: the warp-per-row kernel for the transfer steps and the nearfield,
  // the pipelined block-row kernel for the coupling (measured at 327,680
  // triangles, 16 right-hand sides); double-float: the block-row kernel
  // throughout (its contraction split keeps more of the arithmetic busy)
  const bool wk = std::is_same<T, float>::value;
  // block-row threads: 128 for the double-float transfers and the FP32
  // coupling, 256 for the double-float coupling (measured at 327,680 triangles)
  const int t_tr = 128, t_cpl = std::is_same<T, float>::value ? 128 : 256;
  const int KD = d.gK[D];
  const bool leaf_reg = L <= 32 && KD <= 64 && rp <= 16;
  mk.mark(H2_PH_LEAF_FORWARD);
  if (far && leaf_reg) {
    const size_t sm = (size_t)L * (KD + rp) * sizeof(T);
    k_leaf_fwd_reg<TS, T><<<(unsigned)d.nleaf, 256, sm, st>>>((const TS *)d.V, xpad, nullptr, L, KD, KD, rp,
                                                             X(xhat, D));
    mk.count(H2_PH_LEAF_FORWARD);
  } else if (far) {
    LeafForwardRows<TS, T> rows{(const TS *)d.V, xpad, nullptr, L, KD, rp};
    if ((rc = gca_rows_launch<TS, T>(rows, KD, KD, L, rp, d.nleaf, 0, X(xhat, D), st, wk))) return rc;
    mk.count(H2_PH_LEAF_FORWARD);
  }
  mk.mark(H2_PH_UPWARD);
  for (int l = D; far && l > lmin; --l) {
    GcaUpRows<TS, T> rows{(const TS *)d.gE[l], X(xhat, l), d.gK[l], d.gK[l - 1], rp};
    if ((rc = gca_rows_launch<TS, T>(rows, d.gK[l - 1], d.gK[l - 1], d.gK[l], rp, (int64_t)1 << (l - 1), 0,
                                     X(xhat, l - 1), st, wk, t_tr)))
      return rc;
    mk.count(H2_PH_UPWARD);
  }
  mk.mark(H2_PH_COUPLING);
  for (int l = lmin; far && l <= D; ++l) {
    const int64_t c0 = ((int64_t)1 << l) - 1;
    GcaCouplingRows<TS, T> rows{(const TS *)d.gS[l], d.adm_ptr, d.adm_col, X(xhat, l), d.gK[l], rp, c0};
    if ((rc = gca_rows_launch<TS, T>(rows, d.gK[l], d.gK[l], d.gK[l], rp, (int64_t)1 << l, 0, X(yhat, l), st,
                                     false, t_cpl)))
      return rc;
    mk.count(H2_PH_COUPLING);
  }
  mk.mark(H2_PH_DOWNWARD);
  for (int l = lmin + 1; far && l <= D; ++l) {
    GcaDownRows<TS, T> rows{(const TS *)d.gEt[l], X(yhat, l - 1), d.gK[l], d.gK[l - 1], rp};
    if ((rc = gca_rows_launch<TS, T>(rows, d.gK[l], d.gK[l], d.gK[l - 1], rp, (int64_t)1 << l, 1, X(yhat, l), st,
                                     wk, t_tr)))
      return rc;
    mk.count(H2_PH_DOWNWARD);
  }
  mk.mark(H2_PH_LEAF_NEAR);
  if (far && leaf_reg) {
    const size_t sm = (size_t)KD * (Lp + rp) * sizeof(T);
    k_leaf_bwd_reg<TS, T><<<(unsigned)d.nleaf, 256, sm, st>>>((const TS *)d.Vt, X(yhat, D), nullptr, L, Lp, KD, rp,
                                                             nullptr, xpad, ypad);
    mk.count(H2_PH_LEAF_NEAR);
  } else if (far) {
    LeafBackwardRows<TS, T> rows{(const TS *)d.Vt, X(yhat, D), nullptr, KD, Lp, rp, 0};
    if ((rc = gca_rows_launch<TS, T>(rows, L, Lp, KD, rp, d.nleaf, 0, ypad, st, wk))) return rc;
    mk.count(H2_PH_LEAF_NEAR);
  }
  if (std::is_same<T, dd>::value && d.ntc && rp <= 16) {
    int64_t nl = 0;
    if ((rc = ntc_near(c, xpad, ypad, rp, far ? 1 : 0, &nl))) return rc;
    mk.count(H2_PH_LEAF_NEAR, nl);
  } else {
    NearRows<TS, T> rows{(const TS *)d.near, d.near_ptr, d.near_col, xpad, nullptr, L, Lp, rp, nullptr};
    if ((rc = gca_rows_launch<TS, T>(rows, L, Lp, L, rp, d.nleaf, far ? 1 : 0, ypad, st, wk))) return rc;
    mk.count(H2_PH_LEAF_NEAR);
  }
  mk.mark(H2_PH_PERMUTE_OUT);
  k_permute_out<T, Tio><<<perm_grid, 256, (size_t)kPermRows * (rp + 1) * sizeof(T), st>>>(
      ypad, d.n, nrhs, rp, d.pad_src, d.npad, cmx, acc ? 1 : 0, y);
  mk.count(H2_PH_PERMUTE_OUT);
  mk.mark(H2_NPHASE);
  mk.finish();
  H2_CUDA_TRY(cudaGetLastError());
  d.last_nrhs = nrhs;
  d.last_rp = rp;
  return H2_OK;
}

// ---------------------------------------------------------------- fused
// The whole product of a small FP64-accurate matrix in one cooperative
// launch (a latency path: at a few thousand triangles the separate
// launches of the phases cost more than their work).  Every warp of the
// grid computes whole outputs of a step (warp_dot), each step's outputs
// depending only on the previous steps' (Algorithms 1-3 in order): column
// maxima of x (range guard), x in the padded cluster order, the leaf
// forward step, the upward step level by level, the coupling, the downward
// step level by level, and the leaf backward step with the nearfield,
// written straight into the caller's order.  A
// grid-wide barrier separates the steps: a counter that every CTA
// increments, waited for with an iteration limit (on time-out the device
// error word is raised and every CTA leaves).
struct FusedArgs {
  const double *x;
  double *y;
  int64_t n;
  int nrhs, rp, acc;
  const int32_t *pad_src;
  int L, Lp, k, kp, m, D, lmin;
  int64_t nleaf, leaf0, nclu;
  const dd *V, *Vt, *Ef, *S, *near;
  const int64_t *adm_ptr, *near_ptr;
  const int32_t *adm_col, *near_col;
  dd *xpad, *xhat, *yhat;
  unsigned long long *colmax;
  unsigned *bar;   // [0] arrivals, [1] abort
};

constexpr uint32_t kFusedPolls = 1u << 24;
constexpr int kFusedThreads = 1024;   // one CTA of 32 warps per SM

// grid-wide barrier number g (0, 1, ...): false if it timed out or another CTA
// gave up
__device__ bool fused_barrier(const FusedArgs &a, unsigned g) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    // the CTA's stores of the step (ordered before this thread by the CTA
    // barrier) are made visible device-wide before its arrival counts
    __threadfence();
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(a.bar) : "memory");
    const unsigned target = (g + 1) * gridDim.x;
    uint32_t it = 0;
    unsigned v = 0, ab = 0;
    for (;;) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a.bar) : "memory");
      if (v >= target) break;
      if ((++it & 63) == 0) {
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(ab) : "l"(a.bar + 1) : "memory");
        if (ab || it >= kFusedPolls) break;
      }
    }
    ok = v >= target ? 1 : 0;
    __threadfence();
    if (!ok) {
      atomicExch(&a.bar[1], 1u);
      atomicExch(&g_h2_device_error, 1);
    }
  }
  __syncthreads();
  return ok != 0;
}

// x value of padding row src (-1: zero), column c, scaled by the column's
// range-guard power of two
__device__ __forceinline__ dd fused_x(const FusedArgs &a, int32_t src, int c, int sh) {
  if (src < 0) return zero_of<dd>();
  double v = a.x[src + (int64_t)c * a.n];
  if (sh) v = scale_pow2(v, sh);
  return dd_from_double(v);
}

// values written by other CTAs in an earlier step are read at the L2 level
// (the L1 of an SM is not coherent with the stores of other SMs, and a line
// it cached in an earlier step may hold stale neighbours)
__device__ __forceinline__ dd ld_cg(const dd *p) {
  const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
  return dd{v.x, v.y};
}

// transfer factor E_c[nu'][nu] = Ex[j'x][jx] Ey[j'y][jy] Ez[j'z][jz] (Eq. (9))
__device__ __forceinline__ dd fused_E(const FusedArgs &a, int64_t c, int nup, int nu) {
  const int m = a.m;
  const dd *f = a.Ef + c * 3 * m * m;
  const dd ex = f[(0 * m + nup % m) * m + nu % m];
  const dd ey = f[(1 * m + (nup / m) % m) * m + (nu / m) % m];
  const dd ez = f[(2 * m + nup / (m * m)) * m + nu / (m * m)];
  return ex * ey * ez;
}

// One output of a step, computed by a warp: lane l takes the terms l, l + 32,
// ... of the contraction (two double-float sums each), then the lanes'
// sums are added in a butterfly of fixed order; every lane returns the same
// value.  term(i, a, b) gives the factors of term i.
template <class F>
__device__ __forceinline__ dd warp_dot(int len, F term) {
  const int ln = threadIdx.x & 31;
  dd s0 = zero_of<dd>(), s1 = zero_of<dd>();
  int i = ln;
  for (; i + 32 < len; i += 64) {
    dd a0, b0, a1, b1;
    term(i, a0, b0);
    term(i + 32, a1, b1);
    acc_fma(s0, a0, b0);
    acc_fma(s1, a1, b1);
  }
  if (i < len) {
    dd a0, b0;
    term(i, a0, b0);
    acc_fma(s0, a0, b0);
  }
  acc_norm(s0);
  acc_norm(s1);
  dd s = s0 + s1;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const dd t{__shfl_xor_sync(0xffffffffu, s.hi, o), __shfl_xor_sync(0xffffffffu, s.lo, o)};
    s = s + t;
  }
  return s;
}

__global__ void __launch_bounds__(kFusedThreads) k_fused_dd(FusedArgs a) {
  __shared__ int shift[64];
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
  const int64_t gw = gt >> 5, nw = gs >> 5;
  const bool lead = (threadIdx.x & 31) == 0;
  const int k = a.k, nr = a.nrhs, rp = a.rp, L = a.L;
  const int64_t npad = a.nleaf * L;
  unsigned g = 0;
  // column maxima of x
  for (int c = 0; c < nr; ++c) {
    double mx = 0.0;
    for (int64_t i = gt; i < a.n; i += gs) mx = fmax(mx, fabs(a.x[i + (int64_t)c * a.n]));
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lead && mx > 0.0) atomicMax(&a.colmax[c], (unsigned long long)__double_as_longlong(mx));
  }
  if (!fused_barrier(a, g++)) return;
  if (threadIdx.x < 64) shift[threadIdx.x] = (int)threadIdx.x < nr ? range_shift(__ldcg(a.colmax + threadIdx.x)) : 0;
  __syncthreads();
  // x in the padded cluster order, scaled by the range guard (zero for padding)
  for (int64_t q = gt; q < npad * rp; q += gs) {
    const int64_t p = q / rp;
    const int c = (int)(q - p * rp);
    a.xpad[q] = c < nr ? fused_x(a, a.pad_src[p], c, shift[c]) : zero_of<dd>();
  }
  if (!fused_barrier(a, g++)) return;
  const bool far = a.lmin <= a.D;
  if (far) {
    // leaf forward: x^_j[nu][c] = sum_t V_j[t][nu] x[t][c]
    for (int64_t o = gw; o < a.nleaf * k * nr; o += nw) {
      const int64_t j = o / (k * nr);
      const int r = (int)(o - j * k * nr), nu = r % k, c = r / k;
      const dd v = warp_dot(L, [&](int t, dd &x, dd &y) {
        x = a.V[(j * L + t) * a.kp + nu];
        y = ld_cg(a.xpad + (j * L + t) * rp + c);
      });
      if (lead) a.xhat[((a.leaf0 + j) * k + nu) * rp + c] = v;
    }
    if (!fused_barrier(a, g++)) return;
    // upward: x^_p[nu][c] = sum over the sons s, nu' of E_s[nu'][nu] x^_s[nu'][c]
    for (int l = a.D - 1; l >= a.lmin; --l) {
      const int64_t p0 = ((int64_t)1 << l) - 1, np = (int64_t)1 << l;
      for (int64_t o = gw; o < np * k * nr; o += nw) {
        const int64_t p = p0 + o / (k * nr);
        const int r = (int)(o % (k * nr)), nu = r % k, c = r / k;
        const dd v = warp_dot(2 * k, [&](int i, dd &x, dd &y) {
          const int64_t ch = 2 * p + 1 + (i >= k);
          const int nup = i >= k ? i - k : i;
          x = fused_E(a, ch, nup, nu);
          y = ld_cg(a.xhat + (ch * k + nup) * rp + c);
        });
        if (lead) a.xhat[(p * k + nu) * rp + c] = v;
      }
      if (!fused_barrier(a, g++)) return;
    }
    // coupling: y^_t[nu][c] = sum over the admissible blocks (t, s), mu of S_b[mu][nu] x^_s[mu][c]
    const int64_t t0 = ((int64_t)1 << a.lmin) - 1;
    for (int64_t o = gw; o < (a.nclu - t0) * k * nr; o += nw) {
      const int64_t t = t0 + o / (k * nr);
      const int r = (int)(o % (k * nr)), nu = r % k, c = r / k;
      const int64_t b0 = a.adm_ptr[t];
      const dd v = warp_dot((int)(a.adm_ptr[t + 1] - b0) * k, [&](int i, dd &x, dd &y) {
        const int64_t b = b0 + i / k;
        const int mu = i % k;
        x = a.S[(b * k + mu) * a.kp + nu];
        y = ld_cg(a.xhat + ((int64_t)a.adm_col[b] * k + mu) * rp + c);
      });
      if (lead) a.yhat[(t * k + nu) * rp + c] = v;
    }
    if (!fused_barrier(a, g++)) return;
    // downward: y^_s[nu'][c] += sum_nu E_s[nu'][nu] y^_parent[nu][c]
    for (int l = a.lmin; l < a.D; ++l) {
      const int64_t c0 = ((int64_t)2 << l) - 1, nc = (int64_t)2 << l;
      for (int64_t o = gw; o < nc * k * nr; o += nw) {
        const int64_t ch = c0 + o / (k * nr), p = (ch - 1) / 2;
        const int r = (int)(o % (k * nr)), nup = r % k, c = r / k;
        const dd v = warp_dot(k, [&](int nu, dd &x, dd &y) {
          x = fused_E(a, ch, nup, nu);
          y = ld_cg(a.yhat + (p * k + nu) * rp + c);
        });
        if (lead) {
          dd *out = a.yhat + (ch * k + nup) * rp + c;
          *out = ld_cg(out) + v;
        }
      }
      if (!fused_barrier(a, g++)) return;
    }
  }
  // leaf backward and nearfield: y[t][c] = sum_nu V_j[t][nu] y^_j[nu][c] + sum over the near blocks of G_b x
  for (int64_t o = gw; o < npad * nr; o += nw) {
    const int64_t pr = o / nr;
    const int c = (int)(o - pr * nr);
    const int32_t dst = a.pad_src[pr];
    if (dst < 0) continue;
    const int64_t j = pr / L;
    const int t = (int)(pr - j * L);
    const int kf = far ? k : 0;
    const int64_t nb0 = a.near_ptr[j];
    const dd v = warp_dot(kf + (int)(a.near_ptr[j + 1] - nb0) * L, [&](int i, dd &x, dd &y) {
      if (i < kf) {
        x = a.Vt[(j * k + i) * a.Lp + t];
        y = ld_cg(a.yhat + ((a.leaf0 + j) * k + i) * rp + c);
      } else {
        const int64_t b = nb0 + (i - kf) / L;
        const int u = (i - kf) % L;
        x = a.near[(b * L + u) * a.Lp + t];
        y = ld_cg(a.xpad + ((int64_t)a.near_col[b] * L + u) * rp + c);
      }
    });
    if (lead) {
      double w = dd_to_double(v);
      if (shift[c]) w = scale_pow2(w, -shift[c]);
      double *out = a.y + dst + (int64_t)c * a.n;
      *out = a.acc ? *out + w : w;
    }
  }
}

// y = G~ x by k_fused_dd (one cooperative launch; see the kernel)
int matvec_fused(Ctx &c, const double *x, double *y, int nrhs, bool acc) {
  Dev &d = c.d;
  cudaStream_t st = c.stream;
  const int rp = padded_rhs(nrhs, sizeof(dd));
  Marks mk(c);
  for (int ph = H2_PH_PERMUTE_IN; ph <= H2_PH_COUPLING; ++ph) mk.mark(ph);
  H2_CUDA_TRY(cudaMemsetAsync(d.colmax, 0, sizeof(unsigned long long) * nrhs, st));
  H2_CUDA_TRY(cudaMemsetAsync(d.fbar, 0, 2 * sizeof(unsigned), st));
  FusedArgs a{};
  a.x = x;
  a.y = y;
  a.n = d.n;
  a.nrhs = nrhs;
  a.rp = rp;
  a.acc = acc ? 1 : 0;
  a.pad_src = d.pad_src;
  a.L = (int)d.lmax;
  a.Lp = (int)d.lp;
  a.k = d.k;
  a.kp = d.kp;
  a.m = d.m;
  a.D = d.depth;
  a.lmin = d.first_adm_level;
  a.nleaf = d.nleaf;
  a.leaf0 = d.nleaf - 1;
  a.nclu = d.nclu;
  a.V = (const dd *)d.V;
  a.Vt = (const dd *)d.Vt;
  a.Ef = (const dd *)d.Ef;
  a.S = (const dd *)d.S;
  a.near = (const dd *)d.near;
  a.adm_ptr = d.adm_ptr;
  a.near_ptr = d.near_ptr;
  a.adm_col = d.adm_col;
  a.near_col = d.near_col;
  a.xpad = (dd *)d.xpad;
  a.xhat = (dd *)d.xhat;
  a.yhat = (dd *)d.yhat;
  a.colmax = d.colmax;
  a.bar = d.fbar;
  int dev = 0, sms = 0, per_sm = 0;
  H2_CUDA_TRY(cudaGetDevice(&dev));
  H2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  H2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_dd, kFusedThreads, 0));
  if (per_sm < 1) return fail(H2_EINVAL, "the fused product kernel cannot be resident");
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)sms);
  cfg.blockDim = dim3(kFusedThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  H2_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_fused_dd, a));
  mk.count(H2_PH_COUPLING);
  for (int ph = H2_PH_DOWNWARD; ph <= H2_NPHASE; ++ph) mk.mark(ph);
  mk.finish();
  d.last_nrhs = nrhs;
  d.last_rp = rp;
  return H2_OK;
}

}  // namespace

int column_range_shift(unsigned long long bits) { return range_shift(bits); }

namespace {

// Self-test of the bounded waits: the pipeline of the block-row kernels in
// miniature.  Thread 0 of warp 1 (the producer) fills stages 0 .. kStages-2
// of a shared-memory ring with bulk copies of src, each completing on its
// mbarrier, and with withhold set never fills the last stage; thread 0 of
// warp 0 (the consumer) waits for every stage in order with the bounded
// wait (limit polls).  A withheld stage makes that wait run out: the error
// word is raised and the consumer leaves; the producer always waits for the
// copies it issued (they complete) before it leaves, so no copy is in flight
// when the CTA ends.  out[0] = stages the consumer saw complete.
constexpr int kSelfStages = 4;
constexpr uint32_t kSelfBytes = 4096;
__global__ void k_wait_selftest(const unsigned char *__restrict__ src, int withhold, uint32_t limit,
                                int *__restrict__ out) {
  __shared__ __align__(128) unsigned char buf[kSelfStages][kSelfBytes];
  __shared__ __align__(8) uint64_t full[kSelfStages];
  if (threadIdx.x == 0) {
    for (int i = 0; i < kSelfStages; ++i) mbar_init(&full[i], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 32) {
    const int nfill = withhold ? kSelfStages - 1 : kSelfStages;
    for (int i = 0; i < nfill; ++i) {
      mbar_expect_tx(&full[i], kSelfBytes);
      bulk_g2s(buf[i], src + (size_t)i * kSelfBytes, kSelfBytes, &full[i]);
    }
    for (int i = 0; i < nfill; ++i) mbar_wait_bounded(&full[i], 0);
  } else if (threadIdx.x == 0) {
    int seen = 0;
    for (int i = 0; i < kSelfStages; ++i) {
      if (!mbar_wait_bounded(&full[i], 0, limit)) break;
      ++seen;
    }
    out[0] = seen;
  }
  __syncthreads();
}

}  // namespace

int wait_selftest(Ctx &c, int withhold, uint32_t limit, int *stages_seen) {
  cudaStream_t st = c.stream;
  unsigned char *src = nullptr;
  int *out = nullptr;
  H2_CUDA_TRY(dmalloc(&src, (size_t)kSelfStages * kSelfBytes));
  if (dmalloc(&out, sizeof(int)) != cudaSuccess) {
    cudaFree(src);
    return fail(H2_ENOMEM, "self-test buffer");
  }
  cudaError_t e = cudaMemsetAsync(src, 0x5a, (size_t)kSelfStages * kSelfBytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(out, 0xff, sizeof(int), st);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 64, 0, st>>>(src, withhold, limit ? limit : kWaitPolls, out);
    e = cudaGetLastError();
  }
  int seen = -1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&seen, out, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(src);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
  if (stages_seen) *stages_seen = seen;
  return take_device_error(c);
}

int take_device_error(Ctx &c) {
  int v = 0, zero = 0;
  H2_CUDA_TRY(cudaMemcpyFromSymbolAsync(&v, g_h2_device_error, sizeof(int), 0, cudaMemcpyDeviceToHost, c.stream));
  H2_CUDA_TRY(cudaStreamSynchronize(c.stream));
  if (v) {
    H2_CUDA_TRY(cudaMemcpyToSymbolAsync(g_h2_device_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, c.stream));
    H2_CUDA_TRY(cudaStreamSynchronize(c.stream));
    return fail(H2_ETIMEOUT, "a bounded device wait ran out; the last result is not valid");
  }
  return (c.d.tc || c.d.ntc) ? tc_take_error(c.stream) : H2_OK;
}

int ensure_work(Ctx &c, int nrhs_req) {
  Dev &d = c.d;
  const int nrhs = padded_rhs(nrhs_req, d.esize);
  if (nrhs <= d.cap_nrhs) return H2_OK;
  cudaFree(d.xpad); cudaFree(d.ypad); cudaFree(d.xhat); cudaFree(d.yhat); cudaFree(d.io_x); cudaFree(d.io_y);
  d.xpad = d.ypad = d.xhat = d.yhat = nullptr;
  d.io_x = d.io_y = nullptr;
  d.cap_nrhs = 0;
  size_t es = d.esize;
  auto al = [](void **p, size_t b) { return dmalloc(p, b) == cudaSuccess; };
  bool ok = al(&d.xpad, es * d.npad * nrhs) && al(&d.ypad, es * d.npad * nrhs) &&
            al(&d.xhat, es * d.nclu * d.k * nrhs) && al(&d.yhat, es * d.nclu * d.k * nrhs) &&
            al((void **)&d.io_x, 8 * d.n * nrhs) && al((void **)&d.io_y, 8 * d.n * nrhs);
  if (!ok) {
    cudaGetLastError();
    return fail(H2_ENOMEM, "work buffers for " + std::to_string(nrhs) + " right-hand sides");
  }
  H2_CUDA_TRY(cudaMemsetAsync(d.xhat, 0, es * d.nclu * d.k * nrhs, c.stream));
  H2_CUDA_TRY(cudaMemsetAsync(d.yhat, 0, es * d.nclu * d.k * nrhs, c.stream));
  d.cap_nrhs = nrhs;
  d.work_gen++;
  return H2_OK;
}

int run_matvec(Ctx &c, const void *x, void *y, int nrhs, bool io64, bool acc) {
  Dev &d = c.d;
  if (nrhs < 1 || nrhs > 64) return fail(H2_EINVAL, "nrhs must be in [1, 64]");
  const int rp = padded_rhs(nrhs, d.esize);
  if ((int64_t)d.k * rp > kThreads * kMaxOut || d.lmax * rp > kThreads * kMaxOut)
    return fail(H2_EINVAL, "k * nrhs and leaf_max * nrhs (nrhs padded to 16 bytes) must not exceed 4096");
  int rc = ensure_work(c, nrhs);
  if (rc) return rc;
  using bf = __nv_bfloat16;
  const double *x64 = (const double *)x;
  double *y64 = (double *)y;
  const float *x32 = (const float *)x;
  float *y32 = (float *)y;
  if (d.fused && d.prec == H2_F64 && !d.gca && d.coupling == 0 && d.n <= kFusedMaxN)
    return matvec_fused(c, (const double *)x, (double *)y, nrhs, acc);
  if (d.gca) {
    switch (d.prec) {
      case H2_F64: return matvec_gca<dd, dd, double>(c, x64, y64, nrhs, acc);
      case H2_F64_NATIVE: return matvec_gca<double, double, double>(c, x64, y64, nrhs, acc);
      case H2_F32:
        if (io64) return matvec_gca<float, float, double>(c, x64, y64, nrhs, acc);
        return matvec_gca<float, float, float>(c, x32, y32, nrhs, acc);
      default: return fail(H2_EINVAL, "unknown precision");
    }
  }
  switch (d.prec) {
    case H2_F64: return matvec_typed<dd, dd, dd, dd, double>(c, x64, y64, nrhs, acc);
    case H2_F64_NATIVE: return matvec_typed<double, double, double, double, double>(c, x64, y64, nrhs, acc);
    case H2_F32:
      if (io64) return matvec_typed<float, float, float, float, double>(c, x64, y64, nrhs, acc);
      return matvec_typed<float, float, float, float, float>(c, x32, y32, nrhs, acc);
    case H2_BF16:
      // transfer factors in FP32 under bfloat16 storage (see the set-up); V in FP32 unless asked otherwise
      if (d.v32) {
        if (io64) return matvec_typed<bf, float, float, float, double>(c, x64, y64, nrhs, acc);
        return matvec_typed<bf, float, float, float, float>(c, x32, y32, nrhs, acc);
      }
      if (io64) return matvec_typed<bf, bf, float, float, double>(c, x64, y64, nrhs, acc);
      return matvec_typed<bf, bf, float, float, float>(c, x32, y32, nrhs, acc);
    case H2_F16:
      if (d.v32) {
        if (io64) return matvec_typed<__half, float, float, float, double>(c, x64, y64, nrhs, acc);
        return matvec_typed<__half, float, float, float, float>(c, x32, y32, nrhs, acc);
      }
      if (io64) return matvec_typed<__half, __half, __half, float, double>(c, x64, y64, nrhs, acc);
      return matvec_typed<__half, __half, __half, float, float>(c, x32, y32, nrhs, acc);
    default: return fail(H2_EINVAL, "unknown precision");
  }
}

}  // namespace h2
