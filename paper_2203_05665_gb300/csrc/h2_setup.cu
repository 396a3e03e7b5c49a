// Device-side set-up of the H^2 matrix: coupling matrices (Eq. (6c)) and
// Sauter-Schwab nearfield entries of the Galerkin matrix (Eq. (3)).
//
// Quadrature conventions (shared with nothing; restated from the published
// Sauter-Schwab method):
//   reference triangle {0 <= t <= s <= 1}, map A + s (B - A) + t (C - B),
//   Jacobian 2|T|; regular pairs: collapsed Gauss (s, t) = (u, u v) with
//   weight u and q points per direction, vertices in mesh order; pairs that
//   share vertices: q^4 Gauss points on [0,1]^4 over the method's regions,
//   canonical vertex order (identical: smallest id first, cyclic; edge:
//   smaller shared id, larger shared id, other; vertex: shared, then the
//   triangle's cyclic successors).  Each entry is evaluated with the
//   smaller triangle index as test triangle, so G is symmetric bit for bit.
#include <chrono>
#include <cstdio>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>

#include "h2_dd.cuh"
#include "h2_internal.hpp"
#include "h2_kernel.cuh"

namespace h2 {

namespace {

constexpr int kMaxQ = 16;

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}
__constant__ double c_gx[kMaxQ];
__constant__ double c_gw[kMaxQ];


__device__ __forceinline__ void tri_point(const double *A, const double *B, const double *C, double s, double t,
                                          double *x) {
#pragma unroll
  for (int d = 0; d < 3; ++d) x[d] = A[d] + s * (B[d] - A[d]) + t * (C[d] - B[d]);
}

// ---------------------------------------------------------------- coupling
// S_b stored transposed and padded: S[b][mu][nu], nu < kp, zero for nu >= k
template <class T>
__global__ void k_coupling_fill(const int32_t *__restrict__ row, const int32_t *__restrict__ col,
                                const double *__restrict__ cheb, int m, int kp, int64_t nblk, KernelFn kf,
                                T *__restrict__ S) {
  const int k = m * m * m;
  const int64_t per = (int64_t)k * kp, total = nblk * per;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = e / per;
    int rem = (int)(e - b * per);
    int mu = rem / kp, nu = rem - mu * kp;
    if (nu >= k) { S[e] = zero_of<T>(); continue; }
    int64_t t = row[b], s = col[b];
    double x[3], y[3];
    x[0] = cheb[(3 * t + 0) * m + nu % m];
    x[1] = cheb[(3 * t + 1) * m + (nu / m) % m];
    x[2] = cheb[(3 * t + 2) * m + nu / (m * m)];
    y[0] = cheb[(3 * s + 0) * m + mu % m];
    y[1] = cheb[(3 * s + 1) * m + (mu / m) % m];
    y[2] = cheb[(3 * s + 2) * m + mu / (m * m)];
    S[e] = from_double<T>(kernel_value(kf, x, y));
  }
}

// ---------------------------------------------------------------- nearfield
struct Geo {
  const double *vert;
  const int32_t *tri;
  const double *area;
  const int32_t *pad_src;
  const int32_t *blk_row;   // row leaf of each near block
  const int32_t *blk_col;   // column leaf of each near block
  int64_t lmax, lp;         // leaf height and its padding to a multiple of 4
  KernelFn kf;              // the kernel
};

// Nearfield block layout: entry (t, c) of block b (test triangle t of the
// row leaf, trial triangle c of the column leaf) at b L Lp + c Lp + t,
// i.e. stored transposed with the row index padded to Lp; padding is zero.
__device__ __forceinline__ void near_decode(const Geo &g, int64_t e, int64_t &b, int &t, int &c) {
  const int64_t per = g.lmax * g.lp;
  b = e / per;
  const int rc = (int)(e - b * per);
  c = rc / (int)g.lp;
  t = rc - c * (int)g.lp;
}

__device__ __forceinline__ int shared_count(const int32_t *a, const int32_t *b) {
  int c = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) c += (a[i] == b[j]);
  return c;
}

// Regular entries; entries whose triangles share a vertex are listed for the
// singular pass and left for it.
template <class T>
__global__ void k_near_regular(Geo g, int64_t nblk, int q, T *__restrict__ near, int64_t *__restrict__ sing,
                               unsigned long long *__restrict__ nsing, int64_t sing_cap) {
  const int64_t L = g.lmax, total = nblk * L * g.lp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t b;
    int r, c;
    near_decode(g, e, b, r, c);
    int32_t i = r < L ? g.pad_src[g.blk_row[b] * L + r] : -1, j = g.pad_src[g.blk_col[b] * L + c];
    if (i < 0 || j < 0) { near[e] = zero_of<T>(); continue; }
    if (i > j) { int32_t t = i; i = j; j = t; }
    int32_t ti[3] = {g.tri[3 * i], g.tri[3 * i + 1], g.tri[3 * i + 2]};
    int32_t tj[3] = {g.tri[3 * j], g.tri[3 * j + 1], g.tri[3 * j + 2]};
    if (shared_count(ti, tj) > 0) {
      unsigned long long slot = atomicAdd(nsing, 1ull);
      if ((int64_t)slot < sing_cap) sing[slot] = e;
      near[e] = zero_of<T>();
      continue;
    }
    const double *A1 = g.vert + 3 * ti[0], *B1 = g.vert + 3 * ti[1], *C1 = g.vert + 3 * ti[2];
    const double *A2 = g.vert + 3 * tj[0], *B2 = g.vert + 3 * tj[1], *C2 = g.vert + 3 * tj[2];
    double acc = 0.0;
    for (int a = 0; a < q; ++a)
      for (int bb = 0; bb < q; ++bb) {
        double x[3];
        tri_point(A1, B1, C1, c_gx[a], c_gx[a] * c_gx[bb], x);
        double wx = c_gw[a] * c_gw[bb] * c_gx[a];
        double inner = 0.0;
        for (int cc = 0; cc < q; ++cc)
          for (int dd = 0; dd < q; ++dd) {
            double y[3];
            tri_point(A2, B2, C2, c_gx[cc], c_gx[cc] * c_gx[dd], y);
            inner += c_gw[cc] * c_gw[dd] * c_gx[cc] * kernel_value(g.kf, x, y);
          }
        acc += wx * inner;
      }
    near[e] = from_double<T>(4.0 * g.area[i] * g.area[j] * acc);
  }
}

// Region r of the singular rules at (xi, e1, e2, e3): reference points of the
// test triangle (x1, x2) and of the trial triangle (y1, y2), and the weight.
// kind 3 = identical (6 regions), 2 = common edge (5), 1 = common vertex (2).
__device__ __forceinline__ double sing_region(int kind, int r, double xi, double e1, double e2, double e3,
                                              double *p) {
  if (kind == 3) {
    double w = xi * xi * xi * e1 * e1 * e2;
    double a = xi, b = xi * (1 - e1 + e1 * e2), c = xi * (1 - e1 * e2 * e3), d = xi * (1 - e1);
    double f = xi * e1 * (1 - e2 + e2 * e3), g = xi * (1 - e1 * e2), hh = xi * e1 * (1 - e2);
    double u = xi * e1 * (1 - e2 * e3);
    switch (r) {
      case 0: p[0] = a; p[1] = b; p[2] = c; p[3] = d; break;
      case 1: p[0] = c; p[1] = d; p[2] = a; p[3] = b; break;
      case 2: p[0] = a; p[1] = f; p[2] = g; p[3] = hh; break;
      case 3: p[0] = g; p[1] = hh; p[2] = a; p[3] = f; break;
      case 4: p[0] = c; p[1] = u; p[2] = a; p[3] = hh; break;
      default: p[0] = a; p[1] = hh; p[2] = c; p[3] = u; break;
    }
    return w;
  }
  if (kind == 2) {
    double w1 = xi * xi * xi * e1 * e1;
    switch (r) {
      case 0: p[0] = xi; p[1] = xi * e1 * e3; p[2] = xi * (1 - e1 * e2); p[3] = xi * e1 * (1 - e2); return w1;
      case 1: p[0] = xi; p[1] = xi * e1; p[2] = xi * (1 - e1 * e2 * e3); p[3] = xi * e1 * e2 * (1 - e3); return w1 * e2;
      case 2: p[0] = xi * (1 - e1 * e2); p[1] = xi * e1 * (1 - e2); p[2] = xi; p[3] = xi * e1 * e2 * e3; return w1 * e2;
      case 3: p[0] = xi * (1 - e1 * e2 * e3); p[1] = xi * e1 * e2 * (1 - e3); p[2] = xi; p[3] = xi * e1; return w1 * e2;
      default: p[0] = xi * (1 - e1 * e2 * e3); p[1] = xi * e1 * (1 - e2 * e3); p[2] = xi; p[3] = xi * e1 * e2; return w1 * e2;
    }
  }
  double w = xi * xi * xi * e2;
  if (r == 0) { p[0] = xi; p[1] = xi * e1; p[2] = xi * e2; p[3] = xi * e2 * e3; }
  else { p[0] = xi * e2; p[1] = xi * e2 * e3; p[2] = xi; p[3] = xi * e1; }
  return w;
}

template <class T>
__global__ void k_near_singular(Geo g, const int64_t *__restrict__ sing, int64_t nsing, int q, T *__restrict__ near) {
  const int64_t L = g.lmax;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nsing; s += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = sing[s];
    int64_t b;
    int r, c;
    near_decode(g, e, b, r, c);
    int32_t i = g.pad_src[g.blk_row[b] * L + r], j = g.pad_src[g.blk_col[b] * L + c];
    if (i > j) { int32_t t = i; i = j; j = t; }
    int32_t ti[3] = {g.tri[3 * i], g.tri[3 * i + 1], g.tri[3 * i + 2]};
    int32_t tj[3] = {g.tri[3 * j], g.tri[3 * j + 1], g.tri[3 * j + 2]};
    int ns = shared_count(ti, tj);
    int32_t P[3], Q[3];   // canonical local vertex orders
    if (ns >= 3) {
      int a = 0;
      if (ti[1] < ti[a]) a = 1;
      if (ti[2] < ti[a]) a = 2;
      for (int v = 0; v < 3; ++v) P[v] = Q[v] = ti[(a + v) % 3];
    } else if (ns == 2) {
      int32_t s0 = -1, s1 = -1, oi = -1, oj = -1;
      for (int v = 0; v < 3; ++v) {
        bool in = (ti[v] == tj[0]) || (ti[v] == tj[1]) || (ti[v] == tj[2]);
        if (in) { if (s0 < 0) s0 = ti[v]; else s1 = ti[v]; } else oi = ti[v];
        bool inj = (tj[v] == ti[0]) || (tj[v] == ti[1]) || (tj[v] == ti[2]);
        if (!inj) oj = tj[v];
      }
      int32_t lo_ = s0 < s1 ? s0 : s1, hi_ = s0 < s1 ? s1 : s0;
      P[0] = lo_; P[1] = hi_; P[2] = oi;
      Q[0] = lo_; Q[1] = hi_; Q[2] = oj;
    } else {
      int a = 0, bb = 0;
      for (int u = 0; u < 3; ++u)
        for (int v = 0; v < 3; ++v)
          if (ti[u] == tj[v]) { a = u; bb = v; }
      for (int v = 0; v < 3; ++v) { P[v] = ti[(a + v) % 3]; Q[v] = tj[(bb + v) % 3]; }
    }
    const double *A1 = g.vert + 3 * P[0], *B1 = g.vert + 3 * P[1], *C1 = g.vert + 3 * P[2];
    const double *A2 = g.vert + 3 * Q[0], *B2 = g.vert + 3 * Q[1], *C2 = g.vert + 3 * Q[2];
    int kind = ns >= 3 ? 3 : ns;
    int nreg = kind == 3 ? 6 : (kind == 2 ? 5 : 2);
    double acc = 0.0;
    for (int i0 = 0; i0 < q; ++i0)
      for (int i1 = 0; i1 < q; ++i1)
        for (int i2 = 0; i2 < q; ++i2)
          for (int i3 = 0; i3 < q; ++i3) {
            double part = 0.0;
            for (int rg = 0; rg < nreg; ++rg) {
              double pr[4];
              double w = sing_region(kind, rg, c_gx[i0], c_gx[i1], c_gx[i2], c_gx[i3], pr);
              double x[3], y[3];
              tri_point(A1, B1, C1, pr[0], pr[1], x);
              tri_point(A2, B2, C2, pr[2], pr[3], y);
              part += w * kernel_value(g.kf, x, y);
            }
            acc += c_gw[i0] * c_gw[i1] * c_gw[i2] * c_gw[i3] * part;
          }
    near[e] = from_double<T>(4.0 * g.area[i] * g.area[j] * acc);
  }
}

// rounding of an FP64 value to the stored type
template <class T>
__device__ __forceinline__ T store_as(double v) {
  return from_double<T>(v);
}
template <>
__device__ __forceinline__ __nv_bfloat16 store_as<__nv_bfloat16>(double v) {
  return __double2bfloat16(v);
}
template <>
__device__ __forceinline__ __half store_as<__half>(double v) {
  return __double2half(v);
}

template <class T>
__global__ void k_convert(const double *__restrict__ src, T *__restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = store_as<T>(src[i]);
}

// per nearfield block: the power of two 2^e >= max |entry| (1 for an all-zero block)
__global__ void k_block_scale(const double *__restrict__ near, int64_t per, int64_t nblk, float *__restrict__ scale) {
  for (int64_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    double mx = 0.0;
    for (int64_t i = threadIdx.x; i < per; i += blockDim.x) mx = fmax(mx, fabs(near[b * per + i]));
    __shared__ double part[256];
    part[threadIdx.x] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) part[threadIdx.x] = fmax(part[threadIdx.x], part[threadIdx.x + w]);
      __syncthreads();
    }
    if (threadIdx.x == 0) scale[b] = part[0] > 0.0 ? (float)exp2(ceil(log2(part[0]))) : 1.0f;
    __syncthreads();
  }
}

// stored = value / scale (exact: a power of two) in the stored type
template <class T>
__global__ void k_convert_scaled(const double *__restrict__ src, const float *__restrict__ scale, int64_t per,
                                 T *__restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = store_as<T>(scale ? src[i] / (double)scale[i / per] : src[i]);
}

int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 64) g = 152 * 64;
  return (int)g;
}

template <class T>
int upload_converted(Dev &d, void **dst, const std::vector<double> &src, cudaStream_t st);

// ---------------------------------------------------------------- bases
// 1-D Lagrange polynomial i of the nodes z[0..m) at x, product form
__device__ __forceinline__ double lagrange1(const double *z, int m, int i, double x) {
  double v = 1.0;
  for (int j = 0; j < m; ++j)
    if (j != i) v *= (x - z[j]) / (z[i] - z[j]);
  return v;
}

// Collapsed Gauss rule of the leaf bases (exact for total degree 3(m-1)).
struct BasisRule {
  int q;
  double x[16], w[16];
};

// V64[p][nu] = int_{T} ell_{c,nu} (Eq. (6a)) for padded DoF p (triangle
// pad_src[p] of leaf p / L, cluster leaf0 + p / L), zero for padding rows;
// ell_{c,nu} = ell_x ell_y ell_z on the cluster's Chebyshev nodes.  One
// thread per (p, z index): the 1-D Lagrange values at a quadrature point are
// formed once (in the barycentric form w_i prod_{j != i} (x - z_j)) and serve
// all m^2 entries of that z slab.
template <int M>
__global__ void k_leaf_bases(const double *__restrict__ vert, const int32_t *__restrict__ tri,
                             const double *__restrict__ area, const int32_t *__restrict__ pad_src,
                             const double *__restrict__ cheb, int L, int64_t leaf0, int64_t npad, BasisRule rule,
                             double *__restrict__ V64) {
  constexpr int K = M * M * M;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < npad * M; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / M;
    const int iz = (int)(e - p * M);
    double *row = V64 + p * K + M * M * iz;
    const int32_t t = pad_src[p];
    if (t < 0) {
      for (int q = 0; q < M * M; ++q) row[q] = 0.0;
      continue;
    }
    const int64_t c = leaf0 + p / L;
    double z[3][M], w[3][M];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int i = 0; i < M; ++i) z[d][i] = cheb[(3 * c + d) * M + i];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int i = 0; i < M; ++i) {
        double den = 1.0;
#pragma unroll
        for (int j = 0; j < M; ++j)
          if (j != i) den *= z[d][i] - z[d][j];
        w[d][i] = 1.0 / den;
      }
    const double *A = vert + 3 * (int64_t)tri[3 * (int64_t)t], *B = vert + 3 * (int64_t)tri[3 * (int64_t)t + 1],
                 *C = vert + 3 * (int64_t)tri[3 * (int64_t)t + 2];
    double acc[M * M];
#pragma unroll
    for (int q = 0; q < M * M; ++q) acc[q] = 0.0;
    for (int a = 0; a < rule.q; ++a)
      for (int b = 0; b < rule.q; ++b) {
        const double s = rule.x[a], tt = rule.x[a] * rule.x[b];
        const double wgt = 2.0 * area[t] * rule.w[a] * rule.w[b] * rule.x[a];
        double x[3];
        tri_point(A, B, C, s, tt, x);
        double l[3][M];
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int i = 0; i < M; ++i) {
            double v = w[d][i];
#pragma unroll
            for (int j = 0; j < M; ++j)
              if (j != i) v *= x[d] - z[d][j];
            l[d][i] = v;
          }
        const double wz = wgt * l[2][iz];
#pragma unroll
        for (int iy = 0; iy < M; ++iy)
#pragma unroll
          for (int ix = 0; ix < M; ++ix) acc[iy * M + ix] += wz * (l[0][ix] * l[1][iy]);
      }
#pragma unroll
    for (int q = 0; q < M * M; ++q) row[q] = acc[q];
  }
}

template <int M>
void launch_leaf_bases(const double *vert, const int32_t *tri, const double *area, const int32_t *pad_src,
                       const double *cheb, int L, int64_t leaf0, int64_t npad, const BasisRule &rule, double *V64,
                       cudaStream_t st) {
  k_leaf_bases<M><<<grid_for(npad * M, 128), 128, 0, st>>>(vert, tri, area, pad_src, cheb, L, leaf0, npad, rule, V64);
}

void leaf_bases(int m, const double *vert, const int32_t *tri, const double *area, const int32_t *pad_src,
                const double *cheb, int L, int64_t leaf0, int64_t npad, const BasisRule &rule, double *V64,
                cudaStream_t st) {
  switch (m) {
    case 1: launch_leaf_bases<1>(vert, tri, area, pad_src, cheb, L, leaf0, npad, rule, V64, st); break;
    case 2: launch_leaf_bases<2>(vert, tri, area, pad_src, cheb, L, leaf0, npad, rule, V64, st); break;
    case 3: launch_leaf_bases<3>(vert, tri, area, pad_src, cheb, L, leaf0, npad, rule, V64, st); break;
    case 4: launch_leaf_bases<4>(vert, tri, area, pad_src, cheb, L, leaf0, npad, rule, V64, st); break;
    case 5: launch_leaf_bases<5>(vert, tri, area, pad_src, cheb, L, leaf0, npad, rule, V64, st); break;
    default: launch_leaf_bases<6>(vert, tri, area, pad_src, cheb, L, leaf0, npad, rule, V64, st); break;
  }
}

// per leaf: the power of two 2^e >= max |V| of its rows (half storage)
__global__ void k_leaf_scale(const double *__restrict__ V64, int64_t per, int64_t nleaf, float *__restrict__ scale) {
  for (int64_t j = blockIdx.x; j < nleaf; j += gridDim.x) {
    double mx = 0.0;
    for (int64_t i = threadIdx.x; i < per; i += blockDim.x) mx = fmax(mx, fabs(V64[j * per + i]));
    __shared__ double part[256];
    part[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
      if ((int)threadIdx.x < o) part[threadIdx.x] = fmax(part[threadIdx.x], part[threadIdx.x + o]);
      __syncthreads();
    }
    if (threadIdx.x == 0) scale[j] = part[0] > 0.0 ? (float)exp2(ceil(log2(part[0]))) : 1.0f;
    __syncthreads();
  }
}

// the two stored layouts of V: [leaf][t][kp] (forward) and [leaf][nu][Lp]
// (backward), zero padded, divided by the leaf's scale if there is one
template <class T>
__global__ void k_store_bases(const double *__restrict__ V64, const float *__restrict__ scale, int k, int kp, int L,
                              int Lp, int64_t nleaf, T *__restrict__ V, T *__restrict__ Vt) {
  const int64_t perF = (int64_t)L * kp, perB = (int64_t)k * Lp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nleaf * perF; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / perF;
    const int r = (int)((e - j * perF) / kp), nu = (int)((e - j * perF) % kp);
    const double v = nu < k ? V64[(j * L + r) * k + nu] : 0.0;
    V[e] = store_as<T>(scale ? v / (double)scale[j] : v);
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nleaf * perB; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / perB;
    const int nu = (int)((e - j * perB) / Lp), r = (int)((e - j * perB) % Lp);
    const double v = r < L ? V64[(j * L + r) * k + nu] : 0.0;
    Vt[e] = store_as<T>(scale ? v / (double)scale[j] : v);
  }
}

// transfer factors (Eq. (9)): E_c = Ex (x) Ey (x) Ez, Ed[j'][j] = the parent's
// Lagrange polynomial j at the child's node j'; zero for the root
template <class T>
__global__ void k_transfer_factors(const double *__restrict__ cheb, int m, int64_t nclu, T *__restrict__ Ef) {
  const int64_t per = 3 * (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nclu * per; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / per;
    const int rem = (int)(e - c * per), d = rem / (m * m), jp = (rem / m) % m, j = rem % m;
    double v = 0.0;
    if (c > 0) {
      const int64_t par = (c - 1) / 2;
      v = lagrange1(cheb + (3 * par + d) * m, m, j, cheb[(3 * c + d) * m + jp]);
    }
    Ef[e] = store_as<T>(v);
  }
}

// self[j] = the self block of leaf j (the inadmissible block (j, j), stored
// transposed [c][t], L x Lp entries) rounded to FP32; the block is zeroed in
// the staging array.  selfblk[j] = index of that block.
__global__ void k_split_self(const int32_t *__restrict__ selfblk, int64_t nleaf, int64_t per,
                             double *__restrict__ near, float *__restrict__ self) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nleaf * per; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / per, q = e - j * per;
    double *src = near + (int64_t)selfblk[j] * per + q;
    self[e] = (float)*src;
    *src = 0.0;
  }
}

template <class T>
constexpr bool is_half_type() {
  return std::is_same<T, __nv_bfloat16>::value || std::is_same<T, __half>::value;
}

template <class T>
int upload_converted(Dev &d, void **dst, const std::vector<double> &src, cudaStream_t st) {
  int rc = dev_alloc(d, dst, src.size() * sizeof(T));
  if (rc) return rc;
  if (src.empty()) return H2_OK;
  double *tmp = nullptr;
  H2_CUDA_TRY(dmalloc(&tmp, src.size() * sizeof(double)));
  cudaError_t e = cudaMemcpyAsync(tmp, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_convert<T><<<grid_for((int64_t)src.size(), 256), 256, 0, st>>>(tmp, (T *)*dst, (int64_t)src.size());
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "upload");
  return H2_OK;
}

template <class T>
int build_typed(Ctx &c) {
  Plan &p = c.plan;
  Dev &d = c.d;
  cudaStream_t st = c.stream;
  const int m = p.m, k = p.k;
  const int64_t L = p.lmax;

  // padded DoF layout: leaf j owns rows [j L, j L + size_j)
  std::vector<int32_t> pad(d.npad, -1);
  for (int64_t j = 0; j < p.nleaf; ++j) {
    int64_t c0 = p.leaf0 + j;
    for (int64_t r = 0; r < p.size[c0]; ++r) pad[j * L + r] = (int32_t)p.perm[p.first[c0] + r];
  }
  int rc;
  if ((rc = dev_alloc(d, (void **)&d.pad_src, pad.size() * 4))) return rc;
  H2_CUDA_TRY(cudaMemcpyAsync(d.pad_src, pad.data(), pad.size() * 4, cudaMemcpyHostToDevice, st));
  if ((rc = dev_alloc(d, (void **)&d.cheb, p.cheb.size() * 8))) return rc;
  H2_CUDA_TRY(cudaMemcpyAsync(d.cheb, p.cheb.data(), p.cheb.size() * 8, cudaMemcpyHostToDevice, st));

  // temporary geometry for the set-up kernels
  struct Tmp {
    void *ptr = nullptr;
    ~Tmp() { if (ptr) cudaFree(ptr); }
  } t_arow, t_nrow, t_ncol, t_vert, t_tri, t_area, t_sing, t_cnt, t_v64;
  auto tmp_up = [&](Tmp &t, const void *src, size_t bytes) -> int {
    if (dmalloc(&t.ptr, std::max<size_t>(bytes, 16)) != cudaSuccess) return fail(H2_ENOMEM, "device set-up buffer");
    if (bytes) H2_CUDA_TRY(cudaMemcpyAsync(t.ptr, src, bytes, cudaMemcpyHostToDevice, st));
    return H2_OK;
  };
  if ((rc = tmp_up(t_vert, p.vert.data(), p.vert.size() * 8))) return rc;
  if ((rc = tmp_up(t_tri, p.tri.data(), p.tri.size() * 4))) return rc;
  if ((rc = tmp_up(t_area, p.area.data(), p.area.size() * 8))) return rc;

  // leaf bases V (Eq. (6a)) on the device: FP64 quadrature, then the two
  // stored layouts [L][kp] (forward step, x^ = V^T x) and transposed [k][Lp]
  // (backward step); FP16 storage divides every leaf by a power of two >= its
  // largest entry
  const int64_t kp = d.kp, Lp = d.lp;
  const auto tb0 = std::chrono::steady_clock::now();
  if (!d.gca) {
    BasisRule rule{};
    rule.q = (3 * (m - 1) + 3) / 2 + 1;
    std::vector<double> bx, bw;
    gauss_legendre01(rule.q, bx, bw);
    for (int i = 0; i < rule.q; ++i) {
      rule.x[i] = bx[i];
      rule.w[i] = bw[i];
    }
    if (dmalloc(&t_v64.ptr, std::max<size_t>(16, (size_t)d.npad * k * 8)) != cudaSuccess)
      return fail(H2_ENOMEM, "leaf basis staging buffer");
    leaf_bases(m, (const double *)t_vert.ptr, (const int32_t *)t_tri.ptr, (const double *)t_area.ptr, d.pad_src,
               d.cheb, (int)L, p.leaf0, d.npad, rule, (double *)t_v64.ptr, st);
    H2_CUDA_TRY(cudaGetLastError());
    const bool half_v = std::is_same<T, __half>::value && !d.v32;
    if (half_v) {
      if ((rc = dev_alloc(d, (void **)&d.vscale, p.nleaf * 4))) return rc;
      k_leaf_scale<<<(unsigned)std::min<int64_t>(p.nleaf, 152 * 32), 256, 0, st>>>((const double *)t_v64.ptr, L * k,
                                                                                  p.nleaf, d.vscale);
      H2_CUDA_TRY(cudaGetLastError());
    }
    const int64_t nv = std::max<int64_t>(p.nleaf * L * kp, p.nleaf * k * Lp);
    if (d.v32) {
      if ((rc = dev_alloc(d, &d.V, (size_t)p.nleaf * L * kp * 4))) return rc;
      if ((rc = dev_alloc(d, &d.Vt, (size_t)p.nleaf * k * Lp * 4))) return rc;
      k_store_bases<float><<<grid_for(nv, 256), 256, 0, st>>>((const double *)t_v64.ptr, nullptr, k, (int)kp, (int)L,
                                                              (int)Lp, p.nleaf, (float *)d.V, (float *)d.Vt);
    } else {
      if ((rc = dev_alloc(d, &d.V, (size_t)p.nleaf * L * kp * sizeof(T)))) return rc;
      if ((rc = dev_alloc(d, &d.Vt, (size_t)p.nleaf * k * Lp * sizeof(T)))) return rc;
      k_store_bases<T><<<grid_for(nv, 256), 256, 0, st>>>((const double *)t_v64.ptr, half_v ? d.vscale : nullptr, k,
                                                          (int)kp, (int)L, (int)Lp, p.nleaf, (T *)d.V, (T *)d.Vt);
    }
    H2_CUDA_TRY(cudaGetLastError());
    // transfer factors: FP32 under bfloat16 storage, whose 8-bit significand would
    // compound over the tree levels of the transfer passes (0.2 % of the bytes),
    // and with FP32 leaf bases
    const int64_t ne = p.nclu * 3 * m * m;
    if (std::is_same<T, __nv_bfloat16>::value || d.v32) {
      if ((rc = dev_alloc(d, &d.Ef, (size_t)ne * 4))) return rc;
      k_transfer_factors<float><<<grid_for(ne, 256), 256, 0, st>>>(d.cheb, m, p.nclu, (float *)d.Ef);
    } else {
      if ((rc = dev_alloc(d, &d.Ef, (size_t)ne * sizeof(T)))) return rc;
      k_transfer_factors<T><<<grid_for(ne, 256), 256, 0, st>>>(d.cheb, m, p.nclu, (T *)d.Ef);
    }
    H2_CUDA_TRY(cudaGetLastError());
    H2_CUDA_TRY(cudaStreamSynchronize(st));
  }
  c.build_ms[H2_BUILD_BASES] = ms_since(tb0);
  cudaFree(t_v64.ptr);
  t_v64.ptr = nullptr;
  if ((rc = dev_alloc(d, (void **)&d.adm_ptr, p.adm_ptr.size() * 8))) return rc;
  H2_CUDA_TRY(cudaMemcpyAsync(d.adm_ptr, p.adm_ptr.data(), p.adm_ptr.size() * 8, cudaMemcpyHostToDevice, st));
  if ((rc = dev_alloc(d, (void **)&d.adm_col, std::max<size_t>(1, p.adm_col.size()) * 4))) return rc;
  if (!p.adm_col.empty())
    H2_CUDA_TRY(cudaMemcpyAsync(d.adm_col, p.adm_col.data(), p.adm_col.size() * 4, cudaMemcpyHostToDevice, st));
  if ((rc = dev_alloc(d, (void **)&d.near_ptr, p.near_ptr.size() * 8))) return rc;
  H2_CUDA_TRY(cudaMemcpyAsync(d.near_ptr, p.near_ptr.data(), p.near_ptr.size() * 8, cudaMemcpyHostToDevice, st));
  if ((rc = dev_alloc(d, (void **)&d.near_col, std::max<size_t>(1, p.near_col.size()) * 4))) return rc;
  if (!p.near_col.empty())
    H2_CUDA_TRY(cudaMemcpyAsync(d.near_col, p.near_col.data(), p.near_col.size() * 4, cudaMemcpyHostToDevice, st));
  const auto tc0 = std::chrono::steady_clock::now();
  if (d.coupling == 1) {
    // regenerated coupling: interpolation-box centres (FP64) and half widths (FP32)
    std::vector<float> hw(p.ihalf.begin(), p.ihalf.end());
    if ((rc = dev_alloc(d, (void **)&d.icen, p.icen.size() * 8))) return rc;
    H2_CUDA_TRY(cudaMemcpyAsync(d.icen, p.icen.data(), p.icen.size() * 8, cudaMemcpyHostToDevice, st));
    if ((rc = dev_alloc(d, (void **)&d.ihalf, hw.size() * 4))) return rc;
    H2_CUDA_TRY(cudaMemcpyAsync(d.ihalf, hw.data(), hw.size() * 4, cudaMemcpyHostToDevice, st));
    // per admissible block the gap of the box centres, formed in FP64, rounded once
    std::vector<float> dc(4 * std::max<size_t>(1, p.adm_col.size()), 0.0f);
    for (int64_t t = 0; t < p.nclu; ++t)
      for (int64_t e = p.adm_ptr[t]; e < p.adm_ptr[t + 1]; ++e)
        for (int q = 0; q < 3; ++q) dc[4 * e + q] = (float)(p.icen[3 * t + q] - p.icen[3 * p.adm_col[e] + q]);
    if ((rc = dev_alloc(d, (void **)&d.adm_dc, dc.size() * 4))) return rc;
    H2_CUDA_TRY(cudaMemcpyAsync(d.adm_dc, dc.data(), dc.size() * 4, cudaMemcpyHostToDevice, st));
    H2_CUDA_TRY(cudaStreamSynchronize(st));
  }

  // temporary geometry for the set-up kernels
  std::vector<int32_t> arow(p.adm_col.size()), nrow(p.near_col.size()), ncol(p.near_col.size());
  for (int64_t t = 0; t < p.nclu; ++t)
    for (int64_t e = p.adm_ptr[t]; e < p.adm_ptr[t + 1]; ++e) arow[e] = (int32_t)t;
  for (int64_t j = 0; j < p.nleaf; ++j)
    for (int64_t e = p.near_ptr[j]; e < p.near_ptr[j + 1]; ++e) {
      nrow[e] = (int32_t)j;
      ncol[e] = p.near_col[e];
    }
  if ((rc = tmp_up(t_arow, arow.data(), arow.size() * 4))) return rc;
  if ((rc = tmp_up(t_nrow, nrow.data(), nrow.size() * 4))) return rc;
  if ((rc = tmp_up(t_ncol, ncol.data(), ncol.size() * 4))) return rc;

  // Gauss rule of the nearfield quadrature
  std::vector<double> gx, gw;
  gauss_legendre01(c.quad_order, gx, gw);
  H2_CUDA_TRY(cudaMemcpyToSymbolAsync(c_gx, gx.data(), gx.size() * 8, 0, cudaMemcpyHostToDevice, st));
  H2_CUDA_TRY(cudaMemcpyToSymbolAsync(c_gw, gw.data(), gw.size() * 8, 0, cudaMemcpyHostToDevice, st));

  // GCA-H^2: pivots, leaf bases, transfer and coupling matrices
  if (d.gca) {
    if ((rc = gca_build(c, (const double *)t_vert.ptr, (const int32_t *)t_tri.ptr, (const double *)t_area.ptr)))
      return rc;
  }
  // coupling matrices (stored mode)
  if (!d.gca && d.coupling == 0 &&
      (rc = dev_alloc(d, &d.S, std::max<size_t>(1, (size_t)d.nadm * k * d.kp) * sizeof(T))))
    return rc;
  if (!d.gca && d.coupling == 0 && d.nadm > 0) {
    k_coupling_fill<T><<<grid_for(d.nadm * k * d.kp, 256), 256, 0, st>>>((const int32_t *)t_arow.ptr, d.adm_col,
                                                                          d.cheb, m, d.kp, d.nadm, d.kernel,
                                                                          (T *)d.S);
    H2_CUDA_TRY(cudaGetLastError());
  }
  // FP64 and FP32 handles of order 4: the E4M3 digit planes for the tensor-core coupling
  if (!d.gca && d.tensor == 0 && tc_eligible(d) && (rc = tc_build(c, (const int32_t *)t_arow.ptr))) return rc;
  H2_CUDA_TRY(cudaStreamSynchronize(st));
  c.build_ms[H2_BUILD_COUPLING] = ms_since(tc0) - (d.gca ? c.build_ms[H2_BUILD_BASES] : 0.0);
  const auto tn0 = std::chrono::steady_clock::now();


  // nearfield entries; 16-bit storage: computed in FP64 first, then rounded
  // (FP16: with a power-of-two scale per block)
  if ((rc = dev_alloc(d, &d.near, std::max<size_t>(1, (size_t)d.nnear * L * Lp) * sizeof(T)))) return rc;
  Tmp t_near64;
  using TQ = typename std::conditional<is_half_type<T>(), double, T>::type;
  TQ *qnear = (TQ *)d.near;
  if (is_half_type<T>()) {
    if (dmalloc(&t_near64.ptr, std::max<size_t>(1, (size_t)d.nnear * L * Lp) * 8) != cudaSuccess)
      return fail(H2_ENOMEM, "nearfield staging buffer");
    qnear = (TQ *)t_near64.ptr;
  }
  if (d.nnear > 0) {
    // pairs that share a vertex: at most (n * 3 * valence) ordered pairs; bound by the entry count
    int64_t cap = std::min<int64_t>(d.nnear * L * Lp, 64 * p.n + 1024);
    if (dmalloc(&t_sing.ptr, cap * 8) != cudaSuccess) return fail(H2_ENOMEM, "singular list");
    if (dmalloc(&t_cnt.ptr, 8) != cudaSuccess) return fail(H2_ENOMEM, "singular count");
    H2_CUDA_TRY(cudaMemsetAsync(t_cnt.ptr, 0, 8, st));
    Geo g{(const double *)t_vert.ptr, (const int32_t *)t_tri.ptr, (const double *)t_area.ptr, d.pad_src,
          (const int32_t *)t_nrow.ptr, (const int32_t *)t_ncol.ptr, L, Lp, d.kernel};
    k_near_regular<TQ><<<grid_for(d.nnear * L * Lp, 128), 128, 0, st>>>(
        g, d.nnear, c.quad_order, qnear, (int64_t *)t_sing.ptr, (unsigned long long *)t_cnt.ptr, cap);
    H2_CUDA_TRY(cudaGetLastError());
    unsigned long long ns = 0;
    H2_CUDA_TRY(cudaMemcpyAsync(&ns, t_cnt.ptr, 8, cudaMemcpyDeviceToHost, st));
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    if ((int64_t)ns > cap) return fail(H2_EINVAL, "mesh has more vertex-sharing pairs than supported");
    if (ns > 0) {
      k_near_singular<TQ><<<grid_for((int64_t)ns, 64), 64, 0, st>>>(g, (const int64_t *)t_sing.ptr, (int64_t)ns,
                                                                    c.quad_order, qnear);
      H2_CUDA_TRY(cudaGetLastError());
    }
    if (std::is_same<T, __nv_bfloat16>::value) {
      // bfloat16: the self blocks G_jj (they hold the largest entries of every
      // row, the singular self-interaction g_ii among them) stay in FP32, the
      // other near blocks get a CSR of their own
      std::vector<int64_t> ptr2(p.nleaf + 1, 0), sptr(p.nleaf + 1);
      std::vector<int32_t> col2, blk2, scol(p.nleaf), sblk(p.nleaf, -1);
      for (int64_t j = 0; j < p.nleaf; ++j) {
        for (int64_t e = p.near_ptr[j]; e < p.near_ptr[j + 1]; ++e) {
          if (p.near_col[e] == j) {
            sblk[j] = (int32_t)e;
          } else {
            col2.push_back(p.near_col[e]);
            blk2.push_back((int32_t)e);
          }
        }
        ptr2[j + 1] = (int64_t)col2.size();
        sptr[j] = j;
        scol[j] = (int32_t)j;
        if (sblk[j] < 0) return fail(H2_EINVAL, "a leaf without its self block");
      }
      sptr[p.nleaf] = p.nleaf;
      auto up = [&](void **dst, const void *src, size_t bytes) -> int {
        int r = dev_alloc(d, dst, std::max<size_t>(bytes, 16));
        if (r) return r;
        if (bytes) H2_CUDA_TRY(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st));
        return H2_OK;
      };
      if ((rc = up((void **)&d.near_ptr2, ptr2.data(), ptr2.size() * 8))) return rc;
      if ((rc = up((void **)&d.near_col2, col2.data(), col2.size() * 4))) return rc;
      if ((rc = up((void **)&d.near_blk2, blk2.data(), blk2.size() * 4))) return rc;
      if ((rc = up((void **)&d.self_ptr, sptr.data(), sptr.size() * 8))) return rc;
      if ((rc = up((void **)&d.self_col, scol.data(), scol.size() * 4))) return rc;
      Tmp t_sblk;
      if ((rc = tmp_up(t_sblk, sblk.data(), sblk.size() * 4))) return rc;
      if ((rc = dev_alloc(d, (void **)&d.nself, (size_t)d.nleaf * L * Lp * 4))) return rc;
      k_split_self<<<grid_for(d.nleaf * L * Lp, 256), 256, 0, st>>>((const int32_t *)t_sblk.ptr, d.nleaf,
                                                                    (int64_t)L * Lp, (double *)qnear, d.nself);
      H2_CUDA_TRY(cudaGetLastError());
      H2_CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (is_half_type<T>()) {
      const int64_t per = L * Lp, tot = d.nnear * per;
      if (std::is_same<T, __half>::value) {
        if ((rc = dev_alloc(d, (void **)&d.nscale, d.nnear * 4))) return rc;
        k_block_scale<<<(unsigned)std::min<int64_t>(d.nnear, 152 * 32), 256, 0, st>>>((const double *)qnear, per,
                                                                                      d.nnear, d.nscale);
      }
      k_convert_scaled<T><<<grid_for(tot, 256), 256, 0, st>>>((const double *)qnear, d.nscale, per, (T *)d.near, tot);
      H2_CUDA_TRY(cudaGetLastError());
    }
  }
  // FP64-accurate handles with leaves of at most 21 triangles: the nearfield digits for the tensor cores
  if (ntc_eligible(d) && (rc = ntc_build(c, (const int32_t *)t_nrow.ptr))) return rc;
  H2_CUDA_TRY(cudaStreamSynchronize(st));
  c.build_ms[H2_BUILD_NEAR] = ms_since(tn0);
  return H2_OK;
}

}  // namespace

int dev_alloc(Dev &d, void **ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = dmalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return fail(H2_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  d.bytes += (int64_t)bytes;
  return H2_OK;
}

int device_build(Ctx &c) {
  Plan &p = c.plan;
  Dev &d = c.d;
  if (c.quad_order < 1 || c.quad_order > kMaxQ) return fail(H2_EINVAL, "quad_order must be in [1, 16]");
  d.m = p.m;
  d.k = p.k;
  // stored rows are padded to 16 bytes for 16-bit storage, else to 4 entries
  d.ssize = d.prec == H2_F32 ? 4 : (d.prec == H2_BF16 || d.prec == H2_F16) ? 2 : 8;
  const int rowpad = d.ssize == 2 ? 8 : 4;
  d.kp = (p.k + rowpad - 1) / rowpad * rowpad;
  d.depth = p.depth;
  d.first_adm_level = p.first_adm_level;
  d.n = p.n;
  d.nclu = p.nclu;
  d.nleaf = p.nleaf;
  d.lmax = p.lmax;
  d.npad = p.nleaf * p.lmax;
  d.lp = (p.lmax + rowpad - 1) / rowpad * rowpad;
  d.nadm = (int64_t)p.adm_col.size();
  d.nnear = (int64_t)p.near_col.size();
  if (d.coupling < 0) {
    // automatic: store S unless it would take more than half of the free memory (FP32 only)
    size_t fr = 0, tot = 0;
    H2_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    const double sbytes = (double)d.nadm * d.k * d.kp * d.ssize;
    d.coupling = (d.prec == H2_F32 && sbytes > 0.5 * (double)fr) ? 1 : 0;
  }
  switch (d.prec) {
    case H2_F64: {
      d.esize = 8;
      int rc = dev_alloc(d, (void **)&d.colmax, 64 * sizeof(unsigned long long));
      if (rc) return rc;
      if (d.fused && (rc = dev_alloc(d, (void **)&d.fbar, 2 * sizeof(unsigned)))) return rc;
      return build_typed<dd>(c);
    }
    case H2_F64_NATIVE: d.esize = 8; return build_typed<double>(c);
    case H2_BF16: d.esize = 4; return build_typed<__nv_bfloat16>(c);
    case H2_F16: d.esize = 4; return build_typed<__half>(c);
    default: d.esize = 4; return build_typed<float>(c);
  }
}

}  // namespace h2
