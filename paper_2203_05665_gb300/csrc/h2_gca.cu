// GCA-H^2 construction on the device (Boerm, Section 3, the GCA-H^2
// example): every cluster tau gets pivot elements tau_0 of tau, the pivots
// of a parent chosen among the pivots of its sons, and every admissible
// block the coupling matrix S_{tau sigma} = G|_{tau_0 x sigma_0}, the
// Galerkin matrix on the pivot pairs.  The section states only this; the
// pivots come from the cited Green cross approximation, restated here:
//
//   Green quadrature: Gauss-Legendre rules (green_order nodes per direction,
//   increasing) on the six faces of the box [lo - gamma rho, hi + gamma rho]
//   around the cluster's box (rho = half its diagonal); faces in the order
//   axis 0 low, axis 0 high, axis 1 low, ..., the first remaining axis
//   outermost on a face.
//   Surrogate: one row per candidate triangle, two columns per quadrature
//   point z (weight w, outward normal n): w int_T g(x, z) dx and
//   w int_T n.(x - z) / (4 pi |x - z|^3) dx (the two families of Green's
//   representation formula), integrated by the collapsed Gauss rule with
//   tri_order nodes per direction.
//   Cross approximation with complete pivoting: the pivot of a step is the
//   first entry (row-major) whose modulus is within a relative 2^-30 of the
//   residual's largest; the residual loses the pivot's row and column
//   (R <- R - R[:, j] R[i, :] / R[i, j], row i and column j set to zero);
//   stop when the largest modulus is at most eps times the surrogate's
//   largest, or after min(rows, columns, max_rank) steps.
//   Interpolation: V^ = M[:, J] M[I, J]^{-1}, computed as U L^{-1} from the
//   residual columns U taken at the pivot columns (L = U[I, :] is lower
//   triangular), the pivot rows set to unit vectors.  Leaves keep V^ as V;
//   a parent's candidates are its first son's pivots followed by its second
//   son's, and its V^ splits into the sons' transfer matrices E.
//
// One CTA per cluster of a level runs the surrogate, the cross
// approximation and V^; the levels run from the leaves up to the first
// level that holds an admissible block (higher clusters are never used).
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <vector>

#include "h2_dd.cuh"
#include "h2_internal.hpp"

namespace h2 {

namespace {

constexpr int kGT = 256;          // threads of the per-cluster kernel
constexpr int kMaxGreen = 8;      // green_order <= 8
constexpr int kMaxTri = 16;       // tri_order and the nearfield order <= 16
constexpr double kInv4Pi = 0.0795774715459476678844418816862571810;

__constant__ double c_gq_x[kMaxGreen], c_gq_w[kMaxGreen];   // face rule on [0,1], increasing nodes
__constant__ double c_tq_x[kMaxTri], c_tq_w[kMaxTri];       // triangle rule of the surrogate
__constant__ double c_nq_x[kMaxTri], c_nq_w[kMaxTri];       // regular rule of the Galerkin entries

struct GcaLevel {
  const double *vert;
  const int32_t *tri;
  const double *area;
  const double *lo, *hi;   // cluster boxes [clusters][3]
  double gamma, eps;
  int qg, qt, Q, kcap;
  int64_t c0;              // first cluster of the level
  int nrmax;               // candidate rows per cluster (capacity)
  const int32_t *rows;     // [level cluster][nrmax] candidate triangles
  const int32_t *nrow;     // [level cluster] candidate count
  double *R;               // [level cluster][nrmax][2Q] surrogate, then residual
  double *U;               // [level cluster][nrmax][kcap] residual columns at the pivots
  double *Vh;              // [level cluster][nrmax][kcap] interpolation operator
  int32_t *prow;           // [level cluster][kcap] pivot rows (candidate index)
  int32_t *rank;           // [clusters]
  int32_t *piv;            // [clusters][kcap]
};

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_min(int v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// block-wide maximum (every thread gets it); sred: 33 doubles of shared memory
__device__ double block_max(double v, double *sred) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  if (lane == 0) sred[w] = v;
  __syncthreads();
  if (w == 0) {
    double u = lane < nw ? sred[lane] : 0.0;
    u = warp_max(u);
    if (lane == 0) sred[32] = u;
  }
  __syncthreads();
  const double r = sred[32];
  __syncthreads();
  return r;
}
__device__ int block_min(int v, int *sred) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_min(v);
  if (lane == 0) sred[w] = v;
  __syncthreads();
  if (w == 0) {
    int u = lane < nw ? sred[lane] : INT_MAX;
    u = warp_min(u);
    if (lane == 0) sred[32] = u;
  }
  __syncthreads();
  const int r = sred[32];
  __syncthreads();
  return r;
}

// candidate rows of the clusters of one level: a leaf's triangles in cluster
// order, or the pivots of the first son followed by those of the second
__global__ void k_gca_rows(int64_t c0, int64_t ncl, bool leaves, const int32_t *__restrict__ pad_src, int L,
                           int64_t leaf0, const int64_t *__restrict__ size, const int32_t *__restrict__ rank,
                           const int32_t *__restrict__ piv, int kcap, int nrmax, int32_t *__restrict__ rows,
                           int32_t *__restrict__ nrow) {
  const int64_t total = ncl * nrmax;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cl = e / nrmax;
    const int r = (int)(e - cl * nrmax);
    const int64_t c = c0 + cl;
    int nr;
    int32_t v = -1;
    if (leaves) {
      nr = (int)size[c];
      if (r < nr) v = pad_src[(c - leaf0) * L + r];
    } else {
      const int k1 = rank[2 * c + 1], k2 = rank[2 * c + 2];
      nr = k1 + k2;
      if (r < k1) v = piv[(2 * c + 1) * kcap + r];
      else if (r < nr) v = piv[(2 * c + 2) * kcap + (r - k1)];
    }
    rows[e] = v;
    if (r == 0) nrow[cl] = nr;
  }
}

// Surrogate, cross approximation and interpolation operator of one cluster
// per CTA (see the file comment).
__global__ void __launch_bounds__(kGT) k_gca_cluster(GcaLevel g) {
  extern __shared__ __align__(16) double gsm[];
  const int Q = g.Q, nc = 2 * Q;
  double *Z = gsm;                 // [Q][3]
  double *W = Z + 3 * Q;           // [Q]
  double *wrow = W + Q;            // [nc] pivot row of the residual
  double *ucol = wrow + nc;        // [nrmax] pivot column of the residual
  double *sred = ucol + g.nrmax;   // [33]
  int *nax = reinterpret_cast<int *>(sred + 34);   // [Q] normal: 2 axis + side
  int *sI = nax + Q;               // [kcap] pivot rows
  int *ired = sI + g.kcap;         // [33]
  const int tid = threadIdx.x;
  const int64_t cl = blockIdx.x, c = g.c0 + cl;
  const int nr = g.nrow[cl];
  const int32_t *rows = g.rows + cl * g.nrmax;
  double *R = g.R + cl * (int64_t)g.nrmax * nc;
  double *U = g.U + cl * (int64_t)g.nrmax * g.kcap;
  double *Vh = g.Vh + cl * (int64_t)g.nrmax * g.kcap;

  // Green quadrature on the faces of the enlarged box
  {
    const double *lo = g.lo + 3 * c, *hi = g.hi + 3 * c;
    const double d0 = hi[0] - lo[0], d1 = hi[1] - lo[1], d2 = hi[2] - lo[2];
    const double rho = 0.5 * sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    double olo[3], ohi[3];
    for (int d = 0; d < 3; ++d) {
      olo[d] = lo[d] - g.gamma * rho;
      ohi[d] = hi[d] + g.gamma * rho;
    }
    const int qq = g.qg * g.qg;
    for (int q = tid; q < Q; q += blockDim.x) {
      const int a = q / (2 * qq), side = (q / qq) & 1, i = (q / g.qg) % g.qg, j = q % g.qg;
      const int b = a == 0 ? 1 : 0, cc = a == 2 ? 1 : 2;
      Z[3 * q + a] = side ? ohi[a] : olo[a];
      Z[3 * q + b] = olo[b] + c_gq_x[i] * (ohi[b] - olo[b]);
      Z[3 * q + cc] = olo[cc] + c_gq_x[j] * (ohi[cc] - olo[cc]);
      W[q] = c_gq_w[i] * c_gq_w[j] * (ohi[b] - olo[b]) * (ohi[cc] - olo[cc]);
      nax[q] = 2 * a + side;
    }
  }
  __syncthreads();

  // surrogate rows
  for (int e = tid; e < nr * Q; e += blockDim.x) {
    const int r = e / Q, nu = e - r * Q;
    const int64_t t = rows[r];
    const double *A = g.vert + 3 * (int64_t)g.tri[3 * t], *B = g.vert + 3 * (int64_t)g.tri[3 * t + 1],
                 *C = g.vert + 3 * (int64_t)g.tri[3 * t + 2];
    const double jac = 2.0 * g.area[t];
    const double z0 = Z[3 * nu], z1 = Z[3 * nu + 1], z2 = Z[3 * nu + 2];
    const int ax = nax[nu] >> 1;
    const double sg = (nax[nu] & 1) ? 1.0 : -1.0;
    double s1 = 0.0, s2 = 0.0;
    for (int a = 0; a < g.qt; ++a)
      for (int b = 0; b < g.qt; ++b) {
        const double s = c_tq_x[a], tt = c_tq_x[a] * c_tq_x[b];
        const double x0 = A[0] + s * (B[0] - A[0]) + tt * (C[0] - B[0]);
        const double x1 = A[1] + s * (B[1] - A[1]) + tt * (C[1] - B[1]);
        const double x2 = A[2] + s * (B[2] - A[2]) + tt * (C[2] - B[2]);
        const double w = jac * c_tq_w[a] * c_tq_w[b] * c_tq_x[a];
        const double e0 = x0 - z0, e1 = x1 - z1, e2 = x2 - z2;
        const double rr = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
        const double ea = ax == 0 ? e0 : ax == 1 ? e1 : e2;
        s1 += w / (4.0 * 3.14159265358979323846 * rr);
        s2 += w * (sg * ea) / (4.0 * 3.14159265358979323846 * rr * rr * rr);
      }
    R[(int64_t)r * nc + nu] = W[nu] * s1;
    R[(int64_t)r * nc + Q + nu] = W[nu] * s2;
  }
  __syncthreads();

  // cross approximation with complete pivoting
  const int ntot = nr * nc;
  double lmx = 0.0;
  for (int e = tid; e < ntot; e += blockDim.x) lmx = fmax(lmx, fabs(R[e]));
  double mx = block_max(lmx, sred);
  const double mx0 = mx;
  const int kmax = min(min(nr, nc), g.kcap);
  int k = 0;
  while (k < kmax) {
    if (mx == 0.0 || mx <= g.eps * mx0) break;
    const double thr = mx * (1.0 - 9.313225746154785e-10);   // 1 - 2^-30
    int first = INT_MAX;
    for (int e = tid; e < ntot; e += blockDim.x)
      if (fabs(R[e]) >= thr) {
        first = e;
        break;
      }
    const int pe = block_min(first, ired);
    if (pe == INT_MAX) break;   // not reached for finite data: the largest entry passes its own threshold
    const int i = pe / nc, j = pe - i * nc;
    const double piv = R[pe];
    for (int r = tid; r < nr; r += blockDim.x) {
      const double u = R[(int64_t)r * nc + j];
      ucol[r] = u;
      U[(int64_t)r * g.kcap + k] = u;
    }
    for (int q = tid; q < nc; q += blockDim.x) wrow[q] = R[(int64_t)i * nc + q];
    if (tid == 0) sI[k] = i;
    __syncthreads();
    lmx = 0.0;
    for (int e = tid; e < ntot; e += blockDim.x) {
      const int r = e / nc, q = e - r * nc;
      double v = 0.0;
      if (r != i && q != j) v = R[e] - (ucol[r] / piv) * wrow[q];
      R[e] = v;
      lmx = fmax(lmx, fabs(v));
    }
    ++k;
    mx = block_max(lmx, sred);
  }

  // V^ = U L^{-1} with L[a][b] = U[I_a][b] (lower triangular), pivot rows exact
  for (int r = tid; r < nr; r += blockDim.x) {
    double *vr = Vh + (int64_t)r * g.kcap;
    int pa = -1;
    for (int a = 0; a < k; ++a)
      if (sI[a] == r) pa = a;
    if (pa >= 0) {
      for (int b = 0; b < k; ++b) vr[b] = b == pa ? 1.0 : 0.0;
      continue;
    }
    const double *ur = U + (int64_t)r * g.kcap;
    for (int b = k - 1; b >= 0; --b) {
      double s = ur[b];
      for (int a = b + 1; a < k; ++a) s -= vr[a] * U[(int64_t)sI[a] * g.kcap + b];
      vr[b] = s / U[(int64_t)sI[b] * g.kcap + b];
    }
  }
  if (tid == 0) g.rank[c] = k;
  for (int a = tid; a < k; a += blockDim.x) {
    g.piv[c * g.kcap + a] = rows[sI[a]];
    g.prow[cl * g.kcap + a] = sI[a];
  }
}

// leaf bases: V [leaf][t][K] (forward step) and Vt [leaf][a][Lp] (backward
// step) from the leaves' V^, zero padded
template <class T>
__global__ void k_gca_store_V(const double *__restrict__ Vh, const int32_t *__restrict__ rank,
                              const int64_t *__restrict__ size, int64_t leaf0, int64_t nleaf, int L, int Lp, int kcap,
                              int K, T *__restrict__ V, T *__restrict__ Vt) {
  const int64_t total = nleaf * (int64_t)Lp * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / ((int64_t)Lp * K);
    const int rem = (int)(e - j * Lp * K);
    const int t = rem / K, a = rem - t * K;
    const int64_t c = leaf0 + j;
    const double v = (t < size[c] && a < rank[c]) ? Vh[(j * L + t) * kcap + a] : 0.0;
    if (t < L) V[(j * L + t) * K + a] = from_double<T>(v);
    Vt[(j * K + a) * Lp + t] = from_double<T>(v);
  }
}

// transfer matrices of the sons (level l + 1) of the parents of level l:
// E_s[a][b] = V^_parent[off_s + a][b] (off = 0 for the first son, the first
// son's rank for the second), E [son][Kc][Kp] and Et [son][Kp][Kc]
template <class T>
__global__ void k_gca_store_E(const double *__restrict__ Vh, const int32_t *__restrict__ rank, int64_t cp0,
                              int64_t npar, int nrmax, int kcap, int Kc, int Kp, T *__restrict__ E, T *__restrict__ Et) {
  const int64_t total = 2 * npar * (int64_t)Kc * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = e / ((int64_t)Kc * Kp);
    const int rem = (int)(e - s * Kc * Kp);
    const int a = rem / Kp, b = rem - a * Kp;
    const int64_t p = s >> 1, par = cp0 + p, son = 2 * par + 1 + (s & 1);
    const int off = (s & 1) ? rank[2 * par + 1] : 0;
    const double v = (a < rank[son] && b < rank[par]) ? Vh[(p * nrmax + off + a) * kcap + b] : 0.0;
    E[(s * Kc + a) * Kp + b] = from_double<T>(v);
    Et[(s * Kp + b) * Kc + a] = from_double<T>(v);
  }
}

// g_ij of two triangles without a common vertex: the collapsed Gauss rule
// with q nodes per direction on each triangle (vertices in mesh order), the
// smaller index as test triangle
__device__ double galerkin_regular(const double *vert, const int32_t *tri, const double *area, int32_t i, int32_t j,
                                   int q) {
  if (i > j) {
    const int32_t t = i;
    i = j;
    j = t;
  }
  const double *A1 = vert + 3 * (int64_t)tri[3 * i], *B1 = vert + 3 * (int64_t)tri[3 * i + 1],
               *C1 = vert + 3 * (int64_t)tri[3 * i + 2];
  const double *A2 = vert + 3 * (int64_t)tri[3 * j], *B2 = vert + 3 * (int64_t)tri[3 * j + 1],
               *C2 = vert + 3 * (int64_t)tri[3 * j + 2];
  double acc = 0.0;
  for (int a = 0; a < q; ++a)
    for (int b = 0; b < q; ++b) {
      const double s = c_nq_x[a], t = c_nq_x[a] * c_nq_x[b];
      double x[3];
      for (int d = 0; d < 3; ++d) x[d] = A1[d] + s * (B1[d] - A1[d]) + t * (C1[d] - B1[d]);
      const double wx = c_nq_w[a] * c_nq_w[b] * c_nq_x[a];
      double inner = 0.0;
      for (int cc = 0; cc < q; ++cc)
        for (int dd = 0; dd < q; ++dd) {
          const double s2 = c_nq_x[cc], t2 = c_nq_x[cc] * c_nq_x[dd];
          double y[3];
          for (int d = 0; d < 3; ++d) y[d] = A2[d] + s2 * (B2[d] - A2[d]) + t2 * (C2[d] - B2[d]);
          const double e0 = x[0] - y[0], e1 = x[1] - y[1], e2 = x[2] - y[2];
          inner += c_nq_w[cc] * c_nq_w[dd] * c_nq_x[cc] * (kInv4Pi / sqrt(e0 * e0 + e1 * e1 + e2 * e2));
        }
      acc += wx * inner;
    }
  return 4.0 * area[i] * area[j] * acc;
}

// coupling matrices of one level: S_b = G|_{t_0 x s_0}, stored transposed
// [mu][nu] (nu: row pivot of t, mu: column pivot of s), zero padded to K;
// only the blocks with t < s (the others are their mirrors' transposes,
// k_gca_mirror)
template <class T>
__global__ void k_gca_coupling(const double *__restrict__ vert, const int32_t *__restrict__ tri,
                               const double *__restrict__ area, const int32_t *__restrict__ arow,
                               const int32_t *__restrict__ acol, const int32_t *__restrict__ rank,
                               const int32_t *__restrict__ piv, int kcap, int64_t nb, int K, int q, T *__restrict__ S) {
  const int64_t total = nb * (int64_t)K * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / ((int64_t)K * K);
    const int64_t t = arow[b], s = acol[b];
    if (t > s) continue;
    const int rem = (int)(e - b * K * K);
    const int mu = rem / K, nu = rem - mu * K;
    double v = 0.0;
    if (nu < rank[t] && mu < rank[s])
      v = galerkin_regular(vert, tri, area, piv[t * kcap + nu], piv[s * kcap + mu], q);
    S[e] = from_double<T>(v);
  }
}

// S_{t,s} = S_{s,t}^T for the blocks with t > s of one level (G is symmetric
// bit for bit: every entry is evaluated with the smaller triangle index as
// test triangle); mir[b] = the level-local index of block (s, t)
template <class T>
__global__ void k_gca_mirror(const int32_t *__restrict__ arow, const int32_t *__restrict__ acol,
                             const int32_t *__restrict__ mir, int64_t nb, int K, T *__restrict__ S) {
  const int64_t total = nb * (int64_t)K * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / ((int64_t)K * K);
    if (arow[b] < acol[b]) continue;
    const int rem = (int)(e - b * K * K);
    const int mu = rem / K, nu = rem - mu * K;
    S[e] = S[(int64_t)mir[b] * K * K + (int64_t)nu * K + mu];
  }
}

int grid_of(int64_t n, int threads) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 64));
}

struct DevBuf {
  void *ptr = nullptr;
  ~DevBuf() {
    if (ptr) cudaFree(ptr);
  }
  int get(size_t bytes) {
    if (dmalloc(&ptr, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      ptr = nullptr;
      cudaGetLastError();
      return fail(H2_ENOMEM, "GCA set-up buffer of " + std::to_string(bytes) + " bytes");
    }
    return H2_OK;
  }
};

template <class T>
int gca_build_typed(Ctx &c, const double *vert, const int32_t *tri, const double *area) {
  Plan &p = c.plan;
  Dev &d = c.d;
  const GcaParams &gp = c.gp;
  cudaStream_t st = c.stream;
  const int D = p.depth, lmin = p.first_adm_level, L = (int)p.lmax, Lp = (int)d.lp;
  const int qg = gp.green_order, Q = 6 * qg * qg, nc = 2 * Q, kcap = gp.max_rank;
  const auto t0 = std::chrono::steady_clock::now();
  d.gkcap = kcap;
  int rc;
  if ((rc = dev_alloc(d, (void **)&d.grank, p.nclu * 4))) return rc;
  if ((rc = dev_alloc(d, (void **)&d.gpiv, (size_t)p.nclu * kcap * 4))) return rc;
  H2_CUDA_TRY(cudaMemsetAsync(d.grank, 0, p.nclu * 4, st));
  H2_CUDA_TRY(cudaMemsetAsync(d.gpiv, 0xff, (size_t)p.nclu * kcap * 4, st));
  for (int l = 0; l < kMaxLevels; ++l) d.gK[l] = 0;
  if (lmin > D) {
    // no admissible block: the nearfield is the whole matrix
    d.k = 4;
    d.kp = 4;
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    return H2_OK;
  }

  // quadrature rules (increasing nodes)
  {
    std::vector<double> x, w;
    auto up = [&](int q, const void *sx, const void *sw) -> int {
      gauss_legendre01(q, x, w);   // decreasing nodes
      std::reverse(x.begin(), x.end());
      std::reverse(w.begin(), w.end());
      H2_CUDA_TRY(cudaMemcpyToSymbolAsync(sx, x.data(), q * 8, 0, cudaMemcpyHostToDevice, st));
      H2_CUDA_TRY(cudaMemcpyToSymbolAsync(sw, w.data(), q * 8, 0, cudaMemcpyHostToDevice, st));
      H2_CUDA_TRY(cudaStreamSynchronize(st));
      return H2_OK;
    };
    if ((rc = up(qg, c_gq_x, c_gq_w))) return rc;
    if ((rc = up(gp.tri_order, c_tq_x, c_tq_w))) return rc;
    if ((rc = up(c.quad_order, c_nq_x, c_nq_w))) return rc;
  }
  DevBuf blo, bhi, bsize;
  if ((rc = blo.get(p.lo.size() * 8)) || (rc = bhi.get(p.hi.size() * 8)) || (rc = bsize.get(p.size.size() * 8)))
    return rc;
  H2_CUDA_TRY(cudaMemcpyAsync(blo.ptr, p.lo.data(), p.lo.size() * 8, cudaMemcpyHostToDevice, st));
  H2_CUDA_TRY(cudaMemcpyAsync(bhi.ptr, p.hi.data(), p.hi.size() * 8, cudaMemcpyHostToDevice, st));
  H2_CUDA_TRY(cudaMemcpyAsync(bsize.ptr, p.size.data(), p.size.size() * 8, cudaMemcpyHostToDevice, st));

  const int64_t leaf0 = p.leaf0;
  int maxrank_below = 0;   // largest rank of the level below
  std::vector<int32_t> hrank;
  for (int l = D; l >= lmin; --l) {
    const int64_t ncl = (int64_t)1 << l, c0 = ncl - 1;
    const int nrmax = l == D ? L : 2 * maxrank_below;
    DevBuf brows, bnrow, bR, bU, bVh, bprow;
    if ((rc = brows.get((size_t)ncl * nrmax * 4)) || (rc = bnrow.get((size_t)ncl * 4)) ||
        (rc = bR.get((size_t)ncl * nrmax * nc * 8)) || (rc = bU.get((size_t)ncl * nrmax * kcap * 8)) ||
        (rc = bVh.get((size_t)ncl * nrmax * kcap * 8)) || (rc = bprow.get((size_t)ncl * kcap * 4)))
      return rc;
    k_gca_rows<<<grid_of(ncl * nrmax, 256), 256, 0, st>>>(c0, ncl, l == D, d.pad_src, L, leaf0,
                                                           (const int64_t *)bsize.ptr, d.grank, d.gpiv, kcap, nrmax,
                                                           (int32_t *)brows.ptr, (int32_t *)bnrow.ptr);
    H2_CUDA_TRY(cudaGetLastError());
    GcaLevel g{};
    g.vert = vert;
    g.tri = tri;
    g.area = area;
    g.lo = (const double *)blo.ptr;
    g.hi = (const double *)bhi.ptr;
    g.gamma = gp.gamma;
    g.eps = gp.eps;
    g.qg = qg;
    g.qt = gp.tri_order;
    g.Q = Q;
    g.kcap = kcap;
    g.c0 = c0;
    g.nrmax = nrmax;
    g.rows = (const int32_t *)brows.ptr;
    g.nrow = (const int32_t *)bnrow.ptr;
    g.R = (double *)bR.ptr;
    g.U = (double *)bU.ptr;
    g.Vh = (double *)bVh.ptr;
    g.prow = (int32_t *)bprow.ptr;
    g.rank = d.grank;
    g.piv = d.gpiv;
    const size_t sm = (size_t)(3 * Q + Q + nc + nrmax + 34) * 8 + (size_t)(Q + kcap + 33) * 4;
    if (sm > 48 * 1024)
      H2_CUDA_TRY(cudaFuncSetAttribute((const void *)k_gca_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)std::min<size_t>(sm, 227 * 1024)));
    k_gca_cluster<<<(unsigned)ncl, kGT, sm, st>>>(g);
    H2_CUDA_TRY(cudaGetLastError());
    hrank.assign(ncl, 0);
    H2_CUDA_TRY(cudaMemcpyAsync(hrank.data(), d.grank + c0, ncl * 4, cudaMemcpyDeviceToHost, st));
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    int mr = 0;
    for (int32_t r : hrank) mr = std::max(mr, (int)r);
    d.gK[l] = std::max(4, (mr + 3) / 4 * 4);
    if (l == D) {
      const int K = d.gK[D];
      if ((rc = dev_alloc(d, &d.V, (size_t)p.nleaf * L * K * sizeof(T)))) return rc;
      if ((rc = dev_alloc(d, &d.Vt, (size_t)p.nleaf * K * Lp * sizeof(T)))) return rc;
      k_gca_store_V<T><<<grid_of(p.nleaf * (int64_t)Lp * K, 256), 256, 0, st>>>(
          (const double *)bVh.ptr, d.grank, (const int64_t *)bsize.ptr, leaf0, p.nleaf, L, Lp, kcap, K, (T *)d.V,
          (T *)d.Vt);
    } else {
      const int Kc = d.gK[l + 1], Kp = d.gK[l];
      const size_t ne = (size_t)2 * ncl * Kc * Kp;
      if ((rc = dev_alloc(d, &d.gE[l + 1], ne * sizeof(T)))) return rc;
      if ((rc = dev_alloc(d, &d.gEt[l + 1], ne * sizeof(T)))) return rc;
      k_gca_store_E<T><<<grid_of((int64_t)ne, 256), 256, 0, st>>>((const double *)bVh.ptr, d.grank, c0, ncl, nrmax,
                                                                  kcap, Kc, Kp, (T *)d.gE[l + 1],
                                                                  (T *)d.gEt[l + 1]);
    }
    H2_CUDA_TRY(cudaGetLastError());
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    maxrank_below = mr;
  }
  c.build_ms[H2_BUILD_BASES] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();

  // coefficient offsets and the largest padded rank
  int64_t off = 0;
  int kmax = 4;
  for (int l = 0; l <= D; ++l) {
    d.gX[l] = off;
    off += ((int64_t)1 << l) * d.gK[l];
    kmax = std::max(kmax, d.gK[l]);
  }
  d.k = kmax;
  d.kp = d.gK[D];

  // coupling matrices per level
  std::vector<int32_t> arow(p.adm_col.size());
  for (int64_t t = 0; t < p.nclu; ++t)
    for (int64_t e = p.adm_ptr[t]; e < p.adm_ptr[t + 1]; ++e) arow[e] = (int32_t)t;
  // level-local index of the mirror block (s, t) of every admissible block (t, s)
  std::vector<int32_t> mir(p.adm_col.size(), 0);
  for (int64_t t = 0; t < p.nclu; ++t)
    for (int64_t e = p.adm_ptr[t]; e < p.adm_ptr[t + 1]; ++e) {
      const int64_t sc = p.adm_col[e];
      const auto beg = p.adm_col.begin() + p.adm_ptr[sc], end = p.adm_col.begin() + p.adm_ptr[sc + 1];
      const auto it = std::lower_bound(beg, end, (int32_t)t);
      if (it == end || *it != (int32_t)t) return fail(H2_EINVAL, "block tree is not symmetric");
      int l = 0;
      while (((int64_t)2 << l) - 1 <= sc) ++l;
      mir[e] = (int32_t)((it - p.adm_col.begin()) - p.adm_ptr[((int64_t)1 << l) - 1]);
    }
  DevBuf barow, bmir;
  if ((rc = barow.get(arow.size() * 4)) || (rc = bmir.get(mir.size() * 4))) return rc;
  if (!arow.empty()) {
    H2_CUDA_TRY(cudaMemcpyAsync(barow.ptr, arow.data(), arow.size() * 4, cudaMemcpyHostToDevice, st));
    H2_CUDA_TRY(cudaMemcpyAsync(bmir.ptr, mir.data(), mir.size() * 4, cudaMemcpyHostToDevice, st));
  }
  d.coupling_entries = 0;
  for (int l = lmin; l <= D; ++l) {
    const int64_t c0 = ((int64_t)1 << l) - 1, c1 = ((int64_t)2 << l) - 1;
    const int64_t b0 = p.adm_ptr[c0], nb = p.adm_ptr[c1] - b0;
    const int K = d.gK[l];
    if ((rc = dev_alloc(d, &d.gS[l], (size_t)std::max<int64_t>(nb, 1) * K * K * sizeof(T)))) return rc;
    d.coupling_entries += nb * K * K;
    if (nb == 0) continue;
    k_gca_coupling<T><<<grid_of(nb * K * K, 128), 128, 0, st>>>(vert, tri, area, (const int32_t *)barow.ptr + b0,
                                                               d.adm_col + b0, d.grank, d.gpiv, kcap, nb, K,
                                                               c.quad_order, (T *)d.gS[l]);
    H2_CUDA_TRY(cudaGetLastError());
    k_gca_mirror<T><<<grid_of(nb * K * K, 256), 256, 0, st>>>((const int32_t *)barow.ptr + b0, d.adm_col + b0,
                                                             (const int32_t *)bmir.ptr + b0, nb, K, (T *)d.gS[l]);
    H2_CUDA_TRY(cudaGetLastError());
  }
  H2_CUDA_TRY(cudaStreamSynchronize(st));
  return H2_OK;
}

}  // namespace

int gca_build(Ctx &c, const double *vert, const int32_t *tri, const double *area) {
  const GcaParams &gp = c.gp;
  if (gp.green_order < 1 || gp.green_order > kMaxGreen) return fail(H2_EINVAL, "green_order must be in [1, 8]");
  if (gp.tri_order < 1 || gp.tri_order > kMaxTri) return fail(H2_EINVAL, "tri_order must be in [1, 16]");
  if (c.quad_order > kMaxTri) return fail(H2_EINVAL, "quad_order must be in [1, 16]");
  if (gp.max_rank < 4 || gp.max_rank > 128) return fail(H2_EINVAL, "max_rank must be in [4, 128]");
  if (!(gp.eps >= 0.0) || !(gp.eps < 1.0)) return fail(H2_EINVAL, "eps must be in [0, 1)");
  if (!(gp.gamma > 0.0) || !std::isfinite(gp.gamma)) return fail(H2_EINVAL, "gamma must be positive");
  switch (c.d.prec) {
    case H2_F64: return gca_build_typed<dd>(c, vert, tri, area);
    case H2_F64_NATIVE: return gca_build_typed<double>(c, vert, tri, area);
    case H2_F32: return gca_build_typed<float>(c, vert, tri, area);
    default: return fail(H2_EINVAL, "GCA-H^2 handles support H2_F64, H2_F64_NATIVE and H2_F32");
  }
}

}  // namespace h2
