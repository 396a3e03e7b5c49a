// Restarted GMRES(restart) on the device for G~ z = b, every right-hand side
// an independent Krylov process (Saad, Iterative Methods for Sparse Linear
// Systems, Alg. 6.9, with classical Gram-Schmidt applied twice).  All
// Krylov arithmetic is FP64; the product runs in the handle's precision.
// The paper names Krylov methods for the system Gz = b (Section 1) without
// fixing one.
#include <cmath>
#include <vector>

#include "h2_internal.hpp"

namespace h2 {

namespace {

constexpr int kT = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double part[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) part[w] = v;
  __syncthreads();
  double s = 0;
  if (w == 0) {
    s = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// out[i * nrhs + c] = <X_i[:, c], W[:, c]> for i < nvec; grid (nrhs, nvec)
__global__ void k_dots(const double *__restrict__ X, const double *__restrict__ W, int64_t n, int nrhs,
                       double *__restrict__ out) {
  const int c = blockIdx.x, i = blockIdx.y;
  const double *x = X + ((int64_t)i * nrhs + c) * n, *w = W + (int64_t)c * n;
  double s = 0;
  for (int64_t l = threadIdx.x; l < n; l += blockDim.x) s += x[l] * w[l];
  s = block_sum(s);
  if (threadIdx.x == 0) out[i * nrhs + c] = s;
}

// W[:, c] -= sum_{i < nvec} h[i][c] X_i[:, c]; accumulates h into H column j
__global__ void k_orth(const double *__restrict__ X, const double *__restrict__ h, int nvec, int64_t n, int nrhs,
                       double *__restrict__ W) {
  const int64_t total = n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)(e / n);
    double s = W[e];
    for (int i = 0; i < nvec; ++i) s -= h[i * nrhs + c] * X[(int64_t)i * total + e];
    W[e] = s;
  }
}

// v[:, c] = w[:, c] / nrm[c] for active columns with nrm > 0, else 0
__global__ void k_scale(const double *__restrict__ W, const double *__restrict__ nrm, const int *__restrict__ active,
                        int64_t n, int nrhs, double *__restrict__ Vout) {
  const int64_t total = n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)(e / n);
    double d = nrm[c];
    Vout[e] = (active[c] && d > 0) ? W[e] / d : 0.0;
  }
}

// Hessenberg column j: h1 + h2 from the two Gram-Schmidt passes, then the
// Givens rotations; H[(i * mr + j) * nrhs + c]
__global__ void k_givens(const double *__restrict__ h1, const double *__restrict__ h2, const double *__restrict__ hn,
                         int j, int mr, int nrhs, double *__restrict__ H, double *__restrict__ cs,
                         double *__restrict__ sn, double *__restrict__ g, double *__restrict__ resid,
                         const int *__restrict__ active) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nrhs || !active[c]) return;
  auto Hc = [&](int i) -> double & { return H[((int64_t)i * mr + j) * nrhs + c]; };
  for (int i = 0; i <= j; ++i) Hc(i) = h1[i * nrhs + c] + h2[i * nrhs + c];
  Hc(j + 1) = hn[c];
  for (int i = 0; i < j; ++i) {
    double a = Hc(i), b = Hc(i + 1);
    Hc(i) = cs[i * nrhs + c] * a + sn[i * nrhs + c] * b;
    Hc(i + 1) = -sn[i * nrhs + c] * a + cs[i * nrhs + c] * b;
  }
  double a = Hc(j), b = Hc(j + 1);
  double den = sqrt(a * a + b * b);
  double cj = den > 0 ? a / den : 1.0, sj = den > 0 ? b / den : 0.0;
  cs[j * nrhs + c] = cj;
  sn[j * nrhs + c] = sj;
  Hc(j) = cj * a + sj * b;
  Hc(j + 1) = 0.0;
  double gj = g[j * nrhs + c];
  g[(j + 1) * nrhs + c] = -sj * gj;
  g[j * nrhs + c] = cj * gj;
  resid[c] = fabs(sj * gj);
}

// y = R^{-1} g for the first jc[c] columns, then z[:, c] += sum_i y_i V_i[:, c]
__global__ void k_backsolve(const double *__restrict__ H, const double *__restrict__ g, const int *__restrict__ jc,
                            int mr, int nrhs, double *__restrict__ y) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nrhs) return;
  int J = jc[c];
  for (int i = J - 1; i >= 0; --i) {
    double s = g[i * nrhs + c];
    for (int l = i + 1; l < J; ++l) s -= H[((int64_t)i * mr + l) * nrhs + c] * y[l * nrhs + c];
    double d = H[((int64_t)i * mr + i) * nrhs + c];
    y[i * nrhs + c] = d != 0 ? s / d : 0.0;
  }
}

__global__ void k_update(const double *__restrict__ Vb, const double *__restrict__ y, const int *__restrict__ jc,
                         int64_t n, int nrhs, double *__restrict__ z) {
  const int64_t total = n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)(e / n);
    double s = z[e];
    for (int i = 0; i < jc[c]; ++i) s += y[i * nrhs + c] * Vb[(int64_t)i * total + e];
    z[e] = s;
  }
}

__global__ void k_sqrt(double *__restrict__ v, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = sqrt(v[i]);
}

__global__ void k_residual(const double *__restrict__ b, const double *__restrict__ Az, int64_t total,
                           double *__restrict__ r) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    r[e] = b[e] - Az[e];
}

int grid1(int64_t n) {
  int64_t g = (n + kT - 1) / kT;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

struct DBuf {
  double *p = nullptr;
  ~DBuf() { if (p) cudaFree(p); }
  int alloc(size_t n) {
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * 8) != cudaSuccess) {
      cudaGetLastError();
      return fail(H2_ENOMEM, "GMRES work space");
    }
    return H2_OK;
  }
};
struct IBuf {
  int *p = nullptr;
  ~IBuf() { if (p) cudaFree(p); }
  int alloc(size_t n) {
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(H2_ENOMEM, "GMRES work space");
    }
    return H2_OK;
  }
};

}  // namespace

int run_gmres(Ctx &c, const double *b, double *z, int nrhs, double rtol, int restart, int maxit,
              h2_solve_info *info) {
  const int64_t n = c.d.n, tot = n * nrhs;
  const int mr = restart;
  cudaStream_t st = c.stream;
  int rc;
  DBuf Vb, W, H, cs, sn, g, h1, h2b, hn, resid, yv, bn;
  IBuf active, jc;
  if ((rc = Vb.alloc((size_t)(mr + 1) * tot)) || (rc = W.alloc(tot)) || (rc = H.alloc((size_t)(mr + 1) * mr * nrhs)) ||
      (rc = cs.alloc(mr * nrhs)) || (rc = sn.alloc(mr * nrhs)) || (rc = g.alloc((mr + 1) * nrhs)) ||
      (rc = h1.alloc((mr + 1) * nrhs)) || (rc = h2b.alloc((mr + 1) * nrhs)) || (rc = hn.alloc(nrhs)) ||
      (rc = resid.alloc(nrhs)) || (rc = yv.alloc(mr * nrhs)) || (rc = bn.alloc(nrhs)) ||
      (rc = active.alloc(nrhs)) || (rc = jc.alloc(nrhs)))
    return rc;

  std::vector<double> h_bn(nrhs), h_rn(nrhs), h_res(nrhs), h_g0((mr + 1) * nrhs, 0.0);
  std::vector<int> h_active(nrhs, 1), h_jc(nrhs, 0), h_iters(nrhs, 0), h_done(nrhs, 0);

  // |b|
  k_dots<<<dim3(nrhs, 1), kT, 0, st>>>(b, b, n, nrhs, bn.p);
  H2_CUDA_TRY(cudaMemcpyAsync(h_bn.data(), bn.p, nrhs * 8, cudaMemcpyDeviceToHost, st));
  H2_CUDA_TRY(cudaMemsetAsync(z, 0, tot * 8, st));
  H2_CUDA_TRY(cudaStreamSynchronize(st));
  for (int col = 0; col < nrhs; ++col) {
    h_bn[col] = std::sqrt(h_bn[col]);
    if (h_bn[col] == 0.0) { h_done[col] = 1; h_res[col] = 0.0; }
  }
  // r = b (z0 = 0)
  H2_CUDA_TRY(cudaMemcpyAsync(W.p, b, tot * 8, cudaMemcpyDeviceToDevice, st));
  bool first = true;
  for (;;) {
    if (!first) {
      // true residual r = b - G~ z
      if ((rc = run_matvec(c, z, W.p, nrhs, true))) return rc;
      k_residual<<<grid1(tot), kT, 0, st>>>(b, W.p, tot, W.p);
    }
    k_dots<<<dim3(nrhs, 1), kT, 0, st>>>(W.p, W.p, n, nrhs, hn.p);
    k_sqrt<<<(nrhs + 63) / 64, 64, 0, st>>>(hn.p, nrhs);
    H2_CUDA_TRY(cudaMemcpyAsync(h_rn.data(), hn.p, nrhs * 8, cudaMemcpyDeviceToHost, st));
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    bool any = false;
    for (int col = 0; col < nrhs; ++col) {
      if (h_bn[col] == 0.0) { h_active[col] = 0; continue; }
      h_res[col] = h_rn[col] / h_bn[col];
      if (h_res[col] <= rtol) h_done[col] = 1;
      h_active[col] = (!h_done[col] && h_iters[col] < maxit) ? 1 : 0;
      any = any || h_active[col];
    }
    first = false;
    if (!any) break;
    // start a cycle: V_0 = r / |r|, g = |r| e_1
    H2_CUDA_TRY(cudaMemcpyAsync(active.p, h_active.data(), nrhs * 4, cudaMemcpyHostToDevice, st));
    k_scale<<<grid1(tot), kT, 0, st>>>(W.p, hn.p, active.p, n, nrhs, Vb.p);
    std::fill(h_g0.begin(), h_g0.end(), 0.0);
    for (int col = 0; col < nrhs; ++col) h_g0[col] = h_rn[col];
    H2_CUDA_TRY(cudaMemcpyAsync(g.p, h_g0.data(), (mr + 1) * nrhs * 8, cudaMemcpyHostToDevice, st));
    for (int col = 0; col < nrhs; ++col) h_jc[col] = 0;
    std::vector<double> rs(2 * nrhs);
    for (int j = 0; j < mr; ++j) {
      double *Vj = Vb.p + (int64_t)j * tot, *Vj1 = Vb.p + (int64_t)(j + 1) * tot;
      if ((rc = run_matvec(c, Vj, W.p, nrhs, true))) return rc;
      // classical Gram-Schmidt, twice
      k_dots<<<dim3(nrhs, j + 1), kT, 0, st>>>(Vb.p, W.p, n, nrhs, h1.p);
      k_orth<<<grid1(tot), kT, 0, st>>>(Vb.p, h1.p, j + 1, n, nrhs, W.p);
      k_dots<<<dim3(nrhs, j + 1), kT, 0, st>>>(Vb.p, W.p, n, nrhs, h2b.p);
      k_orth<<<grid1(tot), kT, 0, st>>>(Vb.p, h2b.p, j + 1, n, nrhs, W.p);
      k_dots<<<dim3(nrhs, 1), kT, 0, st>>>(W.p, W.p, n, nrhs, hn.p);
      k_sqrt<<<(nrhs + 63) / 64, 64, 0, st>>>(hn.p, nrhs);
      k_scale<<<grid1(tot), kT, 0, st>>>(W.p, hn.p, active.p, n, nrhs, Vj1);
      k_givens<<<(nrhs + 63) / 64, 64, 0, st>>>(h1.p, h2b.p, hn.p, j, mr, nrhs, H.p, cs.p, sn.p, g.p, resid.p,
                                                active.p);
      H2_CUDA_TRY(cudaGetLastError());
      H2_CUDA_TRY(cudaMemcpyAsync(rs.data(), resid.p, nrhs * 8, cudaMemcpyDeviceToHost, st));
      H2_CUDA_TRY(cudaMemcpyAsync(rs.data() + nrhs, hn.p, nrhs * 8, cudaMemcpyDeviceToHost, st));
      H2_CUDA_TRY(cudaStreamSynchronize(st));
      bool still = false;
      for (int col = 0; col < nrhs; ++col) {
        if (!h_active[col]) continue;
        h_jc[col] = j + 1;
        h_iters[col]++;
        if (rs[col] <= rtol * h_bn[col] || rs[nrhs + col] == 0.0 || h_iters[col] >= maxit) h_active[col] = 0;
        still = still || h_active[col];
      }
      if (!still) break;
      H2_CUDA_TRY(cudaMemcpyAsync(active.p, h_active.data(), nrhs * 4, cudaMemcpyHostToDevice, st));
    }
    H2_CUDA_TRY(cudaMemcpyAsync(jc.p, h_jc.data(), nrhs * 4, cudaMemcpyHostToDevice, st));
    k_backsolve<<<(nrhs + 63) / 64, 64, 0, st>>>(H.p, g.p, jc.p, mr, nrhs, yv.p);
    k_update<<<grid1(tot), kT, 0, st>>>(Vb.p, yv.p, jc.p, n, nrhs, z);
    H2_CUDA_TRY(cudaGetLastError());
  }
  int status = H2_OK;
  for (int col = 0; col < nrhs; ++col) {
    bool ok = h_res[col] <= rtol;
    if (!ok) status = H2_ENOCONV;
    if (info) {
      info[col].iters = h_iters[col];
      info[col].relres = h_res[col];
      info[col].status = ok ? H2_OK : H2_ENOCONV;
    }
  }
  if (status != H2_OK) fail(H2_ENOCONV, "GMRES reached maxit before the residual target");
  return status;
}

}  // namespace h2
