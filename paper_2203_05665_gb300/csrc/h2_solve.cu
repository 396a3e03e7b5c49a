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

}  // namespace

void free_gmres_work(GmresWork &w) {
  double *dp[] = {w.Vb, w.W, w.H, w.cs, w.sn, w.g, w.h1, w.h2, w.hn, w.resid, w.yv, w.bn, w.r, w.d, w.Az};
  for (double *p : dp)
    if (p) cudaFree(p);
  if (w.active) cudaFree(w.active);
  if (w.jc) cudaFree(w.jc);
  w = GmresWork();
}

static int ensure_gmres_work(Ctx &c, int nrhs, int restart) {
  GmresWork &w = c.gw;
  if (nrhs <= w.cols && restart <= w.restart) return H2_OK;
  const int cols = std::max(nrhs, w.cols), mr = std::max(restart, w.restart);
  free_gmres_work(w);
  const size_t n = (size_t)c.d.n, tot = n * cols;
  bool ok = true;
  auto al = [&](double **p, size_t cnt) { ok = ok && cudaMalloc(p, std::max<size_t>(cnt, 1) * 8) == cudaSuccess; };
  al(&w.Vb, (size_t)(mr + 1) * tot);
  al(&w.W, tot);
  al(&w.H, (size_t)(mr + 1) * mr * cols);
  al(&w.cs, (size_t)mr * cols);
  al(&w.sn, (size_t)mr * cols);
  al(&w.g, (size_t)(mr + 1) * cols);
  al(&w.h1, (size_t)(mr + 1) * cols);
  al(&w.h2, (size_t)(mr + 1) * cols);
  al(&w.hn, cols);
  al(&w.resid, cols);
  al(&w.yv, (size_t)mr * cols);
  al(&w.bn, cols);
  al(&w.r, tot);
  al(&w.d, tot);
  al(&w.Az, tot);
  ok = ok && cudaMalloc(&w.active, cols * 4) == cudaSuccess && cudaMalloc(&w.jc, cols * 4) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_gmres_work(w);
    return fail(H2_ENOMEM, "GMRES work space");
  }
  w.cols = cols;
  w.restart = mr;
  return H2_OK;
}

int run_gmres(Ctx &c, const double *b, double *z, int nrhs, double rtol, int restart, int maxit,
              h2_solve_info *info) {
  const int64_t n = c.d.n, tot = n * nrhs;
  const int mr = restart;
  cudaStream_t st = c.stream;
  int rc;
  if ((rc = ensure_gmres_work(c, nrhs, restart))) return rc;
  struct P {
    double *p;
  };
  GmresWork &w = c.gw;
  P Vb{w.Vb}, W{w.W}, H{w.H}, cs{w.cs}, sn{w.sn}, g{w.g}, h1{w.h1}, h2b{w.h2}, hn{w.hn}, resid{w.resid}, yv{w.yv},
      bn{w.bn};
  struct I {
    int *p;
  } active{w.active}, jc{w.jc};

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
  int derr = take_device_error(c);
  return derr ? derr : status;
}

__global__ void k_axpy_cols(const double *__restrict__ d, int64_t total, double *__restrict__ z) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    z[e] += d[e];
}

__global__ void k_mask_cols(const int *__restrict__ keep, int64_t n, int64_t total, double *__restrict__ v) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    if (!keep[e / n]) v[e] = 0.0;
}

// Mixed-precision iterative refinement around GMRES (GMRES-IR, Carson and
// Higham 2018): z = 0; repeat r = b - G~_hi z (hi arithmetic), solve
// G~_lo d = r by GMRES(restart) to inner_rtol, z += d; until |r| <= rtol |b|
// per column.  The Krylov arithmetic is FP64 throughout.
int run_gmres_ir(Ctx &hi, Ctx &lo, const double *b, double *z, int nrhs, double rtol, double inner_rtol,
                 int restart, int maxit_inner, int maxit_outer, h2_solve_info *info) {
  const int64_t n = hi.d.n, tot = n * nrhs;
  cudaStream_t st = hi.stream;
  int rc;
  if ((rc = ensure_gmres_work(hi, nrhs, 1))) return rc;
  double *r = hi.gw.r, *d = hi.gw.d, *Az = hi.gw.Az, *nrm = hi.gw.hn;
  int *keep = hi.gw.active;
  std::vector<double> h_bn(nrhs), h_rn(nrhs), h_res(nrhs, 1.0);
  std::vector<int> h_keep(nrhs, 1), h_iters(nrhs, 0), h_outer(nrhs, 0);
  std::vector<h2_solve_info> inner(nrhs);
  k_dots<<<dim3(nrhs, 1), kT, 0, st>>>(b, b, n, nrhs, nrm);
  k_sqrt<<<(nrhs + 63) / 64, 64, 0, st>>>(nrm, nrhs);
  H2_CUDA_TRY(cudaMemcpyAsync(h_bn.data(), nrm, nrhs * 8, cudaMemcpyDeviceToHost, st));
  H2_CUDA_TRY(cudaMemsetAsync(z, 0, tot * 8, st));
  H2_CUDA_TRY(cudaMemcpyAsync(r, b, tot * 8, cudaMemcpyDeviceToDevice, st));
  H2_CUDA_TRY(cudaStreamSynchronize(st));
  for (int outer = 0;; ++outer) {
    // residual norms and convergence per column
    k_dots<<<dim3(nrhs, 1), kT, 0, st>>>(r, r, n, nrhs, nrm);
    k_sqrt<<<(nrhs + 63) / 64, 64, 0, st>>>(nrm, nrhs);
    H2_CUDA_TRY(cudaMemcpyAsync(h_rn.data(), nrm, nrhs * 8, cudaMemcpyDeviceToHost, st));
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    bool any = false;
    for (int col = 0; col < nrhs; ++col) {
      h_res[col] = h_bn[col] > 0 ? h_rn[col] / h_bn[col] : 0.0;
      h_keep[col] = h_res[col] > rtol && outer < maxit_outer;
      any = any || h_keep[col];
    }
    if (!any) break;
    H2_CUDA_TRY(cudaMemcpyAsync(keep, h_keep.data(), nrhs * 4, cudaMemcpyHostToDevice, st));
    k_mask_cols<<<grid1(tot), kT, 0, st>>>(keep, n, tot, r);
    // inner solve in the low precision (its own stream is the lo handle's)
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    rc = run_gmres(lo, r, d, nrhs, inner_rtol, restart, maxit_inner, inner.data());
    if (rc != H2_OK && rc != H2_ENOCONV) return rc;
    H2_CUDA_TRY(cudaStreamSynchronize(lo.stream));
    for (int col = 0; col < nrhs; ++col)
      if (h_keep[col]) {
        h_iters[col] += inner[col].iters;
        h_outer[col]++;
      }
    k_axpy_cols<<<grid1(tot), kT, 0, st>>>(d, tot, z);
    if ((rc = run_matvec(hi, z, Az, nrhs, true))) return rc;
    k_residual<<<grid1(tot), kT, 0, st>>>(b, Az, tot, r);
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
  if (status != H2_OK) fail(H2_ENOCONV, "refinement reached its step limit before the residual target");
  int derr = take_device_error(hi);
  return derr ? derr : status;
}

}  // namespace h2
