// Restarted GMRES(restart) on the device for G~ z = b, every right-hand side
// an independent Krylov process (Saad, Iterative Methods for Sparse Linear
// Systems, Alg. 6.9, with classical Gram-Schmidt applied twice).  All
// Krylov arithmetic is FP64; the product runs in the handle's precision.
// The paper names Krylov methods for the system Gz = b (Section 1) without
// fixing one.
#include <algorithm>
#include <cmath>
#include <vector>

#include "h2_internal.hpp"

namespace h2 {

namespace {

constexpr int kT = 256;

// Gram-Schmidt dot products, 8 vectors per CTA so that W is read once per 8
// dots: grid (nrhs, ceil(nvec / 8), Z); CTA (c, g, z) sums rows
// [n z / Z, n (z + 1) / Z) and writes part[(z nvec + i) nrhs + c]; with
// Z > 1 k_dots_sum adds the Z chunks in order (no atomics: reproducible).
constexpr int kDotVB = 8;

__global__ void __launch_bounds__(256) k_dots8(const double *__restrict__ X, const double *__restrict__ W, int64_t n,
                                               int nrhs, int nvec, double *__restrict__ part) {
  __shared__ double red[kDotVB][8];
  const int c = blockIdx.x, i0 = blockIdx.y * kDotVB, z = blockIdx.z, Z = gridDim.z;
  const int64_t r0 = n * z / Z, r1 = n * (z + 1) / Z;
  double acc[kDotVB];
#pragma unroll
  for (int k = 0; k < kDotVB; ++k) acc[k] = 0.0;
  const double *wc = W + (int64_t)c * n;
  const double *xc = X + ((int64_t)i0 * nrhs + c) * n;   // vector i0 + k at xc + k nrhs n
  const int64_t vs = (int64_t)nrhs * n, bd = blockDim.x;
  int64_t r = r0 + threadIdx.x;
  // four rows per thread and pass: 36 independent loads in flight instead of 9
  for (; r + 3 * bd < r1; r += 4 * bd) {
    double w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) w[u] = wc[r + u * bd];
#pragma unroll
    for (int k = 0; k < kDotVB; ++k)
      if (i0 + k < nvec) {
        const double *xk = xc + k * vs;
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[k] = fma(xk[r + u * bd], w[u], acc[k]);
      }
  }
  for (; r < r1; r += bd) {
    const double w = wc[r];
#pragma unroll
    for (int k = 0; k < kDotVB; ++k)
      if (i0 + k < nvec) acc[k] = fma(xc[k * vs + r], w, acc[k]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kDotVB; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < kDotVB && i0 + (int)threadIdx.x < nvec) {
    double sum = 0.0;
    for (int w8 = 0; w8 < (int)(blockDim.x >> 5); ++w8) sum += red[threadIdx.x][w8];
    part[((int64_t)z * nvec + i0 + threadIdx.x) * nrhs + c] = sum;
  }
}

__global__ void k_dots_sum(const double *__restrict__ part, int Z, int nvec, int nrhs, double *__restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nvec * nrhs) return;
  double s = 0.0;
  for (int z = 0; z < Z; ++z) s += part[(int64_t)z * nvec * nrhs + e];
  out[e] = s;
}

constexpr int kDotMaxZ = 64;

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

// v[:, c] = w[:, c] / nrm[c] for active columns with nrm > 0, else 0; grid (., nrhs):
// the column's reciprocal is formed once per CTA (FP64 division is slow on this GPU)
__global__ void k_scale(const double *__restrict__ W, const double *__restrict__ nrm, const int *__restrict__ active,
                        int64_t n, int nrhs, double *__restrict__ Vout) {
  const int c = blockIdx.y;
  const double d = nrm[c];
  const double inv = (active[c] && d > 0) ? 1.0 / d : 0.0;
  const double *w = W + (int64_t)c * n;
  double *v = Vout + (int64_t)c * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    v[e] = w[e] * inv;
}

// Hessenberg column j: h1 + h2 from the two Gram-Schmidt passes, then the
// Givens rotations; H[(i * mr + j) * nrhs + c].  The column's convergence
// test runs here too: it leaves the cycle (active = 0) once its residual
// estimate reaches tol, at a breakdown (hn = 0) or at its iteration limit;
// itc counts its iterations and jc its Arnoldi vectors.
__global__ void k_givens(const double *__restrict__ h1, const double *__restrict__ h2, const double *__restrict__ hn,
                         int j, int mr, int nrhs, double *__restrict__ H, double *__restrict__ cs,
                         double *__restrict__ sn, double *__restrict__ g, double *__restrict__ resid,
                         int *__restrict__ active, const double *__restrict__ tolv, const int *__restrict__ maxv,
                         int *__restrict__ itc, int *__restrict__ jc) {
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
  const double rc = fabs(sj * gj);
  resid[c] = rc;
  const int it = itc[c] + 1;
  itc[c] = it;
  jc[c] = j + 1;
  if (rc <= tolv[c] || hn[c] == 0.0 || it >= maxv[c]) active[c] = 0;
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

// out[i nrhs + c] = <X_i[:, c], W[:, c]> for i < nvec (part: kDotMaxZ nvec nrhs doubles of
// scratch, or NULL for one chunk per column)
void dots(const double *X, const double *W, int64_t n, int nrhs, int nvec, double *out, double *part,
          cudaStream_t st) {
  // enough CTAs to fill the GPU, chunks of at least 1024 rows
  const int groups = (nvec + kDotVB - 1) / kDotVB;
  int Z = part ? (int)std::min<int64_t>(kDotMaxZ, std::max<int64_t>(1, n / 1024)) : 1;
  while (Z > 1 && (int64_t)nrhs * groups * Z > 4 * 152) --Z;
  k_dots8<<<dim3(nrhs, groups, Z), 256, 0, st>>>(X, W, n, nrhs, nvec, Z > 1 ? part : out);
  if (Z > 1) k_dots_sum<<<(nvec * nrhs + 127) / 128, 128, 0, st>>>(part, Z, nvec, nrhs, out);
}

// 2-norms of the ncols columns of v (n rows) into out (device)
void norms(const double *v, int64_t n, int ncols, double *out, double *part, cudaStream_t st) {
  dots(v, v, n, ncols, 1, out, part, st);
  k_sqrt<<<(ncols + 63) / 64, 64, 0, st>>>(out, ncols);
}

void launch_scale(const double *W, const double *nrm, const int *active, int64_t n, int nrhs, double *V,
                  cudaStream_t st) {
  const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((n + kT - 1) / kT, std::max(1, 4 * 152 / nrhs)));
  k_scale<<<dim3(gx, nrhs), kT, 0, st>>>(W, nrm, active, n, nrhs, V);
}

}  // namespace

void free_gmres_work(GmresWork &w) {
  double *dp[] = {w.Vb, w.W, w.H, w.cs, w.sn, w.g, w.h1, w.h2, w.hn, w.resid, w.yv, w.bn, w.r, w.d, w.Az, w.dpart};
  for (double *p : dp)
    if (p) cudaFree(p);
  for (int *p : {w.active, w.jc, w.maxv, w.itc})
    if (p) cudaFree(p);
  if (w.tolv) cudaFree(w.tolv);
  if (w.hflag) cudaFreeHost(w.hflag);
  if (w.ev) cudaEventDestroy(w.ev);
  w = GmresWork();
}

static int ensure_gmres_work(Ctx &c, int nrhs, int restart) {
  GmresWork &w = c.gw;
  if (nrhs <= w.cols && restart <= w.restart) return H2_OK;
  return alloc_gmres_work(w, c.d.n, std::max(nrhs, w.cols), std::max(restart, w.restart));
}

int alloc_gmres_work(GmresWork &w, int64_t n_, int cols, int mr) {
  free_gmres_work(w);
  const size_t n = (size_t)n_, tot = n * cols;
  bool ok = true;
  auto al = [&](double **p, size_t cnt) { ok = ok && dmalloc(p, std::max<size_t>(cnt, 1) * 8) == cudaSuccess; };
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
  al(&w.dpart, (size_t)kDotMaxZ * (mr + 1) * cols);
  al(&w.r, tot);
  al(&w.d, tot);
  al(&w.Az, tot);
  al(&w.tolv, cols);
  ok = ok && dmalloc(&w.active, cols * 4) == cudaSuccess && dmalloc(&w.jc, cols * 4) == cudaSuccess &&
       dmalloc(&w.maxv, cols * 4) == cudaSuccess && dmalloc(&w.itc, cols * 4) == cudaSuccess &&
       cudaMallocHost(&w.hflag, cols * 4) == cudaSuccess &&
       cudaEventCreateWithFlags(&w.ev, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_gmres_work(w);
    return fail(H2_ENOMEM, "GMRES work space");
  }
  w.cols = cols;
  w.restart = mr;
  return H2_OK;
}

// One GMRES cycle from a zero initial guess for G~ D = R, column by column:
// Arnoldi with classical Gram-Schmidt applied twice, Givens rotations, and
// the update D = V y.  A column takes part if act[c] and |R_c| > tol[c]; it
// stops when its residual estimate drops to tol[c], at a breakdown, after
// restart iterations or after max_it[c] iterations.  iters[c] receives the
// iterations done.  R may alias w.W.  All host arrays have nrhs entries.
LinOp ctx_op(Ctx &c) {
  LinOp op;
  op.n = c.d.n;
  op.stream = c.stream;
  Ctx *cp = &c;
  op.apply = [cp](const double *x, double *y, int nrhs) { return run_matvec(*cp, x, y, nrhs, true); };
  return op;
}

int gmres_cycle(const LinOp &op, GmresWork &w, const double *R, double *D, int nrhs, int restart,
                const double *tol, const int *act, const int *max_it, int *iters) {
  const int64_t n = op.n, tot = n * nrhs;
  const int mr = restart;
  cudaStream_t st = op.stream;
  int rc;
  std::vector<double> rn(nrhs), g0((size_t)(mr + 1) * nrhs, 0.0);
  std::vector<int> on(nrhs, 0);
  norms(R, n, nrhs, w.hn, w.dpart, st);
  H2_CUDA_TRY(cudaMemcpyAsync(rn.data(), w.hn, nrhs * 8, cudaMemcpyDeviceToHost, st));
  H2_CUDA_TRY(cudaStreamSynchronize(st));
  bool any = false;
  for (int col = 0; col < nrhs; ++col) {
    iters[col] = 0;
    on[col] = act[col] && rn[col] > tol[col] && max_it[col] > 0;
    any = any || on[col];
    g0[col] = rn[col];
  }
  H2_CUDA_TRY(cudaMemsetAsync(D, 0, tot * 8, st));
  if (!any) return H2_OK;
  H2_CUDA_TRY(cudaMemcpyAsync(w.active, on.data(), nrhs * 4, cudaMemcpyHostToDevice, st));
  H2_CUDA_TRY(cudaMemcpyAsync(w.tolv, tol, nrhs * 8, cudaMemcpyHostToDevice, st));
  H2_CUDA_TRY(cudaMemcpyAsync(w.maxv, max_it, nrhs * 4, cudaMemcpyHostToDevice, st));
  H2_CUDA_TRY(cudaMemsetAsync(w.itc, 0, nrhs * 4, st));
  H2_CUDA_TRY(cudaMemsetAsync(w.jc, 0, nrhs * 4, st));
  launch_scale(R, w.hn, w.active, n, nrhs, w.Vb, st);
  H2_CUDA_TRY(cudaMemcpyAsync(w.g, g0.data(), (mr + 1) * nrhs * 8, cudaMemcpyHostToDevice, st));
  // The host looks at the columns' state every `check` iterations only (for
  // small systems an iteration is shorter than a host round trip, for large
  // ones an iteration past the last convergence costs more than the trip),
  // and one check late: the flags of iteration j are copied to pinned memory
  // behind it and read after iteration j + check has been queued, so the GPU
  // never waits for the host.  An iteration queued after every column has
  // stopped changes nothing (all its updates are masked by `active`).
  const int check = tot >= ((int64_t)1 << 20) ? 1 : 4;
  bool pending = false;
  for (int j = 0; j < mr; ++j) {
    double *Vj = w.Vb + (int64_t)j * tot, *Vj1 = w.Vb + (int64_t)(j + 1) * tot;
    if ((rc = op.apply(Vj, w.W, nrhs))) return rc;
    dots(w.Vb, w.W, n, nrhs, j + 1, w.h1, w.dpart, st);
    k_orth<<<grid1(tot), kT, 0, st>>>(w.Vb, w.h1, j + 1, n, nrhs, w.W);
    dots(w.Vb, w.W, n, nrhs, j + 1, w.h2, w.dpart, st);
    k_orth<<<grid1(tot), kT, 0, st>>>(w.Vb, w.h2, j + 1, n, nrhs, w.W);
    dots(w.W, w.W, n, nrhs, 1, w.hn, w.dpart, st);
    k_sqrt<<<(nrhs + 63) / 64, 64, 0, st>>>(w.hn, nrhs);
    launch_scale(w.W, w.hn, w.active, n, nrhs, Vj1, st);
    k_givens<<<(nrhs + 63) / 64, 64, 0, st>>>(w.h1, w.h2, w.hn, j, mr, nrhs, w.H, w.cs, w.sn, w.g, w.resid,
                                              w.active, w.tolv, w.maxv, w.itc, w.jc);
    H2_CUDA_TRY(cudaGetLastError());
    if (pending) {
      H2_CUDA_TRY(cudaEventSynchronize(w.ev));
      pending = false;
      bool still = false;
      for (int col = 0; col < nrhs; ++col) still = still || w.hflag[col];
      if (!still) break;
    }
    if ((j + 1) % check == 0 && j + 1 < mr) {
      H2_CUDA_TRY(cudaMemcpyAsync(w.hflag, w.active, nrhs * 4, cudaMemcpyDeviceToHost, st));
      H2_CUDA_TRY(cudaEventRecord(w.ev, st));
      pending = true;
    }
  }
  H2_CUDA_TRY(cudaMemcpyAsync(iters, w.itc, nrhs * 4, cudaMemcpyDeviceToHost, st));
  k_backsolve<<<(nrhs + 63) / 64, 64, 0, st>>>(w.H, w.g, w.jc, mr, nrhs, w.yv);
  k_update<<<grid1(tot), kT, 0, st>>>(w.Vb, w.yv, w.jc, n, nrhs, D);
  H2_CUDA_TRY(cudaGetLastError());
  H2_CUDA_TRY(cudaStreamSynchronize(st));   // iters (host) is written by the copy above
  return H2_OK;
}

__global__ void k_axpy_cols(const double *__restrict__ d, int64_t total, double *__restrict__ z) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    z[e] += d[e];
}

// Restarted GMRES(restart): z = 0; repeat r = b - G~ z, one cycle for G~ d = r
// with the column tolerance rtol |b|, z += d; a column stops when its true
// relative residual is <= rtol or after maxit iterations.
int run_gmres(Ctx &c, const double *b, double *z, int nrhs, double rtol, int restart, int maxit,
              h2_solve_info *info) {
  int rc;
  if ((rc = ensure_gmres_work(c, nrhs, restart))) return rc;
  const int status = run_gmres_op(ctx_op(c), c.gw, b, z, nrhs, rtol, restart, maxit, info);
  if (status != H2_OK && status != H2_ENOCONV) return status;
  int derr = take_device_error(c);
  return derr ? derr : status;
}

int run_gmres_op(const LinOp &op, GmresWork &w, const double *b, double *z, int nrhs, double rtol, int restart,
                 int maxit, h2_solve_info *info) {
  const int64_t n = op.n, tot = n * nrhs;
  cudaStream_t st = op.stream;
  int rc;
  std::vector<double> bn(nrhs), rn(nrhs), res(nrhs, 0.0), tol(nrhs);
  std::vector<int> act(nrhs), left(nrhs), it(nrhs), iters(nrhs, 0);
  norms(b, n, nrhs, w.bn, w.dpart, st);
  H2_CUDA_TRY(cudaMemcpyAsync(bn.data(), w.bn, nrhs * 8, cudaMemcpyDeviceToHost, st));
  H2_CUDA_TRY(cudaMemsetAsync(z, 0, tot * 8, st));
  H2_CUDA_TRY(cudaMemcpyAsync(w.r, b, tot * 8, cudaMemcpyDeviceToDevice, st));
  for (bool first = true;; first = false) {
    if (!first) {
      if ((rc = op.apply(z, w.Az, nrhs))) return rc;
      k_residual<<<grid1(tot), kT, 0, st>>>(b, w.Az, tot, w.r);
    }
    norms(w.r, n, nrhs, w.hn, w.dpart, st);
    H2_CUDA_TRY(cudaMemcpyAsync(rn.data(), w.hn, nrhs * 8, cudaMemcpyDeviceToHost, st));
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    bool any = false;
    for (int col = 0; col < nrhs; ++col) {
      res[col] = bn[col] > 0 ? rn[col] / bn[col] : 0.0;
      act[col] = res[col] > rtol && iters[col] < maxit;
      left[col] = maxit - iters[col];
      tol[col] = rtol * bn[col];
      any = any || act[col];
    }
    if (!any) break;
    if ((rc = gmres_cycle(op, w, w.r, w.d, nrhs, restart, tol.data(), act.data(), left.data(), it.data())))
      return rc;
    for (int col = 0; col < nrhs; ++col) iters[col] += it[col];
    k_axpy_cols<<<grid1(tot), kT, 0, st>>>(w.d, tot, z);
  }
  int status = H2_OK;
  for (int col = 0; col < nrhs; ++col) {
    bool ok = res[col] <= rtol;
    if (!ok) status = H2_ENOCONV;
    if (info) {
      info[col].iters = iters[col];
      info[col].relres = res[col];
      info[col].status = ok ? H2_OK : H2_ENOCONV;
    }
  }
  if (status != H2_OK) fail(H2_ENOCONV, "GMRES reached maxit before the residual target");
  return status;
}


__global__ void k_mask_cols(const int *__restrict__ keep, int64_t n, int64_t total, double *__restrict__ v) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    if (!keep[e / n]) v[e] = 0.0;
}

void k_launch_residual(const double *b, const double *Az, int64_t total, double *r, cudaStream_t st) {
  k_residual<<<grid1(total), kT, 0, st>>>(b, Az, total, r);
}

void k_launch_axpy(const double *d, int64_t total, double *z, cudaStream_t st) {
  k_axpy_cols<<<grid1(total), kT, 0, st>>>(d, total, z);
}

int column_norms(Ctx &c, const double *v, int64_t n, int ncols, double *dev_tmp, double *host_out) {
  // chunked sums when the handle's GMRES scratch is large enough
  double *part = (c.gw.dpart && ncols <= c.gw.cols) ? c.gw.dpart : nullptr;
  norms(v, n, ncols, dev_tmp, part, c.stream);
  H2_CUDA_TRY(cudaGetLastError());
  H2_CUDA_TRY(cudaMemcpyAsync(host_out, dev_tmp, ncols * 8, cudaMemcpyDeviceToHost, c.stream));
  H2_CUDA_TRY(cudaStreamSynchronize(c.stream));
  return H2_OK;
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
  norms(b, n, nrhs, nrm, hi.gw.dpart, st);
  H2_CUDA_TRY(cudaMemcpyAsync(h_bn.data(), nrm, nrhs * 8, cudaMemcpyDeviceToHost, st));
  H2_CUDA_TRY(cudaMemsetAsync(z, 0, tot * 8, st));
  H2_CUDA_TRY(cudaMemcpyAsync(r, b, tot * 8, cudaMemcpyDeviceToDevice, st));
  H2_CUDA_TRY(cudaStreamSynchronize(st));
  for (int outer = 0;; ++outer) {
    // residual norms and convergence per column
    norms(r, n, nrhs, nrm, hi.gw.dpart, st);
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
