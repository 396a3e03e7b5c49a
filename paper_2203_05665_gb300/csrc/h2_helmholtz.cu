// The Helmholtz single-layer matrix of Section 1 (kernel e^{i kappa r} /
// (4 pi r)) as a pair of real H^2 matrices, G = G_c + i G_s, with the real
// kernels cos(kappa r) / (4 pi r) and sin(kappa r) / (4 pi r): every step of
// Algorithms 1-3 stays real, the complex structure lives in how the two
// products are combined.  A complex product runs the real products of both
// parts on the real and imaginary columns together (2 nrhs columns, one
// launch sequence each) and combines
//   y_re = G_c x_re - G_s x_im,   y_im = G_c x_im + G_s x_re.
// Solves run the real GMRES on the equivalent real system
//   [G_c  -G_s] [z_re]   [b_re]
//   [G_s   G_c] [z_im] = [b_im]
// whose vectors are the complex ones stacked per column (real part, then
// imaginary part): its residual norm is the complex residual's.
#include <algorithm>
#include <cmath>
#include <new>

#include "h2_internal.hpp"

struct h2_zctx {
  h2_ctx *part[2] = {nullptr, nullptr};   // real part (cos kernel), imaginary part (sin kernel)
  int device = 0;
  cudaStream_t stream = nullptr;
  double kappa = 0.0;
  int64_t n = 0;
  int cap = 0;                              // complex right-hand sides the work arrays hold
  double *X = nullptr, *A = nullptr, *B = nullptr;   // n x 2 cap each
  double *sb = nullptr, *sz = nullptr;      // 2 n x cap each: stacked solve vectors
  int scap = 0;
  h2::GmresWork gw;                         // GMRES work space for vectors of length 2 n
};

namespace h2 {
namespace {

int zgrid(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

// X[:, 2c] = Re x[:, c], X[:, 2c + 1] = Im x[:, c] (x interleaved complex)
__global__ void k_z_split(const double *__restrict__ x, int64_t n, int nrhs, double *__restrict__ X) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, i = e - c * n;
    X[2 * c * n + i] = x[2 * e];
    X[(2 * c + 1) * n + i] = x[2 * e + 1];
  }
}

// interleaved y from A = G_c X and B = G_s X
__global__ void k_z_combine(const double *__restrict__ A, const double *__restrict__ B, int64_t n, int nrhs,
                            double *__restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, i = e - c * n;
    const int64_t re = 2 * c * n + i, im = (2 * c + 1) * n + i;
    y[2 * e] = A[re] - B[im];
    y[2 * e + 1] = A[im] + B[re];
  }
}

// the same result in the stacked form: y[c 2n + i] real part, y[c 2n + n + i] imaginary part
__global__ void k_z_combine_st(const double *__restrict__ A, const double *__restrict__ B, int64_t n, int nrhs,
                               double *__restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, i = e - c * n;
    const int64_t re = 2 * c * n + i, im = (2 * c + 1) * n + i;
    y[re] = A[re] - B[im];
    y[im] = A[im] + B[re];
  }
}

// interleaved complex <-> stacked real (per column: real parts, then imaginary parts)
__global__ void k_z_il_to_st(const double *__restrict__ x, int64_t n, int nrhs, double *__restrict__ s) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, i = e - c * n;
    s[2 * c * n + i] = x[2 * e];
    s[(2 * c + 1) * n + i] = x[2 * e + 1];
  }
}
__global__ void k_z_st_to_il(const double *__restrict__ s, int64_t n, int nrhs, double *__restrict__ x) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, i = e - c * n;
    x[2 * e] = s[2 * c * n + i];
    x[2 * e + 1] = s[(2 * c + 1) * n + i];
  }
}

int zwork(h2_zctx &h, int nrhs) {
  if (nrhs <= h.cap) return H2_OK;
  cudaFree(h.X);
  cudaFree(h.A);
  cudaFree(h.B);
  h.X = h.A = h.B = nullptr;
  h.cap = 0;
  const size_t bytes = (size_t)h.n * 2 * nrhs * 8;
  if (dmalloc(&h.X, bytes) != cudaSuccess || dmalloc(&h.A, bytes) != cudaSuccess ||
      dmalloc(&h.B, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(H2_ENOMEM, "Helmholtz work arrays");
  }
  h.cap = nrhs;
  return H2_OK;
}

// the real products of both parts on the n x 2 nrhs array X (real and
// imaginary columns side by side) into A and B
int zproducts(h2_zctx &h, const double *X, int nrhs) {
  int rc;
  if ((rc = run_matvec(*h.part[0], X, h.A, 2 * nrhs, true))) return rc;
  return run_matvec(*h.part[1], X, h.B, 2 * nrhs, true);
}

int ztake_error(h2_zctx &h) {
  int rc = take_device_error(*h.part[0]);
  const int rc2 = take_device_error(*h.part[1]);
  return rc ? rc : rc2;
}

}  // namespace
}  // namespace h2

using namespace h2;

extern "C" {

int h2_zdestroy(h2_zhandle h) {
  if (!h) return H2_OK;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  for (h2_ctx *p : h->part) h2_destroy(p);
  for (double *p : {h->X, h->A, h->B, h->sb, h->sz})
    if (p) cudaFree(p);
  free_gmres_work(h->gw);
  delete h;
  return H2_OK;
}

int h2_zbuild(const double *vert, int64_t nv, const int32_t *tri, int64_t nt, int leaf_size, double eta, int order,
              double kappa, const h2_options *opt, h2_zhandle *out) {
  if (!out) return fail(H2_EINVAL, "out is NULL");
  *out = nullptr;
  if (!(kappa >= 0.0) || !std::isfinite(kappa)) return fail(H2_EINVAL, "kappa must be finite and >= 0");
  h2_options o;
  h2_options_default(&o);
  if (opt) o = *opt;
  if (o.prec != H2_F64 && o.prec != H2_F32 && o.prec != H2_F64_NATIVE)
    return fail(H2_EINVAL, "the Helmholtz matrix takes H2_F64, H2_F32 or H2_F64_NATIVE");
  if (o.coupling == H2_COUPLING_REGEN) return fail(H2_EINVAL, "the Helmholtz matrix stores its coupling matrices");
  o.coupling = H2_COUPLING_STORED;
  h2_zctx *h = new (std::nothrow) h2_zctx();
  if (!h) return fail(H2_ENOMEM, "handle");
  h->device = o.device;
  h->stream = (cudaStream_t)o.stream;
  h->kappa = kappa;
  int rc = build_handle(vert, nv, tri, nt, leaf_size, eta, order, &o, KernelFn{kKernelHelmholtzRe, kappa},
                        &h->part[0]);
  if (!rc)
    rc = build_handle(vert, nv, tri, nt, leaf_size, eta, order, &o, KernelFn{kKernelHelmholtzIm, kappa},
                      &h->part[1]);
  if (rc) {
    h2_zdestroy(h);
    return rc;
  }
  h->n = h->part[0]->d.n;
  *out = h;
  return H2_OK;
}

int h2_zpart(h2_zhandle h, int which, h2_handle *out) {
  if (!h || !out || (which != 0 && which != 1)) return fail(H2_EINVAL, "bad argument");
  *out = h->part[which];
  return H2_OK;
}

int h2_zinfo(h2_zhandle h, h2_stats *out) {
  if (!h || !out) return fail(H2_EINVAL, "NULL argument");
  int rc = h2_info(h->part[0], out);
  if (rc) return rc;
  out->device_bytes = h->part[0]->d.bytes + h->part[1]->d.bytes;
  return H2_OK;
}

int h2_zmatvec(h2_zhandle h, const double *x, double *y, int nrhs) {
  if (!h || !x || !y) return fail(H2_EINVAL, "NULL argument");
  if (nrhs < 1 || nrhs > 32) return fail(H2_EINVAL, "nrhs must be in [1, 32]");
  H2_CUDA_TRY(cudaSetDevice(h->device));
  int rc;
  if ((rc = zwork(*h, nrhs))) return rc;
  const int64_t tot = h->n * nrhs;
  k_z_split<<<zgrid(tot), 256, 0, h->stream>>>(x, h->n, nrhs, h->X);
  if ((rc = zproducts(*h, h->X, nrhs))) return rc;
  k_z_combine<<<zgrid(tot), 256, 0, h->stream>>>(h->A, h->B, h->n, nrhs, y);
  H2_CUDA_TRY(cudaGetLastError());
  return H2_OK;
}

int h2_zmatvec_host(h2_zhandle h, const double *x, double *y, int nrhs) {
  if (!h || !x || !y) return fail(H2_EINVAL, "NULL argument");
  if (nrhs < 1 || nrhs > 32) return fail(H2_EINVAL, "nrhs must be in [1, 32]");
  H2_CUDA_TRY(cudaSetDevice(h->device));
  const size_t bytes = (size_t)h->n * nrhs * 16;
  double *dx = nullptr, *dy = nullptr;
  if (dmalloc(&dx, bytes) != cudaSuccess || dmalloc(&dy, bytes) != cudaSuccess) {
    cudaFree(dx);
    cudaGetLastError();
    return fail(H2_ENOMEM, "Helmholtz staging buffers");
  }
  int rc = H2_OK;
  cudaError_t e = cudaMemcpyAsync(dx, x, bytes, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) rc = cuda_fail(e, "copy x");
  if (!rc) rc = h2_zmatvec(h, dx, dy, nrhs);
  if (!rc) {
    e = cudaMemcpyAsync(y, dy, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "copy y");
  }
  cudaFree(dx);
  cudaFree(dy);
  if (!rc) rc = ztake_error(*h);
  return rc;
}

int h2_zsolve(h2_zhandle h, const double *b, double *z, int nrhs, double rtol, int restart, int maxit,
              h2_solve_info *info) {
  if (!h || !b || !z) return fail(H2_EINVAL, "NULL argument");
  if (nrhs < 1 || nrhs > 32) return fail(H2_EINVAL, "nrhs must be in [1, 32]");
  if (restart < 1 || restart > 200 || maxit < 1 || !(rtol > 0.0)) return fail(H2_EINVAL, "bad solver parameters");
  H2_CUDA_TRY(cudaSetDevice(h->device));
  cudaPointerAttributes ab{}, az{};
  H2_CUDA_TRY(cudaPointerGetAttributes(&ab, b));
  H2_CUDA_TRY(cudaPointerGetAttributes(&az, z));
  const bool db = ab.type == cudaMemoryTypeDevice || ab.type == cudaMemoryTypeManaged;
  const bool dz = az.type == cudaMemoryTypeDevice || az.type == cudaMemoryTypeManaged;
  if (db != dz) return fail(H2_EINVAL, "b and z must both be host or both be device arrays");
  int rc;
  if ((rc = zwork(*h, nrhs))) return rc;
  const int64_t n = h->n, tot = n * nrhs;
  const size_t bytes = (size_t)tot * 16;
  if (nrhs > h->scap) {
    cudaFree(h->sb);
    cudaFree(h->sz);
    h->sb = h->sz = nullptr;
    h->scap = 0;
    if (dmalloc(&h->sb, bytes) != cudaSuccess || dmalloc(&h->sz, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(H2_ENOMEM, "Helmholtz solve vectors");
    }
    h->scap = nrhs;
  }
  if (nrhs > h->gw.cols || restart > h->gw.restart)
    if ((rc = alloc_gmres_work(h->gw, 2 * n, std::max(nrhs, h->gw.cols), std::max(restart, h->gw.restart))))
      return rc;
  // b into the stacked real form (through z's staging when b is on the host)
  if (db) {
    k_z_il_to_st<<<zgrid(tot), 256, 0, h->stream>>>(b, n, nrhs, h->sb);
  } else {
    H2_CUDA_TRY(cudaMemcpyAsync(h->sz, b, bytes, cudaMemcpyHostToDevice, h->stream));
    k_z_il_to_st<<<zgrid(tot), 256, 0, h->stream>>>(h->sz, n, nrhs, h->sb);
  }
  LinOp op;
  op.n = 2 * n;
  op.stream = h->stream;
  h2_zctx *hp = h;
  op.apply = [hp](const double *xs, double *ys, int nr) -> int {
    // a stacked column is the real column followed by the imaginary one: as an
    // n x 2 nr array it is exactly the side-by-side layout of the products
    int r = zproducts(*hp, xs, nr);
    if (r) return r;
    k_z_combine_st<<<zgrid(hp->n * nr), 256, 0, hp->stream>>>(hp->A, hp->B, hp->n, nr, ys);
    return (int)H2_OK;
  };
  rc = run_gmres_op(op, h->gw, h->sb, h->sz, nrhs, rtol, restart, maxit, info);
  if (rc != H2_OK && rc != H2_ENOCONV) return rc;
  const int status = rc;
  // z back to interleaved complex
  if (dz) {
    k_z_st_to_il<<<zgrid(tot), 256, 0, h->stream>>>(h->sz, n, nrhs, z);
  } else {
    k_z_st_to_il<<<zgrid(tot), 256, 0, h->stream>>>(h->sz, n, nrhs, h->sb);
    H2_CUDA_TRY(cudaMemcpyAsync(z, h->sb, bytes, cudaMemcpyDeviceToHost, h->stream));
  }
  H2_CUDA_TRY(cudaStreamSynchronize(h->stream));
  const int derr = ztake_error(*h);
  return derr ? derr : status;
}

}  // extern "C"
