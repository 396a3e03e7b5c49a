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
#include <algorithm>

#include "h2_internal.hpp"

namespace h2 {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxOut = 16;   // outputs per thread in the block-row kernels

template <class Tin, class Tout>
__global__ void k_permute_in(const Tin *__restrict__ x, int64_t n, int nrhs, const int32_t *__restrict__ pad_src,
                             int64_t npad, Tout *__restrict__ xpad) {
  const int64_t total = npad * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = e / nrhs;
    int r = (int)(e - p * nrhs);
    int32_t src = pad_src[p];
    xpad[e] = src >= 0 ? (Tout)x[src + r * n] : (Tout)0;
  }
}

template <class Tin, class Tout>
__global__ void k_permute_out(const Tin *__restrict__ ypad, int64_t n, int nrhs, const int32_t *__restrict__ pad_src,
                              int64_t npad, Tout *__restrict__ y) {
  const int64_t total = npad * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = e / nrhs;
    int r = (int)(e - p * nrhs);
    int32_t src = pad_src[p];
    if (src >= 0) y[src + r * n] = (Tout)ypad[e];
  }
}

// x^_leaf[nu][r] = sum_t V[t][nu] x[t][r]; one CTA per leaf
template <class T>
__global__ void k_leaf_forward(const T *__restrict__ V, const T *__restrict__ xpad, int L, int k, int nrhs,
                               int64_t leaf0, T *__restrict__ xhat) {
  extern __shared__ unsigned char smem_raw[];
  T *sV = reinterpret_cast<T *>(smem_raw);
  T *sx = sV + L * k;
  const int64_t j = blockIdx.x;
  for (int i = threadIdx.x; i < L * k; i += blockDim.x) sV[i] = V[j * L * k + i];
  for (int i = threadIdx.x; i < L * nrhs; i += blockDim.x) sx[i] = xpad[j * L * nrhs + i];
  __syncthreads();
  T *out = xhat + (leaf0 + j) * (int64_t)k * nrhs;
  for (int o = threadIdx.x; o < k * nrhs; o += blockDim.x) {
    int nu = o / nrhs, r = o - nu * nrhs;
    T acc = 0;
    for (int t = 0; t < L; ++t) acc += sV[t * k + nu] * sx[t * nrhs + r];
    out[o] = acc;
  }
}

// one mode product of the factored transfer: axis d, transpose or not.
// in/out: [k][nrhs] tensors with nu = jx + m jy + m^2 jz.
// trans: out[.., j, ..] = sum_{j'} F[j'][j] in[.., j', ..]   (E^T, upward)
// plain: out[.., j', ..] = sum_{j} F[j'][j] in[.., j, ..]    (E, downward)
template <class T>
__device__ __forceinline__ void mode_product(const T *__restrict__ F, const T *in, T *out, int m, int k, int nrhs,
                                             int d, bool trans) {
  const int stride = d == 0 ? 1 : (d == 1 ? m : m * m);
  for (int o = threadIdx.x; o < k * nrhs; o += blockDim.x) {
    int nu = o / nrhs, r = o - nu * nrhs;
    int jd = (nu / stride) % m;
    int base = nu - jd * stride;
    T acc = 0;
    for (int i = 0; i < m; ++i) {
      T f = trans ? F[i * m + jd] : F[jd * m + i];
      acc += f * in[(base + i * stride) * nrhs + r];
    }
    out[o] = acc;
  }
}

// upward: parents of level l; x^_parent = sum_children E_c^T x^_c
template <class T>
__global__ void k_upward(const T *__restrict__ Ef, int m, int k, int nrhs, int64_t par0, T *__restrict__ xhat) {
  extern __shared__ unsigned char smem_raw[];
  T *a = reinterpret_cast<T *>(smem_raw);
  T *b = a + k * nrhs;
  T *acc = b + k * nrhs;
  const int64_t par = par0 + blockIdx.x;
  const int kr = k * nrhs;
  for (int i = threadIdx.x; i < kr; i += blockDim.x) acc[i] = 0;
  for (int ch = 1; ch <= 2; ++ch) {
    const int64_t c = 2 * par + ch;
    for (int i = threadIdx.x; i < kr; i += blockDim.x) a[i] = xhat[c * kr + i];
    __syncthreads();
    const T *F = Ef + c * 3 * m * m;
    mode_product(F + 0 * m * m, a, b, m, k, nrhs, 0, true);
    __syncthreads();
    mode_product(F + 1 * m * m, b, a, m, k, nrhs, 1, true);
    __syncthreads();
    mode_product(F + 2 * m * m, a, b, m, k, nrhs, 2, true);
    __syncthreads();
    for (int i = threadIdx.x; i < kr; i += blockDim.x) acc[i] += b[i];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kr; i += blockDim.x) xhat[par * kr + i] = acc[i];
}

// downward: children of level l+1; y^_c += E_c y^_parent
template <class T>
__global__ void k_downward(const T *__restrict__ Ef, int m, int k, int nrhs, int64_t ch0, T *__restrict__ yhat) {
  extern __shared__ unsigned char smem_raw[];
  T *a = reinterpret_cast<T *>(smem_raw);
  T *b = a + k * nrhs;
  const int64_t c = ch0 + blockIdx.x, par = (c - 1) / 2;
  const int kr = k * nrhs;
  for (int i = threadIdx.x; i < kr; i += blockDim.x) a[i] = yhat[par * kr + i];
  __syncthreads();
  const T *F = Ef + c * 3 * m * m;
  mode_product(F + 0 * m * m, a, b, m, k, nrhs, 0, false);
  __syncthreads();
  mode_product(F + 1 * m * m, b, a, m, k, nrhs, 1, false);
  __syncthreads();
  mode_product(F + 2 * m * m, a, b, m, k, nrhs, 2, false);
  __syncthreads();
  for (int i = threadIdx.x; i < kr; i += blockDim.x) yhat[c * kr + i] += b[i];
}

// coupling: one CTA per row cluster t >= row0; y^_t = sum_b S_b x^_{s_b}
template <class T>
__global__ void k_coupling(const T *__restrict__ S, const int64_t *__restrict__ adm_ptr,
                           const int32_t *__restrict__ adm_col, int k, int nrhs, int64_t row0,
                           const T *__restrict__ xhat, T *__restrict__ yhat) {
  extern __shared__ unsigned char smem_raw[];
  T *sS = reinterpret_cast<T *>(smem_raw);
  T *sx = sS + k * k;
  const int64_t t = row0 + blockIdx.x;
  const int kr = k * nrhs;
  T acc[kMaxOut];
#pragma unroll
  for (int i = 0; i < kMaxOut; ++i) acc[i] = 0;
  for (int64_t e = adm_ptr[t]; e < adm_ptr[t + 1]; ++e) {
    const int64_t s = adm_col[e];
    __syncthreads();
    for (int i = threadIdx.x; i < k * k; i += blockDim.x) sS[i] = S[e * k * k + i];
    for (int i = threadIdx.x; i < kr; i += blockDim.x) sx[i] = xhat[s * kr + i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kMaxOut; ++i) {
      int o = threadIdx.x + i * blockDim.x;
      if (o < kr) {
        int nu = o / nrhs, r = o - nu * nrhs;
        T sum = 0;
        for (int mu = 0; mu < k; ++mu) sum += sS[nu * k + mu] * sx[mu * nrhs + r];
        acc[i] += sum;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < kMaxOut; ++i) {
    int o = threadIdx.x + i * blockDim.x;
    if (o < kr) yhat[t * kr + o] = acc[i];
  }
}

// leaf backward + nearfield: one CTA per leaf t;
// y|t = V_t y^_t + sum_b G_b x|s_b
template <class T>
__global__ void k_leaf_near(const T *__restrict__ V, const T *__restrict__ near, const int64_t *__restrict__ near_ptr,
                            const int32_t *__restrict__ near_col, int L, int k, int nrhs, int64_t leaf0,
                            int use_far, const T *__restrict__ yhat, const T *__restrict__ xpad,
                            T *__restrict__ ypad) {
  extern __shared__ unsigned char smem_raw[];
  T *sA = reinterpret_cast<T *>(smem_raw);         // up to L x max(k, L)
  T *sx = sA + L * (k > L ? k : L);                // up to max(k, L) x nrhs
  const int64_t j = blockIdx.x;
  const int lr = L * nrhs;
  T acc[kMaxOut];
#pragma unroll
  for (int i = 0; i < kMaxOut; ++i) acc[i] = 0;
  if (use_far) {
    for (int i = threadIdx.x; i < L * k; i += blockDim.x) sA[i] = V[j * L * k + i];
    for (int i = threadIdx.x; i < k * nrhs; i += blockDim.x) sx[i] = yhat[(leaf0 + j) * k * nrhs + i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kMaxOut; ++i) {
      int o = threadIdx.x + i * blockDim.x;
      if (o < lr) {
        int t = o / nrhs, r = o - t * nrhs;
        T sum = 0;
        for (int nu = 0; nu < k; ++nu) sum += sA[t * k + nu] * sx[nu * nrhs + r];
        acc[i] += sum;
      }
    }
  }
  for (int64_t e = near_ptr[j]; e < near_ptr[j + 1]; ++e) {
    const int64_t s = near_col[e];
    __syncthreads();
    for (int i = threadIdx.x; i < L * L; i += blockDim.x) sA[i] = near[e * L * L + i];
    for (int i = threadIdx.x; i < lr; i += blockDim.x) sx[i] = xpad[s * lr + i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kMaxOut; ++i) {
      int o = threadIdx.x + i * blockDim.x;
      if (o < lr) {
        int t = o / nrhs, r = o - t * nrhs;
        T sum = 0;
        for (int c = 0; c < L; ++c) sum += sA[t * L + c] * sx[c * nrhs + r];
        acc[i] += sum;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < kMaxOut; ++i) {
    int o = threadIdx.x + i * blockDim.x;
    if (o < lr) ypad[j * lr + o] = acc[i];
  }
}

int grid_for(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

template <class T>
int set_smem(const void *fn, size_t bytes) {
  if (bytes > 48 * 1024) H2_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
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

template <class T, class Tio>
int matvec_typed(Ctx &c, const Tio *x, Tio *y, int nrhs) {
  Dev &d = c.d;
  cudaStream_t st = c.stream;
  Marks mk(c);
  const int k = d.k, m = d.m, L = (int)d.lmax, D = d.depth, lmin = d.first_adm_level;
  const int64_t leaf0 = d.nleaf - 1;
  T *xpad = (T *)d.xpad, *ypad = (T *)d.ypad, *xhat = (T *)d.xhat, *yhat = (T *)d.yhat;
  int rc;

  mk.mark(H2_PH_PERMUTE_IN);
  k_permute_in<Tio, T><<<grid_for(d.npad * nrhs), kThreads, 0, st>>>(x, d.n, nrhs, d.pad_src, d.npad, xpad);
  mk.count(H2_PH_PERMUTE_IN);
  mk.mark(H2_PH_LEAF_FORWARD);
  const bool far = lmin <= D;
  if (far) {
    size_t sm = (size_t)(L * k + L * nrhs) * sizeof(T);
    if ((rc = set_smem<T>((const void *)k_leaf_forward<T>, sm))) return rc;
    k_leaf_forward<T><<<(unsigned)d.nleaf, kThreads, sm, st>>>((const T *)d.V, xpad, L, k, nrhs, leaf0, xhat);
    mk.count(H2_PH_LEAF_FORWARD);
  }
  mk.mark(H2_PH_UPWARD);
  if (far) {
    size_t sm = (size_t)3 * k * nrhs * sizeof(T);
    if ((rc = set_smem<T>((const void *)k_upward<T>, sm))) return rc;
    for (int l = D - 1; l >= lmin; --l) {
      int64_t par0 = ((int64_t)1 << l) - 1;
      k_upward<T><<<(unsigned)((int64_t)1 << l), kThreads, sm, st>>>((const T *)d.Ef, m, k, nrhs, par0, xhat);
      mk.count(H2_PH_UPWARD);
    }
  }
  mk.mark(H2_PH_COUPLING);
  if (far) {
    size_t sm;
    int64_t row0 = ((int64_t)1 << lmin) - 1;
    sm = (size_t)(k * k + k * nrhs) * sizeof(T);
    if ((rc = set_smem<T>((const void *)k_coupling<T>, sm))) return rc;
    k_coupling<T><<<(unsigned)(d.nclu - row0), kThreads, sm, st>>>((const T *)d.S, d.adm_ptr, d.adm_col, k, nrhs,
                                                                   row0, xhat, yhat);
    mk.count(H2_PH_COUPLING);
  }
  mk.mark(H2_PH_DOWNWARD);
  if (far) {
    size_t sm = (size_t)2 * k * nrhs * sizeof(T);
    if ((rc = set_smem<T>((const void *)k_downward<T>, sm))) return rc;
    for (int l = lmin; l < D; ++l) {
      int64_t ch0 = ((int64_t)2 << l) - 1;
      k_downward<T><<<(unsigned)((int64_t)2 << l), kThreads, sm, st>>>((const T *)d.Ef, m, k, nrhs, ch0, yhat);
      mk.count(H2_PH_DOWNWARD);
    }
  }
  mk.mark(H2_PH_LEAF_NEAR);
  {
    int w = std::max(k, L);
    size_t sm = (size_t)(L * w + w * nrhs) * sizeof(T);
    if ((rc = set_smem<T>((const void *)k_leaf_near<T>, sm))) return rc;
    k_leaf_near<T><<<(unsigned)d.nleaf, kThreads, sm, st>>>((const T *)d.V, (const T *)d.near, d.near_ptr,
                                                             d.near_col, L, k, nrhs, leaf0, far ? 1 : 0, yhat, xpad,
                                                             ypad);
    mk.count(H2_PH_LEAF_NEAR);
  }
  mk.mark(H2_PH_PERMUTE_OUT);
  k_permute_out<T, Tio><<<grid_for(d.npad * nrhs), kThreads, 0, st>>>(ypad, d.n, nrhs, d.pad_src, d.npad, y);
  mk.count(H2_PH_PERMUTE_OUT);
  mk.mark(H2_NPHASE);
  mk.finish();
  H2_CUDA_TRY(cudaGetLastError());
  d.last_nrhs = nrhs;
  return H2_OK;
}

}  // namespace

int ensure_work(Ctx &c, int nrhs) {
  Dev &d = c.d;
  if (nrhs <= d.cap_nrhs) return H2_OK;
  cudaFree(d.xpad); cudaFree(d.ypad); cudaFree(d.xhat); cudaFree(d.yhat); cudaFree(d.io_x); cudaFree(d.io_y);
  d.xpad = d.ypad = d.xhat = d.yhat = nullptr;
  d.io_x = d.io_y = nullptr;
  d.cap_nrhs = 0;
  size_t es = d.esize;
  auto al = [](void **p, size_t b) { return cudaMalloc(p, b) == cudaSuccess; };
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
  return H2_OK;
}

int run_matvec(Ctx &c, const void *x, void *y, int nrhs, bool io64) {
  Dev &d = c.d;
  if (nrhs < 1 || nrhs > 64) return fail(H2_EINVAL, "nrhs must be in [1, 64]");
  if ((int64_t)d.k * nrhs > kThreads * kMaxOut || d.lmax * nrhs > kThreads * kMaxOut)
    return fail(H2_EINVAL, "k * nrhs and leaf_max * nrhs must not exceed 4096");
  int rc = ensure_work(c, nrhs);
  if (rc) return rc;
  if (d.prec == H2_F64) return matvec_typed<double, double>(c, (const double *)x, (double *)y, nrhs);
  if (io64) return matvec_typed<float, double>(c, (const double *)x, (double *)y, nrhs);
  return matvec_typed<float, float>(c, (const float *)x, (float *)y, nrhs);
}

}  // namespace h2
