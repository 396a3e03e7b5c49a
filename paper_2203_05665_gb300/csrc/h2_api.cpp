// C ABI of libh2 (declared in include/h2.h): argument checking, handles,
// error reporting, host <-> device staging.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "h2_internal.hpp"

struct h2_plan_ctx {
  h2::Plan plan;
};

namespace h2 {

static thread_local std::string g_last_error;

// allocations left before the injected failure; -1: none pending
static std::atomic<int64_t> g_alloc_countdown{-1};

cudaError_t dmalloc_raw(void **p, size_t bytes) {
  int64_t c = g_alloc_countdown.load();
  while (c >= 0) {
    if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) {
      if (c == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

int fail(int status, const std::string &msg) {
  g_last_error = msg;
  return status;
}

int cuda_fail(cudaError_t e, const char *what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? H2_ENOMEM : H2_ECUDA;
}

static void free_dev(Dev &d) {
  for (int l = 0; l < kMaxLevels; ++l)
    for (void *p : {d.gS[l], d.gE[l], d.gEt[l]})
      if (p) cudaFree(p);
  if (d.fbar) cudaFree(d.fbar);
  if (d.grank) cudaFree(d.grank);
  if (d.gpiv) cudaFree(d.gpiv);
  void *ptrs[] = {d.Vtc, d.tcv_E, d.Ntc, d.xnt, d.ntc_E, d.ntc_xmax, d.Stc, d.xtc, d.tc_E, d.tc_xmax, d.icen, d.adm_dc, d.ihalf, d.colmax, d.nself, d.near_ptr2, d.self_ptr, d.near_col2, d.near_blk2, d.self_col, d.vscale, d.nscale, d.pad_src, d.V, d.Vt, d.Ef,      d.S,       d.near, d.adm_ptr, d.adm_col, d.near_ptr,
                  d.near_col, d.cheb, d.xpad, d.ypad, d.xhat, d.yhat, d.io_x,    d.io_y};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  d = Dev();
}

// H2_F64 keeps every stored value as a pair of FP32 numbers, so the stored
// entries must stay inside FP32's exponent range with room for the low word:
// every nearfield entry is at least amin^2 / (4 pi D) (amin the smallest
// triangle area, D the diameter of the mesh's box), which must not fall below
// 2^-96, and no triangle area may exceed 2^60.
static int check_double_float_range(const Plan &p) {
  double amin = HUGE_VAL, amax = 0.0;
  for (double a : p.area) {
    amin = std::min(amin, a);
    amax = std::max(amax, a);
  }
  double diag = 0.0;
  for (int q = 0; q < 3; ++q) diag += (p.hi[q] - p.lo[q]) * (p.hi[q] - p.lo[q]);
  diag = std::sqrt(diag);
  const double low = amin * amin / (4.0 * 3.14159265358979323846 * std::max(diag, 1e-300));
  if (!(low >= std::ldexp(1.0, -96)) || !(amax <= std::ldexp(1.0, 60)))
    return fail(H2_EINVAL, "mesh scale outside the double-float range of H2_F64 (smallest triangle area " +
                               std::to_string(amin) + ", mesh diameter " + std::to_string(diag) +
                               "); rescale the mesh or use H2_F64_NATIVE");
  return H2_OK;
}

// h2_build with a given kernel (Section 1: Laplace, or a part of Helmholtz)
int build_handle(const double *vert, int64_t nv, const int32_t *tri, int64_t nt, int leaf_size, double eta, int order,
                 const h2_options *opt, KernelFn kf, h2_handle *out, const GcaParams *gca) {
  if (!out) return fail(H2_EINVAL, "out is NULL");
  *out = nullptr;
  h2_options o;
  h2_options_default(&o);
  if (opt) o = *opt;
  if (o.prec < H2_F64 || o.prec > H2_F16) return fail(H2_EINVAL, "unknown precision");
  if (o.coupling < H2_COUPLING_AUTO || o.coupling > H2_COUPLING_REGEN) return fail(H2_EINVAL, "unknown coupling mode");
  const bool half_prec = o.prec == H2_BF16 || o.prec == H2_F16, f64 = o.prec == H2_F64 || o.prec == H2_F64_NATIVE;
  if (o.coupling == H2_COUPLING_REGEN && f64)
    return fail(H2_EINVAL, "the regenerated coupling is FP32; use H2_F32, H2_BF16 or H2_F16");
  if (o.coupling == H2_COUPLING_STORED && half_prec)
    return fail(H2_EINVAL, "16-bit precisions regenerate the coupling");
  if (o.tensor < 0 || o.tensor > 1) return fail(H2_EINVAL, "tensor must be 0 (tensor cores where supported) or 1 (never)");
  if (o.fused < 0 || o.fused > 1) return fail(H2_EINVAL, "fused must be 0 (off) or 1 (single-launch product when eligible)");
  for (int r : o.reserved)
    if (r) return fail(H2_EINVAL, "reserved option fields must be zero");
  if (o.basis_prec != 0) {
    if (!half_prec) return fail(H2_EINVAL, "basis_prec applies to H2_BF16 and H2_F16 handles only; use 0");
    if (o.basis_prec != H2_F32 && o.basis_prec != o.prec)
      return fail(H2_EINVAL, "basis_prec must be 0, H2_F32 or the handle's own 16-bit precision");
  }
  if (gca) {
    if (half_prec) return fail(H2_EINVAL, "GCA-H^2 handles support H2_F64, H2_F64_NATIVE and H2_F32");
    if (o.coupling == H2_COUPLING_REGEN) return fail(H2_EINVAL, "GCA-H^2 handles store their coupling matrices");
  }
  int ndev = 0;
  H2_CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (o.device < 0 || o.device >= ndev) return fail(H2_EINVAL, "device ordinal out of range");
  H2_CUDA_TRY(cudaSetDevice(o.device));
  h2_ctx *c = new (std::nothrow) h2_ctx();
  if (!c) return fail(H2_ENOMEM, "handle");
  c->device = o.device;
  c->stream = (cudaStream_t)o.stream;
  c->quad_order = o.quad_order;
  c->d.prec = o.prec;
  c->d.tensor = o.tensor;
  c->d.kernel = kf;
  c->d.fused = o.fused == 1 && o.prec == H2_F64 && !gca;
  // FP32 leaf bases: explicitly, or by default under bfloat16 storage
  c->d.v32 = half_prec && (o.basis_prec == H2_F32 || (o.basis_prec == 0 && o.prec == H2_BF16));
  c->d.coupling = (o.coupling == H2_COUPLING_REGEN || half_prec) ? 1 : (o.coupling == H2_COUPLING_STORED ? 0 : -1);
  if (gca) {
    c->gp = *gca;
    c->d.gca = true;
    c->d.coupling = 0;
  }
  int rc;
  const auto t0 = std::chrono::steady_clock::now();
  auto ms = [](std::chrono::steady_clock::time_point a) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a).count();
  };
  try {
    // the trees, blocks and interpolation points on the host; V and E are
    // computed on the device by device_build
    rc = make_plan(vert, nv, tri, nt, leaf_size, eta, order, false, c->plan);
    c->build_ms[H2_BUILD_PLAN] = ms(t0);
    if (!rc && o.prec == H2_F64) rc = check_double_float_range(c->plan);
    if (!rc) rc = device_build(*c);
  } catch (const std::bad_alloc &) {
    rc = fail(H2_ENOMEM, "host allocation in set-up");
  }
  c->build_ms[H2_BUILD_TOTAL] = ms(t0);
  if (rc) {
    free_dev(c->d);
    delete c;
    return rc;
  }
  *out = c;
  return H2_OK;
}

}  // namespace h2

using namespace h2;

extern "C" {

const char *h2_last_error(void) { return g_last_error.c_str(); }

int h2_inject_alloc_failure(int64_t after) {
  if (after < -1) return fail(H2_EINVAL, "after must be >= -1");
  g_alloc_countdown.store(after);
  return H2_OK;
}

int h2_options_default(h2_options *opt) {
  if (!opt) return fail(H2_EINVAL, "opt is NULL");
  std::memset(opt, 0, sizeof(*opt));
  opt->prec = H2_F64;
  opt->quad_order = 3;
  opt->device = 0;
  opt->stream = nullptr;
  return H2_OK;
}

int h2_plan_create(const double *vert, int64_t nv, const int32_t *tri, int64_t nt, int leaf_size, double eta,
                   int order, h2_plan *out) {
  if (!out) return fail(H2_EINVAL, "out is NULL");
  *out = nullptr;
  h2_plan_ctx *p = new (std::nothrow) h2_plan_ctx();
  if (!p) return fail(H2_ENOMEM, "plan");
  int rc;
  try {
    rc = make_plan(vert, nv, tri, nt, leaf_size, eta, order, true, p->plan);
  } catch (const std::bad_alloc &) {
    rc = fail(H2_ENOMEM, "host allocation in planning");
  }
  if (rc) {
    delete p;
    return rc;
  }
  *out = p;
  return H2_OK;
}

int h2_plan_destroy(h2_plan p) {
  delete p;
  return H2_OK;
}

int h2_plan_counts(h2_plan pp, int64_t *counts) {
  if (!pp || !counts) return fail(H2_EINVAL, "NULL argument");
  const Plan &p = pp->plan;
  counts[0] = p.n;
  counts[1] = p.depth;
  counts[2] = p.nclu;
  counts[3] = p.lmax;
  counts[4] = (int64_t)p.adm_col.size();
  counts[5] = (int64_t)p.near_col.size();
  counts[6] = p.near_entries;
  counts[7] = p.first_adm_level;
  return H2_OK;
}

int h2_plan_tree(h2_plan pp, int64_t *perm, int64_t *first, int64_t *size, double *lo, double *hi) {
  if (!pp) return fail(H2_EINVAL, "NULL plan");
  const Plan &p = pp->plan;
  if (perm) std::memcpy(perm, p.perm.data(), p.n * 8);
  if (first) std::memcpy(first, p.first.data(), p.nclu * 8);
  if (size) std::memcpy(size, p.size.data(), p.nclu * 8);
  if (lo) std::memcpy(lo, p.lo.data(), p.nclu * 24);
  if (hi) std::memcpy(hi, p.hi.data(), p.nclu * 24);
  return H2_OK;
}

int h2_plan_blocks(h2_plan pp, int32_t *adm_t, int32_t *adm_s, int32_t *near_t, int32_t *near_s) {
  if (!pp) return fail(H2_EINVAL, "NULL plan");
  const Plan &p = pp->plan;
  for (int64_t t = 0; t < p.nclu; ++t)
    for (int64_t e = p.adm_ptr[t]; e < p.adm_ptr[t + 1]; ++e) {
      if (adm_t) adm_t[e] = (int32_t)t;
      if (adm_s) adm_s[e] = p.adm_col[e];
    }
  for (int64_t j = 0; j < p.nleaf; ++j)
    for (int64_t e = p.near_ptr[j]; e < p.near_ptr[j + 1]; ++e) {
      if (near_t) near_t[e] = (int32_t)(p.leaf0 + j);
      if (near_s) near_s[e] = (int32_t)(p.leaf0 + p.near_col[e]);
    }
  return H2_OK;
}

int h2_plan_bases(h2_plan pp, double *V, double *E) {
  if (!pp) return fail(H2_EINVAL, "NULL plan");
  const Plan &p = pp->plan;
  if (V) std::memcpy(V, p.V.data(), p.V.size() * 8);
  if (E) std::memcpy(E, p.Ef.data(), p.Ef.size() * 8);
  return H2_OK;
}

int h2_build(const double *vert, int64_t nv, const int32_t *tri, int64_t nt, int leaf_size, double eta, int order,
             const h2_options *opt, h2_handle *out) {
  return build_handle(vert, nv, tri, nt, leaf_size, eta, order, opt, KernelFn{kKernelLaplace, 0.0}, out);
}

int h2_gca_options_default(h2_gca_options *g) {
  if (!g) return fail(H2_EINVAL, "NULL argument");
  std::memset(g, 0, sizeof(*g));
  const GcaParams d;
  g->eps = d.eps;
  g->gamma = d.gamma;
  g->green_order = d.green_order;
  g->tri_order = d.tri_order;
  g->max_rank = d.max_rank;
  return H2_OK;
}

int h2_build_gca(const double *vert, int64_t nv, const int32_t *tri, int64_t nt, int leaf_size, double eta,
                 const h2_gca_options *gopt, const h2_options *opt, h2_handle *out) {
  GcaParams gp;
  if (gopt) {
    for (int r : gopt->reserved)
      if (r) return fail(H2_EINVAL, "reserved GCA option fields must be zero");
    gp.eps = gopt->eps;
    gp.gamma = gopt->gamma;
    gp.green_order = gopt->green_order;
    gp.tri_order = gopt->tri_order;
    gp.max_rank = gopt->max_rank;
  }
  return build_handle(vert, nv, tri, nt, leaf_size, eta, 1, opt, KernelFn{kKernelLaplace, 0.0}, out, &gp);
}

int h2_gca_pivots(h2_handle h, int32_t *rank, int32_t *pivots, int64_t cap) {
  if (!h) return fail(H2_EINVAL, "NULL handle");
  if (!h->d.gca) return fail(H2_EINVAL, "not a GCA-H^2 handle");
  const Dev &d = h->d;
  if (pivots && cap < d.k) return fail(H2_EINVAL, "cap must be at least the handle's rank (h2_stats.rank)");
  H2_CUDA_TRY(cudaSetDevice(h->device));
  H2_CUDA_TRY(cudaStreamSynchronize(h->stream));
  std::vector<int32_t> r(d.nclu), pv((size_t)d.nclu * d.gkcap);
  H2_CUDA_TRY(cudaMemcpy(r.data(), d.grank, d.nclu * 4, cudaMemcpyDeviceToHost));
  if (rank) std::memcpy(rank, r.data(), d.nclu * 4);
  if (pivots) {
    H2_CUDA_TRY(cudaMemcpy(pv.data(), d.gpiv, pv.size() * 4, cudaMemcpyDeviceToHost));
    for (int64_t c = 0; c < d.nclu; ++c)
      for (int64_t a = 0; a < cap; ++a) pivots[c * cap + a] = a < r[c] ? pv[c * d.gkcap + a] : -1;
  }
  return H2_OK;
}

namespace {

void free_stream_work(StreamWork &w) {
  for (int b = 0; b < 2; ++b) {
    if (w.x[b]) cudaFree(w.x[b]);
    if (w.y[b]) cudaFree(w.y[b]);
    for (cudaEvent_t e : {w.ev_in[b], w.ev_done[b], w.ev_out[b]})
      if (e) cudaEventDestroy(e);
  }
  if (w.in) cudaStreamDestroy(w.in);
  if (w.out) cudaStreamDestroy(w.out);
  w = StreamWork();
}

int ensure_stream_work(StreamWork &w, size_t bytes) {
  if (w.in && bytes <= w.bytes) return H2_OK;
  free_stream_work(w);
  auto al = [](double **p, size_t b) { return dmalloc(p, b) == cudaSuccess; };
  if (!al(&w.x[0], bytes) || !al(&w.x[1], bytes) || !al(&w.y[0], bytes) || !al(&w.y[1], bytes)) {
    cudaGetLastError();
    free_stream_work(w);
    return fail(H2_ENOMEM, "buffers of h2_matvec_host_stream");
  }
  cudaError_t e = cudaStreamCreateWithFlags(&w.in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w.out, cudaStreamNonBlocking);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b)
    for (cudaEvent_t *ev : {&w.ev_in[b], &w.ev_done[b], &w.ev_out[b]})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_stream_work(w);
    return cuda_fail(e, "streams of h2_matvec_host_stream");
  }
  w.bytes = bytes;
  return H2_OK;
}

}  // namespace

static void drop_events(Prof &p) {
  for (auto e : p.ev) cudaEventDestroy(e);
  p.ev.clear();
}

int h2_destroy(h2_handle h) {
  if (!h) return H2_OK;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  drop_events(h->prof);
  free_gmres_work(h->gw);
  free_stream_work(h->sw);
  free_dev(h->d);
  delete h;
  return H2_OK;
}

int h2_info(h2_handle h, h2_stats *out) {
  if (!h || !out) return fail(H2_EINVAL, "NULL argument");
  const Plan &p = h->plan;
  out->n = p.n;
  out->depth = p.depth;
  out->clusters = p.nclu;
  out->leaf_max = p.lmax;
  out->order = p.m;
  out->rank = p.k;
  out->adm_blocks = (int64_t)p.adm_col.size();
  out->near_blocks = (int64_t)p.near_col.size();
  out->near_entries = p.near_entries;
  out->first_adm_level = p.first_adm_level;
  out->device_bytes = h->d.bytes;
  out->prec = h->d.prec;
  out->coupling = h->d.coupling == 1 ? H2_COUPLING_REGEN : H2_COUPLING_STORED;
  out->tensor = h->d.tc ? 1 : 0;
  out->tensor_near = h->d.ntc ? 1 : 0;
  out->tensor_leaf = h->d.Vtc ? 1 : 0;
  out->basis_prec = h->d.v32 ? H2_F32 : h->d.prec;
  out->gca = h->d.gca ? 1 : 0;
  out->coupling_entries = h->d.gca ? h->d.coupling_entries : (int64_t)p.adm_col.size() * p.k * p.k;
  if (h->d.gca) {
    out->order = h->gp.green_order;
    out->rank = h->d.k;
  }
  return H2_OK;
}

int h2_profile(h2_handle h, int enable) {
  if (!h) return fail(H2_EINVAL, "NULL handle");
  H2_CUDA_TRY(cudaSetDevice(h->device));
  H2_CUDA_TRY(cudaStreamSynchronize(h->stream));
  drop_events(h->prof);
  h->prof.on = enable != 0;
  h->prof.launches.assign(H2_NPHASE, 0);
  h->prof.products = 0;
  for (double &v : h->prof.ms) v = 0.0;
  return H2_OK;
}

int h2_phase_times(h2_handle h, double *ms, int64_t *launches, int64_t *products) {
  if (!h) return fail(H2_EINVAL, "NULL handle");
  H2_CUDA_TRY(cudaSetDevice(h->device));
  H2_CUDA_TRY(cudaStreamSynchronize(h->stream));
  Prof &p = h->prof;
  const size_t per = H2_NPHASE + 1;
  for (size_t b = 0; b + per <= p.ev.size(); b += per)
    for (int i = 0; i < H2_NPHASE; ++i) {
      float t = 0;
      H2_CUDA_TRY(cudaEventElapsedTime(&t, p.ev[b + i], p.ev[b + i + 1]));
      p.ms[i] += t;
    }
  drop_events(p);
  int derr = take_device_error(*h);
  if (derr) return derr;
  if (ms)
    for (int i = 0; i < H2_NPHASE; ++i) ms[i] = p.ms[i];
  if (launches)
    for (int i = 0; i < H2_NPHASE; ++i) launches[i] = i < (int)p.launches.size() ? p.launches[i] : 0;
  if (products) *products = p.products;
  return H2_OK;
}

int h2_matvec(h2_handle h, const void *x, void *y, int nrhs) {
  if (!h || !x || !y) return fail(H2_EINVAL, "NULL argument");
  H2_CUDA_TRY(cudaSetDevice(h->device));
  return run_matvec(*h, x, y, nrhs, false);
}

int h2_wait_selftest(h2_handle h, int withhold, uint32_t poll_limit, int *stages_seen) {
  if (!h) return fail(H2_EINVAL, "NULL handle");
  if (withhold != 0 && withhold != 1) return fail(H2_EINVAL, "withhold must be 0 or 1");
  H2_CUDA_TRY(cudaSetDevice(h->device));
  return wait_selftest(*h, withhold, poll_limit, stages_seen);
}

int h2_build_times(h2_handle h, double *ms) {
  if (!h || !ms) return fail(H2_EINVAL, "NULL argument");
  for (int i = 0; i < H2_NBUILD; ++i) ms[i] = h->build_ms[i];
  return H2_OK;
}

int h2_matvec_acc(h2_handle h, const void *x, void *y, int nrhs) {
  if (!h || !x || !y) return fail(H2_EINVAL, "NULL argument");
  H2_CUDA_TRY(cudaSetDevice(h->device));
  return run_matvec(*h, x, y, nrhs, false, true);
}

}  // extern "C"

struct h2_graph_s {
  h2_ctx *h = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t work_gen = 0;    // the handle's work-space generation at capture
  int nrhs = 0, rp = 0;    // the captured product's right-hand sides and padded width
};

extern "C" {

int h2_graph_create(h2_handle h, const void *x, void *y, int nrhs, h2_graph *out) {
  if (!out) return fail(H2_EINVAL, "out is NULL");
  *out = nullptr;
  if (!h || !x || !y) return fail(H2_EINVAL, "NULL argument");
  if (nrhs < 1 || nrhs > 64) return fail(H2_EINVAL, "nrhs must be in [1, 64]");
  H2_CUDA_TRY(cudaSetDevice(h->device));
  int rc = ensure_work(*h, nrhs);   // any allocation happens before the capture
  if (rc) return rc;
  if (h->stream) H2_CUDA_TRY(cudaStreamSynchronize(h->stream));
  else H2_CUDA_TRY(cudaDeviceSynchronize());
  cudaStream_t cap = nullptr;
  H2_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaStream_t own = h->stream;
  const bool prof = h->prof.on;
  const int slast = h->d.last_nrhs, slast_rp = h->d.last_rp;
  h->stream = cap;
  h->prof.on = false;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  int cap_nrhs = 0, cap_rp = 0;
  if (e == cudaSuccess) {
    rc = run_matvec(*h, x, y, nrhs, false);
    cap_nrhs = h->d.last_nrhs;
    cap_rp = h->d.last_rp;
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    if (!rc && e2 != cudaSuccess) rc = cuda_fail(e2, "capture of the product");
  } else {
    rc = cuda_fail(e, "cudaStreamBeginCapture");
  }
  h->stream = own;
  h->prof.on = prof;
  h->d.last_nrhs = slast;
  h->d.last_rp = slast_rp;
  cudaStreamDestroy(cap);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  h2_graph_s *G = new (std::nothrow) h2_graph_s();
  if (!G) {
    cudaGraphDestroy(g);
    return fail(H2_ENOMEM, "graph");
  }
  e = cudaGraphInstantiate(&G->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    delete G;
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  G->h = h;
  G->work_gen = h->d.work_gen;
  G->nrhs = cap_nrhs;
  G->rp = cap_rp;
  *out = G;
  return H2_OK;
}

int h2_graph_launch(h2_graph g) {
  if (!g) return fail(H2_EINVAL, "NULL graph");
  if (g->h->d.work_gen != g->work_gen)
    return fail(H2_EINVAL, "the handle's work space was reallocated since the capture; create the graph again");
  H2_CUDA_TRY(cudaSetDevice(g->h->device));
  H2_CUDA_TRY(cudaGraphLaunch(g->exec, g->h->stream));
  g->h->d.last_nrhs = g->nrhs;   // h2_coefficients now describes this product
  g->h->d.last_rp = g->rp;
  return H2_OK;
}

int h2_graph_destroy(h2_graph g) {
  if (!g) return H2_OK;
  cudaSetDevice(g->h->device);
  if (g->h->stream) cudaStreamSynchronize(g->h->stream);
  else cudaDeviceSynchronize();
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
  return H2_OK;
}

int h2_matvec_host(h2_handle h, const double *x, double *y, int nrhs) {
  if (!h || !x || !y) return fail(H2_EINVAL, "NULL argument");
  if (nrhs < 1 || nrhs > 64) return fail(H2_EINVAL, "nrhs must be in [1, 64]");
  H2_CUDA_TRY(cudaSetDevice(h->device));
  int rc = ensure_work(*h, nrhs);
  if (rc) return rc;
  size_t bytes = (size_t)h->d.n * nrhs * 8;
  H2_CUDA_TRY(cudaMemcpyAsync(h->d.io_x, x, bytes, cudaMemcpyHostToDevice, h->stream));
  if ((rc = run_matvec(*h, h->d.io_x, h->d.io_y, nrhs, true))) return rc;
  H2_CUDA_TRY(cudaMemcpyAsync(y, h->d.io_y, bytes, cudaMemcpyDeviceToHost, h->stream));
  H2_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return take_device_error(*h);
}

int h2_matvec_host_stream(h2_handle h, const double *x, double *y, int nrhs, int count) {
  if (!h || !x || !y) return fail(H2_EINVAL, "NULL argument");
  if (nrhs < 1 || nrhs > 64) return fail(H2_EINVAL, "nrhs must be in [1, 64]");
  if (count < 1) return fail(H2_EINVAL, "count must be at least 1");
  H2_CUDA_TRY(cudaSetDevice(h->device));
  int rc = ensure_work(*h, nrhs);
  if (rc) return rc;
  const size_t bytes = (size_t)h->d.n * nrhs * 8;
  StreamWork &w = h->sw;
  if ((rc = ensure_stream_work(w, bytes))) return rc;
  // the copy streams start after everything already queued on the handle's stream
  cudaEvent_t start = nullptr;
  H2_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(start, h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(w.in, start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(w.out, start, 0);
  cudaEventDestroy(start);
  if (e != cudaSuccess) return cuda_fail(e, "h2_matvec_host_stream set-up");
  for (int i = 0; i < count && !rc; ++i) {
    const int b = i & 1;
    const double *xi = x + (size_t)i * h->d.n * nrhs;
    double *yi = y + (size_t)i * h->d.n * nrhs;
    // block i in: once the product of block i - 2 has read the buffer
    if (i >= 2) H2_CUDA_TRY(cudaStreamWaitEvent(w.in, w.ev_done[b], 0));
    H2_CUDA_TRY(cudaMemcpyAsync(w.x[b], xi, bytes, cudaMemcpyHostToDevice, w.in));
    H2_CUDA_TRY(cudaEventRecord(w.ev_in[b], w.in));
    // the product of block i: its input has landed and block i - 2's result has left
    H2_CUDA_TRY(cudaStreamWaitEvent(h->stream, w.ev_in[b], 0));
    if (i >= 2) H2_CUDA_TRY(cudaStreamWaitEvent(h->stream, w.ev_out[b], 0));
    rc = run_matvec(*h, w.x[b], w.y[b], nrhs, true);
    if (rc) break;
    H2_CUDA_TRY(cudaEventRecord(w.ev_done[b], h->stream));
    // block i out
    H2_CUDA_TRY(cudaStreamWaitEvent(w.out, w.ev_done[b], 0));
    H2_CUDA_TRY(cudaMemcpyAsync(yi, w.y[b], bytes, cudaMemcpyDeviceToHost, w.out));
    H2_CUDA_TRY(cudaEventRecord(w.ev_out[b], w.out));
  }
  H2_CUDA_TRY(cudaStreamSynchronize(w.in));
  H2_CUDA_TRY(cudaStreamSynchronize(h->stream));
  H2_CUDA_TRY(cudaStreamSynchronize(w.out));
  if (rc) return rc;
  return take_device_error(*h);
}

int h2_coefficients(h2_handle h, int which, double *out) {
  if (!h || !out || (which != 0 && which != 1)) return fail(H2_EINVAL, "bad argument");
  if (h->d.gca) return fail(H2_EINVAL, "GCA-H^2 handles have per-level ranks; use h2_export");
  if (h->d.last_nrhs < 1) return fail(H2_EINVAL, "no product has run on this handle");
  H2_CUDA_TRY(cudaSetDevice(h->device));
  H2_CUDA_TRY(cudaStreamSynchronize(h->stream));
  const Dev &d = h->d;
  // the coefficients of the last product: [clusters][k][last_rp], the first last_nrhs columns are returned
  const size_t rows = (size_t)d.nclu * d.k, rp = d.last_rp, nr = d.last_nrhs;
  const void *src = which == 0 ? d.xhat : d.yhat;
  std::vector<double> tmp(rows * rp);
  if (d.prec == H2_F64_NATIVE) {
    H2_CUDA_TRY(cudaMemcpy(tmp.data(), src, rows * rp * 8, cudaMemcpyDeviceToHost));
  } else if (d.prec == H2_F64) {
    std::vector<float> tf(2 * rows * rp);
    H2_CUDA_TRY(cudaMemcpy(tf.data(), src, rows * rp * 8, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < rows * rp; ++i) tmp[i] = (double)tf[2 * i] + (double)tf[2 * i + 1];
  } else {
    std::vector<float> tf(rows * rp);
    H2_CUDA_TRY(cudaMemcpy(tf.data(), src, rows * rp * 4, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < tf.size(); ++i) tmp[i] = tf[i];
  }
  // columns scaled by the double-float range guard are reported unscaled
  double unscale[64];
  for (size_t c = 0; c < nr; ++c) unscale[c] = 1.0;
  if (d.colmax) {
    unsigned long long bits[64];
    H2_CUDA_TRY(cudaMemcpy(bits, d.colmax, nr * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    for (size_t c = 0; c < nr; ++c) unscale[c] = std::ldexp(1.0, -column_range_shift(bits[c]));
  }
  for (size_t r = 0; r < rows; ++r)
    for (size_t c = 0; c < nr; ++c) out[r * nr + c] = tmp[r * rp + c] * unscale[c];
  return H2_OK;
}

namespace {

enum StoredType { ST_DD, ST_F64, ST_F32, ST_BF16, ST_F16 };

// one stored value as a double (IEEE binary16 and bfloat16 decoded from
// their bit fields; a double-float pair summed)
double stored_value(const unsigned char *p, int type) {
  switch (type) {
    case ST_DD: {
      float hl[2];
      std::memcpy(hl, p, 8);
      return (double)hl[0] + (double)hl[1];
    }
    case ST_F64: {
      double v;
      std::memcpy(&v, p, 8);
      return v;
    }
    case ST_F32: {
      float v;
      std::memcpy(&v, p, 4);
      return v;
    }
    case ST_BF16: {
      uint16_t b;
      std::memcpy(&b, p, 2);
      const uint32_t u = (uint32_t)b << 16;
      float v;
      std::memcpy(&v, &u, 4);
      return v;
    }
    default: {
      uint16_t b;
      std::memcpy(&b, p, 2);
      const int sgn = b >> 15, ex = (b >> 10) & 31, man = b & 1023;
      double v = ex == 0 ? std::ldexp((double)man, -24)
                         : ex == 31 ? (man ? NAN : HUGE_VAL) : std::ldexp((double)(man + 1024), ex - 25);
      return sgn ? -v : v;
    }
  }
}

int stored_type_of(int prec) {
  switch (prec) {
    case H2_F64: return ST_DD;
    case H2_F64_NATIVE: return ST_F64;
    case H2_BF16: return ST_BF16;
    case H2_F16: return ST_F16;
    default: return ST_F32;
  }
}

size_t stored_size(int type) { return type == ST_DD || type == ST_F64 ? 8 : type == ST_F32 ? 4 : 2; }

// copy count * per stored values starting at element first * per of a device array to the host
int fetch(const void *src, size_t esz, int64_t first, int64_t count, int64_t per, std::vector<unsigned char> &buf) {
  buf.resize((size_t)(count * per) * esz);
  if (count == 0) return H2_OK;
  H2_CUDA_TRY(cudaMemcpy(buf.data(), static_cast<const unsigned char *>(src) + (size_t)(first * per) * esz,
                         buf.size(), cudaMemcpyDeviceToHost));
  return H2_OK;
}

}  // namespace

int h2_export(h2_handle h, int what, int64_t first, int64_t count, double *out) {
  if (!h || (!out && count > 0) || first < 0 || count < 0) return fail(H2_EINVAL, "bad argument");
  H2_CUDA_TRY(cudaSetDevice(h->device));
  H2_CUDA_TRY(cudaStreamSynchronize(h->stream));
  const Dev &d = h->d;
  const Plan &p = h->plan;
  const int64_t L = d.lmax, Lp = d.lp, k = d.k, kp = d.kp, m = d.m;
  const int ts = stored_type_of(d.prec);
  std::vector<unsigned char> buf;
  int rc;
  switch (what) {
    case H2_EXPORT_NEAR: {
      if (first + count > d.nnear) return fail(H2_EINVAL, "near block range out of bounds");
      if ((rc = fetch(d.near, stored_size(ts), first, count, L * Lp, buf))) return rc;
      std::vector<float> sc;
      if (d.nscale) {
        sc.resize(count);
        if (count) H2_CUDA_TRY(cudaMemcpy(sc.data(), d.nscale + first, count * 4, cudaMemcpyDeviceToHost));
      }
      for (int64_t i = 0; i < count; ++i)
        for (int64_t t = 0; t < L; ++t)
          for (int64_t c = 0; c < L; ++c) {
            double v = stored_value(buf.data() + ((i * L + c) * Lp + t) * stored_size(ts), ts);
            out[(i * L + t) * L + c] = d.nscale ? v * sc[i] : v;
          }
      if (d.nself) {
        // bfloat16 handles: the self blocks are held in FP32
        for (int64_t i = 0; i < count; ++i) {
          const int64_t b = first + i;
          const int64_t j = std::upper_bound(p.near_ptr.begin(), p.near_ptr.end(), b) - p.near_ptr.begin() - 1;
          if (p.near_col[b] != j) continue;
          std::vector<unsigned char> sb;
          if ((rc = fetch(d.nself, 4, j, 1, L * Lp, sb))) return rc;
          for (int64_t t = 0; t < L; ++t)
            for (int64_t c = 0; c < L; ++c) out[(i * L + t) * L + c] = stored_value(sb.data() + (c * Lp + t) * 4, ST_F32);
        }
      }
      return H2_OK;
    }
    case H2_EXPORT_COUPLING: {
      if (d.gca) return fail(H2_EINVAL, "GCA-H^2 handles: use H2_EXPORT_GCA_S");
      if (!d.S) return fail(H2_EINVAL, "the coupling matrices are regenerated, not stored");
      if (first + count > d.nadm) return fail(H2_EINVAL, "admissible block range out of bounds");
      if ((rc = fetch(d.S, stored_size(ts), first, count, k * kp, buf))) return rc;
      for (int64_t i = 0; i < count; ++i)
        for (int64_t nu = 0; nu < k; ++nu)
          for (int64_t mu = 0; mu < k; ++mu)
            out[(i * k + nu) * k + mu] = stored_value(buf.data() + ((i * k + mu) * kp + nu) * stored_size(ts), ts);
      return H2_OK;
    }
    case H2_EXPORT_V: {
      if (d.gca) return fail(H2_EINVAL, "GCA-H^2 handles: use H2_EXPORT_GCA_V");
      if (first + count > d.npad) return fail(H2_EINVAL, "padded DoF range out of bounds");
      const int tv = d.v32 ? ST_F32 : ts;
      if ((rc = fetch(d.V, stored_size(tv), first, count, kp, buf))) return rc;
      std::vector<float> vs;
      if (d.vscale) {
        vs.resize(d.nleaf);
        H2_CUDA_TRY(cudaMemcpy(vs.data(), d.vscale, d.nleaf * 4, cudaMemcpyDeviceToHost));
      }
      for (int64_t i = 0; i < count; ++i)
        for (int64_t nu = 0; nu < k; ++nu) {
          double v = stored_value(buf.data() + (i * kp + nu) * stored_size(tv), tv);
          out[i * k + nu] = d.vscale ? v * vs[(first + i) / L] : v;
        }
      return H2_OK;
    }
    case H2_EXPORT_E: {
      if (d.gca) return fail(H2_EINVAL, "GCA-H^2 handles: use H2_EXPORT_GCA_E");
      if (first + count > d.nclu) return fail(H2_EINVAL, "cluster range out of bounds");
      const int te = (d.prec == H2_BF16 || d.v32) ? ST_F32 : ts;
      if ((rc = fetch(d.Ef, stored_size(te), first, count, 3 * m * m, buf))) return rc;
      for (int64_t i = 0; i < count * 3 * m * m; ++i) out[i] = stored_value(buf.data() + i * stored_size(te), te);
      return H2_OK;
    }
    case H2_EXPORT_GCA_S:
    case H2_EXPORT_GCA_V:
    case H2_EXPORT_GCA_E: {
      if (!d.gca) return fail(H2_EINVAL, "not a GCA-H^2 handle");
      const int64_t K = d.k;
      const int64_t lim = what == H2_EXPORT_GCA_S ? d.nadm : what == H2_EXPORT_GCA_V ? d.nleaf : d.nclu;
      if (first + count > lim) return fail(H2_EINVAL, "export range out of bounds");
      const size_t es = stored_size(ts);
      auto level_of = [](int64_t c) {
        int l = 0;
        while (((int64_t)2 << l) - 1 <= c) ++l;
        return l;
      };
      for (int64_t i = 0; i < count; ++i) {
        double *o = out + i * (what == H2_EXPORT_GCA_V ? L * K : K * K);
        std::fill(o, o + (what == H2_EXPORT_GCA_V ? L * K : K * K), 0.0);
        if (what == H2_EXPORT_GCA_S) {
          const int64_t b = first + i;
          const int64_t t = std::upper_bound(p.adm_ptr.begin(), p.adm_ptr.end(), b) - p.adm_ptr.begin() - 1;
          const int l = level_of(t);
          const int64_t Kl = d.gK[l], bl = b - p.adm_ptr[((int64_t)1 << l) - 1];
          if ((rc = fetch(d.gS[l], es, bl, 1, Kl * Kl, buf))) return rc;
          for (int64_t mu = 0; mu < Kl; ++mu)
            for (int64_t nu = 0; nu < Kl; ++nu) o[nu * K + mu] = stored_value(buf.data() + (mu * Kl + nu) * es, ts);
        } else if (what == H2_EXPORT_GCA_V) {
          const int64_t KD = d.gK[d.depth];
          if (KD == 0) continue;
          if ((rc = fetch(d.V, es, first + i, 1, L * KD, buf))) return rc;
          for (int64_t t = 0; t < L; ++t)
            for (int64_t a = 0; a < KD; ++a) o[t * K + a] = stored_value(buf.data() + (t * KD + a) * es, ts);
        } else {
          const int64_t c = first + i;
          if (c == 0) continue;
          const int l = level_of(c);
          if (!d.gE[l]) continue;
          const int64_t Kc = d.gK[l], Kq = d.gK[l - 1];
          if ((rc = fetch(d.gE[l], es, c - (((int64_t)1 << l) - 1), 1, Kc * Kq, buf))) return rc;
          for (int64_t a = 0; a < Kc; ++a)
            for (int64_t b = 0; b < Kq; ++b) o[a * K + b] = stored_value(buf.data() + (a * Kq + b) * es, ts);
        }
      }
      return H2_OK;
    }
    default: return fail(H2_EINVAL, "unknown export item");
  }
}

int h2_solve(h2_handle h, const double *b, double *z, int nrhs, double rtol, int restart, int maxit,
             h2_solve_info *info) {
  if (!h || !b || !z) return fail(H2_EINVAL, "NULL argument");
  if (nrhs < 1 || nrhs > 64) return fail(H2_EINVAL, "nrhs must be in [1, 64]");
  if (restart < 1 || restart > 200 || maxit < 1 || !(rtol > 0.0)) return fail(H2_EINVAL, "bad solver parameters");
  H2_CUDA_TRY(cudaSetDevice(h->device));
  cudaPointerAttributes ab{}, az{};
  H2_CUDA_TRY(cudaPointerGetAttributes(&ab, b));
  H2_CUDA_TRY(cudaPointerGetAttributes(&az, z));
  bool db = ab.type == cudaMemoryTypeDevice || ab.type == cudaMemoryTypeManaged;
  bool dz = az.type == cudaMemoryTypeDevice || az.type == cudaMemoryTypeManaged;
  if (db != dz) return fail(H2_EINVAL, "b and z must both be host or both be device arrays");
  if (db) return run_gmres(*h, b, z, nrhs, rtol, restart, maxit, info);
  size_t bytes = (size_t)h->d.n * nrhs * 8;
  double *db_ = nullptr, *dz_ = nullptr;
  if (dmalloc(&db_, bytes) != cudaSuccess || dmalloc(&dz_, bytes) != cudaSuccess) {
    cudaFree(db_);
    cudaGetLastError();
    return fail(H2_ENOMEM, "solve staging buffers");
  }
  int rc = H2_OK;
  cudaError_t e = cudaMemcpyAsync(db_, b, bytes, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) rc = cuda_fail(e, "copy b");
  if (!rc || rc == H2_ENOCONV) rc = run_gmres(*h, db_, dz_, nrhs, rtol, restart, maxit, info);
  if (!rc || rc == H2_ENOCONV) {
    e = cudaMemcpyAsync(z, dz_, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "copy z");
  }
  cudaFree(db_);
  cudaFree(dz_);
  return rc;
}

int h2_solve_ir(h2_handle hi, h2_handle lo, const double *b, double *z, int nrhs, double rtol, double inner_rtol,
                int restart, int maxit_inner, int maxit_outer, h2_solve_info *info) {
  if (!hi || !lo || !b || !z) return fail(H2_EINVAL, "NULL argument");
  if (nrhs < 1 || nrhs > 64) return fail(H2_EINVAL, "nrhs must be in [1, 64]");
  if (restart < 1 || restart > 200 || maxit_inner < 1 || maxit_outer < 1 || !(rtol > 0.0) || !(inner_rtol > 0.0) ||
      !(inner_rtol < 1.0))
    return fail(H2_EINVAL, "bad solver parameters");
  if (hi->device != lo->device) return fail(H2_EINVAL, "both handles must live on one device");
  if (hi->plan.n != lo->plan.n || hi->plan.nclu != lo->plan.nclu || hi->plan.adm_col.size() != lo->plan.adm_col.size() ||
      hi->plan.near_col.size() != lo->plan.near_col.size())
    return fail(H2_EINVAL, "the two handles must represent the same matrix structure");
  H2_CUDA_TRY(cudaSetDevice(hi->device));
  cudaPointerAttributes ab{}, az{};
  H2_CUDA_TRY(cudaPointerGetAttributes(&ab, b));
  H2_CUDA_TRY(cudaPointerGetAttributes(&az, z));
  bool db = ab.type == cudaMemoryTypeDevice || ab.type == cudaMemoryTypeManaged;
  bool dz = az.type == cudaMemoryTypeDevice || az.type == cudaMemoryTypeManaged;
  if (db != dz) return fail(H2_EINVAL, "b and z must both be host or both be device arrays");
  if (db) return run_gmres_ir(*hi, *lo, b, z, nrhs, rtol, inner_rtol, restart, maxit_inner, maxit_outer, info);
  size_t bytes = (size_t)hi->d.n * nrhs * 8;
  double *db_ = nullptr, *dz_ = nullptr;
  if (dmalloc(&db_, bytes) != cudaSuccess || dmalloc(&dz_, bytes) != cudaSuccess) {
    cudaFree(db_);
    cudaGetLastError();
    return fail(H2_ENOMEM, "solve staging buffers");
  }
  int rc = H2_OK;
  cudaError_t e = cudaMemcpyAsync(db_, b, bytes, cudaMemcpyHostToDevice, hi->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(hi->stream);
  if (e != cudaSuccess) rc = cuda_fail(e, "copy b");
  if (!rc) rc = run_gmres_ir(*hi, *lo, db_, dz_, nrhs, rtol, inner_rtol, restart, maxit_inner, maxit_outer, info);
  if (!rc || rc == H2_ENOCONV) {
    e = cudaMemcpyAsync(z, dz_, bytes, cudaMemcpyDeviceToHost, hi->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(hi->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "copy z");
  }
  cudaFree(db_);
  cudaFree(dz_);
  return rc;
}

}  // extern "C"
