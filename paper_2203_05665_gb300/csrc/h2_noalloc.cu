// h2_matvec_noalloc: the H^2 product without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// product: code that runs while an allocator is locked or pooled by another
// runtime, a real-time loop that must not block on cudaMalloc, or a process
// whose device memory has been handed out completely ahead of time.  For
// them this entry point runs the same kernels as h2_matvec but takes its work
// buffers (the padded input and output vectors and the cluster coefficients)
// from one fixed array in device memory that is part of the library itself.
#include <mutex>

#include "h2_internal.hpp"

namespace h2 {
namespace {

// Work space of h2_matvec_noalloc.  Every GPU that loads the library keeps
// these kH2NoallocBytes until the process exits.
constexpr size_t kH2NoallocBytes = (size_t)64 << 20;
static __device__ __align__(256) unsigned char g_h2_noalloc_scratch[kH2NoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch[kMaxDevices] = {};   // device address of the array, per device (set up once)

inline size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace
}  // namespace h2

using namespace h2;

extern "C" int h2_matvec_noalloc(h2_handle h, const void *x, void *y, int nrhs) {
  if (!h || !x || !y) return fail(H2_EINVAL, "NULL argument");
  if (nrhs < 1 || nrhs > 64) return fail(H2_EINVAL, "nrhs must be in [1, 64]");
  if (h->device < 0 || h->device >= kMaxDevices) return fail(H2_EINVAL, "device ordinal out of range");
  H2_CUDA_TRY(cudaSetDevice(h->device));
  void *base = nullptr;
  {
    // once per device, with the device current: the address of the array
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch[h->device]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_h2_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the no-alloc work space");
      g_scratch[h->device] = p;
    }
    base = g_scratch[h->device];
  }
  Dev &d = h->d;
  const int rp = padded_rhs(nrhs, d.esize);
  const size_t vec = round256((size_t)d.npad * rp * d.esize);
  const size_t coef = round256((size_t)d.nclu * d.k * rp * d.esize);
  const size_t need = 2 * vec + 2 * coef;
  if (need > kH2NoallocBytes)
    return fail(H2_EINVAL, "h2_matvec_noalloc: this matrix and nrhs need " + std::to_string(need) +
                               " bytes of work space; the fixed limit is " + std::to_string(kH2NoallocBytes) +
                               " bytes (use h2_matvec)");
  // Run the product with the work buffers pointed into the array; the
  // handle's own buffers are put back afterwards.  No entry is read before
  // the same call has written it, so nothing has to be cleared.
  unsigned char *b = static_cast<unsigned char *>(base);
  void *sv[4] = {d.xpad, d.ypad, d.xhat, d.yhat};
  const int scap = d.cap_nrhs, slast = d.last_nrhs, slast_rp = d.last_rp;
  const bool sprof = h->prof.on;
  d.xpad = b;
  d.ypad = b + vec;
  d.xhat = b + 2 * vec;
  d.yhat = b + 2 * vec + coef;
  d.cap_nrhs = rp;        // the buffers fit rp columns: no growth, no allocation
  h->prof.on = false;     // no timing events either
  int rc = run_matvec(*h, x, y, nrhs, false);
  d.xpad = sv[0];
  d.ypad = sv[1];
  d.xhat = sv[2];
  d.yhat = sv[3];
  d.cap_nrhs = scap;
  h->prof.on = sprof;
  d.last_nrhs = slast;    // h2_coefficients keeps reporting the last h2_matvec product
  d.last_rp = slast_rp;
  return rc;
}
