// Internal declarations of libh2 (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/h2.h"

namespace h2 {

// Sets the calling thread's error message and returns the status.
int fail(int status, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define H2_CUDA_TRY(call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return ::h2::cuda_fail(e_, #call); \
  } while (0)

// Every device allocation of the library goes through dmalloc: cudaMalloc,
// except that h2_inject_alloc_failure can make one chosen allocation fail as
// if the device were out of memory (test hook for the error paths).
cudaError_t dmalloc_raw(void **p, size_t bytes);
template <class T>
inline cudaError_t dmalloc(T **p, size_t bytes) {
  return dmalloc_raw(reinterpret_cast<void **>(p), bytes);
}

// Kernel of a real H^2 matrix (Section 1): the Laplace kernel, or the real
// or imaginary part of the Helmholtz kernel with wave number kappa.
constexpr int kKernelLaplace = 0, kKernelHelmholtzRe = 1, kKernelHelmholtzIm = 2;
struct KernelFn {
  int kind;
  double kappa;
};

// Gauss-Legendre nodes and weights on [0,1] (Newton on the Legendre recurrence).
void gauss_legendre01(int q, std::vector<double> &x, std::vector<double> &w);

// Host-side plan: cluster tree (Definition 1 with median bisection), block
// tree (Eq. (8)), Chebyshev points, leaf bases V (Eq. (6a)) and the factors
// of the transfer matrices (Eq. (9)).
struct Plan {
  int64_t n = 0, nv = 0;
  std::vector<double> vert;    // nv x 3
  std::vector<int32_t> tri;    // n x 3
  std::vector<double> area;    // n
  std::vector<double> cen;     // n x 3
  int leaf = 0, m = 0, k = 0, depth = 0;
  double eta = 0;
  int64_t nclu = 0, nleaf = 0, lmax = 0, leaf0 = 0;
  std::vector<int64_t> perm;   // cluster order -> triangle
  std::vector<int64_t> first, size;
  std::vector<double> lo, hi;  // nclu x 3
  std::vector<double> cheb;    // nclu x 3 x m
  std::vector<double> icen, ihalf;   // nclu x 3: interpolation-box centre and half width
  // admissible blocks in CSR by row cluster (columns sorted)
  std::vector<int64_t> adm_ptr;   // nclu + 1
  std::vector<int32_t> adm_col;
  // inadmissible blocks in CSR by row leaf (leaf-local indices, sorted)
  std::vector<int64_t> near_ptr;  // nleaf + 1
  std::vector<int32_t> near_col;
  int first_adm_level = 0;
  int64_t near_entries = 0;
  std::vector<double> V;       // n x k, cluster order
  std::vector<double> Ef;      // nclu x 3 x m x m
};

int make_plan(const double *vert, int64_t nv, const int32_t *tri, int64_t nt, int leaf_size, double eta, int order,
              bool with_bases, Plan &p);

constexpr int kMaxLevels = 40;
// largest problem (triangles) that the single-launch product takes
constexpr int64_t kFusedMaxN = 65536;

// Parameters of the GCA-H^2 construction (h2_build_gca)
struct GcaParams {
  double eps = 1e-4, gamma = 1.0;
  int green_order = 4, tri_order = 3, max_rank = 128;
};

// Device representation of one H^2 matrix.
struct Dev {
  int prec = H2_F64;
  KernelFn kernel{kKernelLaplace, 0.0};   // the real kernel of this matrix
  int coupling = 0;             // 0: S stored, 1: S regenerated in FP32 in the product
  size_t esize = 8;             // bytes of an arithmetic / vector value
  size_t ssize = 8;             // bytes of a stored value (V, E, S, nearfield)
  int m = 0, k = 0, kp = 0, depth = 0, first_adm_level = 0;
  int64_t n = 0, nclu = 0, nleaf = 0, lmax = 0, lp = 0, npad = 0;
  int64_t nadm = 0, nnear = 0;
  int32_t *pad_src = nullptr;   // npad: original triangle index of padded DoF, or -1
  void *V = nullptr;            // nleaf x lmax x kp (forward step)
  void *Vt = nullptr;           // nleaf x k x lp, transposed (backward step)
  void *Ef = nullptr;           // nclu x 3 x m x m
  void *S = nullptr;            // nadm x k x kp: S_b stored transposed, [mu][nu], nu padded to kp = 4 ceil(k/4)
  void *near = nullptr;         // nnear x lmax x lp, stored transposed: entry (t, c) at c lp + t
  int64_t *adm_ptr = nullptr;   // nclu + 1
  int32_t *adm_col = nullptr;
  int64_t *near_ptr = nullptr;  // nleaf + 1
  int32_t *near_col = nullptr;  // leaf-local
  double *cheb = nullptr;       // nclu x 3 x m (FP64 always)
  double *icen = nullptr;       // nclu x 3 interpolation-box centres (regenerated coupling)
  float *adm_dc = nullptr;      // nadm x 4: centre of the row cluster minus centre of the column cluster
  float *ihalf = nullptr;       // nclu x 3 interpolation-box half widths
  // Coupling on the tensor cores (order 4, FP64 or FP32 handles): the E4M3
  // digit planes of every S_b ([nadm][tc_nd][64 x 64] bytes, K-major
  // core-matrix layout), the row exponents ([nclu][64]), the digit planes of
  // the coefficients of one product ([nclu][tc_nd][16 x 64]) and the column
  // maxima per level ([32][16])
  int tensor = 0;               // 0: use the tensor cores where supported, 1: never
  bool tc = false;              // the digits exist
  int tc_nd = 0;                // digits per value: 10 (FP64-accurate) or 6 (FP32 handles)
  void *Stc = nullptr, *xtc = nullptr;
  int32_t *tc_E = nullptr;
  unsigned *tc_xmax = nullptr;
  // FP64-accurate nearfield on the tensor cores (leaves of at most 21
  // triangles): the digit planes of every near block (ntc_ablk bytes each,
  // two stacked groups of K-major rows), the row exponents ([nleaf][lmax]),
  // the digit planes of the permuted input of one product ([nleaf][10][16 x
  // 32]) and its column maxima ([16])
  bool ntc = false;
  void *Ntc = nullptr, *xnt = nullptr;
  int32_t *ntc_E = nullptr;
  unsigned *ntc_xmax = nullptr;
  uint32_t ntc_ablk = 0;
  // tensor-core leaf forward step: the ten E4M3 digit planes of every V_t^T
  // ([leaf][10][64 x 32] bytes, K-major core matrices) and their row powers
  // of two [leaf][64]
  void *Vtc = nullptr;
  int32_t *tcv_E = nullptr;
  unsigned long long *colmax = nullptr;   // H2_F64: 64 column maxima of x (range guard of double-float)
  bool v32 = false;             // 16-bit handle whose V, Vt and transfer factors are stored in FP32
  float *vscale = nullptr;      // per leaf: power of two dividing the stored V (FP16), or NULL
  float *nscale = nullptr;      // per nearfield block: the same for G_b, or NULL
  // bfloat16 handles: the self blocks G_jj of the leaves in FP32 ([nleaf][lmax][lp], zero in `near`),
  // the CSR of the other near blocks (near_ptr2 [nleaf + 1], near_col2, stored block near_blk2) and
  // the one-term CSR of the self blocks (self_ptr [nleaf + 1], self_col [nleaf])
  float *nself = nullptr;
  int64_t *near_ptr2 = nullptr, *self_ptr = nullptr;
  int32_t *near_col2 = nullptr, *near_blk2 = nullptr, *self_col = nullptr;
  // GCA-H^2 (Section 3's GCA-H^2 example): the rank and the pivot triangles
  // of every cluster (gpiv [clusters][gkcap], pivot order), per tree level l
  // the padded rank gK[l] (a multiple of 4; 0 above the first admissible
  // level), the coupling matrices of the level's admissible blocks (gS[l]:
  // [block][K_l][K_l], S_b stored transposed [mu][nu]), the transfer
  // matrices E_c of the level's clusters (gE[l]: [c][K_l][K_{l-1}]) and their
  // transposes (gEt[l]: [c][K_{l-1}][K_l]), and the offset of the level's
  // coefficients in units of rp values (gX[l]); k is the largest gK.  The
  // leaf bases use V and Vt with kp = gK[depth]; the nearfield is the same.
  // single-launch product for small FP64-accurate matrices (h2_options.fused):
  // the flag and the grid-barrier words of that launch
  bool fused = false;
  unsigned *fbar = nullptr;
  bool gca = false;
  int gK[kMaxLevels] = {0};
  int64_t gX[kMaxLevels] = {0};
  void *gS[kMaxLevels] = {nullptr}, *gE[kMaxLevels] = {nullptr}, *gEt[kMaxLevels] = {nullptr};
  int gkcap = 0;
  int32_t *grank = nullptr, *gpiv = nullptr;
  int64_t coupling_entries = 0;  // stored coupling entries (padded; GCA handles)
  // work buffers for up to cap_nrhs right-hand sides
  int cap_nrhs = 0;
  void *xpad = nullptr, *ypad = nullptr, *xhat = nullptr, *yhat = nullptr;
  double *io_x = nullptr, *io_y = nullptr;   // FP64 staging for host / solver I/O
  int last_nrhs = 0, last_rp = 0;  // last product: right-hand sides and padded coefficient width
  int64_t work_gen = 0;            // incremented whenever the work buffers are reallocated
  int64_t bytes = 0;
};

struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> ev;      // (H2_NPHASE + 1) events per recorded product
  std::vector<int64_t> launches;    // per phase, accumulated
  int64_t products = 0;
  double ms[H2_NPHASE] = {0};
};

// GMRES work space kept on the handle (grown on demand, freed with it)
struct GmresWork {
  int cols = 0, restart = 0;
  double *Vb = nullptr, *W = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr;
  double *h1 = nullptr, *h2 = nullptr, *hn = nullptr, *resid = nullptr, *yv = nullptr, *bn = nullptr;
  double *r = nullptr, *d = nullptr, *Az = nullptr;   // refinement vectors
  int *active = nullptr, *jc = nullptr;
  double *tolv = nullptr;                 // per column: residual target of the cycle
  double *dpart = nullptr;                // chunk sums of the Gram-Schmidt dot products
  int *maxv = nullptr, *itc = nullptr;    // per column: iteration limit, iterations done
  int *hflag = nullptr;                   // pinned host copy of `active` (convergence checks)
  cudaEvent_t ev = nullptr;               // recorded behind that copy
};
void free_gmres_work(GmresWork &w);

// Buffers of h2_matvec_host_stream (grown on demand, freed with the handle):
// two device block pairs, the input and output copy streams and the events
// that order copies and products
struct StreamWork {
  size_t bytes = 0;
  double *x[2] = {nullptr, nullptr}, *y[2] = {nullptr, nullptr};
  cudaStream_t in = nullptr, out = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
};

struct Ctx {
  double build_ms[H2_NBUILD] = {0};   // wall time of the build phases (h2_build_times)
  StreamWork sw;                      // h2_matvec_host_stream
  GcaParams gp;                       // GCA-H^2 handles: construction parameters
  GmresWork gw;
  Prof prof;
  int device = 0;
  cudaStream_t stream = nullptr;
  int quad_order = 3;
  Plan plan;
  Dev d;
};

// padded coefficient width: right-hand sides rounded up to 16 bytes
inline int padded_rhs(int nrhs, size_t esize) {
  int v = (int)(16 / esize);
  return (nrhs + v - 1) / v * v;
}

// power of two applied to a column of x whose largest entry (bits of the
// double) lies outside the double-float range guard [2^-40, 2^40]; 0 inside
int column_range_shift(unsigned long long bits);

// device-side error word (a bounded wait ran out); read and cleared by the host
int take_device_error(Ctx &c);
// the bounded-wait self-test of h2_wait_selftest (h2_matvec.cu)
int wait_selftest(Ctx &c, int withhold, uint32_t limit, int *stages_seen);

// FP64-accurate coupling on the tensor cores (h2_tc.cu): eligibility,
// set-up of the slices (arow_dev: row cluster of every admissible block, on
// the device), the coupling phase of one product (xhat, yhat: double-float
// coefficient arrays [clusters][k][rp]) and that file's device error word
bool tc_eligible(const Dev &d);
int tc_build(Ctx &c, const int32_t *arow_dev);
// leaf_max: the leaf coefficients' column maxima are in place (written by
// the tensor-core leaf forward step)
int tc_upward(Ctx &c, void *xhat, int rp, int64_t *launches, bool leaf_max = false);
int tc_coupling(Ctx &c, const void *xhat, void *yhat, int rp);
int tc_take_error(cudaStream_t st);
bool ntc_eligible(const Dev &d);
int ntc_build(Ctx &c, const int32_t *nrow_dev);
int ntc_near(Ctx &c, const void *xpad, void *ypad, int rp, int accumulate, int64_t *launches,
             bool have_input = false);
// input column maxima and digit planes per leaf (nearfield, tensor-core leaf step)
// have_max: the column maxima are in place (taken by the permutation)
int ntc_input(Ctx &c, const void *xpad, int rp, int64_t *launches, bool have_max = false);
// leaf forward step on the tensor cores (after ntc_input); requires d.Vtc
int tc_leaf_forward(Ctx &c, void *xhat, int rp);

// h2_build for a given kernel (h2_api.cpp)
int build_handle(const double *vert, int64_t nv, const int32_t *tri, int64_t nt, int leaf_size, double eta, int order,
                 const h2_options *opt, KernelFn kf, h2_handle *out, const GcaParams *gca = nullptr);

// device allocation helper (tracks bytes)
int dev_alloc(Dev &d, void **ptr, size_t bytes);
int ensure_work(Ctx &c, int nrhs);

// build steps on the device (h2_setup.cu)
int device_build(Ctx &c);
// GCA-H^2 pivots, leaf bases, transfer and coupling matrices on the device
// (h2_gca.cu); vert, tri, area: the mesh on the device
int gca_build(Ctx &c, const double *vert, const int32_t *tri, const double *area);
// y = G~ x with device arrays of the handle's precision (h2_matvec.cu);
// if x64/y64 are given instead the product reads/writes FP64 arrays.
// Threads per CTA of a transfer launch (one CTA per parent) at tree level l:
// the wide levels (1024 parents and more) take 128 threads, so that more CTAs
// stay resident per SM to hide the global-memory latency of each parent's
// step; the narrow top levels keep 256 to shorten each CTA.
inline int transfer_threads(int l) { return l >= 10 ? 128 : 256; }
// accumulate: y += G~ x instead of y = G~ x (the final scatter adds)
int run_matvec(Ctx &c, const void *x, void *y, int nrhs, bool io64, bool accumulate = false);
// GMRES (h2_solve.cu); b, z device FP64 arrays
int run_gmres(Ctx &c, const double *b, double *z, int nrhs, double rtol, int restart, int maxit,
              h2_solve_info *info);
// A linear operator y = A x on column-major n x nrhs FP64 device arrays, as
// GMRES sees it: the product of one handle (ctx_op), or a composite such as
// the real form of a complex Helmholtz matrix.
struct LinOp {
  int64_t n = 0;
  cudaStream_t stream = nullptr;
  std::function<int(const double *, double *, int)> apply;
};
LinOp ctx_op(Ctx &c);
// one GMRES cycle for A D = R (see h2_solve.cu); host arrays of nrhs entries
int gmres_cycle(const LinOp &op, GmresWork &w, const double *R, double *D, int nrhs, int restart,
                const double *tol, const int *act, const int *max_it, int *iters);
// restarted GMRES for A z = b with work space w (at least nrhs columns and restart)
int run_gmres_op(const LinOp &op, GmresWork &w, const double *b, double *z, int nrhs, double rtol, int restart,
                 int maxit, h2_solve_info *info);
int alloc_gmres_work(GmresWork &w, int64_t n, int cols, int restart);
// GMRES-IR: outer residuals with hi, inner GMRES with lo (same mesh and tree)
int run_gmres_ir(Ctx &hi, Ctx &lo, const double *b, double *z, int nrhs, double rtol, double inner_rtol,
                 int restart, int maxit_inner, int maxit_outer, h2_solve_info *info);

// vector helpers of the solver (h2_solve.cu) on the context's stream
void k_launch_residual(const double *b, const double *Az, int64_t total, double *r, cudaStream_t st);
void k_launch_axpy(const double *d, int64_t total, double *z, cudaStream_t st);
int column_norms(Ctx &c, const double *v, int64_t n, int ncols, double *dev_tmp, double *host_out);

}  // namespace h2

// the opaque handle of the C ABI
struct h2_ctx : h2::Ctx {};
