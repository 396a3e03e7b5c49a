// Coupling and nearfield phases on the tensor cores (tcgen05, FP8 E4M3
// operands, FP32 accumulation in tensor memory), up to 16 right-hand sides:
// the coupling of order-4 handles (k = 64) in FP64 accuracy (ten digits per
// value) or FP32 accuracy (six digits), and the FP64-accurate nearfield of
// handles whose leaves hold at most 21 triangles (second part of the file).
//
// GB300 runs FP64 at 1/58 of its FP32 rate, and double-float arithmetic on
// the FP32 pipe leaves the coupling (Algorithm 3, y^_t = sum S_ts x^_s)
// bound by instruction issue far below the memory roofline.  This path
// computes the same sums exactly enough for FP64 parity with integer digits
// on the tensor cores (the splitting scheme of Ozaki et al.):
//
//  * every row nu of the coupling matrices of row cluster t gets a power of
//    two 2^E (E[t][nu], common to all blocks of the row, |S| < 2^E), every
//    column j of the coefficients of tree level l a power of two 2^F;
//  * a value v becomes the integer X = round(v 2^(49-E)), |X| <= 2^49,
//    split into ten signed 5-bit digits, X = sum_i s_i 2^(50-5i),
//    |s_i| <= 16: every digit is exact in FP8 E4M3 (one byte);
//  * D_ik = sum_blocks sum_mu s_i[nu][mu] t_k[mu][j] is a sum of at most
//    64 x 64 products of magnitude <= 2^8, an integer of at most 2^20: the
//    tensor cores accumulate it exactly in FP32, and the at most five D_ik
//    of one level i + k add exactly in FP32 too;
//  * y^_t[nu][j] = 2^(E + F) sum_{i + k <= 11} 2^(2-5(i+k)) D_ik, the ten
//    levels summed in double-float; the dropped pairs and the rounding of X
//    stay below 2^-46 of the row's scale.  With six digits (FP32 handles):
//    |X| <= 2^29, pairs i + k <= 7, below 2^-27.
//
// The digits of S are cut once at set-up, straight into the layout the
// tensor cores read from shared memory (K-major, 8 x 16-byte core matrices,
// no swizzle), 10 bytes per entry, so bulk copies (TMA engine) move a block
// as it is stored; the coefficients are cut once per product.  One MMA
// instruction (kind::f8f6f4, K = 32) multiplies two stacked digit planes of
// S (M = 128 rows: digits i and i+1) by the digit planes of x^ it pairs with
// (N = 16 columns per plane, 160 down to 32): five such groups, two K steps
// each, 10 instructions per block.  The groups write their pairs so that the
// pairs of one level i + k land in the same accumulator columns (the tensor
// cores add them, exactly), so a segment's results take 160 columns and
// three accumulator sets rotate: the MMAs of one row segment overlap the
// epilogue of the previous one.
//
// Kernel roles (one CTA per SM, 6 warps): warp 0 streams the digits of each
// block through a shared-memory ring (bulk copies completing on mbarriers;
// the digit stream evict-first in L2, the coefficient tiles evict-last),
// warp 1 allocates tensor memory and issues the MMAs of a row segment (at
// most 64 blocks) into the next free accumulator set, warps 2-5 read it back
// (tcgen05.ld), add the levels in double-float, and write y^_t.  Every wait is bounded; on a timeout the
// device error word is raised, every role stops, copies and MMAs in flight
// are waited for and the tensor memory is released before the CTA exits.
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "h2_dd.cuh"
#include "h2_digits.hpp"
#include "h2_internal.hpp"
#include "h2_kernel.cuh"
#include "h2_ptx.cuh"
#include "h2_transfer.cuh"

namespace h2 {
namespace {

constexpr int kTcK = 64;                 // rank k = m^3, m = 4
constexpr int kTcN = 16;                 // right-hand sides of one product (padded)
constexpr int kTcSlices = 10;            // 5-bit digits of an FP64-accurate value
constexpr int kTcFixBits = 49;           // |X| <= 2^49
constexpr int kTcTop = 11;               // digit pairs with i + k <= 11 are summed
constexpr int kTcSegBlocks = 64;         // blocks accumulated in one exact segment (sums <= 2^20)
constexpr uint32_t kSliceA = kTcK * kTcK;              // 4096 bytes: one digit plane of S_b (64 x 64 E4M3)
constexpr uint32_t kSliceB = kTcN * kTcK;              // 1024 bytes: one digit plane of x^_s (16 x 64 E4M3)

// The coupling's digit layout for ND digits per value: ND = 10 for FP64
// accuracy (|X| <= 2^49, pairs i + k <= 11), ND = 6 for FP32 accuracy (|X| <=
// 2^29, pairs i + k <= 7: the dropped pairs stay below 2^-27 of the row's
// scale).  Group g pairs S digits 2g+1 (accumulator lanes 0-63) and 2g+2
// (lanes 64-127) with x^ digits k = 1 .. ND - 2g (N = 16 (ND - 2g)) and
// writes them from accumulator column 32 g on: x^ digit k of group g lands in
// column block 2g + k - 1, so column block c holds, in lanes 0-63, the sum of
// every pair of level i + k = c + 2 and, in lanes 64-127, of level c + 3.  The
// tensor cores thus add the pairs of one level themselves (exactly: at most
// five sums of at most 2^20 each), an accumulator set is 16 ND columns wide
// (160 or 96) and kSets sets rotate, so that the MMAs of the next row segment
// run while the epilogue reads the previous one.
//
// KB is the contraction length of one block in bytes: 64 for the coupling
// matrices (two MMA K steps), 32 for the leaf bases V_t^T of the leaf forward
// step (the L <= 32 triangles of a leaf, zero padded; one K step).
template <int ND, int KB = kTcK>
struct Dig {
  static constexpr int kFix = 5 * ND - 1;
  static constexpr int kTop = ND + 1;
  static constexpr int kGroups = ND / 2;
  static constexpr int kKSteps = KB / 32;
  static constexpr uint32_t kPlaneA = kTcK * KB;   // one digit plane of a block: 64 rows x KB
  static constexpr uint32_t kPlaneB = kTcN * KB;   // one digit plane of the coefficients: 16 rows x KB
  static constexpr uint32_t kTileA = ND * kPlaneA;
  static constexpr uint32_t kTileB = ND * kPlaneB;
  static constexpr uint32_t kStage = kTileA + kTileB;
  static constexpr int kStages = (ND == 10 ? 4 : 6) * (kTcK / KB);
  static constexpr uint32_t kW = kTcN * ND;      // columns of an accumulator set
  static constexpr int kSets = 3;
  __host__ __device__ static constexpr int nx(int g) { return ND - 2 * g; }
  __host__ __device__ static constexpr uint32_t col(int g) { return (uint32_t)(2 * kTcN * g); }
};
static_assert(Dig<10>::kSets * Dig<10>::kW <= 512 && Dig<6>::kSets * Dig<6>::kW <= 512, "accumulator sets");
constexpr uint32_t kTmemCols = 512;      // the accumulator sets
constexpr int kTcThreads = 192;          // producer, MMA, four epilogue warps
constexpr uint32_t kXch = 64 * kTcN * 8; // epilogue exchange: 64 rows x 16 double-float values
// EG: epilogue warp groups (2 for one-block rows, whose epilogue is not
// hidden behind the MMAs of many blocks), each with its own exchange area
template <int ND, int KB = kTcK, int EG = 1>
__host__ __device__ constexpr uint32_t tc_bar_off() {
  return Dig<ND, KB>::kStages * Dig<ND, KB>::kStage + EG * kXch;
}
template <int ND, int KB = kTcK, int EG = 1>
__host__ __device__ constexpr uint32_t tc_smem() { return tc_bar_off<ND, KB, EG>() + 40 * 8 + 16; }

// instruction descriptor of tcgen05.mma kind::f8f6f4: D FP32 (bits 4-5 =
// 1), A and B E4M3 (bits 7-9 = 0, bits 10-12 = 0), both K-major (bits 15, 16
// = 0), N / 8 at bits 17-22, M / 16 at bits 24-28
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}


// byte offset of (row r, contraction index c) in a K-major one-byte operand
// of 64 contraction values per row: core matrices of 8 rows x 16 bytes, four
// along K (128 bytes apart), then the next 8 rows (512 bytes on)
__host__ __device__ __forceinline__ int core_off(int r, int c) {
  return ((r >> 3) * 4 + (c >> 4)) * 128 + (r & 7) * 16 + (c & 15);
}

// shared-memory matrix descriptor (no swizzle): start address, leading
// byte offset 128 (next core matrix along K), stride byte offset 512 (next
// 8 rows), descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(512u >> 4) << 32) |
         (1ull << 46);
}
// the same for rows of KB contraction bytes (the next 8 rows 8 KB bytes on)
template <int KB>
__device__ __forceinline__ uint64_t sdesc_kb(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)((8u * KB) >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// arrive on bar once every MMA issued so far by this thread has completed
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive 32-bit columns of this warp's 32 tensor-memory lanes; the
// registers are valid after tmem_wait()
__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Column indices of the blocks a producer streams, loaded 8 blocks ahead so
// that the address of a bulk copy never waits on a global load.
// Without a column array (col = NULL) block e lies in column e.
struct ColAhead {
  const int32_t *col;
  int64_t end;
  int32_t c[8];
  __device__ __forceinline__ int32_t at(int64_t e) const { return col ? col[e] : (int32_t)e; }
  __device__ __forceinline__ ColAhead(const int32_t *cl, int64_t e0, int64_t e1) : col(cl), end(e1) {
#pragma unroll
    for (int u = 0; u < 8; ++u) c[u] = e0 + u < e1 ? at(e0 + u) : 0;
  }
  // the column of block e; afterwards block e + 8 is in flight
  __device__ __forceinline__ int32_t next(int64_t e) {
    const int32_t v = c[0];
#pragma unroll
    for (int u = 0; u < 7; ++u) c[u] = c[u + 1];
    c[7] = e + 8 < end ? at(e + 8) : 0;
    return v;
  }
};

__device__ __forceinline__ void named_sync_id(uint32_t id, uint32_t nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// 2^e as a float for -126 <= e <= 127 (exact; used for power-of-two scaling)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }


// interpolation point nu of cluster c (tensor Chebyshev points, Eq. (6c))
__device__ __forceinline__ void tc_point(const double *cheb, int64_t c, int nu, double *x) {
  x[0] = cheb[(3 * c + 0) * 4 + (nu & 3)];
  x[1] = cheb[(3 * c + 1) * 4 + ((nu >> 2) & 3)];
  x[2] = cheb[(3 * c + 2) * 4 + (nu >> 4)];
}

// ---------------------------------------------------------------- set-up
// E[t][nu]: 1 + floor(log2 max |S_ts[nu][mu]|) over the blocks of row t (0 if none)
__global__ void k_tc_rowexp(const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                            const double *__restrict__ cheb, int64_t row0, int64_t nclu, KernelFn kf,
                            int32_t *__restrict__ E) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (nclu - row0) * kTcK) return;
  const int64_t t = row0 + e / kTcK;
  const int nu = (int)(e % kTcK);
  double x[3], y[3], mx = 0.0;
  tc_point(cheb, t, nu, x);
  for (int64_t b = ptr[t]; b < ptr[t + 1]; ++b)
    for (int mu = 0; mu < kTcK; ++mu) {
      tc_point(cheb, col[b], mu, y);
      mx = fmax(mx, fabs(kernel_value(kf, x, y)));
    }
  E[t * kTcK + nu] = mx > 0.0 ? ilogb(mx) + 1 : 0;
}

// a digit (|s| <= 16, an integer) as its exact FP8 E4M3 byte
__device__ __forceinline__ unsigned char e4m3(int s) {
  return (unsigned char)__nv_cvt_float_to_fp8((float)s, __NV_SATFINITE, __NV_E4M3);
}

// the ND E4M3 digit planes of S_b, row nu, contraction indices 16 cg .. 16 cg + 15
template <int ND>
__global__ void k_tc_slice_s(const int32_t *__restrict__ brow, const int32_t *__restrict__ col,
                             const double *__restrict__ cheb, const int32_t *__restrict__ E, int64_t nblk,
                             KernelFn kf, unsigned char *__restrict__ Stc) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nblk * kTcK * 4) return;
  const int64_t b = e / (kTcK * 4);
  const int nu = (int)((e / 4) % kTcK), cg = (int)(e % 4);
  const int64_t t = brow[b], s = col[b];
  double x[3], y[3];
  tc_point(cheb, t, nu, x);
  const int sc = Dig<ND>::kFix - E[t * kTcK + nu];
  __align__(16) unsigned char out[ND][16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    tc_point(cheb, s, 16 * cg + q, y);
    const long long X = llrint(ldexp(kernel_value(kf, x, y), sc));
    int sl[ND];
    split_digits<ND>(X, sl);
#pragma unroll
    for (int i = 0; i < ND; ++i) out[i][q] = e4m3(sl[i]);
  }
  unsigned char *base = Stc + b * (int64_t)Dig<ND>::kTileA + core_off(nu, 16 * cg);
#pragma unroll
  for (int i = 0; i < ND; ++i)
    *reinterpret_cast<uint4 *>(base + i * kSliceA) = *reinterpret_cast<const uint4 *>(out[i]);
}

// ---------------------------------------------------------------- per product
__device__ __forceinline__ int tc_level(int64_t c) { return 63 - __clzll(c + 1); }

// xmax[j] = largest |x| (double-float: |hi|) of column j over rows [0, rows) of x
// ([rows][rp], as float bits).  A warp reads 32 / LPR rows at a time with 16-byte
// loads (LPR lanes per row of 16 columns, lane l: row l / LPR, its EPV columns
// from EPV (l % LPR)), so the reads are contiguous and every lane keeps fixed
// columns; rp is a multiple of EPV (rows are padded to 16 bytes).
__device__ __forceinline__ float mag(float v) { return fabsf(v); }
__device__ __forceinline__ float mag(dd v) { return fabsf(v.hi); }

template <class T>
__global__ void k_tc_levmax(const T *__restrict__ x, int64_t rows, int rp, unsigned *__restrict__ xmax) {
  constexpr int EPV = 16 / (int)sizeof(T), LPR = kTcN / EPV, RPW = 32 / LPR;
  __shared__ unsigned loc[kTcN];
  if (threadIdx.x < kTcN) loc[threadIdx.x] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31, sub = lane % LPR, nv = rp / EPV;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t w = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  float m[EPV];
#pragma unroll
  for (int e = 0; e < EPV; ++e) m[e] = 0.0f;
  if (sub < nv)
    for (int64_t r = RPW * w + lane / LPR; r < rows; r += RPW * warps) {
      const T *p = x + r * rp + EPV * sub;
#pragma unroll
      for (int e = 0; e < EPV; ++e) m[e] = fmaxf(m[e], mag(p[e]));
    }
#pragma unroll
  for (int e = 0; e < EPV; ++e)
    for (int o = LPR; o < 32; o <<= 1) m[e] = fmaxf(m[e], __shfl_xor_sync(0xffffffffu, m[e], o));
  if (lane < nv)
#pragma unroll
    for (int e = 0; e < EPV; ++e)
      if (m[e] > 0.0f) atomicMax(&loc[EPV * lane + e], __float_as_uint(m[e]));
  __syncthreads();
  if (threadIdx.x < kTcN && loc[threadIdx.x]) atomicMax(&xmax[threadIdx.x], loc[threadIdx.x]);
}

// F = 2 + floor(log2 max): |hi + lo| < 2^(F-1)
__device__ __forceinline__ int tc_colexp(unsigned bits) {
  return bits ? (int)((bits >> 23) & 0xFF) - 127 + 2 : 0;
}

// v 2^sc for the coefficient scalings (|v 2^sc| <= 2^49, |sc| < 252): two
// power-of-two factors that are normal floats, so the product is exact
// unless it is far below 1/2, where it rounds to the integer 0 anyway
__device__ __forceinline__ float scale2(float v, int sc) {
  const int h = sc >> 1;
  return v * pow2f(h) * pow2f(sc - h);
}

// the ND digits (exact floats) of round(v 2^sc) for a double-float or FP32 value
template <int ND>
__device__ __forceinline__ void digits_of(dd v, int sc, float (&f)[ND]) {
  split_digits_f<ND>(scale2(v.hi, sc), scale2(v.lo, sc), f);
}
template <int ND>
__device__ __forceinline__ void digits_of(float v, int sc, float (&f)[ND]) {
  split_digits_f<ND>(scale2(v, sc), 0.0f, f);
}

// two digits as their E4M3 bytes, the first in the low byte
__device__ __forceinline__ uint32_t e4m3x2(float a, float b) {
  return (uint32_t)__nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
}

// The digit planes of 16 consecutive values v[0..15] of one column, each
// scaled by 2^sc: plane i as one 16-byte word (the bytes in value order), a
// row of one core matrix of the MMA layout.
template <int ND, class T>
__device__ __forceinline__ void cut_row16(const T (&v)[16], int sc, uint4 (&w)[ND]) {
  uint32_t u[ND][4];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float f0[ND], f1[ND];
    digits_of<ND>(v[2 * q], sc, f0);
    digits_of<ND>(v[2 * q + 1], sc, f1);
#pragma unroll
    for (int i = 0; i < ND; ++i) {
      const uint32_t h = e4m3x2(f0[i], f1[i]);
      u[i][q >> 1] = (q & 1) ? (u[i][q >> 1] | (h << 16)) : h;
    }
  }
#pragma unroll
  for (int i = 0; i < ND; ++i) w[i] = make_uint4(u[i][0], u[i][1], u[i][2], u[i][3]);
}

// The ND E4M3 digit planes of the coefficients x^_c ([64][rp]) of clusters
// c0 .. c0 + ncl - 1, each with the column maxima of its own tree level:
// 64 threads per cluster (four per CTA), thread (g, j) cuts the values
// mu = 16 g .. 16 g + 15 of column j in registers and writes one 16-byte row
// of a core matrix per plane (zero digits for the columns j >= rp).
template <class T, int ND>
__global__ void __launch_bounds__(256) k_tc_slice_x(const T *__restrict__ xhat, int64_t c0, int64_t ncl, int rp,
                                                    const unsigned *__restrict__ xmax, unsigned char *__restrict__ xtc) {
  const int64_t ci = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 6);
  if (ci >= ncl) return;
  const int64_t c = c0 + ci;
  const int g = (threadIdx.x >> 4) & 3, j = threadIdx.x & 15;
  const T *xc = xhat + c * kTcK * rp;
  const int sc = Dig<ND>::kFix - tc_colexp(xmax[tc_level(c) * kTcN + j]);
  T v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = j < rp ? xc[(16 * g + q) * rp + j] : T{};
  uint4 w[ND];
  cut_row16<ND>(v, sc, w);
  unsigned char *dst = xtc + c * (int64_t)Dig<ND>::kTileB + core_off(j, 16 * g);
#pragma unroll
  for (int i = 0; i < ND; ++i) *reinterpret_cast<uint4 *>(dst + i * Dig<ND>::kPlaneB) = w[i];
}

__device__ __forceinline__ dd dd_scale(dd v, int e) {
  if (e >= -126 && e <= 127) {
    const float w = pow2f(e);
    return dd{v.hi * w, v.lo * w};
  }
  return dd{ldexpf(v.hi, e), ldexpf(v.lo, e)};
}

// The coupling kernel (see the top of the file).  Rows t = row0 + r for r
// in [0, nrows); each CTA takes a contiguous range of rows holding about
// 1/gridDim of the blocks.
// T: the coefficient type (dd with ND = 10, float with ND = 6).
// DIAG: row r holds the single block r in column r (ptr = col = NULL), its
// row powers of two are E[r][nu] and the column powers xmax[j] (one level):
// the leaf forward step x^_t = V_t^T x|t with KB = 32, the V_t^T digit
// planes as the blocks and the input digit planes of leaf t as the
// coefficients (with ymax, the largest |hi| of every column of the results
// is taken too, as float bits).  Three epilogue warp groups then take every
// third row, and two
// neighbouring digit levels are combined exactly in FP32 before entering
// double-float: a level sum of one block is at most 5 x 32 x 16^2 < 2^15.4,
// so 32 D_L + D_(L+1) < 2^21.
__device__ __forceinline__ dd to_dd(dd v) { return v; }
__device__ __forceinline__ dd to_dd(float v) { return dd{v, 0.0f}; }
__device__ __forceinline__ void store_as(dd v, dd *p) { *p = v; }
__device__ __forceinline__ void store_as(dd v, float *p) { *p = v.hi + v.lo; }

constexpr int kDiagGroups = 3;   // epilogue warp groups of one-block rows
template <int ND, class T, int KB = kTcK, bool DIAG = false>
__global__ void __launch_bounds__(DIAG ? 64 + kDiagGroups * 128 : kTcThreads, 1)
    k_coupling_tc(const unsigned char *__restrict__ Stc, const unsigned char *__restrict__ xtc,
                  const int64_t *__restrict__ ptr, const int32_t *__restrict__ col, const int32_t *__restrict__ E,
                  const unsigned *__restrict__ xmax, int64_t row0, int64_t nrows, int rp, T *__restrict__ yhat,
                  unsigned *__restrict__ ymax = nullptr) {
  using D = Dig<ND, KB>;
  // first block of row t (t = row0 + r); one block per row without ptr
  auto pt = [&](int64_t t) -> int64_t { return DIAG ? t - row0 : ptr[t]; };
  constexpr int kTcStages = D::kStages, kTcGroups = D::kGroups;
  constexpr uint32_t kStage = D::kStage, kTileA = D::kTileA, kTileB = D::kTileB;
  extern __shared__ __align__(1024) unsigned char smem[];
  dd *xch = reinterpret_cast<dd *>(smem + kTcStages * kStage);
  constexpr int kSets = D::kSets;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + tc_bar_off<ND, KB, DIAG ? kDiagGroups : 1>());
  uint64_t *empty = full + kTcStages;
  uint64_t *accf = empty + kTcStages;   // [kSets]: the MMAs of a segment have completed
  uint64_t *acce = accf + kSets;        // [kSets]: the epilogue has read the set
  uint64_t *done = acce + kSets;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort = reinterpret_cast<volatile int *>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // rows of this CTA: from the first row whose blocks start at or after its share
  const int64_t b_all0 = pt(row0), total = pt(row0 + nrows) - b_all0;
  auto row_at = [&](int64_t w) -> int64_t {
    if (w >= (int64_t)gridDim.x) return nrows;
    const int64_t target = total * w / gridDim.x;
    int64_t lo = 0, hi = nrows;
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if (pt(row0 + mid) - b_all0 >= target) hi = mid;
      else lo = mid + 1;
    }
    return lo;
  };
  const int64_t r_begin = blockIdx.x == 0 ? 0 : row_at(blockIdx.x);
  const int64_t r_end = row_at(blockIdx.x + 1);
  const int64_t e_begin = pt(row0 + r_begin), e_end = pt(row0 + r_end);

  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int u = 0; u < kSets; ++u) {
      mbar_init(&accf[u], 1);
      mbar_init(&acce[u], 4);
    }
    mbar_init(done, 1);
    *abort = 0;
    mbar_fence_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;

  if (warp == 0) {
    // ---------------- producer: the slices of every block of the range
    if (lane == 0) {
      int64_t e = e_begin;
      ColAhead ca(col, e, e_end);
      const uint64_t pol_stream = l2_evict_first(), pol_keep = l2_evict_last();
      for (; e < e_end; ++e) {
        const int64_t i = e - e_begin;
        const int s = (int)(i % kTcStages);
        const int32_t cb = ca.next(e);
        if (i >= kTcStages && !mbar_wait_or_abort(&empty[s], (uint32_t)((i / kTcStages - 1) & 1), abort)) break;
        unsigned char *st = smem + (size_t)s * kStage;
        mbar_expect_tx(&full[s], kStage);
        // the coefficient digits first (read by every block of their column: kept in
        // L2), then S two planes at a time (read once: evicted first)
        bulk_g2s_hint(st + kTileA, xtc + (int64_t)cb * kTileB, kTileB, &full[s], pol_keep);
        const unsigned char *src = Stc + e * (int64_t)kTileA;
#pragma unroll
        for (int g = 0; g < kTcGroups; ++g)
          bulk_g2s_hint(st + 2 * g * D::kPlaneA, src + 2 * g * D::kPlaneA, 2 * D::kPlaneA, &full[s], pol_stream);
      }
      if (*abort) {
        // let the copies in flight land before the CTA leaves (bounded)
        const int64_t j0 = e - kTcStages > e_begin ? e - kTcStages : e_begin;
        for (int64_t j = j0; j < e; ++j) {
          const int64_t ij = j - e_begin;
          mbar_wait_bounded(&full[ij % kTcStages], (uint32_t)((ij / kTcStages) & 1));
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int64_t i = 0, q = 0;
      bool ok = true;
      int64_t pnext = pt(row0 + r_begin);   // row pointers loaded one row ahead
      for (int64_t r = r_begin; r < r_end && ok; ++r) {
        const int64_t b0 = pnext;
        pnext = pt(row0 + r + 1);
        const int64_t nb = pnext - b0;
        for (int64_t s0 = 0; s0 < nb && ok; s0 += kTcSegBlocks, ++q) {
          // accumulator set q mod kSets is free once the epilogue has read its previous use
          const int set = (int)(q % kSets);
          if (q >= kSets && !mbar_wait_or_abort(&acce[set], (uint32_t)((q / kSets - 1) & 1), abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dset = tbase + (uint32_t)set * D::kW;
          const int64_t sn = nb - s0 < kTcSegBlocks ? nb - s0 : kTcSegBlocks;
          for (int64_t t = 0; t < sn; ++t, ++i) {
            const int s = (int)(i % kTcStages);
            if (!mbar_wait_or_abort(&full[s], (uint32_t)((i / kTcStages) & 1), abort)) {
              ok = false;
              break;
            }
            tc_fence_after();
            // descriptors of the stage; offsets below 256 KB add to the 14-bit address field.
            // Group g: S digits 2g+1, 2g+2 (M = 128 rows) times x^ digits 1 .. ND - 2g into
            // column blocks 2g .. ND - 1 of the set.  Group 0 covers every column, so its
            // first MMA of a segment overwrites the set and all later ones accumulate.
            // K steps (32 bytes, two core matrices) outermost.
            const uint32_t A0 = smem_u32(smem + (size_t)s * kStage), B0 = A0 + kTileA;
            const uint64_t dA = sdesc_kb<KB>(A0), dB = sdesc_kb<KB>(B0);
#pragma unroll
            for (int kk = 0; kk < D::kKSteps; ++kk)
#pragma unroll
              for (int g = 0; g < kTcGroups; ++g)
                tc_mma(dset + D::col(g), dA + (uint64_t)((2 * g * D::kPlaneA + kk * 256) >> 4),
                       dB + (uint64_t)(kk * 16), tc_idesc(kTcN * D::nx(g)), (t > 0 || kk > 0 || g > 0) ? 1u : 0u);
            tc_commit(&empty[s]);   // the stage is free once these MMAs have read it
          }
          if (ok) tc_commit(&accf[set]);
        }
      }
      // every MMA issued has completed before the tensor memory is released
      tc_commit(done);
      mbar_wait_bounded(done, 0);
    }
    __syncwarp();
  } else if (DIAG) {
    // ---------------- one-block rows: warps 2-5 (group 0), 6-9 (group 1) and
    // 10-13 (group 2) take every third row; each reads tensor-memory lanes
    // 32 (warp % 4) ..
    const int grp = (warp - 2) >> 2;
    const int quad = warp & 3, tl = quad * 32 + lane, half = tl >> 6, nu = tl & 63;
    dd *xg = xch + grp * (64 * kTcN);
    const uint32_t bar_or = 1 + 2 * grp, bar_x = 2 + 2 * grp;
    int cx[kTcN];
    float cm[kTcN];   // column maxima of the rows this thread writes
#pragma unroll
    for (int j = 0; j < kTcN; ++j) {
      cx[j] = tc_colexp(xmax[j]);
      cm[j] = 0.0f;
    }
    int64_t r = r_begin + grp;
    int Enext = r < r_end ? E[r * kTcK + nu] : 0;   // the row's powers, loaded a row ahead
    for (; r < r_end; r += kDiagGroups) {
      const int64_t q = r - r_begin, t = row0 + r;
      const int Er = Enext;
      if (r + kDiagGroups < r_end) Enext = E[(r + kDiagGroups) * kTcK + nu];
      T *yrow = yhat + (t * kTcK + nu) * rp;
      const int set = (int)(q % kSets);
      const bool ready = !*abort && mbar_wait_or_abort(&accf[set], (uint32_t)((q / kSets) & 1), abort);
      if (named_sync_or_id(bar_or, 128, ready ? 0 : 1)) break;
      tc_fence_after();
      dd acc[kTcN];
#pragma unroll
      for (int j = 0; j < kTcN; ++j) acc[j] = dd{0.0f, 0.0f};
      // column block c holds level L = c + 2 + half; blocks c, c + 1 combine as
      // (32 D_L + D_(L+1)) 2^(2 - 5 (L + 1)), in increasing L
      const uint32_t tset = tbase + ((uint32_t)(quad * 32) << 16) + (uint32_t)set * D::kW;
#pragma unroll
      for (int c0 = 0; c0 < ND; c0 += 4) {
        uint32_t raw[4][16];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (c0 + u < ND) tmem_ld16_nw(tset + (uint32_t)((c0 + u) * kTcN), raw[u]);
        tmem_wait();
#pragma unroll
        for (int u = 0; u < 4; u += 2) {
          const int L = c0 + u + 2 + half;
          if (c0 + u < ND && L <= D::kTop) {
            const float w = pow2f(2 - 5 * (L + 1));
            const float c1 = L + 1 <= D::kTop ? 1.0f : 0.0f;
#pragma unroll
            for (int j = 0; j < kTcN; ++j) {
              const float v = 32.0f * __uint_as_float(raw[u][j]) + c1 * __uint_as_float(raw[u + 1][j]);
              acc[j] = acc[j] + dd{v * w, 0.0f};
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[set]);
      if (half == 1)
#pragma unroll
        for (int j = 0; j < kTcN; ++j) xg[j * 64 + nu] = acc[j];
      named_sync_id(bar_x, 128);
      if (half == 0) {
#pragma unroll
        for (int j = 0; j < kTcN; ++j) {
          if (j >= rp) break;
          const dd v = dd_scale(acc[j] + xg[j * 64 + nu], Er + cx[j]);
          store_as(v, yrow + j);
          cm[j] = fmaxf(cm[j], fabsf(v.hi));
        }
      }
      named_sync_id(bar_x, 128);
    }
    if (ymax && half == 0) {
#pragma unroll
      for (int j = 0; j < kTcN; ++j) {
        float m = cm[j];
#pragma unroll
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0 && j < rp && m > 0.0f) atomicMax(&ymax[j], __float_as_uint(m));
      }
    }
  } else {
    // ---------------- epilogue: warps 2-5 read tensor-memory lanes 32 (warp % 4) ..
    const int quad = warp & 3, tl = quad * 32 + lane, half = tl >> 6, nu = tl & 63;
    int64_t q = 0;
    for (int64_t r = r_begin; r < r_end; ++r) {
      const int64_t t = row0 + r;
      const int64_t nb = pt(t + 1) - pt(t);
      T *yrow = yhat + (t * kTcK + nu) * rp;
      if (nb == 0) {
        if (half == 0)
          for (int j = 0; j < rp; ++j) store_as(dd{0.0f, 0.0f}, yrow + j);
        continue;
      }
      const int Er = E[t * kTcK + nu];
      const int lvl = tc_level(t);
      int Fc[kTcN];
#pragma unroll
      for (int j = 0; j < kTcN; ++j) Fc[j] = Er + tc_colexp(xmax[lvl * kTcN + j]);
      bool stop = false;
      for (int64_t s0 = 0; s0 < nb; s0 += kTcSegBlocks, ++q) {
        const int set = (int)(q % kSets);
        const bool ready = !*abort && mbar_wait_or_abort(&accf[set], (uint32_t)((q / kSets) & 1), abort);
        if (named_sync_or(128, ready ? 0 : 1)) {   // all epilogue warps agree to stop
          stop = true;
          break;
        }
        tc_fence_after();
        dd acc[kTcN];
#pragma unroll
        for (int j = 0; j < kTcN; ++j) acc[j] = dd{0.0f, 0.0f};
        // column block c of lane nu (+ 64) holds the sum of every digit pair of level
        // L = c + 2 (+ 1) (integers, exact in FP32); the levels share the weight
        // 2^(2-5L) and enter the double-float result once each, in increasing order
        // (L <= ND + 1: lanes 64-127 skip their last block)
        const uint32_t tset = tbase + ((uint32_t)(quad * 32) << 16) + (uint32_t)set * D::kW;
#pragma unroll
        for (int c0 = 0; c0 < ND; c0 += 5) {
          uint32_t raw[5][16];
#pragma unroll
          for (int u = 0; u < 5; ++u)
            if (c0 + u < ND) tmem_ld16_nw(tset + (uint32_t)((c0 + u) * kTcN), raw[u]);
          tmem_wait();
#pragma unroll
          for (int u = 0; u < 5; ++u) {
            const int L = c0 + u + 2 + half;
            if (c0 + u < ND && L <= D::kTop) {
              const float w = pow2f(2 - 5 * L);
#pragma unroll
              for (int j = 0; j < kTcN; ++j) acc[j] = acc[j] + dd{__uint_as_float(raw[u][j]) * w, 0.0f};
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[set]);
        if (half == 1)
#pragma unroll
          for (int j = 0; j < kTcN; ++j) xch[j * 64 + nu] = acc[j];   // consecutive lanes, consecutive words
        named_sync_id(2, 128);
        if (half == 0) {
#pragma unroll
          for (int j = 0; j < kTcN; ++j) {
            if (j >= rp) break;
            dd v = dd_scale(acc[j] + xch[j * 64 + nu], Fc[j]);
            if (s0 > 0) v = v + to_dd(yrow[j]);
            store_as(v, yrow + j);
          }
        }
        named_sync_id(2, 128);
      }
      if (stop) break;
    }
  }
  // tensor memory is released once every role is done
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols) : "memory");
}


// ---------------------------------------------------------------- nearfield
// The nearfield phase (Algorithm 3 over the inadmissible leaf pairs,
// y|t += G_ts x|s) with the same exact digit products: every row nu of leaf
// t gets a power of two 2^E over its near blocks, every column j of the
// permuted input x a power of two 2^F over all leaves, and both sides are
// cut into the ten E4M3 digits above.  A block G_ts is L x L (L <= 21
// triangles per leaf); its contraction index (the triangles of s) is padded
// with zeros to K = 32 bytes, one MMA K step.  The digit planes of a block
// are stacked along M: digits 1-6 in rows (i - 1) L + nu of the first
// 128-row group, digits 7-10 in rows (i - 7) L + nu of the second; the
// input digits of leaf s are the N side (16 columns per plane).  Two MMAs
// per block: group 1 against input digits 1-10 (N = 160), group 2 against
// input digits 1-4 (N = 64), so every pair with i + k <= 11 is formed.  Two
// accumulator sets of 224 columns let the epilogue of one row run while the
// MMAs of the next fill the other set.  Rows longer than 32 blocks are cut
// into segments: a sum D_ik then stays below 32 x 21 x 2^8 < 2^17.4, so two
// neighbouring input digits combine exactly in FP32 (32 D_ik + D_i,k+1 <
// 2^23) before entering double-float.
constexpr int kNtLmax = 21;                      // six planes of 21 rows fit in 128
constexpr int kNtPlanes1 = 6;                    // digits 1-6 in the first group, 7-10 in the second
constexpr uint32_t kNtRowB = 32;                 // bytes per operand row (K = 32)
constexpr uint32_t kNtG1 = 128 * kNtRowB;        // 4096: the first group of a block
// the A region of a stage holds the stored block (at most 4096 + 88 x 32 bytes); the
// second MMA reads 128 rows from 4096 on, i.e. past the block's 4 L rows into the
// input digits that follow (or the next stage, or the exchange area after the last
// stage): rows whose accumulators the epilogue never reads
constexpr uint32_t kNtAreg = kNtG1 + 88 * kNtRowB;      // 6912
constexpr uint32_t kNtX = kTcSlices * kTcN * kNtRowB;   // 5120: the input digits of one leaf
constexpr uint32_t kNtStage = kNtAreg + kNtX;           // 12032
constexpr int kNtStages = 16;
constexpr int kNtSeg = 32;                       // blocks per exact segment
constexpr int kNtN1 = kTcSlices * kTcN;          // 160
constexpr int kNtN2 = 4 * kTcN;                  // 64
constexpr uint32_t kNtSet = 256;                 // tensor-memory columns per accumulator set
constexpr uint32_t kNtXch = kTcSlices * kNtLmax * kTcN * 8;   // 26880: [digit][nu][j] double-float
constexpr uint32_t kNtBarOff = kNtStages * kNtStage + kNtXch;
constexpr uint32_t kNtSmem = kNtBarOff + 512;
static_assert(kNtSmem <= 227 * 1024, "nearfield tensor-core kernel does not fit in shared memory");

// byte offset of (row r, contraction index c) in a K-major one-byte operand
// of 32 contraction values per row: two core matrices along K (128 bytes
// apart), then the next 8 rows (256 bytes on)
__host__ __device__ __forceinline__ int core_off32(int r, int c) {
  return ((r >> 3) * 2 + (c >> 4)) * 128 + (r & 7) * 16 + (c & 15);
}
__device__ __forceinline__ uint64_t sdesc32(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(256u >> 4) << 32) |
         (1ull << 46);
}

// bytes of the stored digits of one block: group 1 (128 rows) and the 4 L rows of group 2
__host__ __device__ __forceinline__ uint32_t ntc_block_bytes(int L) {
  return kNtG1 + (uint32_t)((4 * L + 7) / 8 * 8) * kNtRowB;
}

// E[t][nu] = 1 + floor(log2 max |G_b[nu][mu]|) over the near blocks b of leaf row t (0 if none)
__global__ void k_ntc_rowexp(const dd *__restrict__ near, const int64_t *__restrict__ ptr, int64_t nleaf, int L,
                             int Lp, int32_t *__restrict__ E) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nleaf * L) return;
  const int64_t t = e / L;
  const int nu = (int)(e % L);
  float mx = 0.0f;
  for (int64_t b = ptr[t]; b < ptr[t + 1]; ++b)
    for (int mu = 0; mu < L; ++mu) mx = fmaxf(mx, fabsf(near[(b * L + mu) * Lp + nu].hi));
  E[e] = mx > 0.0f ? ilogbf(mx) + 1 : 0;
}

// the ten digit planes of block b, row nu, contraction indices 16 cg .. 16 cg + 15
__global__ void k_ntc_slice(const dd *__restrict__ near, const int32_t *__restrict__ brow,
                            const int32_t *__restrict__ E, int64_t nnear, int L, int Lp, uint32_t ablk,
                            unsigned char *__restrict__ Ntc) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nnear * L * 2) return;
  const int64_t b = e / (2 * L);
  const int nu = (int)((e / 2) % L), cg = (int)(e % 2);
  const int sc = kTcFixBits - E[(int64_t)brow[b] * L + nu];
  __align__(16) unsigned char out[kTcSlices][16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int mu = 16 * cg + q;
    long long X = 0;
    if (mu < L) {
      const dd v = near[(b * L + mu) * Lp + nu];
      X = llrint(ldexp((double)v.hi + (double)v.lo, sc));
    }
    int sl[kTcSlices];
    split_digits(X, sl);
#pragma unroll
    for (int i = 0; i < kTcSlices; ++i) out[i][q] = e4m3(sl[i]);
  }
  unsigned char *base = Ntc + b * (int64_t)ablk;
#pragma unroll
  for (int i = 0; i < kTcSlices; ++i) {
    const int r = i < kNtPlanes1 ? i * L + nu : (i - kNtPlanes1) * L + nu;
    const uint32_t g = i < kNtPlanes1 ? 0u : kNtG1;
    *reinterpret_cast<uint4 *>(base + g + core_off32(r, 16 * cg)) = *reinterpret_cast<const uint4 *>(out[i]);
  }
}

// the digit planes of the input of leaf s (x_pad rows s L .. s L + L - 1): 16
// rows j x 32 bytes each; 32 threads per leaf (four per CTA), thread (g, j)
// cuts rows mu = 16 g .. 16 g + 15 of column j (zero beyond L and rp)
__global__ void __launch_bounds__(128) k_ntc_slice_x(const dd *__restrict__ xpad, int64_t nleaf, int L, int rp,
                                                     const unsigned *__restrict__ xmax,
                                                     unsigned char *__restrict__ xnt) {
  const int64_t t = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
  if (t >= nleaf) return;
  const int g = (threadIdx.x >> 4) & 1, j = threadIdx.x & 15;
  const int sc = kTcFixBits - tc_colexp(xmax[j]);
  dd v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int mu = 16 * g + q;
    v[q] = mu < L && j < rp ? xpad[(t * L + mu) * rp + j] : dd{0.0f, 0.0f};
  }
  uint4 w[kTcSlices];
  cut_row16<kTcSlices>(v, sc, w);
  unsigned char *dst = xnt + t * (int64_t)kNtX + core_off32(j, 16 * g);
#pragma unroll
  for (int i = 0; i < kTcSlices; ++i) *reinterpret_cast<uint4 *>(dst + i * (kTcN * kNtRowB)) = w[i];
}

// Leaf forward step on the tensor cores (Algorithm 1 at the leaves,
// x^_t = V_t^T x|t, FP64-accurate handles of order 4 with leaves of at most
// 32 triangles): the blocks are V_t^T (64 rows nu, the leaf's triangles r as
// the contraction index, zero padded to 32 bytes), cut once into the ten
// digit planes of the coupling with a power of two per row,
// Ev[t][nu] = 1 + floor(log2 max_r |V_t[r][nu]|); the coefficients are the
// input digit planes of leaf t that the nearfield cuts (k_ntc_slice_x).
__global__ void k_tcv_rowexp(const dd *__restrict__ V, int64_t nleaf, int L, int kp, int32_t *__restrict__ Ev) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nleaf * kTcK) return;
  const int64_t t = e / kTcK;
  const int nu = (int)(e % kTcK);
  float mx = 0.0f;
  for (int r = 0; r < L; ++r) mx = fmaxf(mx, fabsf(V[(t * L + r) * kp + nu].hi));
  Ev[e] = mx > 0.0f ? ilogbf(mx) + 1 : 0;
}

// the ten digit planes of V_t^T, row nu, contraction indices 16 cg .. 16 cg + 15
__global__ void k_tcv_slice(const dd *__restrict__ V, const int32_t *__restrict__ Ev, int64_t nleaf, int L, int kp,
                            unsigned char *__restrict__ Vtc) {
  using D = Dig<kTcSlices, 32>;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nleaf * kTcK * 2) return;
  const int64_t t = e / (kTcK * 2);
  const int nu = (int)((e / 2) % kTcK), cg = (int)(e % 2);
  const int sc = kTcFixBits - Ev[t * kTcK + nu];
  __align__(16) unsigned char out[kTcSlices][16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int r = 16 * cg + q;
    long long X = 0;
    if (r < L) {
      const dd v = V[(t * L + r) * kp + nu];
      X = llrint(ldexp((double)v.hi + (double)v.lo, sc));
    }
    int sl[kTcSlices];
    split_digits(X, sl);
#pragma unroll
    for (int i = 0; i < kTcSlices; ++i) out[i][q] = e4m3(sl[i]);
  }
  unsigned char *base = Vtc + t * (int64_t)D::kTileA + core_off32(nu, 16 * cg);
#pragma unroll
  for (int i = 0; i < kTcSlices; ++i)
    *reinterpret_cast<uint4 *>(base + i * D::kPlaneA) = *reinterpret_cast<const uint4 *>(out[i]);
}

// The nearfield kernel: rows t in [0, nrows) (leaves), each CTA a contiguous
// range of rows holding about 1/gridDim of the blocks; roles as in
// k_coupling_tc (producer warp, MMA warp, four epilogue warps).
__global__ void __launch_bounds__(kTcThreads, 1)
    k_near_tc(const unsigned char *__restrict__ Ntc, uint32_t ablk, const unsigned char *__restrict__ xnt,
              const int64_t *__restrict__ ptr, const int32_t *__restrict__ col, const int32_t *__restrict__ E,
              const unsigned *__restrict__ xmax, int64_t nrows, int L, int rp, int accumulate,
              dd *__restrict__ ypad) {
  extern __shared__ __align__(1024) unsigned char smem[];
  dd *xch = reinterpret_cast<dd *>(smem + kNtStages * kNtStage);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + kNtBarOff);
  uint64_t *empty = full + kNtStages;
  uint64_t *accf = empty + kNtStages;   // [2]
  uint64_t *acce = accf + 2;            // [2]
  uint64_t *done = acce + 2;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort = reinterpret_cast<volatile int *>(tslot + 1);
  int *fexp = reinterpret_cast<int *>(smem + kNtBarOff + 320);   // column exponents F_j
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < kTcN) fexp[tid] = tc_colexp(xmax[tid]);

  const int64_t total = ptr[nrows];
  auto row_at = [&](int64_t w) -> int64_t {
    if (w >= (int64_t)gridDim.x) return nrows;
    const int64_t target = total * w / gridDim.x;
    int64_t lo = 0, hi = nrows;
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if (ptr[mid] >= target) hi = mid;
      else lo = mid + 1;
    }
    return lo;
  };
  const int64_t r_begin = blockIdx.x == 0 ? 0 : row_at(blockIdx.x);
  const int64_t r_end = row_at(blockIdx.x + 1);
  const int64_t e_begin = ptr[r_begin], e_end = ptr[r_end];

  if (tid == 0) {
    for (int s = 0; s < kNtStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&accf[s], 1);
      mbar_init(&acce[s], 4);
    }
    mbar_init(done, 1);
    *abort = 0;
    mbar_fence_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;

  if (warp == 0) {
    // ---------------- producer: the digits of every block of the range and of its column leaf
    if (lane == 0) {
      int64_t e = e_begin;
      ColAhead ca(col, e, e_end);
      const uint64_t pol_stream = l2_evict_first(), pol_keep = l2_evict_last();
      for (; e < e_end; ++e) {
        const int64_t i = e - e_begin;
        const int s = (int)(i % kNtStages);
        const int32_t cb = ca.next(e);
        if (i >= kNtStages && !mbar_wait_or_abort(&empty[s], (uint32_t)((i / kNtStages - 1) & 1), abort)) break;
        unsigned char *st = smem + (size_t)s * kNtStage;
        mbar_expect_tx(&full[s], ablk + kNtX);
        bulk_g2s_hint(st + kNtAreg, xnt + (int64_t)cb * kNtX, kNtX, &full[s], pol_keep);
        bulk_g2s_hint(st, Ntc + e * (int64_t)ablk, ablk, &full[s], pol_stream);
      }
      if (*abort) {
        const int64_t j0 = e - kNtStages > e_begin ? e - kNtStages : e_begin;
        for (int64_t j = j0; j < e; ++j) {
          const int64_t ij = j - e_begin;
          mbar_wait_bounded(&full[ij % kNtStages], (uint32_t)((ij / kNtStages) & 1));
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int64_t i = 0, q = 0;
      bool ok = true;
      int64_t pnext = ptr[r_begin];   // row pointers loaded one row ahead
      for (int64_t r = r_begin; r < r_end && ok; ++r) {
        const int64_t b0 = pnext;
        pnext = ptr[r + 1];
        const int64_t nb = pnext - b0;
        for (int64_t s0 = 0; s0 < nb && ok; s0 += kNtSeg, ++q) {
          const uint32_t set = (uint32_t)(q & 1);
          // this set is free once the epilogue has read the segment before last
          if (q >= 2 && !mbar_wait_or_abort(&acce[set], (uint32_t)(((q - 2) >> 1) & 1), abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int64_t sn = nb - s0 < kNtSeg ? nb - s0 : kNtSeg;
          for (int64_t t = 0; t < sn; ++t, ++i) {
            const int s = (int)(i % kNtStages);
            if (!mbar_wait_or_abort(&full[s], (uint32_t)((i / kNtStages) & 1), abort)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t A0 = smem_u32(smem + (size_t)s * kNtStage), B0 = A0 + kNtAreg;
            const uint64_t dA = sdesc32(A0), dB = sdesc32(B0);
            const uint32_t acc = t > 0 ? 1u : 0u;
            tc_mma(tbase + set * kNtSet, dA, dB, tc_idesc(kNtN1), acc);
            tc_mma(tbase + set * kNtSet + (uint32_t)kNtN1, dA + (uint64_t)(kNtG1 >> 4), dB, tc_idesc(kNtN2), acc);
            tc_commit(&empty[s]);
          }
          if (ok) tc_commit(&accf[set]);
        }
      }
      tc_commit(done);
      mbar_wait_bounded(done, 0);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: warps 2-5 read tensor-memory lanes 32 (warp % 4) ..
    const int quad = warp & 3, tl = quad * 32 + lane;
    const bool v1 = tl < kNtPlanes1 * L, v2 = tl < (kTcSlices - kNtPlanes1) * L;
    const int i1 = tl / L + 1, i2 = tl / L + 1 + kNtPlanes1, nu = tl % L;   // digit and row of this lane
    const int km1 = v1 ? kTcTop - i1 : 0, km2 = v2 ? kTcTop - i2 : 0;       // input digits paired with it
    const int km1w = __reduce_max_sync(0xffffffffu, km1), km2w = __reduce_max_sync(0xffffffffu, km2);
    const uint32_t lrow = (uint32_t)(quad * 32) << 16;
    int64_t q = 0;
    int64_t pnext = ptr[r_begin];
    for (int64_t r = r_begin; r < r_end; ++r) {
      const int64_t b0 = pnext;
      pnext = ptr[r + 1];
      const int64_t nb = pnext - b0;
      dd *yrow = ypad + r * (int64_t)L * rp;
      if (nb == 0) {
        if (!accumulate)
          for (int o = tl; o < L * rp; o += 128) yrow[o] = dd{0.0f, 0.0f};
        continue;
      }
      bool stop = false;
      for (int64_t s0 = 0; s0 < nb; s0 += kNtSeg, ++q) {
        const uint32_t set = (uint32_t)(q & 1);
        // this thread's outputs o = tl + 128 u: row o % L, column o / L; their row
        // exponents and previous values are loaded before the wait
        int eo[3];
        dd yold[3];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int o = tl + 128 * u, rn = o % L, j = o / L;
          eo[u] = 0;
          yold[u] = dd{0.0f, 0.0f};
          if (o < L * kTcN && j < rp) {
            eo[u] = E[r * L + rn] + fexp[j];
            if (s0 > 0 || accumulate) yold[u] = yrow[rn * rp + j];
          }
        }
        const bool ready = !*abort && mbar_wait_or_abort(&accf[set], (uint32_t)((q >> 1) & 1), abort);
        if (named_sync_or(128, ready ? 0 : 1)) {
          stop = true;
          break;
        }
        tc_fence_after();
        dd p1[kTcN], p2[kTcN];
#pragma unroll
        for (int j = 0; j < kTcN; ++j) p1[j] = p2[j] = dd{0.0f, 0.0f};
        // group 1: input digits k, k + 1 combined exactly, weight 2^(2 - 5 (i + k + 1))
#pragma unroll 1
        for (int k = 1; k <= km1w; k += 2) {
          uint32_t ra[16], rb[16];
          tmem_ld16_nw(tbase + lrow + set * kNtSet + (uint32_t)((k - 1) * kTcN), ra);
          if (k + 1 <= km1w) tmem_ld16_nw(tbase + lrow + set * kNtSet + (uint32_t)(k * kTcN), rb);
          tmem_wait();
          const float ca = k <= km1 ? 32.0f : 0.0f, cb = k + 1 <= km1 ? 1.0f : 0.0f;
          const float w = pow2f(2 - 5 * (i1 + k + 1));
#pragma unroll
          for (int j = 0; j < kTcN; ++j) {
            const float v = ca * __uint_as_float(ra[j]) + (k + 1 <= km1w ? cb * __uint_as_float(rb[j]) : 0.0f);
            p1[j] = p1[j] + dd{v * w, 0.0f};
          }
        }
        // group 2: digits 7-10 against input digits 1-4
#pragma unroll 1
        for (int k = 1; k <= km2w; k += 2) {
          uint32_t ra[16], rb[16];
          tmem_ld16_nw(tbase + lrow + set * kNtSet + (uint32_t)(kNtN1 + (k - 1) * kTcN), ra);
          if (k + 1 <= km2w) tmem_ld16_nw(tbase + lrow + set * kNtSet + (uint32_t)(kNtN1 + k * kTcN), rb);
          tmem_wait();
          const float ca = k <= km2 ? 32.0f : 0.0f, cb = k + 1 <= km2 ? 1.0f : 0.0f;
          const float w = pow2f(2 - 5 * (i2 + k + 1));
#pragma unroll
          for (int j = 0; j < kTcN; ++j) {
            const float v = ca * __uint_as_float(ra[j]) + (k + 1 <= km2w ? cb * __uint_as_float(rb[j]) : 0.0f);
            p2[j] = p2[j] + dd{v * w, 0.0f};
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[set]);
        // exchange [j][digit][row]: consecutive lanes write consecutive words
        const int dl = kTcSlices * L;
        if (v1)
#pragma unroll
          for (int j = 0; j < kTcN; ++j) xch[j * dl + (i1 - 1) * L + nu] = p1[j];
        if (v2)
#pragma unroll
          for (int j = 0; j < kTcN; ++j) xch[j * dl + (i2 - 1) * L + nu] = p2[j];
        named_sync_id(2, 128);
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int o = tl + 128 * u, rn = o % L, j = o / L;
          if (o >= L * kTcN || j >= rp) continue;
          const dd *xc = xch + j * dl + rn;
          dd v = xc[0];
#pragma unroll
          for (int i = 1; i < kTcSlices; ++i) v = v + xc[i * L];
          v = dd_scale(v, eo[u]);
          if (s0 > 0 || accumulate) v = v + yold[u];
          yrow[rn * rp + j] = v;
        }
        named_sync_id(2, 128);
      }
      if (stop) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols) : "memory");
}
}  // namespace

// ---------------------------------------------------------------- host side
// CTAs of k_tc_levmax: 8 warps of 4 rows each per pass, at most 8 CTAs per SM
static unsigned levmax_grid(int64_t rows) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + 31) / 32, 152 * 8));
}

// FP64-accurate (ten digits) or FP32-accurate (six digits) coupling of an
// order-4 handle with stored coupling matrices
bool tc_eligible(const Dev &d) {
  return (d.prec == H2_F64 || d.prec == H2_F32) && d.coupling == 0 && d.m == 4 && d.kp == kTcK;
}

namespace {

template <int ND>
int tc_build_nd(Ctx &c, const int32_t *arow_dev) {
  Dev &d = c.d;
  cudaStream_t st = c.stream;
  const int64_t row0 = ((int64_t)1 << d.first_adm_level) - 1;
  int rc;
  if ((rc = dev_alloc(d, (void **)&d.tc_E, sizeof(int32_t) * (size_t)d.nclu * kTcK))) return rc;
  if ((rc = dev_alloc(d, &d.Stc, (size_t)d.nadm * Dig<ND>::kTileA))) return rc;
  if ((rc = dev_alloc(d, &d.xtc, (size_t)d.nclu * Dig<ND>::kTileB))) return rc;
  if ((rc = dev_alloc(d, (void **)&d.tc_xmax, sizeof(unsigned) * 32 * kTcN))) return rc;
  H2_CUDA_TRY(cudaMemsetAsync(d.tc_E, 0, sizeof(int32_t) * (size_t)d.nclu * kTcK, st));
  H2_CUDA_TRY(cudaMemsetAsync(d.xtc, 0, (size_t)d.nclu * Dig<ND>::kTileB, st));
  const int64_t nr = (d.nclu - row0) * kTcK;
  k_tc_rowexp<<<(unsigned)((nr + 127) / 128), 128, 0, st>>>(d.adm_ptr, d.adm_col, d.cheb, row0, d.nclu, d.kernel,
                                                             d.tc_E);
  const int64_t ns = d.nadm * kTcK * 4;
  k_tc_slice_s<ND><<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(arow_dev, d.adm_col, d.cheb, d.tc_E, d.nadm,
                                                                 d.kernel, (unsigned char *)d.Stc);
  H2_CUDA_TRY(cudaGetLastError());
  H2_CUDA_TRY(cudaStreamSynchronize(st));
  d.tc_nd = ND;
  d.tc = true;
  return H2_OK;
}

// Upward pass of a product on the tensor-core path: the transfers of
// Algorithm 1, each level's column maxima taken on the way (k_up_reg /
// k_up_split; the leaves' by k_tc_levmax), then the coefficient digits of
// every far-field level in one launch (k_tc_slice_x, each cluster with its
// level's maxima).  Cutting a level's digits inside the next level's
// transfer launch was slower: the transfer threads are latency bound.
// Returns the launches made.
template <class T, int ND>
int tc_upward_t(Ctx &c, T *xhat, int rp, int64_t *launches, bool leaf_max) {
  Dev &d = c.d;
  cudaStream_t st = c.stream;
  const int D = d.depth, lmin = d.first_adm_level;
  if (lmin > D) return H2_OK;
  const int64_t leaf0 = d.nleaf - 1;
  int64_t nl = 0;
  if (!leaf_max) {
    H2_CUDA_TRY(cudaMemsetAsync(d.tc_xmax, 0, sizeof(unsigned) * 32 * kTcN, st));
    const int64_t lrows = d.nleaf * kTcK;
    k_tc_levmax<T><<<levmax_grid(lrows), 256, 0, st>>>(xhat + leaf0 * kTcK * rp, lrows, rp, d.tc_xmax + D * kTcN);
    ++nl;
  }
  for (int l = D - 1; l >= lmin; --l) {
    // level l from level l + 1, with the column maxima of level l
    const int64_t np = (int64_t)1 << l;
    if (np <= kUpSplitMax)
      k_up_split<T, T, 4><<<(unsigned)((np + kSplitParents - 1) / kSplitParents), 256, 0, st>>>(
          (const T *)d.Ef, rp, np - 1, np, xhat, d.tc_xmax + l * kTcN);
    else
      k_up_reg<T, T, 4><<<(unsigned)((np + kRegParents - 1) / kRegParents), 256, 0, st>>>(
          (const T *)d.Ef, rp, np - 1, np, xhat, d.tc_xmax + l * kTcN);
    ++nl;
  }
  // the digits of every level at once (all maxima are complete)
  const int64_t c0 = ((int64_t)1 << lmin) - 1, ncl = d.nclu - c0;
  k_tc_slice_x<T, ND><<<(unsigned)((ncl + 3) / 4), 256, 0, st>>>(xhat, c0, ncl, rp, d.tc_xmax,
                                                                 (unsigned char *)d.xtc);
  ++nl;
  H2_CUDA_TRY(cudaGetLastError());
  if (launches) *launches = nl;
  return H2_OK;
}

template <class T, int ND>
int tc_coupling_t(Ctx &c, T *yhat, int rp) {
  Dev &d = c.d;
  cudaStream_t st = c.stream;
  const int64_t row0 = ((int64_t)1 << d.first_adm_level) - 1, nrows = d.nclu - row0;
  if (nrows <= 0) return H2_OK;
  static_assert(tc_smem<ND>() <= 227 * 1024, "tensor-core coupling does not fit in shared memory");
  H2_CUDA_TRY(cudaFuncSetAttribute((const void *)k_coupling_tc<ND, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(227 * 1024)));
  int sms = 0, dev = 0;
  H2_CUDA_TRY(cudaGetDevice(&dev));
  H2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = (int)std::min<int64_t>(sms, nrows);
  k_coupling_tc<ND, T><<<grid, kTcThreads, tc_smem<ND>(), st>>>((const unsigned char *)d.Stc,
                                                                (const unsigned char *)d.xtc, d.adm_ptr, d.adm_col,
                                                                d.tc_E, d.tc_xmax, row0, nrows, rp, yhat);
  H2_CUDA_TRY(cudaGetLastError());
  return H2_OK;
}

}  // namespace

int tc_build(Ctx &c, const int32_t *arow_dev) {
  Dev &d = c.d;
  if (d.first_adm_level > d.depth || d.nadm == 0) return H2_OK;
  return d.prec == H2_F64 ? tc_build_nd<10>(c, arow_dev) : tc_build_nd<6>(c, arow_dev);
}

int tc_upward(Ctx &c, void *xhat, int rp, int64_t *launches, bool leaf_max) {
  if (rp > kTcN) return fail(H2_EINVAL, "the tensor-core coupling takes at most 16 right-hand sides");
  if (c.d.tc_nd == 10) return tc_upward_t<dd, 10>(c, static_cast<dd *>(xhat), rp, launches, leaf_max);
  return tc_upward_t<float, 6>(c, static_cast<float *>(xhat), rp, launches, leaf_max);
}

// the coupling phase: the coefficient digits exist (tc_upward)
int tc_coupling(Ctx &c, const void *xhat, void *yhat, int rp) {
  (void)xhat;
  if (rp > kTcN) return fail(H2_EINVAL, "the tensor-core coupling takes at most 16 right-hand sides");
  if (c.d.tc_nd == 10) return tc_coupling_t<dd, 10>(c, static_cast<dd *>(yhat), rp);
  return tc_coupling_t<float, 6>(c, static_cast<float *>(yhat), rp);
}

// ---------------------------------------------------------------- nearfield host side
bool ntc_eligible(const Dev &d) {
  return d.prec == H2_F64 && d.tensor == 0 && d.lmax <= kNtLmax && d.nnear > 0;
}

int ntc_build(Ctx &c, const int32_t *nrow_dev) {
  Dev &d = c.d;
  cudaStream_t st = c.stream;
  if (!ntc_eligible(d)) return H2_OK;
  const int L = (int)d.lmax, Lp = (int)d.lp;
  const uint32_t ablk = ntc_block_bytes(L);
  int rc;
  if ((rc = dev_alloc(d, (void **)&d.ntc_E, sizeof(int32_t) * (size_t)d.nleaf * L))) return rc;
  if ((rc = dev_alloc(d, &d.Ntc, (size_t)d.nnear * ablk))) return rc;
  if ((rc = dev_alloc(d, &d.xnt, (size_t)d.nleaf * kNtX))) return rc;
  if ((rc = dev_alloc(d, (void **)&d.ntc_xmax, sizeof(unsigned) * kTcN))) return rc;
  H2_CUDA_TRY(cudaMemsetAsync(d.Ntc, 0, (size_t)d.nnear * ablk, st));
  const int64_t nr = d.nleaf * L;
  k_ntc_rowexp<<<(unsigned)((nr + 127) / 128), 128, 0, st>>>((const dd *)d.near, d.near_ptr, d.nleaf, L, Lp,
                                                             d.ntc_E);
  const int64_t ns = d.nnear * L * 2;
  k_ntc_slice<<<(unsigned)((ns + 255) / 256), 256, 0, st>>>((const dd *)d.near, nrow_dev, d.ntc_E, d.nnear, L, Lp,
                                                            ablk, (unsigned char *)d.Ntc);
  H2_CUDA_TRY(cudaGetLastError());
  if (d.tc && d.tc_nd == kTcSlices && d.k == kTcK && d.kp == kTcK && L <= 32) {
    // the V_t^T digit planes of the tensor-core leaf forward step
    using DV = Dig<kTcSlices, 32>;
    if ((rc = dev_alloc(d, (void **)&d.tcv_E, sizeof(int32_t) * (size_t)d.nleaf * kTcK))) return rc;
    if ((rc = dev_alloc(d, &d.Vtc, (size_t)d.nleaf * DV::kTileA))) return rc;
    const int64_t nv = d.nleaf * kTcK;
    k_tcv_rowexp<<<(unsigned)((nv + 127) / 128), 128, 0, st>>>((const dd *)d.V, d.nleaf, L, (int)d.kp, d.tcv_E);
    k_tcv_slice<<<(unsigned)((2 * nv + 255) / 256), 256, 0, st>>>((const dd *)d.V, d.tcv_E, d.nleaf, L, (int)d.kp,
                                                                  (unsigned char *)d.Vtc);
    H2_CUDA_TRY(cudaGetLastError());
  }
  H2_CUDA_TRY(cudaStreamSynchronize(st));
  d.ntc_ablk = ablk;
  d.ntc = true;
  return H2_OK;
}

// the input's column maxima and its digit planes per leaf (read by the
// nearfield and by the tensor-core leaf forward step)
int ntc_input(Ctx &c, const void *xpad_v, int rp, int64_t *launches, bool have_max) {
  const dd *xpad = static_cast<const dd *>(xpad_v);
  Dev &d = c.d;
  cudaStream_t st = c.stream;
  if (rp > kTcN) return fail(H2_EINVAL, "the tensor-core nearfield takes at most 16 right-hand sides");
  const int L = (int)d.lmax;
  if (!have_max) {
    H2_CUDA_TRY(cudaMemsetAsync(d.ntc_xmax, 0, sizeof(unsigned) * kTcN, st));
    const int64_t rows = d.nleaf * L;
    k_tc_levmax<dd><<<levmax_grid(rows), 256, 0, st>>>(xpad, rows, rp, d.ntc_xmax);
  }
  k_ntc_slice_x<<<(unsigned)((d.nleaf + 3) / 4), 128, 0, st>>>(xpad, d.nleaf, L, rp, d.ntc_xmax,
                                                               (unsigned char *)d.xnt);
  H2_CUDA_TRY(cudaGetLastError());
  if (launches) *launches = have_max ? 1 : 2;
  return H2_OK;
}

// the leaf forward step on the tensor cores: x^ of the leaf clusters from the
// input digits (ntc_input) and the stored V_t^T digits, with their column
// maxima for the upward pass
int tc_leaf_forward(Ctx &c, void *xhat_v, int rp) {
  Dev &d = c.d;
  cudaStream_t st = c.stream;
  if (rp > kTcN || !d.Vtc) return fail(H2_EINVAL, "no tensor-core leaf forward step for this handle");
  constexpr int KB = 32;
  constexpr uint32_t sm = tc_smem<kTcSlices, KB, kDiagGroups>();
  static_assert(sm <= 227 * 1024, "tensor-core leaf step does not fit in shared memory");
  H2_CUDA_TRY(cudaFuncSetAttribute((const void *)k_coupling_tc<kTcSlices, dd, KB, true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(227 * 1024)));
  int sms = 0, dev = 0;
  H2_CUDA_TRY(cudaGetDevice(&dev));
  H2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = (int)std::min<int64_t>(sms, d.nleaf);
  // the leaf level's column maxima of the upward pass are taken here
  // (tc_upward with leaf_max); every level's maxima start from zero
  H2_CUDA_TRY(cudaMemsetAsync(d.tc_xmax, 0, sizeof(unsigned) * 32 * kTcN, st));
  k_coupling_tc<kTcSlices, dd, KB, true><<<grid, 64 + kDiagGroups * 128, sm, st>>>(
      (const unsigned char *)d.Vtc, (const unsigned char *)d.xnt, nullptr, nullptr, d.tcv_E, d.ntc_xmax,
      d.nleaf - 1, d.nleaf, rp, static_cast<dd *>(xhat_v), d.tc_xmax + d.depth * kTcN);
  H2_CUDA_TRY(cudaGetLastError());
  return H2_OK;
}

// the nearfield phase on the tensor cores: the input's column maxima, its
// digit planes per leaf, then the block rows (y_pad += or = the near sums)
int ntc_near(Ctx &c, const void *xpad_v, void *ypad_v, int rp, int accumulate, int64_t *launches, bool have_input) {
  dd *ypad = static_cast<dd *>(ypad_v);
  Dev &d = c.d;
  cudaStream_t st = c.stream;
  if (rp > kTcN) return fail(H2_EINVAL, "the tensor-core nearfield takes at most 16 right-hand sides");
  const int L = (int)d.lmax;
  int64_t nin = 0;
  int rc;
  if (!have_input && (rc = ntc_input(c, xpad_v, rp, &nin))) return rc;
  H2_CUDA_TRY(cudaFuncSetAttribute((const void *)k_near_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(227 * 1024)));
  int sms = 0, dev = 0;
  H2_CUDA_TRY(cudaGetDevice(&dev));
  H2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = (int)std::min<int64_t>(sms, d.nleaf);
  k_near_tc<<<grid, kTcThreads, kNtSmem, st>>>((const unsigned char *)d.Ntc, d.ntc_ablk,
                                               (const unsigned char *)d.xnt, d.near_ptr, d.near_col, d.ntc_E,
                                               d.ntc_xmax, d.nleaf, L, rp, accumulate, ypad);
  H2_CUDA_TRY(cudaGetLastError());
  if (launches) *launches = nin + 1;
  return H2_OK;
}

// the tensor-core path's own device error word (bounded waits of this file)
int tc_take_error(cudaStream_t st) {
  int v = 0, zero = 0;
  H2_CUDA_TRY(cudaMemcpyFromSymbolAsync(&v, g_h2_device_error, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
  H2_CUDA_TRY(cudaStreamSynchronize(st));
  if (v) {
    H2_CUDA_TRY(cudaMemcpyToSymbolAsync(g_h2_device_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    return fail(H2_ETIMEOUT, "a bounded device wait of the tensor-core coupling ran out");
  }
  return H2_OK;
}

}  // namespace h2
