// Batched H^2 products over independent matrices of uneven sizes (FP32
// storage and arithmetic, stored coupling).
//
// Every block-row phase of the product (leaf forward, coupling, leaf
// backward, nearfield: Algorithms 1-3) runs as ONE persistent launch over
// the rows of all problems.  Rows differ in shape from problem to problem
// (rank k = m^3 for m = 3 or 4, leaf sizes up to 64, 1 to 16 right-hand
// sides), so the kernel is warp-per-row: every warp owns a contiguous range
// of rows holding about 1/(number of warps) of the work, in problem order,
// and streams the stored tiles of its rows through its own ring of shared-
// memory slots with bulk copies (TMA engine, one mbarrier per slot).  A slot
// holds several whole terms A X of one row, or one piece of a term cut along
// the contraction index when a term is larger than a slot.  Lane l owns the
// output rows 2l and 2l + 1 (row l for tiles of at most 32 rows) of the
// current row for all right-hand sides, multiplies in packed FP32 pairs and
// sums its terms in a fixed order: results are bit-reproducible.
//
// The transfer passes run level-synchronously across problems: step s of the
// upward pass treats level D_p - 1 - s of every problem p, step s of the
// downward pass level lmin_p + s.  The permutations in and out are one
// launch each over the packed vectors of all problems.  The whole sequence
// is captured once in a CUDA graph and replayed.
//
// The slot size, slots per warp and warps per CTA of every block-row phase
// are chosen by measurement (h2_batch_tune).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "h2_internal.hpp"
#include "h2_ptx.cuh"
#include "h2_transfer.cuh"

namespace h2 {
namespace {

// One problem's rows in one block-row phase.
struct BRows {
  const float *A;        // stored tiles: term b at A + b a_stride, [K][Mp] (contraction index major)
  const float *X;        // input tiles: unit u at X + u x_stride, [K][rp]
  const int64_t *ptr;    // terms of row r: [ptr[row0 + r], ptr[row0 + r + 1]); NULL: the single term r
  const int64_t *pend;   // if set, row r's terms end at pend[r] instead (rows made of chunks)
  const int32_t *col;    // unit of term b; NULL: unit = r
  float *out;            // output row r at out + r out_stride, [M][rp]
  int64_t a_stride, x_stride, out_stride, row0, nrows;
  int64_t w0;            // work of all earlier problems in this phase
  int64_t wterm, wrow;   // work of a term and of a row (bytes moved, plus a fixed overhead)
  int64_t cap;           // at most cap terms of a row are taken here (the rest goes to chunk rows)
  int64_t wfix;          // if > 0, every row counts wfix work (chunk rows)
  int M, Mp, K, rp;
  int tps;               // whole terms per slot; 0: terms are cut in pieces of P contraction rows
  int P, ppt;            // rows per piece, pieces per term (cut terms)
  int accumulate;
};

// One problem's parents in one transfer step.
struct BTr {
  const float *Ef;
  float *hat;
  int64_t par0, g0;      // first parent of the entry, its global parent index
  int m, k, rp, pad;
};

// One problem's part of the packed input / output vectors.
struct BPerm {
  const int32_t *pad_src;
  float *pad;
  int64_t n, npad, xoff, e0;
  int nrhs, rp;
};

constexpr int kBatchMaxRows = 64;   // output rows of a tile (k or the leaf size)
constexpr int kBatchMaxRp = 16;     // padded right-hand sides

// ---------------------------------------------------------------------------
// work partition: position (problem, row) of the first row whose work starts
// at or after W
struct Pos {
  int p;
  int64_t r;
};
__device__ __forceinline__ bool pos_less(Pos a, Pos b) { return a.p < b.p || (a.p == b.p && a.r < b.r); }

__device__ __forceinline__ int64_t row_work(const BRows &q, int64_t r) {
  if (q.wfix > 0) return q.w0 + r * q.wfix;
  const int64_t terms = q.ptr ? q.ptr[q.row0 + r] - q.ptr[q.row0] : r;
  return q.w0 + terms * q.wterm + r * q.wrow;
}

// first term and number of terms of row r
__device__ __forceinline__ void row_terms(const BRows &q, int64_t r, int64_t &b0, int64_t &nt) {
  if (!q.ptr) {
    b0 = r;
    nt = 1;
    return;
  }
  b0 = q.ptr[q.row0 + r];
  const int64_t e = q.pend ? q.pend[r] : q.ptr[q.row0 + r + 1];
  nt = min(e - b0, q.cap);
}

__device__ Pos find_pos(const BRows *__restrict__ pr, int np, int64_t W) {
  int lo = 0, hi = np - 1;   // largest p with w0 <= W
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (pr[mid].w0 <= W) lo = mid;
    else hi = mid - 1;
  }
  Pos ps{lo, 0};
  const BRows &q = pr[lo];
  int64_t a = 0, b = q.nrows;   // smallest r with row_work >= W
  while (a < b) {
    const int64_t mid = (a + b) / 2;
    if (row_work(q, mid) >= W) b = mid;
    else a = mid + 1;
  }
  ps.r = a;
  while (ps.p < np && ps.r >= pr[ps.p].nrows) {
    ps.p++;
    ps.r = 0;
  }
  return ps;
}

// issue cursor over the slots of a warp
struct Cur {
  int p;
  int64_t r, e, b0, nt;
  int q;
};

__device__ __forceinline__ void cur_load(const BRows *__restrict__ pr, Cur &c) {
  row_terms(pr[c.p], c.r, c.b0, c.nt);
  c.e = 0;
  c.q = 0;
}

// next row that has terms, or a position at or after end
__device__ __forceinline__ void cur_next_row(const BRows *__restrict__ pr, int np, Pos end, Cur &c) {
  for (;;) {
    c.r++;
    while (c.p < np && c.r >= pr[c.p].nrows) {
      c.p++;
      c.r = 0;
    }
    if (c.p >= np || !pos_less(Pos{c.p, c.r}, end)) return;
    cur_load(pr, c);
    if (c.nt > 0) return;
  }
}

__device__ __forceinline__ bool cur_valid(int np, Pos end, const Cur &c) {
  return c.p < np && pos_less(Pos{c.p, c.r}, end);
}

// lane 0 issues the copies of the cursor's slot into `slot`; all lanes advance the cursor
__device__ __forceinline__ void issue_slot(const BRows *__restrict__ pr, int np, Pos end, Cur &c,
                                           unsigned char *slot, uint64_t *bar, int lane) {
  const BRows &q = pr[c.p];
  if (q.tps > 0) {
    const int cnt = (int)min((int64_t)q.tps, c.nt - c.e);
    const uint32_t ab = 4u * q.K * q.Mp, xb = 4u * q.K * q.rp;
    if (lane == 0) {
      mbar_expect_tx(bar, (uint32_t)cnt * (ab + xb));
      for (int t = 0; t < cnt; ++t) {
        const int64_t b = c.b0 + c.e + t;
        const int64_t u = q.col ? (int64_t)q.col[b] : c.r;
        bulk_g2s(slot + t * (ab + xb), q.A + b * q.a_stride, ab, bar);
        bulk_g2s(slot + t * (ab + xb) + ab, q.X + u * q.x_stride, xb, bar);
      }
    }
    c.e += cnt;
  } else {
    const int r0 = c.q * q.P, rows = min(q.P, q.K - r0);
    const uint32_t ab = 4u * rows * q.Mp, xb = 4u * rows * q.rp;
    if (lane == 0) {
      const int64_t b = c.b0 + c.e;
      const int64_t u = q.col ? (int64_t)q.col[b] : c.r;
      mbar_expect_tx(bar, ab + xb);
      bulk_g2s(slot, q.A + b * q.a_stride + (int64_t)r0 * q.Mp, ab, bar);
      bulk_g2s(slot + ab, q.X + u * q.x_stride + (int64_t)r0 * q.rp, xb, bar);
    }
    if (++c.q == q.ppt) {
      c.q = 0;
      c.e++;
    }
  }
  if (c.e >= c.nt) cur_next_row(pr, np, end, c);
}

// Packed FP32 pairs: (lo, hi) in one 64-bit register pair.  fma.rn.f32x2
// rounds each half exactly like fmaf, so results equal the scalar form.
__device__ __forceinline__ uint64_t dup2(float a) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ void fma2(uint64_t &d, uint64_t a, uint64_t b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

// acc[i] += sum_mu A[mu][row_i] X[mu][:] over one segment of a slot, the
// columns of X in packed pairs.  QR = 2 (tiles of more than 32 rows): lane l
// owns rows 2l and 2l + 1 and reads both with one 8-byte load; QR = 1: row l.
template <int QR, int CP>
__device__ __forceinline__ void seg_fma(const float *sA, const float *sX, int rows, int Mp, int lane,
                                        uint64_t (&acc)[2][kBatchMaxRp / 2]) {
  const bool v = QR == 2 ? 2 * lane < Mp : lane < Mp;
#pragma unroll 4
  for (int mu = 0; mu < rows; ++mu) {
    uint64_t a0, a1 = 0;
    if (QR == 2) {
      const float2 av = v ? *reinterpret_cast<const float2 *>(sA + mu * Mp + 2 * lane) : make_float2(0.f, 0.f);
      a0 = dup2(av.x);
      a1 = dup2(av.y);
    } else {
      a0 = dup2(v ? sA[mu * Mp + lane] : 0.0f);
    }
#pragma unroll
    for (int c = 0; c < CP; c += 4) {
      const ulonglong2 xv = *reinterpret_cast<const ulonglong2 *>(sX + mu * CP + c);
      fma2(acc[0][c / 2], a0, xv.x);
      fma2(acc[0][c / 2 + 1], a0, xv.y);
      if (QR == 2) {
        fma2(acc[1][c / 2], a1, xv.x);
        fma2(acc[1][c / 2 + 1], a1, xv.y);
      }
    }
  }
}

__device__ __forceinline__ void seg_any(bool two, int rp, const float *sA, const float *sX, int rows, int Mp, int lane,
                                        uint64_t (&acc)[2][kBatchMaxRp / 2]) {
  switch (rp) {
    case 4: two ? seg_fma<2, 4>(sA, sX, rows, Mp, lane, acc) : seg_fma<1, 4>(sA, sX, rows, Mp, lane, acc); break;
    case 8: two ? seg_fma<2, 8>(sA, sX, rows, Mp, lane, acc) : seg_fma<1, 8>(sA, sX, rows, Mp, lane, acc); break;
    case 12: two ? seg_fma<2, 12>(sA, sX, rows, Mp, lane, acc) : seg_fma<1, 12>(sA, sX, rows, Mp, lane, acc); break;
    default: two ? seg_fma<2, 16>(sA, sX, rows, Mp, lane, acc) : seg_fma<1, 16>(sA, sX, rows, Mp, lane, acc); break;
  }
}

__device__ __forceinline__ float lo_of(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi_of(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }

// The batched block-row kernel (see the top of the file).  nslot slots of
// zbytes per warp, then nslot mbarriers per warp.
__global__ void __launch_bounds__(512) k_batch_rows(const BRows *__restrict__ pr, int np, int64_t wtotal, int nslot,
                                                    int zbytes) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  unsigned char *ring = smem + (size_t)wib * nslot * zbytes;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (size_t)wpb * nslot * zbytes) + (size_t)wib * nslot;
  const int64_t gw = (int64_t)blockIdx.x * wpb + wib, nw = (int64_t)gridDim.x * wpb;
  const Pos beg = find_pos(pr, np, wtotal * gw / nw);
  const Pos end = find_pos(pr, np, wtotal * (gw + 1) / nw);
  if (!pos_less(beg, end)) return;

  if (lane == 0) {
    for (int s = 0; s < nslot; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncwarp();

  // issue cursor: first row of the range that has terms
  Cur ic{beg.p, beg.r, 0, 0, 0, 0};
  cur_load(pr, ic);
  if (ic.nt == 0) cur_next_row(pr, np, end, ic);
  int64_t issued = 0, consumed = 0;
  while (issued < nslot && cur_valid(np, end, ic)) {
    issue_slot(pr, np, end, ic, ring + (size_t)issued * zbytes, &bar[issued], lane);
    ++issued;
  }

  Pos ps = beg;
  while (pos_less(ps, end)) {
    const BRows &q = pr[ps.p];
    int64_t b0, nt;
    row_terms(q, ps.r, b0, nt);
    const int64_t ns = q.tps > 0 ? (nt + q.tps - 1) / q.tps : nt * q.ppt;
    const bool two = q.M > 32;
    uint64_t acc[2][kBatchMaxRp / 2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int c = 0; c < kBatchMaxRp / 2; ++c) acc[i][c] = 0;
    for (int64_t j = 0; j < ns; ++j) {
      const int s = (int)(consumed % nslot);
      if (!mbar_wait_bounded(&bar[s], (uint32_t)((consumed / nslot) & 1))) {
        // a copy did not arrive: let the others in flight land, then leave
        for (int64_t i = consumed + 1; i < issued; ++i)
          mbar_wait_bounded(&bar[i % nslot], (uint32_t)((i / nslot) & 1));
        return;
      }
      const unsigned char *slot = ring + (size_t)s * zbytes;
      if (q.tps > 0) {
        const int cnt = (int)min((int64_t)q.tps, nt - j * q.tps);
        const int tb = 4 * q.K * (q.Mp + q.rp);
        for (int t = 0; t < cnt; ++t) {
          const float *sA = reinterpret_cast<const float *>(slot + t * tb);
          seg_any(two, q.rp, sA, sA + q.K * q.Mp, q.K, q.Mp, lane, acc);
        }
      } else {
        const int rows = min(q.P, q.K - (int)(j % q.ppt) * q.P);
        const float *sA = reinterpret_cast<const float *>(slot);
        seg_any(two, q.rp, sA, sA + rows * q.Mp, rows, q.Mp, lane, acc);
      }
      __syncwarp();
      ++consumed;
      if (cur_valid(np, end, ic)) {
        // the slot just read is refilled by the TMA engine: order the reads first
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue_slot(pr, np, end, ic, ring + (size_t)s * zbytes, &bar[s], lane);
        ++issued;
      }
    }
    // write the row: lane owns rows 2 lane and 2 lane + 1 (tiles of more than 32 rows) or row lane
    float *o = q.out + ps.r * q.out_stride;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int row = two ? 2 * lane + i : (i == 0 ? lane : q.M);
      if (row < q.M) {
        float4 *o4 = reinterpret_cast<float4 *>(o + (int64_t)row * q.rp);
#pragma unroll
        for (int c4 = 0; c4 < kBatchMaxRp / 4; ++c4) {
          if (4 * c4 < q.rp) {
            const uint64_t p0 = acc[i][2 * c4], p1 = acc[i][2 * c4 + 1];
            float4 v = make_float4(lo_of(p0), hi_of(p0), lo_of(p1), hi_of(p1));
            if (q.accumulate) {
              const float4 u = o4[c4];
              v.x += u.x;
              v.y += u.y;
              v.z += u.z;
              v.w += u.w;
            }
            o4[c4] = v;
          }
        }
      }
    }
    ps.r++;
    while (ps.p < np && ps.r >= pr[ps.p].nrows) {
      ps.p++;
      ps.r = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// transfers: warp per parent; global parent g -> (entry, parent) by the
// entries' first global parent index
constexpr int kTrWarps = 4;

__device__ __forceinline__ int find_entry(const BTr *__restrict__ te, int ne, int64_t g) {
  int lo = 0, hi = ne - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (te[mid].g0 <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(32 * kTrWarps) k_batch_upward(const BTr *__restrict__ te, int ne, int64_t total,
                                                                 int wfloats) {
  extern __shared__ __align__(16) float trs[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t g = (int64_t)blockIdx.x * kTrWarps + w;
  if (g >= total) return;
  const BTr &t = te[find_entry(te, ne, g)];
  upward_parent_warp<float, float>(t.Ef, t.m, t.k, t.rp, t.par0 + (g - t.g0), t.hat, trs + (size_t)w * wfloats, lane);
}

__global__ void __launch_bounds__(32 * kTrWarps) k_batch_downward(const BTr *__restrict__ te, int ne, int64_t total,
                                                                   int wfloats) {
  extern __shared__ __align__(16) float trs[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t g = (int64_t)blockIdx.x * kTrWarps + w;
  if (g >= total) return;
  const BTr &t = te[find_entry(te, ne, g)];
  downward_parent_warp<float, float>(t.Ef, t.m, t.k, t.rp, t.par0 + (g - t.g0), t.hat, trs + (size_t)w * wfloats,
                                     lane);
}

// rows cut in chunks: out (+)= the partial sums of the chunk rows, in chunk order
struct BRed {
  float *out;            // the output row (already holding the first chunk's sum)
  const float *part;     // nch partial rows of len values each
  int nch, len;
};

__global__ void k_batch_reduce(const BRed *__restrict__ rd) {
  const BRed &q = rd[blockIdx.x];
  for (int i = threadIdx.x; i < q.len; i += blockDim.x) {
    float v = q.out[i];
    for (int j = 0; j < q.nch; ++j) v += q.part[(int64_t)j * q.len + i];
    q.out[i] = v;
  }
}

// ---------------------------------------------------------------------------
// permutations over the packed vectors: element e of the padded space of all
// problems; each thread walks increasing e, so its problem index only grows
__device__ __forceinline__ int perm_problem(const BPerm *__restrict__ pp, int np, int64_t e) {
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (pp[mid].e0 <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_batch_permute_in(const BPerm *__restrict__ pp, int np, int64_t total, const float *__restrict__ x) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  int p = perm_problem(pp, np, e);
  for (; e < total; e += stride) {
    while (p + 1 < np && pp[p + 1].e0 <= e) ++p;
    const BPerm &q = pp[p];
    const int64_t l = e - q.e0, i = l / q.rp;
    const int c = (int)(l - i * q.rp);
    const int32_t src = q.pad_src[i];
    q.pad[l] = (src >= 0 && c < q.nrhs) ? x[q.xoff + src + (int64_t)c * q.n] : 0.0f;
  }
}

__global__ void k_batch_permute_out(const BPerm *__restrict__ pp, int np, int64_t total, float *__restrict__ y) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  int p = perm_problem(pp, np, e);
  for (; e < total; e += stride) {
    while (p + 1 < np && pp[p + 1].e0 <= e) ++p;
    const BPerm &q = pp[p];
    const int64_t l = e - q.e0, i = l / q.rp;
    const int c = (int)(l - i * q.rp);
    const int32_t src = q.pad_src[i];
    if (src >= 0 && c < q.nrhs) y[q.xoff + src + (int64_t)c * q.n] = q.pad[l];
  }
}

int take_batch_error(cudaStream_t st) {
  int v = 0, zero = 0;
  H2_CUDA_TRY(cudaMemcpyFromSymbolAsync(&v, g_h2_device_error, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
  H2_CUDA_TRY(cudaStreamSynchronize(st));
  if (v) {
    H2_CUDA_TRY(cudaMemcpyToSymbolAsync(g_h2_device_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    return fail(H2_ETIMEOUT, "a bounded device wait ran out; the last batched result is not valid");
  }
  return H2_OK;
}

constexpr int kRowPhases = 4;   // leaf forward, coupling, leaf backward, nearfield
constexpr int64_t kChunkTerms = 24;   // rows with more terms are cut in chunks of this many terms
constexpr int64_t kNoCap = (int64_t)1 << 62;
constexpr int kPermThreads = 256;
constexpr size_t kBatchSmemMax = 227 * 1024;

// launch shapes of the block-row kernel the tuner chooses from
struct Shape {
  int wpb, nslot, zbytes;
};
constexpr Shape kShapes[] = {
    {4, 6, 8192}, {8, 6, 4096}, {8, 4, 6144}, {4, 6, 4096}, {12, 4, 4096}, {16, 3, 4096}, {6, 4, 8192}, {2, 8, 6144},
};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

size_t shape_smem(const Shape &s) { return (size_t)s.wpb * s.nslot * (s.zbytes + 8); }

}  // namespace
}  // namespace h2

using namespace h2;

struct h2_batch_s {
  struct Prob {
    h2_ctx *h = nullptr;
    int nrhs = 0, rp = 0;
    int64_t xoff = 0;
    float *xpad = nullptr, *ypad = nullptr, *xhat = nullptr, *yhat = nullptr;
  };
  int device = 0;
  cudaStream_t stream = nullptr;       // launches (NULL: the legacy default stream)
  cudaStream_t cap = nullptr;          // capture stream
  std::vector<Prob> probs;
  int64_t packed = 0;                  // elements of the packed x and y
  int64_t dofs = 0;                    // sum of n nrhs
  void *work = nullptr;                // all work vectors
  int64_t work_bytes = 0;
  // block-row phases
  std::vector<BRows> rows[kRowPhases];
  BRows *d_rows[kRowPhases] = {};
  int64_t wtotal[kRowPhases] = {};
  int shape[kRowPhases] = {0, 0, 0, 0};
  int grid[kRowPhases] = {};
  // rows cut in chunks (coupling and nearfield): chunk bounds, partial sums, reductions
  int64_t *d_chunks[kRowPhases] = {};
  float *scratch[kRowPhases] = {};
  BRed *d_red[kRowPhases] = {};
  int nred[kRowPhases] = {};
  // transfers: per step, entries (device arrays) and parents
  std::vector<BTr *> d_up, d_down;
  std::vector<int> n_up, n_down;
  std::vector<int64_t> tot_up, tot_down;
  int tr_wfloats = 0;
  // permutations
  BPerm *d_perm_in = nullptr, *d_perm_out = nullptr;
  int64_t perm_total = 0;
  // graph
  cudaGraphExec_t exec = nullptr;
  const float *gx = nullptr;
  float *gy = nullptr;
  bool gprof = false;
  // profiling
  bool prof = false;
  cudaEvent_t ev[H2_NPHASE + 1] = {};
  double ms[H2_NPHASE] = {0};
  int64_t launches[H2_NPHASE] = {0};
  int64_t products = 0;
  int64_t graph_launches = 0;          // kernel launches per product
};

namespace h2 {
namespace {

// work per term / row: bytes moved plus a fixed overhead
void set_rows_shape(BRows &q, int zbytes) {
  const int64_t tb = 4LL * q.K * (q.Mp + q.rp);
  q.wterm = tb + 64;
  q.wrow = 4LL * q.M * q.rp * (1 + q.accumulate) + 128;
  if (tb <= zbytes) {
    q.tps = (int)(zbytes / tb);
    q.P = q.K;
    q.ppt = 1;
  } else {
    q.tps = 0;
    q.P = std::max(1, (int)(zbytes / (4LL * (q.Mp + q.rp))));
    q.ppt = (q.K + q.P - 1) / q.P;
  }
}

int upload_rows(h2_batch_s &b, int ph) {
  const Shape &s = kShapes[b.shape[ph]];
  // work prefix over the problems, from the host copies of the block lists
  int64_t w = 0;
  for (size_t p = 0; p < b.rows[ph].size(); ++p) {
    BRows &q = b.rows[ph][p];
    set_rows_shape(q, s.zbytes);
    q.w0 = w;
    if (q.pend) {   // chunk rows
      q.wfix = kChunkTerms * q.wterm + q.wrow;
      w += q.nrows * q.wfix;
      continue;
    }
    const Plan &pl = b.probs[p].h->plan;
    int64_t terms = q.nrows;
    if (q.nrows > 0 && q.ptr) {
      if (ph == 1) terms = pl.adm_ptr[q.row0 + q.nrows] - pl.adm_ptr[q.row0];
      else terms = pl.near_ptr[q.nrows] - pl.near_ptr[0];
    }
    w += terms * q.wterm + q.nrows * q.wrow;
  }
  b.wtotal[ph] = w;
  H2_CUDA_TRY(cudaMemcpy(b.d_rows[ph], b.rows[ph].data(), sizeof(BRows) * b.rows[ph].size(), cudaMemcpyHostToDevice));
  // persistent grid: as many CTAs as stay resident
  const size_t sm = shape_smem(s);
  H2_CUDA_TRY(cudaFuncSetAttribute((const void *)k_batch_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kBatchSmemMax));
  int per_sm = 0, sms = 0;
  H2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b.device));
  H2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_batch_rows, 32 * s.wpb, sm));
  if (per_sm < 1) return fail(H2_EINVAL, "batched block-row kernel cannot be resident");
  b.grid[ph] = per_sm * sms;
  return H2_OK;
}

void launch_rows_phase(h2_batch_s &b, int ph, cudaStream_t st) {
  if (b.wtotal[ph] == 0) return;
  const Shape &s = kShapes[b.shape[ph]];
  k_batch_rows<<<b.grid[ph], 32 * s.wpb, shape_smem(s), st>>>(b.d_rows[ph], (int)b.rows[ph].size(), b.wtotal[ph],
                                                              s.nslot, s.zbytes);
}

// enqueue one product on st; returns the number of kernel launches
int64_t enqueue(h2_batch_s &b, const float *x, float *y, cudaStream_t st, bool events) {
  int64_t nl = 0;
  const int np = (int)b.probs.size();
  // inside a capture, external event nodes stay visible to the host (timing)
  auto mark = [&](int ph) {
    if (events) cudaEventRecordWithFlags(b.ev[ph], st, cudaEventRecordExternal);
  };
  const int pgrid = (int)std::max<int64_t>(1, std::min<int64_t>((b.perm_total + kPermThreads - 1) / kPermThreads, 152 * 16));
  mark(H2_PH_PERMUTE_IN);
  k_batch_permute_in<<<pgrid, kPermThreads, 0, st>>>(b.d_perm_in, np, b.perm_total, x);
  ++nl;
  mark(H2_PH_LEAF_FORWARD);
  if (b.wtotal[0]) launch_rows_phase(b, 0, st), ++nl;
  const size_t trs = (size_t)kTrWarps * b.tr_wfloats * sizeof(float);
  mark(H2_PH_UPWARD);
  for (size_t s = 0; s < b.d_up.size(); ++s) {
    k_batch_upward<<<(unsigned)((b.tot_up[s] + kTrWarps - 1) / kTrWarps), 32 * kTrWarps, trs, st>>>(
        b.d_up[s], b.n_up[s], b.tot_up[s], b.tr_wfloats);
    ++nl;
  }
  mark(H2_PH_COUPLING);
  if (b.wtotal[1]) launch_rows_phase(b, 1, st), ++nl;
  if (b.nred[1]) k_batch_reduce<<<b.nred[1], 128, 0, st>>>(b.d_red[1]), ++nl;
  mark(H2_PH_DOWNWARD);
  for (size_t s = 0; s < b.d_down.size(); ++s) {
    k_batch_downward<<<(unsigned)((b.tot_down[s] + kTrWarps - 1) / kTrWarps), 32 * kTrWarps, trs, st>>>(
        b.d_down[s], b.n_down[s], b.tot_down[s], b.tr_wfloats);
    ++nl;
  }
  mark(H2_PH_LEAF_NEAR);
  if (b.wtotal[2]) launch_rows_phase(b, 2, st), ++nl;
  if (b.wtotal[3]) launch_rows_phase(b, 3, st), ++nl;
  if (b.nred[3]) k_batch_reduce<<<b.nred[3], 128, 0, st>>>(b.d_red[3]), ++nl;
  mark(H2_PH_PERMUTE_OUT);
  k_batch_permute_out<<<pgrid, kPermThreads, 0, st>>>(b.d_perm_out, np, b.perm_total, y);
  ++nl;
  mark(H2_NPHASE);
  return nl;
}

void drop_graph(h2_batch_s &b) {
  if (b.exec) cudaGraphExecDestroy(b.exec);
  b.exec = nullptr;
  b.gx = nullptr;
  b.gy = nullptr;
}

int capture(h2_batch_s &b, const float *x, float *y) {
  drop_graph(b);
  cudaGraph_t g = nullptr;
  H2_CUDA_TRY(cudaStreamBeginCapture(b.cap, cudaStreamCaptureModeThreadLocal));
  b.graph_launches = enqueue(b, x, y, b.cap, b.prof);
  cudaError_t e = cudaStreamEndCapture(b.cap, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e, "capture of the batched product");
  }
  e = cudaGraphInstantiate(&b.exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b.exec = nullptr;
    return cuda_fail(e, "instantiation of the batched product graph");
  }
  b.gx = x;
  b.gy = y;
  b.gprof = b.prof;
  return H2_OK;
}

void free_batch(h2_batch_s *b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  drop_graph(*b);
  for (auto &d : b->d_rows)
    if (d) cudaFree(d);
  for (int ph = 0; ph < kRowPhases; ++ph) {
    if (b->d_chunks[ph]) cudaFree(b->d_chunks[ph]);
    if (b->scratch[ph]) cudaFree(b->scratch[ph]);
    if (b->d_red[ph]) cudaFree(b->d_red[ph]);
  }
  for (auto p : b->d_up) cudaFree(p);
  for (auto p : b->d_down) cudaFree(p);
  if (b->d_perm_in) cudaFree(b->d_perm_in);
  if (b->d_perm_out) cudaFree(b->d_perm_out);
  if (b->work) cudaFree(b->work);
  for (auto e : b->ev)
    if (e) cudaEventDestroy(e);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

}  // namespace
}  // namespace h2

extern "C" {

int h2_batch_create(const h2_handle *hs, int nprob, const int *nrhs, void *stream, h2_batch *out) {
  if (!out) return fail(H2_EINVAL, "out is NULL");
  *out = nullptr;
  if (!hs || !nrhs || nprob < 1) return fail(H2_EINVAL, "a batch needs at least one handle and its nrhs");
  for (int p = 0; p < nprob; ++p) {
    const h2_ctx *h = hs[p];
    if (!h) return fail(H2_EINVAL, "NULL handle in the batch");
    if (h->d.prec != H2_F32) return fail(H2_EINVAL, "batched products need H2_F32 handles");
    if (h->d.gca) return fail(H2_EINVAL, "batched products need interpolation handles (not GCA-H^2)");
    if (h->d.coupling != 0) return fail(H2_EINVAL, "batched products need stored coupling matrices");
    if (h->d.k > kBatchMaxRows || h->d.lmax > kBatchMaxRows)
      return fail(H2_EINVAL, "batched products need rank k <= 64 (order <= 4) and leaves of at most 64 triangles");
    if (nrhs[p] < 1 || padded_rhs(nrhs[p], 4) > kBatchMaxRp) return fail(H2_EINVAL, "batched nrhs must be in [1, 16]");
    if (h->device != hs[0]->device) return fail(H2_EINVAL, "all handles of a batch must live on one device");
  }
  h2_batch_s *b = new (std::nothrow) h2_batch_s();
  if (!b) return fail(H2_ENOMEM, "batch");
  b->device = hs[0]->device;
  b->stream = (cudaStream_t)stream;
  auto bail = [&](int rc) {
    free_batch(b);
    return rc;
  };
  cudaError_t ce = cudaSetDevice(b->device);
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaSetDevice"));
  if ((ce = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(cuda_fail(ce, "capture stream"));
  for (auto &e : b->ev)
    if ((ce = cudaEventCreate(&e)) != cudaSuccess) return bail(cuda_fail(ce, "events"));

  // work vectors of every problem in one allocation (256-byte aligned parts)
  b->probs.resize(nprob);
  auto r256 = [](int64_t v) { return (v + 63) / 64 * 64; };   // floats
  int64_t off = 0, xoff = 0;
  std::vector<int64_t> offs(4 * (size_t)nprob);
  for (int p = 0; p < nprob; ++p) {
    auto &P = b->probs[p];
    P.h = hs[p];
    P.nrhs = nrhs[p];
    P.rp = padded_rhs(nrhs[p], 4);
    P.xoff = xoff;
    const Dev &d = P.h->d;
    xoff += d.n * P.nrhs;
    b->dofs += d.n * P.nrhs;
    const int64_t vec = r256(d.npad * P.rp), coef = r256(d.nclu * (int64_t)d.k * P.rp);
    offs[4 * p] = off;
    offs[4 * p + 1] = off + vec;
    offs[4 * p + 2] = off + 2 * vec;
    offs[4 * p + 3] = off + 2 * vec + coef;
    off += 2 * vec + 2 * coef;
  }
  b->packed = xoff;
  b->work_bytes = off * 4;
  if ((ce = dmalloc(&b->work, (size_t)b->work_bytes)) != cudaSuccess)
    return bail(cuda_fail(ce, "batched work vectors"));
  if ((ce = cudaMemset(b->work, 0, (size_t)b->work_bytes)) != cudaSuccess) return bail(cuda_fail(ce, "memset"));
  float *wf = static_cast<float *>(b->work);
  for (int p = 0; p < nprob; ++p) {
    auto &P = b->probs[p];
    P.xpad = wf + offs[4 * p];
    P.ypad = wf + offs[4 * p + 1];
    P.xhat = wf + offs[4 * p + 2];
    P.yhat = wf + offs[4 * p + 3];
  }

  // block-row phases
  for (int ph = 0; ph < kRowPhases; ++ph) b->rows[ph].resize(nprob);
  int max_steps = 0;
  for (int p = 0; p < nprob; ++p) {
    const auto &P = b->probs[p];
    const Dev &d = P.h->d;
    const int k = d.k, kp = d.kp, L = (int)d.lmax, Lp = (int)d.lp, rp = P.rp;
    const bool far = d.first_adm_level <= d.depth;
    const int64_t leaf0 = d.nleaf - 1, row0 = ((int64_t)1 << d.first_adm_level) - 1;
    BRows z{};
    z.rp = rp;
    BRows &fw = b->rows[0][p];
    fw = z;
    fw.A = (const float *)d.V;
    fw.a_stride = (int64_t)L * kp;
    fw.X = P.xpad;
    fw.x_stride = (int64_t)L * rp;
    fw.out = P.xhat + leaf0 * k * rp;
    fw.out_stride = (int64_t)k * rp;
    fw.nrows = far ? d.nleaf : 0;
    fw.M = k, fw.Mp = kp, fw.K = L;
    BRows &cp = b->rows[1][p];
    cp = z;
    cp.A = (const float *)d.S;
    cp.a_stride = (int64_t)k * kp;
    cp.X = P.xhat;
    cp.x_stride = (int64_t)k * rp;
    cp.ptr = d.adm_ptr;
    cp.col = d.adm_col;
    cp.out = P.yhat + row0 * k * rp;
    cp.out_stride = (int64_t)k * rp;
    cp.row0 = row0;
    cp.nrows = far ? d.nclu - row0 : 0;
    cp.M = k, cp.Mp = kp, cp.K = k;
    BRows &bw = b->rows[2][p];
    bw = z;
    bw.A = (const float *)d.Vt;
    bw.a_stride = (int64_t)k * Lp;
    bw.X = P.yhat + leaf0 * k * rp;
    bw.x_stride = (int64_t)k * rp;
    bw.out = P.ypad;
    bw.out_stride = (int64_t)L * rp;
    bw.nrows = far ? d.nleaf : 0;
    bw.M = L, bw.Mp = Lp, bw.K = k;
    BRows &nr = b->rows[3][p];
    nr = z;
    nr.A = (const float *)d.near;
    nr.a_stride = (int64_t)L * Lp;
    nr.X = P.xpad;
    nr.x_stride = (int64_t)L * rp;
    nr.ptr = d.near_ptr;
    nr.col = d.near_col;
    nr.out = P.ypad;
    nr.out_stride = (int64_t)L * rp;
    nr.nrows = d.nleaf;
    nr.M = L, nr.Mp = Lp, nr.K = L;
    nr.accumulate = far ? 1 : 0;
    if (far) max_steps = std::max(max_steps, d.depth - d.first_adm_level);
    b->tr_wfloats = std::max(b->tr_wfloats, (3 * k * rp + 6 * d.m * d.m + 3) / 4 * 4);
    for (int ph = 0; ph < kRowPhases; ++ph) b->rows[ph][p].cap = kNoCap;
  }

  // rows of the coupling and the nearfield with more than kChunkTerms terms
  // (cube surfaces produce clusters with hundreds of blocks): the row keeps
  // its first kChunkTerms terms, the rest become chunk rows of their own that
  // write partial sums, added to the row afterwards in chunk order
  for (int ph : {1, 3}) {
    std::vector<int64_t> cb, ce_;
    std::vector<BRed> red;
    std::vector<BRows> extra;
    for (int p = 0; p < nprob; ++p) {
      BRows &q = b->rows[ph][p];
      if (q.nrows == 0) continue;
      const Plan &pl = b->probs[p].h->plan;
      const int64_t *hp = ph == 1 ? pl.adm_ptr.data() + q.row0 : pl.near_ptr.data();
      BRows x = q;
      x.nrows = 0;
      const int64_t first_chunk = (int64_t)cb.size();
      for (int64_t r = 0; r < q.nrows; ++r) {
        const int64_t nt = hp[r + 1] - hp[r];
        if (nt <= kChunkTerms) continue;
        const int64_t nch = (nt - 1) / kChunkTerms;   // chunks beyond the first
        BRed rd{};
        rd.out = q.out + r * q.out_stride;
        rd.part = nullptr;   // set once the partial rows are allocated
        rd.nch = (int)nch;
        rd.len = q.M * q.rp;
        red.push_back(rd);
        for (int64_t j = 1; j <= nch; ++j) {
          cb.push_back(hp[r] + j * kChunkTerms);
          ce_.push_back(std::min(hp[r + 1], hp[r] + (j + 1) * kChunkTerms));
        }
        x.nrows += nch;
      }
      if (x.nrows == 0) continue;
      q.cap = kChunkTerms;
      x.ptr = reinterpret_cast<const int64_t *>(first_chunk);   // rebased below
      x.row0 = 0;
      x.pend = nullptr;
      x.accumulate = 0;
      x.out_stride = (int64_t)q.M * q.rp;
      x.cap = kNoCap;
      extra.push_back(x);
    }
    if (extra.empty()) continue;
    // partial rows: float offsets of every extra entry (rows of M rp values)
    int64_t floats = 0;
    std::vector<int64_t> fl_off(extra.size());
    for (size_t i = 0; i < extra.size(); ++i) {
      fl_off[i] = floats;
      floats += extra[i].nrows * extra[i].M * extra[i].rp;
    }
    const size_t nc = cb.size();
    if ((ce = dmalloc((void **)&b->d_chunks[ph], 2 * nc * sizeof(int64_t))) != cudaSuccess ||
        (ce = dmalloc((void **)&b->scratch[ph], (size_t)floats * sizeof(float))) != cudaSuccess ||
        (ce = dmalloc((void **)&b->d_red[ph], red.size() * sizeof(BRed))) != cudaSuccess)
      return bail(cuda_fail(ce, "chunk rows"));
    std::vector<int64_t> both(cb);
    both.insert(both.end(), ce_.begin(), ce_.end());
    if ((ce = cudaMemcpy(b->d_chunks[ph], both.data(), both.size() * sizeof(int64_t), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return bail(cuda_fail(ce, "chunk rows"));
    // rebase: chunk bounds and partial rows of each extra entry
    size_t ri = 0;
    for (size_t i = 0; i < extra.size(); ++i) {
      BRows &x = extra[i];
      const int64_t c0 = reinterpret_cast<int64_t>(x.ptr);
      x.ptr = b->d_chunks[ph] + c0;
      x.pend = b->d_chunks[ph] + nc + c0;
      x.out = b->scratch[ph] + fl_off[i];
      // the reductions of this entry's rows, in row order
      int64_t row_in_entry = 0;
      while (ri < red.size() && row_in_entry < x.nrows) {
        red[ri].part = x.out + row_in_entry * x.M * x.rp;
        row_in_entry += red[ri].nch;
        ++ri;
      }
      b->rows[ph].push_back(x);
    }
    if ((ce = cudaMemcpy(b->d_red[ph], red.data(), red.size() * sizeof(BRed), cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(cuda_fail(ce, "chunk reductions"));
    b->nred[ph] = (int)red.size();
  }
  for (int ph = 0; ph < kRowPhases; ++ph) {
    if ((ce = dmalloc((void **)&b->d_rows[ph], sizeof(BRows) * b->rows[ph].size())) != cudaSuccess)
      return bail(cuda_fail(ce, "batch descriptors"));
    int rc = upload_rows(*b, ph);
    if (rc) return bail(rc);
  }

  // transfer steps
  for (int up = 0; up < 2; ++up) {
    for (int s = 0; s < max_steps; ++s) {
      std::vector<BTr> ent;
      int64_t tot = 0;
      for (int p = 0; p < nprob; ++p) {
        const auto &P = b->probs[p];
        const Dev &d = P.h->d;
        if (d.first_adm_level > d.depth || s >= d.depth - d.first_adm_level) continue;
        const int l = up ? d.depth - 1 - s : d.first_adm_level + s;   // parent level
        BTr t{};
        t.Ef = (const float *)d.Ef;
        t.hat = up ? P.xhat : P.yhat;
        t.par0 = ((int64_t)1 << l) - 1;
        t.g0 = tot;
        t.m = d.m;
        t.k = d.k;
        t.rp = P.rp;
        ent.push_back(t);
        tot += (int64_t)1 << l;
      }
      BTr *dp = nullptr;
      if ((ce = dmalloc((void **)&dp, sizeof(BTr) * ent.size())) != cudaSuccess)
        return bail(cuda_fail(ce, "transfer descriptors"));
      (up ? b->d_up : b->d_down).push_back(dp);
      if ((ce = cudaMemcpy(dp, ent.data(), sizeof(BTr) * ent.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(cuda_fail(ce, "transfer descriptors"));
      (up ? b->n_up : b->n_down).push_back((int)ent.size());
      (up ? b->tot_up : b->tot_down).push_back(tot);
    }
  }
  {
    const int trs = kTrWarps * b->tr_wfloats * (int)sizeof(float);
    if ((size_t)trs > kBatchSmemMax) return bail(fail(H2_EINVAL, "transfer work space does not fit in shared memory"));
    if (trs > 48 * 1024) {   // one value for all batches (they may be created from several threads)
      cudaFuncSetAttribute((const void *)k_batch_upward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmemMax);
      cudaFuncSetAttribute((const void *)k_batch_downward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kBatchSmemMax);
    }
  }

  // permutations
  std::vector<BPerm> pin(nprob), pout(nprob);
  int64_t e0 = 0;
  for (int p = 0; p < nprob; ++p) {
    const auto &P = b->probs[p];
    const Dev &d = P.h->d;
    BPerm q{d.pad_src, P.xpad, d.n, d.npad, P.xoff, e0, P.nrhs, P.rp};
    pin[p] = q;
    q.pad = P.ypad;
    pout[p] = q;
    e0 += d.npad * P.rp;
  }
  b->perm_total = e0;
  if ((ce = dmalloc((void **)&b->d_perm_in, sizeof(BPerm) * nprob)) != cudaSuccess ||
      (ce = dmalloc((void **)&b->d_perm_out, sizeof(BPerm) * nprob)) != cudaSuccess)
    return bail(cuda_fail(ce, "permutation descriptors"));
  if ((ce = cudaMemcpy(b->d_perm_in, pin.data(), sizeof(BPerm) * nprob, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (ce = cudaMemcpy(b->d_perm_out, pout.data(), sizeof(BPerm) * nprob, cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(cuda_fail(ce, "permutation descriptors"));
  *out = b;
  return H2_OK;
}

int h2_batch_offsets(h2_batch b, int64_t *offsets) {
  if (!b || !offsets) return fail(H2_EINVAL, "NULL argument");
  for (size_t p = 0; p < b->probs.size(); ++p) offsets[p] = b->probs[p].xoff;
  offsets[b->probs.size()] = b->packed;
  return H2_OK;
}

int h2_batch_matvec(h2_batch b, const float *x, float *y) {
  if (!b || !x || !y) return fail(H2_EINVAL, "NULL argument");
  H2_CUDA_TRY(cudaSetDevice(b->device));
  if (!b->exec || b->gx != x || b->gy != y || b->gprof != b->prof) {
    int rc = capture(*b, x, y);
    if (rc) return rc;
  }
  H2_CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));
  if (b->prof) {
    H2_CUDA_TRY(cudaEventSynchronize(b->ev[H2_NPHASE]));
    for (int i = 0; i < H2_NPHASE; ++i) {
      float t = 0;
      H2_CUDA_TRY(cudaEventElapsedTime(&t, b->ev[i], b->ev[i + 1]));
      b->ms[i] += t;
    }
    b->products++;
  }
  return H2_OK;
}

int h2_batch_tune(h2_batch b, int reps, int *choice) {
  if (!b) return fail(H2_EINVAL, "NULL batch");
  if (reps < 1) reps = 3;
  H2_CUDA_TRY(cudaSetDevice(b->device));
  H2_CUDA_TRY(cudaStreamSynchronize(b->stream));
  drop_graph(*b);
  // the kernels of one phase only read their inputs and (over)write their
  // outputs, so a phase can be launched on its own repeatedly; the work
  // vectors hold whatever the last product left
  cudaEvent_t t0, t1;
  H2_CUDA_TRY(cudaEventCreate(&t0));
  H2_CUDA_TRY(cudaEventCreate(&t1));
  int rc = H2_OK;
  for (int ph = 0; ph < kRowPhases && !rc; ++ph) {
    if (b->wtotal[ph] == 0) continue;
    int best = b->shape[ph];
    float best_ms = 1e30f;
    for (int s = 0; s < kNumShapes && !rc; ++s) {
      if (shape_smem(kShapes[s]) > kBatchSmemMax) continue;
      b->shape[ph] = s;
      if ((rc = upload_rows(*b, ph))) break;
      launch_rows_phase(*b, ph, b->cap);   // warm-up
      cudaEventRecord(t0, b->cap);
      for (int i = 0; i < reps; ++i) launch_rows_phase(*b, ph, b->cap);
      cudaEventRecord(t1, b->cap);
      cudaError_t e = cudaEventSynchronize(t1);
      if (e != cudaSuccess) {
        rc = cuda_fail(e, "tuning run");
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, t0, t1);
      if (ms < best_ms) {
        best_ms = ms;
        best = s;
      }
    }
    b->shape[ph] = best;
    if (!rc) rc = upload_rows(*b, ph);
    // a phase that accumulates was run repeatedly: the next product rewrites it
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (rc) return rc;
  if ((rc = take_batch_error(b->cap))) return rc;
  if (choice)
    for (int ph = 0; ph < kRowPhases; ++ph) choice[ph] = b->shape[ph];
  return H2_OK;
}

int h2_batch_set_shapes(h2_batch b, const int *choice) {
  if (!b || !choice) return fail(H2_EINVAL, "NULL argument");
  for (int ph = 0; ph < kRowPhases; ++ph)
    if (choice[ph] < 0 || choice[ph] >= kNumShapes || shape_smem(kShapes[choice[ph]]) > kBatchSmemMax)
      return fail(H2_EINVAL, "unknown launch shape");
  H2_CUDA_TRY(cudaSetDevice(b->device));
  H2_CUDA_TRY(cudaStreamSynchronize(b->stream));
  drop_graph(*b);
  for (int ph = 0; ph < kRowPhases; ++ph) {
    b->shape[ph] = choice[ph];
    int rc = upload_rows(*b, ph);
    if (rc) return rc;
  }
  return H2_OK;
}

int h2_batch_profile(h2_batch b, int enable) {
  if (!b) return fail(H2_EINVAL, "NULL batch");
  b->prof = enable != 0;
  for (double &v : b->ms) v = 0.0;
  b->products = 0;
  return H2_OK;
}

int h2_batch_phase_times(h2_batch b, double *ms, int64_t *launches, int64_t *products) {
  if (!b) return fail(H2_EINVAL, "NULL batch");
  H2_CUDA_TRY(cudaSetDevice(b->device));
  H2_CUDA_TRY(cudaStreamSynchronize(b->stream));
  int rc = take_batch_error(b->cap);
  if (rc) return rc;
  if (ms)
    for (int i = 0; i < H2_NPHASE; ++i) ms[i] = b->ms[i];
  if (launches) {
    launches[H2_PH_PERMUTE_IN] = 1;
    launches[H2_PH_LEAF_FORWARD] = b->wtotal[0] ? 1 : 0;
    launches[H2_PH_UPWARD] = (int64_t)b->d_up.size();
    launches[H2_PH_COUPLING] = (b->wtotal[1] ? 1 : 0) + (b->nred[1] ? 1 : 0);
    launches[H2_PH_DOWNWARD] = (int64_t)b->d_down.size();
    launches[H2_PH_LEAF_NEAR] = (b->wtotal[2] ? 1 : 0) + (b->wtotal[3] ? 1 : 0) + (b->nred[3] ? 1 : 0);
    launches[H2_PH_PERMUTE_OUT] = 1;
  }
  if (products) *products = b->products;
  return H2_OK;
}

int h2_batch_info(h2_batch b, int64_t *info) {
  if (!b || !info) return fail(H2_EINVAL, "NULL argument");
  info[0] = (int64_t)b->probs.size();
  info[1] = b->packed;
  info[2] = b->dofs;
  info[3] = b->work_bytes;
  int64_t nl = 2 + (int64_t)b->d_up.size() + (int64_t)b->d_down.size();
  for (int ph = 0; ph < kRowPhases; ++ph) nl += (b->wtotal[ph] ? 1 : 0) + (b->nred[ph] ? 1 : 0);
  info[4] = nl;
  for (int ph = 0; ph < kRowPhases; ++ph) info[5 + ph] = b->shape[ph];
  return H2_OK;
}

int h2_batch_sync(h2_batch b) {
  if (!b) return fail(H2_EINVAL, "NULL batch");
  H2_CUDA_TRY(cudaSetDevice(b->device));
  H2_CUDA_TRY(cudaStreamSynchronize(b->stream));
  return take_batch_error(b->cap);
}

int h2_batch_destroy(h2_batch b) {
  free_batch(b);
  return H2_OK;
}

}  // extern "C"
