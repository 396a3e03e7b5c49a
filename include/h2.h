/*
 * h2.h -- C ABI of libh2: the H^2-matrix approximation of the Galerkin
 * single-layer matrix (Laplace kernel, piecewise-constant basis on flat
 * triangles) and its matrix-vector product on one NVIDIA GB300 GPU.
 *
 * The operation follows Boerm, "Distributed H^2-matrices for boundary element
 * methods", Section 2: the matrix G of Eq. (3) is approximated on admissible
 * blocks (Eq. (8)) by V_t S_ts W_s^T (Eq. (7)) with interpolation bases
 * (Eq. (6a-c)) and nested transfer matrices (Eqs. (9), (10)); the product runs
 * as forward transformation (Algorithm 1), interaction (Algorithm 3) and
 * backward transformation (Algorithm 2).  Test and trial bases coincide
 * (piecewise constants on one mesh), so W = V and F = E.
 *
 * Conventions for every entry point:
 *   - The return value is an h2_status; H2_OK is 0.  No call aborts, exits
 *     or traps the GPU.  h2_last_error() gives a message for the calling
 *     thread's most recent failure.
 *   - The library copies every host array it is given and keeps no caller
 *     pointer.  Handles own all device memory they allocate.
 *   - Vectors are column-major n x nrhs arrays (leading dimension n) in the
 *     caller's triangle order.
 *   - A handle is not thread-safe; use one handle per host thread or
 *     serialise calls.
 */
#ifndef H2_H
#define H2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct h2_ctx *h2_handle;
typedef struct h2_plan_ctx *h2_plan;

enum h2_status {
  H2_OK = 0,
  H2_EINVAL = 1,   /* invalid argument (sizes, pointers, options) */
  H2_ENOMEM = 2,   /* device or host allocation failed */
  H2_ECUDA = 3,    /* a CUDA runtime call failed; see h2_last_error() */
  H2_ENOCONV = 4,  /* iterative solve stopped at maxit; best iterate written */
  H2_ETIMEOUT = 5, /* a bounded device wait ran out */
  H2_PENDING = 6,  /* asynchronous result not ready yet */
  H2_EBUSY = 7     /* resource in use */
};

/* arithmetic of the stored representation and of the product:
 *   H2_F64        FP64-accurate: every stored value is kept as an unevaluated
 *                 sum of two FP32 numbers (about 48 significant bits) and the
 *                 product runs in double-float arithmetic on the FP32 pipe;
 *                 vectors are double.
 *   H2_F32        FP32 storage and arithmetic; vectors are float.
 *   H2_F64_NATIVE FP64 storage and arithmetic on the FP64 pipe (1/58 of the
 *                 FP32 rate on GB300); vectors are double.
 *   H2_BF16       nearfield stored in bfloat16 except the self blocks G_jj of
 *                 the leaves (they hold the largest entries of every row, the
 *                 singular g_ii among them; FP32, about a tenth of the
 *                 nearfield), leaf bases and transfer factors in FP32 unless
 *                 basis_prec asks for bfloat16 V, FP32 accumulation, coupling
 *                 regenerated in FP32; vectors float.
 *   H2_F16        nearfield, leaf bases and transfer factors in IEEE half
 *                 (basis_prec may ask for FP32 bases), FP32 accumulation,
 *                 coupling regenerated in FP32; every nearfield block and
 *                 every half-precision leaf basis carries a power-of-two scale
 *                 so that its entries (of size h^2 to h^4) stay in the half
 *                 range. */
enum h2_prec { H2_F64 = 0, H2_F32 = 1, H2_F64_NATIVE = 2, H2_BF16 = 3, H2_F16 = 4 };

/* coupling matrices S_ts (Eq. (6c)):
 *   H2_COUPLING_AUTO   stored, except regenerated for H2_BF16 / H2_F16 and for
 *                      H2_F32 when storing them would take more than half of
 *                      the free device memory;
 *   H2_COUPLING_STORED computed once at build time and streamed by the product;
 *   H2_COUPLING_REGEN  recomputed in FP32 inside the product from the
 *                      interpolation points (not for H2_F64 / H2_F64_NATIVE). */
enum h2_coupling { H2_COUPLING_AUTO = 0, H2_COUPLING_STORED = 1, H2_COUPLING_REGEN = 2 };

typedef struct h2_options {
  int prec;          /* enum h2_prec; default H2_F64 */
  int quad_order;    /* Gauss points per coordinate of the nearfield quadrature; default 3 */
  int device;        /* CUDA device ordinal; default 0 */
  void *stream;      /* cudaStream_t used by every call on the handle; NULL = the legacy default stream */
  int coupling;      /* enum h2_coupling; default H2_COUPLING_AUTO */
  int tensor;        /* 0 (default): an H2_F64 handle with stored coupling and order 4 also keeps its
                      * coupling matrices as 10 signed 5-bit digits in FP8 E4M3 (10 bytes per
                      * entry, a power of two per row) and runs the coupling phase of products with
                      * up to 16 right-hand sides on the tensor cores (integer digit products summed
                      * exactly, combined in double-float; agrees with the double-float path to
                      * about 1e-13); an H2_F32 handle of order 4 with stored coupling does the
                      * same with 6 digits (6 bytes per entry, FP32 accuracy); any H2_F64 handle
                      * with leaves of at most 21 triangles keeps its nearfield blocks as 10-digit
                      * planes and runs the nearfield phase on the tensor cores; 1: never */
  int basis_prec;    /* storage of the leaf bases V (Eq. (6a)) and the transfer factors (Eq. (9))
                      * of H2_BF16 / H2_F16 handles: 0 = the default, H2_F32 for H2_BF16 (V in
                      * bfloat16 costs about 1e-3 of relative accuracy, amplified by the Lebesgue
                      * constant of the interpolation, which leaves no room under 2e-3) and the
                      * handle's own type for H2_F16; H2_F32 or the handle's own 16-bit type may
                      * be asked for explicitly (H2_BF16 keeps its transfer factors in FP32
                      * either way).  Other precisions store V and E in their own type and
                      * accept only 0.  The nearfield is always stored in prec, and the coupling
                      * is stored in prec or regenerated in FP32 (field coupling). */
  int fused;         /* 1: products of an H2_F64 handle with stored coupling and at most 65,536
                      * triangles run as one cooperative launch (a grid-wide barrier between the
                      * steps of Algorithms 1-3; for small problems, whose time the separate
                      * launches of the phases dominate); 0 (default): the launch per phase */
  int reserved[4];   /* must be zero */
} h2_options;

/* Statistics of a built matrix (h2_info). */
typedef struct h2_stats {
  int64_t n;              /* triangles = degrees of freedom */
  int64_t depth;          /* leaf level of the cluster tree (root = level 0) */
  int64_t clusters;       /* 2^(depth+1) - 1 */
  int64_t leaf_max;       /* largest leaf, the padded leaf height */
  int64_t order;          /* interpolation points per axis m */
  int64_t rank;           /* k = m^3 */
  int64_t adm_blocks;     /* admissible leaves of the block tree */
  int64_t near_blocks;    /* inadmissible leaves */
  int64_t near_entries;   /* sum over inadmissible leaves of |t| |s| */
  int64_t first_adm_level;/* smallest level holding an admissible block */
  int64_t device_bytes;   /* device memory held by the handle (without work buffers) */
  int64_t prec;           /* enum h2_prec */
  int64_t coupling;       /* H2_COUPLING_STORED or H2_COUPLING_REGEN as built */
  int64_t tensor;         /* 1 if the tensor-core digits of the coupling were built */
  int64_t tensor_near;    /* 1 if the tensor-core digits of the nearfield were built */
  int64_t basis_prec;     /* enum h2_prec of the stored leaf bases V */
  int64_t gca;            /* 1 for a GCA-H^2 handle (h2_build_gca): then order is the Green
                           * quadrature order and rank the largest padded rank of a level */
  int64_t coupling_entries; /* stored coupling entries (interpolation: adm_blocks x rank^2; GCA-H^2:
                           * the sum over levels of blocks x padded rank^2) */
  int64_t tensor_leaf;    /* 1 if the tensor-core digits of the leaf bases were built (the leaf
                           * forward step of Algorithm 1 on the tensor cores, FP64-accurate
                           * handles with both tensor-core coupling and nearfield) */
} h2_stats;

/* Per right-hand side result of h2_solve. */
typedef struct h2_solve_info {
  int iters;          /* GMRES iterations (matrix-vector products in the Arnoldi process) */
  int status;         /* H2_OK or H2_ENOCONV */
  double relres;      /* true relative residual |b - G~ z| / |b| of the returned z */
} h2_solve_info;

/* Fill *opt with the defaults (FP64, quadrature order 3, device 0, default stream). */
int h2_options_default(h2_options *opt);

/* ---------------------------------------------------------------------------
 * Host-only planning: cluster tree (Definition 1), block tree (Eq. (8)),
 * interpolation points, leaf bases V (Eq. (6a)) and transfer factors (Eq. (9)).
 * Needs no GPU.
 *
 * vert: nv x 3 row-major coordinates; tri: nt x 3 row-major 0-based vertex
 * indices.  leaf_size >= 2, eta > 0, 1 <= order <= 6.
 * Errors: H2_EINVAL for bad sizes, NULL pointers or out-of-range vertex
 * indices; H2_ENOMEM.
 * ------------------------------------------------------------------------- */
int h2_plan_create(const double *vert, int64_t nv, const int32_t *tri, int64_t nt, int leaf_size, double eta,
                   int order, h2_plan *out);
int h2_plan_destroy(h2_plan p);

/* Query items of a plan.  Each call copies into caller memory of the size
 * given; pass NULL to skip an item.
 *   counts[8]  : n, depth, clusters, leaf_max, adm_blocks, near_blocks, near_entries, first_adm_level
 *   perm[n]    : perm[p] = triangle index of degree of freedom p in cluster order
 *   first[clusters], size[clusters] : index range of each cluster in cluster order
 *   lo[clusters*3], hi[clusters*3]  : cluster boxes
 *   adm_t/adm_s[adm_blocks]   : admissible blocks (row cluster, column cluster), sorted by (t, s)
 *   near_t/near_s[near_blocks]: inadmissible blocks (cluster indices), sorted by (t, s)
 *   V[n*k]     : leaf basis rows in cluster order (row p belongs to DoF p), Eq. (6a)
 *   E[clusters*3*m*m] : per cluster and axis the m x m factor E_d[j'][j] of
 *                the transfer matrix E_c = E_x (x) E_y (x) E_z, Eq. (9); root zero. */
int h2_plan_counts(h2_plan p, int64_t *counts);
int h2_plan_tree(h2_plan p, int64_t *perm, int64_t *first, int64_t *size, double *lo, double *hi);
int h2_plan_blocks(h2_plan p, int32_t *adm_t, int32_t *adm_s, int32_t *near_t, int32_t *near_s);
int h2_plan_bases(h2_plan p, double *V, double *E);

/* ---------------------------------------------------------------------------
 * Build the H^2 matrix on the device: plan as above, coupling matrices
 * S_ts = g(xi_t, xi_s) (Eq. (6c)) and Sauter-Schwab nearfield entries of
 * Eq. (3), stored in opt->prec.  opt may be NULL (defaults).
 * Range of H2_F64 (pairs of FP32 numbers, FP32's exponent range): the mesh
 * must satisfy amin^2 / (4 pi D) >= 2^-96 and amax <= 2^60 (amin, amax the
 * smallest and largest triangle area, D the diameter of the mesh's bounding
 * box), else H2_EINVAL; rescale the mesh or use H2_F64_NATIVE.
 * Errors: H2_EINVAL, H2_ENOMEM (device memory), H2_ECUDA.
 * ------------------------------------------------------------------------- */
int h2_build(const double *vert, int64_t nv, const int32_t *tri, int64_t nt, int leaf_size, double eta, int order,
             const h2_options *opt, h2_handle *out);
int h2_destroy(h2_handle h);
int h2_info(h2_handle h, h2_stats *out);

/* Phases of h2_build (h2_build_times): the cluster tree, block tree and
 * interpolation points on the host (Definition 1, Eq. (8)); then on the
 * device the leaf bases V and transfer factors E (Eqs. (6a), (9)), the
 * coupling matrices S (Eq. (6c)) with their tensor-core digits or the data
 * of their regeneration, and the nearfield (Sauter-Schwab quadrature of
 * Eq. (3)) with its conversion and digits. */
enum h2_build_phase { H2_BUILD_PLAN = 0, H2_BUILD_BASES, H2_BUILD_COUPLING, H2_BUILD_NEAR, H2_BUILD_TOTAL, H2_NBUILD };
/* Wall-clock milliseconds of every build phase of the handle (ms[H2_NBUILD];
 * the device phases include their synchronisation). */
int h2_build_times(h2_handle h, double *ms);

/* y = G~ x (overwrites y) for nrhs right-hand sides, Section 2 (the
 * paper's y <- y + G x with y cleared first).  x, y: DEVICE pointers to
 * column-major n x nrhs arrays of the handle's vector type (double for H2_F64
 * and H2_F64_NATIVE, float for H2_F32); they must not overlap.  Asynchronous on the handle's
 * stream.  1 <= nrhs <= 64.  H2_F64 handles accept any finite double: a
 * column whose largest entry lies outside [2^-40, 2^40] is scaled by a power
 * of two on the way in and back on the way out (exact), so it keeps FP64-level
 * relative accuracy; zero, infinite and NaN columns are passed as they are.
 * Errors: H2_EINVAL (NULL, nrhs out of range), H2_ENOMEM (work buffers),
 * H2_ECUDA (launch failure). */
int h2_matvec(h2_handle h, const void *x, void *y, int nrhs);

/* y <- y + G~ x: the product in the accumulating form in which Section 2
 * states it (Algorithms 1-3 add into the output).  Arguments, layout, types,
 * stream and errors as for h2_matvec; y must hold valid values of the
 * vector type on entry.  The sum is formed once, in the last step that
 * writes the caller's y (cluster order -> caller order), so it costs one
 * extra read of y and no extra launch. */
int h2_matvec_acc(h2_handle h, const void *x, void *y, int nrhs);

/* The same product as h2_matvec for callers that cannot allocate device
 * memory when they multiply (an allocator owned by another runtime, a
 * real-time loop that must not block in cudaMalloc, memory handed out in
 * full ahead of time).  It allocates nothing: its work buffers live in one
 * fixed array of 64 MiB of device memory inside the library, which every GPU
 * that loads the library keeps until the process exits.  The paper has no
 * counterpart; this is an interface of this library only.
 *   - x, y, nrhs and the result are as for h2_matvec, on the handle's stream.
 *   - Matrices that need more work space than 64 MiB for the given nrhs
 *     (2 (n_leaves leaf_max + clusters k) nrhs_padded value bytes) are
 *     rejected with H2_EINVAL and a message giving both sizes.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call outside any stream capture.
 *   - All calls share the one array: calls that can overlap on the GPU (on
 *     different streams, from different threads or handles) race and must be
 *     serialised by the caller.
 *   - h2_coefficients keeps describing the last h2_matvec product. */
int h2_matvec_noalloc(h2_handle h, const void *x, void *y, int nrhs);

/* The product captured once into a CUDA graph for fixed device buffers x, y
 * (as for h2_matvec) and replayed: h2_graph_launch runs y = G~ x
 * asynchronously on the handle's stream with the launch cost of one graph
 * (the product is 20 to 40 kernels).  The paper has no counterpart: a CUDA
 * graph takes the place a tracing compiler would take elsewhere.
 * The graph refers to the handle's work space: a later product with more
 * right-hand sides than any before reallocates it, after which
 * h2_graph_launch returns H2_EINVAL.  Destroy graphs before their handle;
 * a handle's graphs and products must not overlap on the GPU (one stream). */
typedef struct h2_graph_s *h2_graph;
int h2_graph_create(h2_handle h, const void *x, void *y, int nrhs, h2_graph *out);
int h2_graph_launch(h2_graph g);
int h2_graph_destroy(h2_graph g);

/* The same product with HOST double arrays whatever the handle's precision:
 * copies x to the device, multiplies, copies y back and synchronises the
 * stream. */
int h2_matvec_host(h2_handle h, const double *x, double *y, int nrhs);

/* A sequence of count products with HOST double arrays: block i of x (at
 * x + i n nrhs, column-major n x nrhs) gives block i of y.  The copy of block
 * i + 1 in and of block i - 1 out run beside the product of block i (two
 * device buffer pairs kept on the handle, two copy streams, events between
 * them), so a stream of inputs moves at the rate of the products when the
 * host arrays are pinned.  Blocks are independent; each result equals
 * h2_matvec_host's.  Synchronises before returning.  Errors as for
 * h2_matvec_host; count >= 1. */
int h2_matvec_host_stream(h2_handle h, const double *x, double *y, int nrhs, int count);

/* Coefficients of the last product (diagnostics): which = 0 gives x^ after
 * the forward transformation, 1 gives y^ after the interaction and the
 * downward transfer (as used by the leaf backward step).  out: HOST double
 * array [clusters][k][nrhs] of the last product's nrhs. */
int h2_coefficients(h2_handle h, int which, double *out);

/* The stored representation as built on the device, converted to double
 * (diagnostics: it lets the set-up be checked entry by entry).  Items:
 *   H2_EXPORT_NEAR      nearfield blocks G_b (Eq. (3), Sauter-Schwab quadrature)
 *                       first .. first+count-1 in the order of h2_plan_blocks'
 *                       inadmissible list; out[(i lmax + t) lmax + c] = entry
 *                       (test triangle t, trial triangle c) in leaf-local
 *                       cluster order, zero for padding.
 *   H2_EXPORT_COUPLING  coupling matrices S_b (Eq. (6c)) of admissible blocks
 *                       first .. in h2_plan_blocks' admissible order (stored
 *                       coupling only); out[(i k + nu) k + mu].
 *   H2_EXPORT_V         leaf basis rows (Eq. (6a)) of padded degrees of freedom
 *                       first .. (leaf j owns rows j lmax .. j lmax + lmax - 1);
 *                       out[i k + nu].
 *   H2_EXPORT_E         transfer factors (Eq. (9)) of clusters first ..;
 *                       out[((i 3 + axis) m + j') m + j].
 * Synchronises the handle's stream.  Errors: H2_EINVAL for an unknown item
 * or a range out of bounds. */
enum h2_export_item {
  H2_EXPORT_NEAR = 0,
  H2_EXPORT_COUPLING = 1,
  H2_EXPORT_V = 2,
  H2_EXPORT_E = 3,
  /* GCA-H^2 handles (K = h2_stats.rank, zero padded):
   *   H2_EXPORT_GCA_S  S_b = G|_{t_0 x s_0} of admissible blocks first .. (h2_plan_blocks'
   *                    admissible order): out[(i K + a) K + b], a the row pivot of t, b the
   *                    column pivot of s (h2_gca_pivots' order)
   *   H2_EXPORT_GCA_V  leaf bases of leaves first ..: out[(i lmax + t) K + a], t in
   *                    leaf-local cluster order
   *   H2_EXPORT_GCA_E  transfer matrices of clusters first ..: out[(i K + a) K + b], a a pivot
   *                    of the cluster, b one of its parent (zero where not built) */
  H2_EXPORT_GCA_S = 4,
  H2_EXPORT_GCA_V = 5,
  H2_EXPORT_GCA_E = 6
};
int h2_export(h2_handle h, int what, int64_t first, int64_t count, double *out);

/* Solve G~ z = b by restarted GMRES(restart) per column, z0 = 0, in FP64
 * arithmetic around the handle's product.  b, z: column-major n x nrhs
 * double arrays, both on the host or both on the device (detected).  A
 * column stops when its true relative residual |b - G~ z| / |b| <= rtol or
 * after maxit iterations (status H2_ENOCONV, best iterate written).  info
 * (host, nrhs entries) may be NULL.  Returns H2_OK when every column
 * converged, H2_ENOCONV otherwise. */
int h2_solve(h2_handle h, const double *b, double *z, int nrhs, double rtol, int restart, int maxit,
             h2_solve_info *info);

/* Mixed-precision iterative refinement around GMRES (GMRES-IR): the outer
 * residual r = b - G~ z is formed with handle hi (e.g. H2_F64), the
 * correction solves G~ d = r by GMRES(restart) with handle lo (e.g. H2_F32)
 * to the relative tolerance inner_rtol, z += d, until |r| <= rtol |b| per
 * column or maxit_outer refinement steps.  The paper names Krylov solvers for
 * Gz = b (Section 1) without fixing one; the refinement scheme is Carson and
 * Higham's GMRES-IR.  hi and lo must be built from the same mesh and tree
 * parameters on one device; b, z as for h2_solve.  info[c].iters counts the
 * inner GMRES iterations over all refinement steps, info[c].relres is the
 * residual with hi.  Returns H2_OK or H2_ENOCONV (best iterate written). */
int h2_solve_ir(h2_handle hi, h2_handle lo, const double *b, double *z, int nrhs, double rtol, double inner_rtol,
                int restart, int maxit_inner, int maxit_outer, h2_solve_info *info);

/* ---------------------------------------------------------------------------
 * Serving with continuous batching.  A server solves queued right-hand
 * sides on registered matrices.  Each registered matrix gets an engine with
 * its own worker thread and CUDA stream (engines of different matrices run
 * concurrently) and `slots` column slots; the columns of all its
 * requests share one batched product per Arnoldi step, and at every restart
 * cycle finished columns leave and queued requests are admitted into the
 * free slots.  With a low-precision partner handle lo the engine runs
 * GMRES-IR (inner cycles with lo to inner_rtol, residuals with hi), else
 * restarted GMRES with hi.  A column finishes when |b - G~_hi z| <= rtol |b|
 * or after maxit iterations.  Admission is by device memory: an engine's work
 * space (about (restart + 9) n slots doubles) is allocated when its first
 * request is admitted, within hbm_budget bytes (0 = 90 % of the free device
 * memory at creation), and released when the engine is idle and another
 * needs the room.  Registered handles belong to the server until it is
 * destroyed: they must not be used by other threads meanwhile, a handle can
 * be registered once (as hi or lo), and their streams are replaced by the
 * engine's stream and restored by h2_serve_destroy.
 * ------------------------------------------------------------------------- */
typedef struct h2_srv *h2_server;
int h2_serve_create(int device, size_t hbm_budget, h2_server *out);
/* Register matrix hi (and optionally its low-precision copy lo) with the
 * server.  1 <= slots <= 64, 1 <= restart <= 200, maxit >= 1; inner_rtol in
 * (0, 1) when lo is given.  H2_ENOMEM if one engine exceeds the budget. */
int h2_serve_register(h2_server s, h2_handle hi, h2_handle lo, int slots, int restart, int maxit, double inner_rtol);
/* Queue a solve of G~ z = b on the registered matrix hi: b is a HOST
 * column-major n x nrhs array (copied), 1 <= nrhs <= slots.  *ticket
 * identifies the request. */
int h2_serve_submit(h2_server s, h2_handle hi, const double *b, int nrhs, double rtol, uint64_t *ticket);
/* H2_PENDING while the request runs; once done, copies z (host n x nrhs)
 * and info (nrhs entries, either may be NULL), forgets the ticket and
 * returns H2_OK or H2_ENOCONV. */
int h2_serve_poll(h2_server s, uint64_t ticket, double *z, h2_solve_info *info);
/* Block until the request is done or timeout_s seconds pass (H2_PENDING). */
int h2_serve_wait(h2_server s, uint64_t ticket, double timeout_s);
/* stats[6]: queued requests, running columns, completed requests, engine
 * steps, device bytes in use by engines, budget. */
int h2_serve_stats(h2_server s, int64_t *stats);
/* Stop the engines' workers (running requests are abandoned), free the
 * engines and give the handles back their streams. */
int h2_serve_destroy(h2_server s);

/* Phases of the product, in launch order (h2_phase_times). */
enum h2_phase {
  H2_PH_PERMUTE_IN = 0,  /* caller order -> leaf-padded cluster order */
  H2_PH_LEAF_FORWARD,    /* x^ = V^T x on the leaves (Algorithm 1) */
  H2_PH_UPWARD,          /* x^_parent = sum E^T x^_child (Algorithm 1, Eq. (10)) */
  H2_PH_COUPLING,        /* y^_t = sum S_ts x^_s (Algorithm 3, Eq. (6c)) */
  H2_PH_DOWNWARD,        /* y^_child += E y^_parent (Algorithm 2) */
  H2_PH_LEAF_NEAR,       /* y = V y^ + nearfield (Algorithms 2 and 3) */
  H2_PH_PERMUTE_OUT,     /* cluster order -> caller order */
  H2_NPHASE
};

/* Enable (1) or disable (0) per-phase timing: while enabled every product
 * records CUDA events around each phase on the handle's stream.  Enabling
 * clears the accumulated times. */
int h2_profile(h2_handle h, int enable);

/* Accumulated device time in milliseconds (ms[H2_NPHASE]) and kernel
 * launches (launches[H2_NPHASE]) per phase since profiling was enabled,
 * and the number of products timed (*products).  Synchronises the stream.
 * Any output pointer may be NULL. */
int h2_phase_times(h2_handle h, double *ms, int64_t *launches, int64_t *products);

/* ---------------------------------------------------------------------------
 * Batched products over independent matrices of uneven sizes.
 *
 * The paper multiplies one H^2 matrix at a time (Section 2, Algorithms 1-3);
 * the batch runs the same steps for many matrices at once: each block-row
 * phase (leaf forward, coupling, leaf backward, nearfield) is ONE persistent
 * kernel launch over the rows of all matrices, the transfer passes run level
 * by level across the matrices, and the whole product is captured in a CUDA
 * graph on first use and replayed afterwards.
 *
 * Requirements: every handle is H2_F32 with stored coupling, order <= 4 and
 * leaves of at most 64 triangles, all on one device; nrhs[p] in [1, 16]; a
 * handle appears at most once.  The batch keeps pointers to the handles: they
 * must outlive it, and must not be destroyed while it exists.  It owns its
 * own work vectors, so products on the member handles do not disturb it.
 *
 * Vectors are PACKED: problem p's x (and y) is a column-major n_p x nrhs[p]
 * float block at element offset offsets[p] of one device array of
 * offsets[nprob] floats (h2_batch_offsets), in the caller's triangle order.
 * stream: the CUDA stream the products run on (NULL: the legacy default
 * stream).  Returns H2_EINVAL for a violated requirement, H2_ENOMEM if the
 * work vectors do not fit. */
typedef struct h2_batch_s *h2_batch;
int h2_batch_create(const h2_handle *hs, int nprob, const int *nrhs, void *stream, h2_batch *out);
/* offsets[nprob + 1]: element offset of every problem in the packed vectors,
 * offsets[nprob] = total length. */
int h2_batch_offsets(h2_batch b, int64_t *offsets);
/* y = G~_p x_p for every problem p; x, y device float arrays in the packed
 * layout, asynchronous on the batch's stream.  The first call with a given
 * (x, y) pair captures the CUDA graph (and so does the first call after
 * h2_batch_tune, h2_batch_set_shapes or h2_batch_profile); later calls
 * replay it.  A capture uses a private stream: do not call this function
 * while another capture is in progress on the calling thread. */
int h2_batch_matvec(h2_batch b, const float *x, float *y);
/* Autotuner of the launch shapes: times every candidate shape (slot size,
 * slots per warp, warps per CTA) of every block-row phase, reps launches
 * each, on the work vectors as the last product left them, and keeps the
 * fastest.  choice (4 ints, may be NULL) receives the chosen shape indices
 * of leaf forward, coupling, leaf backward and nearfield.  Synchronises. */
int h2_batch_tune(h2_batch b, int reps, int *choice);
/* Set the four shape indices directly (as returned by h2_batch_tune). */
int h2_batch_set_shapes(h2_batch b, const int *choice);
/* Per-phase timing of the following products (CUDA events inside the graph;
 * every product then synchronises); enabling clears the accumulated times. */
int h2_batch_profile(h2_batch b, int enable);
/* As h2_phase_times, for the batch (launches: per product). */
int h2_batch_phase_times(h2_batch b, double *ms, int64_t *launches, int64_t *products);
/* info[9]: problems, packed length, sum of n_p nrhs_p, work bytes, kernel
 * launches per product, the four shape indices. */
int h2_batch_info(h2_batch b, int64_t *info);
/* Wait for the batch's products; H2_ETIMEOUT if a bounded device wait ran out. */
int h2_batch_sync(h2_batch b);
int h2_batch_destroy(h2_batch b);

/* ---------------------------------------------------------------------------
 * The Helmholtz single-layer matrix (Section 1: g(x, y) = e^{i kappa |x-y|} /
 * (4 pi |x-y|), wave number kappa >= 0), approximated as in Section 2.  Its
 * real and imaginary parts, cos(kappa r) / (4 pi r) and sin(kappa r) /
 * (4 pi r), are two real kernels; a complex handle holds one real H^2 matrix
 * of each (the same trees, interpolation bases and quadrature; coupling
 * matrices and nearfield per part), G = G_c + i G_s, and multiplies complex
 * vectors as y_re = G_c x_re - G_s x_im, y_im = G_c x_im + G_s x_re, both
 * real products taking the real and imaginary columns together (2 nrhs
 * columns).  The interpolation needs kappa diam of the clusters to stay
 * moderate (low-frequency regime): accuracy falls as kappa grows.
 *
 * Complex vectors are column-major n x nrhs arrays of interleaved (real,
 * imaginary) double pairs (C99 double complex, std::complex<double>).
 * Precisions: H2_F64 (with the tensor-core coupling and nearfield where
 * eligible: order 4, at most 8 complex right-hand sides), H2_F32,
 * H2_F64_NATIVE; the coupling is always stored.
 * ------------------------------------------------------------------------- */
typedef struct h2_zctx *h2_zhandle;
/* Build; arguments as for h2_build plus kappa >= 0 (finite).  opt->coupling
 * must be AUTO or STORED and opt->prec one of the three above (H2_EINVAL
 * otherwise). */
int h2_zbuild(const double *vert, int64_t nv, const int32_t *tri, int64_t nt, int leaf_size, double eta, int order,
              double kappa, const h2_options *opt, h2_zhandle *out);
int h2_zdestroy(h2_zhandle h);
/* The real H^2 matrix of part `which` (0: real part G_c, 1: imaginary part
 * G_s), owned by h (do not destroy it): for h2_info, h2_export and products
 * of one part alone. */
int h2_zpart(h2_zhandle h, int which, h2_handle *out);
/* Statistics of the real part's matrix (the imaginary part has the same
 * structure); device_bytes counts both parts. */
int h2_zinfo(h2_zhandle h, h2_stats *out);
/* y = G~ x for nrhs complex right-hand sides, 1 <= nrhs <= 32; x, y DEVICE
 * pointers (interleaved complex doubles), asynchronous on the handle's
 * stream.  Errors as for h2_matvec. */
int h2_zmatvec(h2_zhandle h, const double *x, double *y, int nrhs);
/* The same with HOST arrays (copies included, synchronises). */
int h2_zmatvec_host(h2_zhandle h, const double *x, double *y, int nrhs);
/* Solve G~ z = b by restarted GMRES(restart), z0 = 0, per complex column, on
 * the equivalent real system [G_c -G_s; G_s G_c] [z_re; z_im] = [b_re;
 * b_im] (its residual norm is the complex residual's), in FP64 around the
 * handle's products.  b, z both host or both device (interleaved complex);
 * rtol, restart, maxit and info as for h2_solve (relres is the complex
 * relative residual |b - G~ z| / |b|). */
int h2_zsolve(h2_zhandle h, const double *b, double *z, int nrhs, double rtol, int restart, int maxit,
              h2_solve_info *info);

/* ---------------------------------------------------------------------------
 * GCA-H^2 (Section 3, the GCA-H^2 example): an H^2 matrix of the Laplace
 * single-layer operator whose cluster bases interpolate at pivot elements.
 * Every cluster tau has pivot triangles tau_0 of tau (a parent's pivots are
 * chosen among its sons' pivots, so the bases are nested, Eq. (10)), and
 * every admissible block the coupling matrix S_{tau sigma} =
 * G|_{tau_0 x sigma_0}, the Galerkin matrix on the pivot pairs (Eq. (3),
 * the nearfield's regular quadrature).  The section states only this; the
 * pivots come from the cited Green cross approximation:
 *   - a quadrature rule on the boundary of the cluster's box enlarged by
 *     gamma times its half diagonal (green_order Gauss nodes per direction on
 *     each face) gives a surrogate of the cluster's rows: for every candidate
 *     triangle the weighted integrals of g(x, z) and of its normal derivative
 *     in z at every quadrature point z (Green's representation formula),
 *     each by the collapsed Gauss rule with tri_order nodes per direction;
 *   - cross approximation with complete pivoting of the surrogate to the
 *     relative accuracy eps (at most max_rank pivots) picks the pivot rows;
 *     ties (within a relative 2^-30) go to the first entry in row-major order;
 *   - the interpolation operator V^ = M[:, J] M[I, J]^{-1} (pivot rows exactly
 *     unit vectors) is the leaf basis V of a leaf, and splits into the
 *     transfer matrices E of the sons for a parent, whose candidates are its
 *     first son's pivots followed by its second son's.
 * The trees, blocks (eta) and nearfield are those of h2_build.  The product,
 * solvers and graphs take GCA-H^2 handles like any other (h2_matvec,
 * h2_matvec_acc, h2_matvec_host, h2_matvec_noalloc, h2_solve, h2_solve_ir,
 * h2_graph_*, h2_serve_*); h2_batch_* and h2_coefficients do not.
 * ------------------------------------------------------------------------- */
typedef struct h2_gca_options {
  double eps;        /* relative accuracy of the cross approximation; default 1e-4, in [0, 1) */
  double gamma;      /* enlargement of the auxiliary box in half diagonals; default 1, > 0 */
  int green_order;   /* Gauss nodes per direction on each face; default 4, in [1, 8] */
  int tri_order;     /* collapsed Gauss nodes per direction on a triangle; default 3, in [1, 16] */
  int max_rank;      /* pivots per cluster at most; default 128, in [4, 128] */
  int reserved[5];   /* must be zero */
} h2_gca_options;
int h2_gca_options_default(h2_gca_options *g);
/* Build a GCA-H^2 matrix.  Arguments as for h2_build (no order); gopt NULL =
 * defaults; opt->prec one of H2_F64, H2_F64_NATIVE, H2_F32 and opt->coupling
 * AUTO or STORED (H2_EINVAL otherwise).  Pivots, bases, transfer and
 * coupling matrices are computed on the device (FP64), for the levels from
 * the leaves up to the first level with an admissible block. */
int h2_build_gca(const double *vert, int64_t nv, const int32_t *tri, int64_t nt, int leaf_size, double eta,
                 const h2_gca_options *gopt, const h2_options *opt, h2_handle *out);
/* Ranks and pivots of a GCA-H^2 handle: rank[clusters] (0 above the first
 * admissible level), pivots[c * cap + a] = triangle index (caller's order) of
 * pivot a of cluster c in pivot order, -1 beyond the rank; cap >= h2_stats.rank.
 * Either output may be NULL. */
int h2_gca_pivots(h2_handle h, int32_t *rank, int32_t *pivots, int64_t cap);

/* ---------------------------------------------------------------------------
 * Failure injection and self-tests of the error paths (no counterpart in the
 * paper; they make failures happen on the host or inside a bounded wait,
 * never as a GPU fault).
 * ------------------------------------------------------------------------- */
/* Make the device allocation `after` allocations from now (0 = the next one)
 * of any thread fail as if the device were out of memory; -1 cancels a
 * pending injection.  One failure per call.  Every entry point that
 * allocates must then return H2_ENOMEM and release what it had allocated. */
int h2_inject_alloc_failure(int64_t after);

/* Run the library's bounded-wait machinery in miniature on the handle's
 * stream: a producer thread fills a ring of four shared-memory stages with
 * bulk copies completing on mbarriers, a consumer thread waits for each stage
 * with at most poll_limit polls (0 = the limit the product kernels use).
 * withhold = 1: the producer never fills the last stage, so that wait runs
 * out, raises the device error word and the call returns H2_ETIMEOUT (the
 * error is read and cleared, the handle stays usable); withhold = 0: H2_OK.
 * *stages_seen (may be NULL) receives the stages the consumer saw complete. */
int h2_wait_selftest(h2_handle h, int withhold, uint32_t poll_limit, int *stages_seen);

/* Message describing the calling thread's most recent failure ("" if none). */
const char *h2_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* H2_H */
