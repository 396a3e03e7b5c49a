/*
 * h2oracle.c -- plain, slow FP64 CPU oracle for the interpolation-based
 * H^2-matrix approximation of the Galerkin single-layer matrix
 * (Laplace kernel, piecewise-constant basis on flat triangles).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant with the CUDA library; both read the same
 * seeded input arrays and nothing else.
 *
 * Sources (Boerm, "Distributed H^2-matrices for boundary element methods"):
 *   Galerkin matrix g_ij and right-hand side b_i ........ Section 1, Eq. (3)
 *   Laplace kernel g(x,y) = 1/(4 pi |x-y|) .............. Section 1
 *   Helmholtz kernel e^{i kappa |x-y|}/(4 pi |x-y|) ..... Section 1: its
 *     real part cos(kappa r)/(4 pi r) and imaginary part sin(kappa r)/(4 pi r)
 *     are two real kernels (kinds 2 and 3) approximated the same way
 *   tensor interpolation of g on box pairs .............. Section 2, Eq. (4)
 *   cluster index sets, minimal boxes ................... Section 2, Eq. (5)
 *   leaf bases V (= W here), coupling S ................. Section 2, Eq. (6a-c)
 *   cluster tree ........................................ Section 2, Definition 1
 *   block tree, admissibility ........................... Section 2, Eq. (8)
 *   transfer matrices E (= F here), nested bases ........ Section 2, Eqs. (9), (10)
 *   forward / backward / interaction phases ............. Section 2, Algorithms 1-3
 *   GCA-H^2: pivot elements, S = G on pivot pairs ....... Section 3 (GCA-H^2 example)
 * Nearfield entries use the Sauter-Schwab quadrature that the paper's
 * experiments name (Section 3, experiments paragraph), restated from the
 * published method (Sauter & Schwab, Boundary Element Methods, 2011, Sec. 5.2).
 * GMRES is Saad's restarted GMRES with modified Gram-Schmidt and Givens
 * rotations (Saad, Iterative Methods for Sparse Linear Systems, Alg. 6.9).
 *
 * Readings where the paper is silent (the library follows the same ones):
 *   R1 characteristic point = centroid ((a+b)+c)/3; box = min/max of vertices.
 *   R2 binary tree, every cluster above depth D is split, D the smallest depth
 *      with ceil(n/2^D) <= leaf_size; split axis = longest extent of the
 *      centroid bounding box (lowest axis on ties); sort by (centroid, index);
 *      first floor(|t|/2) go to child 0; children of c are 2c+1, 2c+2.
 *   R3 diam = box diagonal, dist = norm of per-axis gaps, admissible iff
 *      max(diam_t, diam_s) <= (2 eta) dist.
 *   R4 Chebyshev nodes c + h cos((2j+1) pi / (2m)); nu = jx + m jy + m^2 jz;
 *      an axis with extent <= 1e-12 * (largest extent) is widened to half
 *      width 1e-6 * (largest extent) for interpolation only.
 *   R5 reference triangle {0 <= t <= s <= 1}, chi(s,t) = A + s(B-A) + t(C-B);
 *      collapsed Gauss rule (s,t) = (u, u v) with weight u.
 *   R6 V exact: q_V = ceil((3(m-1)+2)/2) points per direction.
 *   R7 nearfield: shared global vertices decide identical / edge / vertex /
 *      regular; regular pairs use the collapsed rule with q points per
 *      direction on each triangle in mesh vertex order; singular pairs use
 *      q points per coordinate on [0,1]^4; canonical local vertex order:
 *      identical -> rotate smallest id first; edge -> (smaller shared, larger
 *      shared, other); vertex -> (shared, next, next-next) cyclically; each
 *      unordered pair is computed once with the smaller index as test
 *      triangle and mirrored.
 *   R8 matvec overwrites: y = G~ x.
 *
 * GCA-H^2 (Section 3 names it and states only that pivot elements are
 * chosen per cluster and that S_{tau sigma} is computed from G on the
 * pivots); the construction follows the cited Green cross approximation
 * with these readings:
 *   G1 Green quadrature on the boundary of the box [lo - gamma rho, hi +
 *      gamma rho], rho = half diagonal of the cluster's box, gamma = 1 by
 *      default: per face a tensor Gauss rule with qg nodes per direction
 *      (qg = 4, the paper's "quadrature order m = 4" of its GCA runs);
 *      faces in the order (axis 0 low, high, axis 1 ..., axis 2 ...).
 *   G2 the surrogate of a cluster: rows = candidate triangles, columns = the
 *      single-layer and the double-layer family of Green's representation
 *      formula at every quadrature point, weighted, each integrated over the
 *      triangle by the collapsed rule with qt = 3.
 *   G3 cross approximation with complete pivoting, relative accuracy eps
 *      (1e-4, the paper's value) against the largest entry of the surrogate,
 *      at most 128 pivots per cluster.
 *   G4 ties: the first entry (row-major) within a relative 2^-30 of the
 *      largest modulus.
 *   G5 V^ = M[:, J] M[I, J]^{-1} with its pivot rows set to unit vectors:
 *      leaves keep it as V, parents cut it into their sons' E.
 *   G6 nested pivots: the candidates of a parent are the pivots of its first
 *      son, then those of its second son; leaves take their triangles in
 *      cluster order.  S_{tau sigma} = G|_{tau_0 x sigma_0} by R7.
 *
 * Compile with -ffp-contract=off so that the tree-building comparisons are
 * evaluated without fused multiply-adds.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------ */
/* Gauss-Legendre rule on [0,1]: Newton iteration on P_n, whose value and
 * derivative come from the three-term recurrence (n+1)P_{n+1} =
 * (2n+1) x P_n - n P_{n-1}.                                            */
/* ------------------------------------------------------------------ */
void or_gauss01(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(OR_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    /* node on [-1,1] is z; weight 2/((1-z^2) P_n'(z)^2); map to [0,1] */
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* ------------------------------------------------------------------ */
/* Kernels.  kind 0: Laplace 1/(4 pi |x-y|) (Section 1).  kind 1: a
 * smooth symmetric test polynomial of per-axis degree <= m-1 in x and in
 * y, which tensor interpolation of order m reproduces exactly.  kinds 2
 * and 3: the real and imaginary parts of the Helmholtz kernel of Section 1,
 * cos(kappa r) / (4 pi r) and sin(kappa r) / (4 pi r), r = |x - y| (the
 * second is smooth: kappa / (4 pi) at r = 0).                           */
/* ------------------------------------------------------------------ */
static double kernel_eval(int kind, int m, double kappa, const double *x, const double *y) {
  if (kind == 0 || kind == 2 || kind == 3) {
    double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    if (kind == 0) return 1.0 / (4.0 * OR_PI * r);
    if (kind == 2) return cos(kappa * r) * (1.0 / (4.0 * OR_PI * r));
    return r > 0.0 ? sin(kappa * r) * (1.0 / (4.0 * OR_PI * r)) : kappa / (4.0 * OR_PI);
  }
  double prod = 1.0;
  for (int d = 0; d < 3; ++d) {
    double s = 0.0, xa = 1.0;
    for (int a = 0; a < m; ++a) {
      double yb = 1.0;
      for (int b = 0; b < m; ++b) {
        s += xa * yb / (1.0 + a + b);
        yb *= y[d];
      }
      xa *= x[d];
    }
    prod *= s;
  }
  return prod;
}

/* ------------------------------------------------------------------ */
/* The oracle's H^2 matrix.                                            */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t nt, nv;
  double *vert;   /* nv x 3 */
  int32_t *tri;   /* nt x 3 */
  double *cen;    /* nt x 3 centroids (R1) */
  double *area;   /* nt */
  int leaf, m, k, q, kind, depth;
  double kappa;   /* wave number of kinds 2 and 3 */
  double eta;
  int64_t nclu;
  int64_t *idx;   /* cluster order -> triangle index */
  int64_t *first, *size;
  double *lo, *hi;        /* true boxes */
  double *pts;            /* Chebyshev points [nclu][3][m] */
  /* block tree leaves in recursion order */
  int64_t nblk, cap;
  int32_t *bt, *bs;
  uint8_t *badm;
  /* blocks grouped by row cluster (recursion order inside a row) */
  int64_t *rowptr, *rowblk;
  double *V;              /* nt x k, row p = DoF in cluster order */
  double *E;              /* nclu x k x k, E[c][nu'][nu] */
  int store_near;
  int64_t *noff;          /* per block offset into nval (inadmissible only) */
  double *nval;
} orh2;

static int level_of(int64_t c) {
  int l = 0;
  while (c > 0) { c = (c - 1) / 2; ++l; }
  return l;
}

/* triangle area, |(b-a) x (c-a)| / 2 */
static double tri_area(const double *a, const double *b, const double *c) {
  double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  double n0 = u[1] * v[2] - u[2] * v[1];
  double n1 = u[2] * v[0] - u[0] * v[2];
  double n2 = u[0] * v[1] - u[1] * v[0];
  return 0.5 * sqrt(n0 * n0 + n1 * n1 + n2 * n2);
}

/* sort context for the median split (R2) */
static const double *g_sort_cen;
static int g_sort_axis;
static int cmp_axis(const void *pa, const void *pb) {
  int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
  double ca = g_sort_cen[3 * a + g_sort_axis], cb = g_sort_cen[3 * b + g_sort_axis];
  if (ca < cb) return -1;
  if (ca > cb) return 1;
  return (a < b) ? -1 : (a > b) ? 1 : 0;
}

/* Definition 1 via bisection of characteristic points (Section 2, R2) */
static void build_cluster(orh2 *h, int64_t c, int level, int64_t first, int64_t size) {
  h->first[c] = first;
  h->size[c] = size;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t p = first; p < first + size; ++p) {
    int64_t t = h->idx[p];
    for (int v = 0; v < 3; ++v) {
      const double *x = h->vert + 3 * (int64_t)h->tri[3 * t + v];
      for (int d = 0; d < 3; ++d) {
        if (x[d] < lo[d]) lo[d] = x[d];
        if (x[d] > hi[d]) hi[d] = x[d];
      }
    }
  }
  for (int d = 0; d < 3; ++d) { h->lo[3 * c + d] = lo[d]; h->hi[3 * c + d] = hi[d]; }
  if (level >= h->depth) return;
  double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t p = first; p < first + size; ++p) {
    const double *x = h->cen + 3 * h->idx[p];
    for (int d = 0; d < 3; ++d) {
      if (x[d] < clo[d]) clo[d] = x[d];
      if (x[d] > chi[d]) chi[d] = x[d];
    }
  }
  int axis = 0;
  for (int d = 1; d < 3; ++d)
    if (chi[d] - clo[d] > chi[axis] - clo[axis]) axis = d;
  g_sort_cen = h->cen;
  g_sort_axis = axis;
  qsort(h->idx + first, (size_t)size, sizeof(int64_t), cmp_axis);
  int64_t half = size / 2;
  build_cluster(h, 2 * c + 1, level + 1, first, half);
  build_cluster(h, 2 * c + 2, level + 1, first + half, size - half);
}

/* R4: interpolation points of a cluster box */
static void cheb_points(orh2 *h, int64_t c) {
  const double *lo = h->lo + 3 * c, *hi = h->hi + 3 * c;
  double maxext = 0.0;
  for (int d = 0; d < 3; ++d)
    if (hi[d] - lo[d] > maxext) maxext = hi[d] - lo[d];
  for (int d = 0; d < 3; ++d) {
    double mid = 0.5 * (lo[d] + hi[d]);
    double half = 0.5 * (hi[d] - lo[d]);
    if (hi[d] - lo[d] <= 1e-12 * maxext) half = 1e-6 * maxext;
    for (int j = 0; j < h->m; ++j)
      h->pts[(c * 3 + d) * h->m + j] = mid + half * cos((2.0 * j + 1.0) * OR_PI / (2.0 * h->m));
  }
}

/* 1-D Lagrange polynomial j of cluster c on axis d, product form */
static double lagrange1(const orh2 *h, int64_t c, int d, int j, double t) {
  const double *p = h->pts + (c * 3 + d) * h->m;
  double v = 1.0;
  for (int i = 0; i < h->m; ++i)
    if (i != j) v *= (t - p[i]) / (p[j] - p[i]);
  return v;
}

/* tensor Lagrange polynomial ell_{c,nu}(x), Eq. (4) */
static double lagrange3(const orh2 *h, int64_t c, int nu, const double *x) {
  int m = h->m;
  int jx = nu % m, jy = (nu / m) % m, jz = nu / (m * m);
  return lagrange1(h, c, 0, jx, x[0]) * lagrange1(h, c, 1, jy, x[1]) * lagrange1(h, c, 2, jz, x[2]);
}

static void cheb_point3(const orh2 *h, int64_t c, int nu, double *x) {
  int m = h->m;
  x[0] = h->pts[(c * 3 + 0) * m + nu % m];
  x[1] = h->pts[(c * 3 + 1) * m + (nu / m) % m];
  x[2] = h->pts[(c * 3 + 2) * m + nu / (m * m)];
}

/* R3: standard admissibility, Eq. (8) */
static int admissible(const orh2 *h, int64_t t, int64_t s) {
  const double *lt = h->lo + 3 * t, *ht = h->hi + 3 * t;
  const double *ls = h->lo + 3 * s, *hs = h->hi + 3 * s;
  double e0 = ht[0] - lt[0], e1 = ht[1] - lt[1], e2 = ht[2] - lt[2];
  double dt = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
  e0 = hs[0] - ls[0]; e1 = hs[1] - ls[1]; e2 = hs[2] - ls[2];
  double ds = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
  double g[3];
  for (int d = 0; d < 3; ++d) {
    double a = lt[d] - hs[d], b = ls[d] - ht[d];
    double v = a > b ? a : b;
    g[d] = v > 0.0 ? v : 0.0;
  }
  double dist = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  double dmax = dt > ds ? dt : ds;
  return dmax <= (2.0 * h->eta) * dist;
}

static void push_block(orh2 *h, int64_t t, int64_t s, int adm) {
  if (h->nblk == h->cap) {
    h->cap = h->cap ? 2 * h->cap : 1024;
    h->bt = (int32_t *)realloc(h->bt, h->cap * sizeof(int32_t));
    h->bs = (int32_t *)realloc(h->bs, h->cap * sizeof(int32_t));
    h->badm = (uint8_t *)realloc(h->badm, h->cap);
  }
  h->bt[h->nblk] = (int32_t)t;
  h->bs[h->nblk] = (int32_t)s;
  h->badm[h->nblk] = (uint8_t)adm;
  h->nblk++;
}

/* block tree recursion (Section 2, after Eq. (8)) */
static void build_blocks(orh2 *h, int64_t t, int64_t s) {
  int lt = level_of(t), ls = level_of(s);
  int ct = lt < h->depth, cs = ls < h->depth;
  if (admissible(h, t, s)) {
    push_block(h, t, s, 1);
  } else if (ct && cs) {
    for (int a = 1; a <= 2; ++a)
      for (int b = 1; b <= 2; ++b) build_blocks(h, 2 * t + a, 2 * s + b);
  } else if (cs) {
    for (int b = 1; b <= 2; ++b) build_blocks(h, t, 2 * s + b);
  } else if (ct) {
    for (int a = 1; a <= 2; ++a) build_blocks(h, 2 * t + a, s);
  } else {
    push_block(h, t, s, 0);
  }
}

/* R5: reference map chi(s,t) = A + s (B-A) + t (C-B) */
static void ref_map(const double *A, const double *B, const double *C, double s, double t, double *x) {
  for (int d = 0; d < 3; ++d) x[d] = A[d] + s * (B[d] - A[d]) + t * (C[d] - B[d]);
}

/* V_tau for a leaf, Eq. (6a), exact collapsed Gauss quadrature (R6) */
static void leaf_basis(orh2 *h, int64_t c) {
  int qv = (3 * (h->m - 1) + 2 + 1) / 2;
  if (qv < 1) qv = 1;
  double gx[32], gw[32];
  or_gauss01(qv, gx, gw);
  for (int64_t p = h->first[c]; p < h->first[c] + h->size[c]; ++p) {
    int64_t t = h->idx[p];
    const double *A = h->vert + 3 * (int64_t)h->tri[3 * t + 0];
    const double *B = h->vert + 3 * (int64_t)h->tri[3 * t + 1];
    const double *C = h->vert + 3 * (int64_t)h->tri[3 * t + 2];
    double jac = 2.0 * h->area[t];
    for (int nu = 0; nu < h->k; ++nu) {
      double acc = 0.0;
      for (int a = 0; a < qv; ++a)
        for (int b = 0; b < qv; ++b) {
          double x[3];
          ref_map(A, B, C, gx[a], gx[a] * gx[b], x);
          acc += gw[a] * gw[b] * gx[a] * lagrange3(h, c, nu, x);
        }
      h->V[p * h->k + nu] = jac * acc;
    }
  }
}

/* transfer matrix of a non-root cluster, Eq. (9): E[nu'][nu] = ell_{parent,nu}(xi_{c,nu'}) */
static void transfer_matrix(orh2 *h, int64_t c) {
  int64_t par = (c - 1) / 2;
  for (int nup = 0; nup < h->k; ++nup) {
    double x[3];
    cheb_point3(h, c, nup, x);
    for (int nu = 0; nu < h->k; ++nu)
      h->E[(c * h->k + nup) * h->k + nu] = lagrange3(h, par, nu, x);
  }
}

/* ------------------------------------------------------------------ */
/* Galerkin entries (Eq. (3)) by Sauter-Schwab quadrature (R7).        */
/* ------------------------------------------------------------------ */
static double quad_regular(const orh2 *h, const double *A1, const double *B1, const double *C1,
                           const double *A2, const double *B2, const double *C2, int q) {
  double gx[32], gw[32];
  or_gauss01(q, gx, gw);
  double acc = 0.0;
  for (int a = 0; a < q; ++a)
    for (int b = 0; b < q; ++b) {
      double x[3];
      ref_map(A1, B1, C1, gx[a], gx[a] * gx[b], x);
      double wx = gw[a] * gw[b] * gx[a];
      for (int c = 0; c < q; ++c)
        for (int d = 0; d < q; ++d) {
          double y[3];
          ref_map(A2, B2, C2, gx[c], gx[c] * gx[d], y);
          acc += wx * gw[c] * gw[d] * gx[c] * kernel_eval(h->kind, h->m, h->kappa, x, y);
        }
    }
  return acc;
}

/* one region of a singular rule: weight W, reference points (x1,x2), (y1,y2) */
static double sing_term(const orh2 *h, const double *A1, const double *B1, const double *C1,
                        const double *A2, const double *B2, const double *C2,
                        double W, double x1, double x2, double y1, double y2) {
  double x[3], y[3];
  ref_map(A1, B1, C1, x1, x2, x);
  ref_map(A2, B2, C2, y1, y2, y);
  return W * kernel_eval(h->kind, h->m, h->kappa, x, y);
}

/* identical panels: six regions, weight xi^3 e1^2 e2 */
static double quad_identical(const orh2 *h, const double *A, const double *B, const double *C, int q) {
  double g[32], w[32];
  or_gauss01(q, g, w);
  double acc = 0.0;
  for (int i0 = 0; i0 < q; ++i0)
    for (int i1 = 0; i1 < q; ++i1)
      for (int i2 = 0; i2 < q; ++i2)
        for (int i3 = 0; i3 < q; ++i3) {
          double xi = g[i0], e1 = g[i1], e2 = g[i2], e3 = g[i3];
          double W = xi * xi * xi * e1 * e1 * e2;
          double s = 0.0;
          s += sing_term(h, A, B, C, A, B, C, W, xi, xi * (1 - e1 + e1 * e2), xi * (1 - e1 * e2 * e3), xi * (1 - e1));
          s += sing_term(h, A, B, C, A, B, C, W, xi * (1 - e1 * e2 * e3), xi * (1 - e1), xi, xi * (1 - e1 + e1 * e2));
          s += sing_term(h, A, B, C, A, B, C, W, xi, xi * e1 * (1 - e2 + e2 * e3), xi * (1 - e1 * e2), xi * e1 * (1 - e2));
          s += sing_term(h, A, B, C, A, B, C, W, xi * (1 - e1 * e2), xi * e1 * (1 - e2), xi, xi * e1 * (1 - e2 + e2 * e3));
          s += sing_term(h, A, B, C, A, B, C, W, xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), xi, xi * e1 * (1 - e2));
          s += sing_term(h, A, B, C, A, B, C, W, xi, xi * e1 * (1 - e2), xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3));
          acc += w[i0] * w[i1] * w[i2] * w[i3] * s;
        }
  return acc;
}

/* common edge A-B (the image of t = 0 in both maps): five regions */
static double quad_edge(const orh2 *h, const double *A1, const double *B1, const double *C1,
                        const double *A2, const double *B2, const double *C2, int q) {
  double g[32], w[32];
  or_gauss01(q, g, w);
  double acc = 0.0;
  for (int i0 = 0; i0 < q; ++i0)
    for (int i1 = 0; i1 < q; ++i1)
      for (int i2 = 0; i2 < q; ++i2)
        for (int i3 = 0; i3 < q; ++i3) {
          double xi = g[i0], e1 = g[i1], e2 = g[i2], e3 = g[i3];
          double W1 = xi * xi * xi * e1 * e1;
          double W2 = W1 * e2;
          double s = 0.0;
          s += sing_term(h, A1, B1, C1, A2, B2, C2, W1, xi, xi * e1 * e3, xi * (1 - e1 * e2), xi * e1 * (1 - e2));
          s += sing_term(h, A1, B1, C1, A2, B2, C2, W2, xi, xi * e1, xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3));
          s += sing_term(h, A1, B1, C1, A2, B2, C2, W2, xi * (1 - e1 * e2), xi * e1 * (1 - e2), xi, xi * e1 * e2 * e3);
          s += sing_term(h, A1, B1, C1, A2, B2, C2, W2, xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3), xi, xi * e1);
          s += sing_term(h, A1, B1, C1, A2, B2, C2, W2, xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), xi, xi * e1 * e2);
          acc += w[i0] * w[i1] * w[i2] * w[i3] * s;
        }
  return acc;
}

/* common vertex A (the image of (0,0) in both maps): two regions */
static double quad_vertex(const orh2 *h, const double *A1, const double *B1, const double *C1,
                          const double *A2, const double *B2, const double *C2, int q) {
  double g[32], w[32];
  or_gauss01(q, g, w);
  double acc = 0.0;
  for (int i0 = 0; i0 < q; ++i0)
    for (int i1 = 0; i1 < q; ++i1)
      for (int i2 = 0; i2 < q; ++i2)
        for (int i3 = 0; i3 < q; ++i3) {
          double xi = g[i0], e1 = g[i1], e2 = g[i2], e3 = g[i3];
          double W = xi * xi * xi * e2;
          double s = 0.0;
          s += sing_term(h, A1, B1, C1, A2, B2, C2, W, xi, xi * e1, xi * e2, xi * e2 * e3);
          s += sing_term(h, A1, B1, C1, A2, B2, C2, W, xi * e2, xi * e2 * e3, xi, xi * e1);
          acc += w[i0] * w[i1] * w[i2] * w[i3] * s;
        }
  return acc;
}

/* g_ij for triangles i, j with quadrature order q (R7) */
static double galerkin_entry_q(const orh2 *h, int64_t i, int64_t j, int q) {
  if (i > j) { int64_t t = i; i = j; j = t; }
  const int32_t *ti = h->tri + 3 * i, *tj = h->tri + 3 * j;
  const double *V = h->vert;
  double jac = 4.0 * h->area[i] * h->area[j];
  if (h->kind == 1) {
    /* smooth test kernel: the exact collapsed rule for every pair */
    int qv = (3 * (h->m - 1) + 2 + 1) / 2 + 1;
    return jac * quad_regular(h, V + 3 * (int64_t)ti[0], V + 3 * (int64_t)ti[1], V + 3 * (int64_t)ti[2],
                              V + 3 * (int64_t)tj[0], V + 3 * (int64_t)tj[1], V + 3 * (int64_t)tj[2], qv);
  }
  int common = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      if (ti[a] == tj[b]) common++;
  if (common == 0)
    return jac * quad_regular(h, V + 3 * (int64_t)ti[0], V + 3 * (int64_t)ti[1], V + 3 * (int64_t)ti[2],
                              V + 3 * (int64_t)tj[0], V + 3 * (int64_t)tj[1], V + 3 * (int64_t)tj[2], q);
  if (common == 3) {
    int r = 0;
    for (int a = 1; a < 3; ++a)
      if (ti[a] < ti[r]) r = a;
    return jac * quad_identical(h, V + 3 * (int64_t)ti[r], V + 3 * (int64_t)ti[(r + 1) % 3],
                                V + 3 * (int64_t)ti[(r + 2) % 3], q);
  }
  if (common == 2) {
    int32_t sh[2], n = 0, oi = -1, oj = -1;
    for (int a = 0; a < 3; ++a) {
      int in = 0;
      for (int b = 0; b < 3; ++b) if (ti[a] == tj[b]) in = 1;
      if (in) sh[n++] = ti[a]; else oi = ti[a];
    }
    for (int b = 0; b < 3; ++b) {
      int in = 0;
      for (int a = 0; a < 3; ++a) if (ti[a] == tj[b]) in = 1;
      if (!in) oj = tj[b];
    }
    int32_t e0 = sh[0] < sh[1] ? sh[0] : sh[1], e1 = sh[0] < sh[1] ? sh[1] : sh[0];
    return jac * quad_edge(h, V + 3 * (int64_t)e0, V + 3 * (int64_t)e1, V + 3 * (int64_t)oi,
                           V + 3 * (int64_t)e0, V + 3 * (int64_t)e1, V + 3 * (int64_t)oj, q);
  }
  /* common == 1 */
  int ai = 0, bj = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      if (ti[a] == tj[b]) { ai = a; bj = b; }
  return jac * quad_vertex(h, V + 3 * (int64_t)ti[ai], V + 3 * (int64_t)ti[(ai + 1) % 3], V + 3 * (int64_t)ti[(ai + 2) % 3],
                           V + 3 * (int64_t)tj[bj], V + 3 * (int64_t)tj[(bj + 1) % 3], V + 3 * (int64_t)tj[(bj + 2) % 3], q);
}

/* ------------------------------------------------------------------ */
/* public API                                                          */
/* ------------------------------------------------------------------ */
void or_free(orh2 *h) {
  if (!h) return;
  free(h->vert); free(h->tri); free(h->cen); free(h->area); free(h->idx);
  free(h->first); free(h->size); free(h->lo); free(h->hi); free(h->pts);
  free(h->bt); free(h->bs); free(h->badm); free(h->rowptr); free(h->rowblk);
  free(h->V); free(h->E); free(h->noff); free(h->nval);
  free(h);
}

int or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Build the H^2 approximation.  kind: 0 Laplace, 1 smooth polynomial test
 * kernel, 2 / 3 real / imaginary part of the Helmholtz kernel with wave
 * number kappa.  store_near: assemble and keep the nearfield blocks.
 * with_bases: compute V and E (needed by the matvec).  Returns NULL on
 * invalid arguments. */
orh2 *or_build(const double *vert, int64_t nv, const int32_t *tri, int64_t nt, int leaf, double eta,
               int m, int q, int kind, double kappa, int store_near, int with_bases) {
  if (nt < 1 || nv < 3 || leaf < 2 || m < 1 || m > 8 || q < 1 || q > 30 || !(eta > 0.0)) return NULL;
  orh2 *h = (orh2 *)calloc(1, sizeof(orh2));
  h->nt = nt; h->nv = nv; h->leaf = leaf; h->eta = eta; h->m = m; h->k = m * m * m; h->q = q; h->kind = kind;
  h->kappa = kappa;
  h->vert = (double *)malloc(nv * 3 * sizeof(double));
  memcpy(h->vert, vert, nv * 3 * sizeof(double));
  h->tri = (int32_t *)malloc(nt * 3 * sizeof(int32_t));
  memcpy(h->tri, tri, nt * 3 * sizeof(int32_t));
  h->cen = (double *)malloc(nt * 3 * sizeof(double));
  h->area = (double *)malloc(nt * sizeof(double));
  for (int64_t t = 0; t < nt; ++t) {
    const double *a = vert + 3 * (int64_t)tri[3 * t], *b = vert + 3 * (int64_t)tri[3 * t + 1],
                 *c = vert + 3 * (int64_t)tri[3 * t + 2];
    for (int d = 0; d < 3; ++d) h->cen[3 * t + d] = (a[d] + b[d] + c[d]) / 3.0;
    h->area[t] = tri_area(a, b, c);
  }
  int D = 0;
  while ((nt + ((int64_t)1 << D) - 1) / ((int64_t)1 << D) > leaf) D++;
  h->depth = D;
  h->nclu = ((int64_t)2 << D) - 1;
  h->idx = (int64_t *)malloc(nt * sizeof(int64_t));
  for (int64_t t = 0; t < nt; ++t) h->idx[t] = t;
  h->first = (int64_t *)calloc(h->nclu, sizeof(int64_t));
  h->size = (int64_t *)calloc(h->nclu, sizeof(int64_t));
  h->lo = (double *)calloc(h->nclu * 3, sizeof(double));
  h->hi = (double *)calloc(h->nclu * 3, sizeof(double));
  build_cluster(h, 0, 0, 0, nt);
  h->pts = (double *)calloc(h->nclu * 3 * m, sizeof(double));
  for (int64_t c = 0; c < h->nclu; ++c) cheb_points(h, c);
  build_blocks(h, 0, 0);
  /* group blocks by row cluster, keeping recursion order */
  h->rowptr = (int64_t *)calloc(h->nclu + 1, sizeof(int64_t));
  h->rowblk = (int64_t *)malloc((h->nblk > 0 ? h->nblk : 1) * sizeof(int64_t));
  for (int64_t b = 0; b < h->nblk; ++b) h->rowptr[h->bt[b] + 1]++;
  for (int64_t c = 0; c < h->nclu; ++c) h->rowptr[c + 1] += h->rowptr[c];
  {
    size_t nfill = h->nclu > 0 ? (size_t)h->nclu : 1;
    int64_t *fill = (int64_t *)calloc(nfill, sizeof(int64_t));
    for (int64_t b = 0; b < h->nblk; ++b) {
      int64_t t = h->bt[b];
      h->rowblk[h->rowptr[t] + fill[t]++] = b;
    }
    free(fill);
  }
  if (with_bases) {
    int k = h->k;
    h->V = (double *)calloc(nt * k, sizeof(double));
    int64_t leaf0 = ((int64_t)1 << D) - 1;
    int64_t nleaf = (int64_t)1 << D;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < nleaf; ++j) leaf_basis(h, leaf0 + j);
    h->E = (double *)calloc(h->nclu * (int64_t)k * k, sizeof(double));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 1; c < h->nclu; ++c) transfer_matrix(h, c);
  }
  h->store_near = store_near;
  if (store_near) {
    h->noff = (int64_t *)calloc(h->nblk + 1, sizeof(int64_t));
    int64_t tot = 0;
    for (int64_t b = 0; b < h->nblk; ++b) {
      h->noff[b] = tot;
      if (!h->badm[b]) tot += h->size[h->bt[b]] * h->size[h->bs[b]];
    }
    h->noff[h->nblk] = tot;
    h->nval = (double *)calloc(tot > 0 ? tot : 1, sizeof(double));
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t b = 0; b < h->nblk; ++b) {
      if (h->badm[b]) continue;
      int64_t t = h->bt[b], s = h->bs[b];
      for (int64_t r = 0; r < h->size[t]; ++r)
        for (int64_t c = 0; c < h->size[s]; ++c)
          h->nval[h->noff[b] + r * h->size[s] + c] =
              galerkin_entry_q(h, h->idx[h->first[t] + r], h->idx[h->first[s] + c], h->q);
    }
  }
  return h;
}

void or_info(const orh2 *h, int64_t *out) {
  int64_t nadm = 0, nnear = 0, near_entries = 0;
  for (int64_t b = 0; b < h->nblk; ++b) {
    if (h->badm[b]) nadm++;
    else { nnear++; near_entries += h->size[h->bt[b]] * h->size[h->bs[b]]; }
  }
  out[0] = h->depth; out[1] = h->nclu; out[2] = h->nblk; out[3] = nadm; out[4] = nnear;
  out[5] = near_entries; out[6] = h->k;
}

void or_tree(const orh2 *h, int64_t *idx, int64_t *first, int64_t *size, double *lo, double *hi, double *pts) {
  if (idx) memcpy(idx, h->idx, h->nt * sizeof(int64_t));
  if (first) memcpy(first, h->first, h->nclu * sizeof(int64_t));
  if (size) memcpy(size, h->size, h->nclu * sizeof(int64_t));
  if (lo) memcpy(lo, h->lo, h->nclu * 3 * sizeof(double));
  if (hi) memcpy(hi, h->hi, h->nclu * 3 * sizeof(double));
  if (pts) memcpy(pts, h->pts, h->nclu * 3 * h->m * sizeof(double));
}

void or_blocks(const orh2 *h, int32_t *t, int32_t *s, uint8_t *adm) {
  memcpy(t, h->bt, h->nblk * sizeof(int32_t));
  memcpy(s, h->bs, h->nblk * sizeof(int32_t));
  memcpy(adm, h->badm, h->nblk);
}

/* V rows (cluster order) and E of one cluster */
void or_V(const orh2 *h, double *V) { memcpy(V, h->V, h->nt * h->k * sizeof(double)); }
void or_E(const orh2 *h, int64_t c, double *E) { memcpy(E, h->E + c * h->k * h->k, h->k * h->k * sizeof(double)); }

/* coupling matrix S_{t,s}, Eq. (6c): S[nu][mu] = g(xi_{t,nu}, xi_{s,mu}) */
void or_S(const orh2 *h, int64_t t, int64_t s, double *S) {
  for (int nu = 0; nu < h->k; ++nu) {
    double x[3];
    cheb_point3(h, t, nu, x);
    for (int mu = 0; mu < h->k; ++mu) {
      double y[3];
      cheb_point3(h, s, mu, y);
      S[nu * h->k + mu] = kernel_eval(h->kind, h->m, h->kappa, x, y);
    }
  }
}

/* tensor Lagrange polynomial of cluster c at points x (for pins) */
void or_lagrange(const orh2 *h, int64_t c, int nu, const double *x, int64_t np, double *out) {
  for (int64_t i = 0; i < np; ++i) out[i] = lagrange3(h, c, nu, x + 3 * i);
}

double or_entry(const orh2 *h, int64_t i, int64_t j, int q) { return galerkin_entry_q(h, i, j, q); }

/* the reference-map quadratures for two explicit triangles (pins):
 * mode 0 regular, 1 identical (uses triangle 1), 2 edge, 3 vertex. */
double or_pair_quad(const double *T1, const double *T2, int mode, int q, int kind, int m, double kappa) {
  orh2 tmp;
  memset(&tmp, 0, sizeof(tmp));
  tmp.kind = kind;
  tmp.kappa = kappa;
  tmp.m = m;
  switch (mode) {
    case 0: return quad_regular(&tmp, T1, T1 + 3, T1 + 6, T2, T2 + 3, T2 + 6, q);
    case 1: return quad_identical(&tmp, T1, T1 + 3, T1 + 6, q);
    case 2: return quad_edge(&tmp, T1, T1 + 3, T1 + 6, T2, T2 + 3, T2 + 6, q);
    default: return quad_vertex(&tmp, T1, T1 + 3, T1 + 6, T2, T2 + 3, T2 + 6, q);
  }
}

/* dense Galerkin matrix, column-major n x n, every pair by the same rule */
void or_dense(const orh2 *h, double *G) {
  int64_t n = h->nt;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i <= j; ++i) {
      double g = galerkin_entry_q(h, i, j, h->q);
      G[i + j * n] = g;
      G[j + i * n] = g;
    }
}

/* ---------------- H^2 matvec, Algorithms 1-3 ---------------- */

/* Algorithm 1 (post-order): xh[c][nu][r] */
static void forward_rec(const orh2 *h, int64_t c, int lev, const double *x, int nrhs, double *xh) {
  int k = h->k;
  double *xc = xh + c * k * nrhs;
  if (lev == h->depth) {
    for (int nu = 0; nu < k; ++nu)
      for (int r = 0; r < nrhs; ++r) {
        double acc = 0.0;
        for (int64_t p = h->first[c]; p < h->first[c] + h->size[c]; ++p)
          acc += h->V[p * k + nu] * x[h->idx[p] + r * h->nt];
        xc[nu * nrhs + r] = acc;
      }
    return;
  }
  for (int i = 0; i < k * nrhs; ++i) xc[i] = 0.0;
  for (int a = 1; a <= 2; ++a) {
    int64_t ch = 2 * c + a;
    forward_rec(h, ch, lev + 1, x, nrhs, xh);
    const double *E = h->E + ch * k * k;
    const double *xs = xh + ch * k * nrhs;
    for (int nu = 0; nu < k; ++nu)
      for (int r = 0; r < nrhs; ++r) {
        double acc = 0.0;
        for (int nup = 0; nup < k; ++nup) acc += E[nup * k + nu] * xs[nup * nrhs + r];
        xc[nu * nrhs + r] += acc;
      }
  }
}

/* Algorithm 2 (pre-order) */
static void backward_rec(const orh2 *h, int64_t c, int lev, double *yh, int nrhs, double *y) {
  int k = h->k;
  double *yc = yh + c * k * nrhs;
  if (lev == h->depth) {
    for (int64_t p = h->first[c]; p < h->first[c] + h->size[c]; ++p)
      for (int r = 0; r < nrhs; ++r) {
        double acc = 0.0;
        for (int nu = 0; nu < k; ++nu) acc += h->V[p * k + nu] * yc[nu * nrhs + r];
        y[h->idx[p] + r * h->nt] += acc;
      }
    return;
  }
  for (int a = 1; a <= 2; ++a) {
    int64_t ch = 2 * c + a;
    const double *E = h->E + ch * k * k;
    double *ys = yh + ch * k * nrhs;
    for (int nup = 0; nup < k; ++nup)
      for (int r = 0; r < nrhs; ++r) {
        double acc = 0.0;
        for (int nu = 0; nu < k; ++nu) acc += E[nup * k + nu] * yc[nu * nrhs + r];
        ys[nup * nrhs + r] += acc;
      }
    backward_rec(h, ch, lev + 1, yh, nrhs, y);
  }
}

/* Algorithm 3 over the leaves of the block tree, grouped by row cluster so
 * that rows can run in parallel; within a row the recursion order is kept. */
static void interaction(const orh2 *h, const double *xh, const double *x, int nrhs, double *yh, double *y) {
  int k = h->k;
#pragma omp parallel
  {
    double *S = (double *)malloc((size_t)k * k * sizeof(double));
#pragma omp for schedule(dynamic, 4)
    for (int64_t t = 0; t < h->nclu; ++t) {
      for (int64_t e = h->rowptr[t]; e < h->rowptr[t + 1]; ++e) {
        int64_t b = h->rowblk[e], s = h->bs[b];
        if (h->badm[b]) {
          or_S(h, t, s, S);
          const double *xs = xh + s * k * nrhs;
          double *yt = yh + t * k * nrhs;
          for (int nu = 0; nu < k; ++nu)
            for (int r = 0; r < nrhs; ++r) {
              double acc = 0.0;
              for (int mu = 0; mu < k; ++mu) acc += S[nu * k + mu] * xs[mu * nrhs + r];
              yt[nu * nrhs + r] += acc;
            }
        } else {
          for (int64_t i = 0; i < h->size[t]; ++i)
            for (int r = 0; r < nrhs; ++r) {
              double acc = 0.0;
              for (int64_t j = 0; j < h->size[s]; ++j) {
                double g = h->store_near ? h->nval[h->noff[b] + i * h->size[s] + j]
                                         : galerkin_entry_q(h, h->idx[h->first[t] + i], h->idx[h->first[s] + j], h->q);
                acc += g * x[h->idx[h->first[s] + j] + r * h->nt];
              }
              y[h->idx[h->first[t] + i] + r * h->nt] += acc;
            }
        }
      }
    }
    free(S);
  }
}

/* y = G~ x, x and y column-major nt x nrhs in the caller's triangle order.
 * xh_out / yh_out (optional, [nclu][k][nrhs]) receive the coefficients
 * after the forward phase and after the interaction phase. */
int or_matvec(const orh2 *h, const double *x, double *y, int nrhs, double *xh_out, double *yh_out) {
  if (!h->V || !h->E) return 1;
  size_t nc = (size_t)h->nclu * h->k * nrhs;
  double *xh = (double *)calloc(nc, sizeof(double));
  double *yh = (double *)calloc(nc, sizeof(double));
  forward_rec(h, 0, 0, x, nrhs, xh);
  memset(y, 0, (size_t)h->nt * nrhs * sizeof(double));
  interaction(h, xh, x, nrhs, yh, y);
  if (xh_out) memcpy(xh_out, xh, nc * sizeof(double));
  if (yh_out) memcpy(yh_out, yh, nc * sizeof(double));
  backward_rec(h, 0, 0, yh, nrhs, y);
  free(xh);
  free(yh);
  return 0;
}

/* Rows of y = G~ x one by one, for problems too large to multiply whole:
 * the forward phase (Algorithm 1) runs over the whole tree, then for every
 * requested row i the interaction phase is restricted to the blocks whose
 * row cluster contains i and the backward phase (Algorithm 2) to the path
 * from the root to the leaf of i.  Nearfield entries are computed on the
 * fly.  rows are original triangle indices; yrows is nrows x nrhs
 * column-major. */
int or_matvec_rows(const orh2 *h, const double *x, int nrhs, const int64_t *rows, int64_t nrows, double *yrows) {
  if (!h->V || !h->E) return 1;
  int k = h->k;
  size_t nc = (size_t)h->nclu * k * nrhs;
  double *xh = (double *)calloc(nc, sizeof(double));
  forward_rec(h, 0, 0, x, nrhs, xh);
  int64_t *pos = (int64_t *)malloc(h->nt * sizeof(int64_t));
  for (int64_t p = 0; p < h->nt; ++p) pos[h->idx[p]] = p;
  int64_t leaf0 = ((int64_t)1 << h->depth) - 1;
#pragma omp parallel
  {
    double *S = (double *)malloc((size_t)k * k * sizeof(double));
    double *acc = (double *)malloc((size_t)k * nrhs * sizeof(double));
    double *tmp = (double *)malloc((size_t)k * nrhs * sizeof(double));
    int64_t path[64];
#pragma omp for schedule(dynamic, 1)
    for (int64_t ri = 0; ri < nrows; ++ri) {
      int64_t i = rows[ri], p = pos[i];
      int64_t leaf = leaf0;
      while (!(p >= h->first[leaf] && p < h->first[leaf] + h->size[leaf])) leaf++;
      int np = 0;
      for (int64_t c = leaf;; c = (c - 1) / 2) {
        path[np++] = c;
        if (c == 0) break;
      }
      for (int r = 0; r < nrhs; ++r) yrows[ri + r * nrows] = 0.0;
      /* nearfield part of row i */
      for (int64_t e = h->rowptr[leaf]; e < h->rowptr[leaf + 1]; ++e) {
        int64_t b = h->rowblk[e], s = h->bs[b];
        if (h->badm[b]) continue;
        for (int64_t j = 0; j < h->size[s]; ++j) {
          int64_t tj = h->idx[h->first[s] + j];
          double g = galerkin_entry_q(h, i, tj, h->q);
          for (int r = 0; r < nrhs; ++r) yrows[ri + r * nrows] += g * x[tj + r * h->nt];
        }
      }
      /* farfield: yhat along the path, root first, pushed down by E */
      for (int q = 0; q < k * nrhs; ++q) acc[q] = 0.0;
      for (int a = np - 1; a >= 0; --a) {
        int64_t t = path[a];
        if (a != np - 1) {
          const double *E = h->E + t * k * k;
          for (int nup = 0; nup < k; ++nup)
            for (int r = 0; r < nrhs; ++r) {
              double s_ = 0.0;
              for (int nu = 0; nu < k; ++nu) s_ += E[nup * k + nu] * acc[nu * nrhs + r];
              tmp[nup * nrhs + r] = s_;
            }
          memcpy(acc, tmp, (size_t)k * nrhs * sizeof(double));
        }
        for (int64_t e = h->rowptr[t]; e < h->rowptr[t + 1]; ++e) {
          int64_t b = h->rowblk[e], s = h->bs[b];
          if (!h->badm[b]) continue;
          or_S(h, t, s, S);
          const double *xs = xh + s * k * nrhs;
          for (int nu = 0; nu < k; ++nu)
            for (int r = 0; r < nrhs; ++r) {
              double s_ = 0.0;
              for (int mu = 0; mu < k; ++mu) s_ += S[nu * k + mu] * xs[mu * nrhs + r];
              acc[nu * nrhs + r] += s_;
            }
        }
      }
      for (int r = 0; r < nrhs; ++r) {
        double s_ = 0.0;
        for (int nu = 0; nu < k; ++nu) s_ += h->V[p * k + nu] * acc[nu * nrhs + r];
        yrows[ri + r * nrows] += s_;
      }
    }
    free(S);
    free(acc);
    free(tmp);
  }
  free(pos);
  free(xh);
  return 0;
}


/* ------------------------------------------------------------------ */
/* GCA-H^2: nested cross approximation with Green quadrature (Section 3,
 * the GCA-H^2 example).  Every cluster tau gets pivot elements
 * tau_0 of tau (pivots of a parent are chosen among its sons' pivots), and
 * every admissible block the coupling S_{tau sigma} = G|_{tau_0 x sigma_0},
 * the Galerkin submatrix on the pivots.  The section states only this much;
 * the construction of the pivots follows the cited Green cross
 * approximation with the readings G1-G6 listed in the header.            */
/* ------------------------------------------------------------------ */

/* G1: quadrature on the boundary of the auxiliary box omega = [lo - gamma
 * rho, hi + gamma rho] (rho = half the diagonal of [lo, hi]): for axis
 * a = 0, 1, 2, the face at the low end (outward normal -e_a) then the face
 * at the high end (+e_a); on a face the other two axes b < c carry the
 * tensor Gauss-Legendre rule with qg nodes in increasing order, node i on
 * axis b outermost.  Returns the point count Q = 6 qg^2; Z, N: Q x 3,
 * W: Q. */
int or_gca_green_rule(const double *lo, const double *hi, double gamma, int qg, double *Z, double *N, double *W) {
  double gx[64], gw[64];
  or_gauss01(qg, gx, gw);
  double d0 = hi[0] - lo[0], d1 = hi[1] - lo[1], d2 = hi[2] - lo[2];
  double rho = 0.5 * sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  double olo[3], ohi[3];
  for (int d = 0; d < 3; ++d) { olo[d] = lo[d] - gamma * rho; ohi[d] = hi[d] + gamma * rho; }
  int q = 0;
  for (int a = 0; a < 3; ++a) {
    int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
    for (int side = 0; side < 2; ++side)
      for (int i = 0; i < qg; ++i)
        for (int j = 0; j < qg; ++j) {
          double *z = Z + 3 * q, *n = N + 3 * q;
          z[a] = side ? ohi[a] : olo[a];
          z[b] = olo[b] + gx[i] * (ohi[b] - olo[b]);
          z[c] = olo[c] + gx[j] * (ohi[c] - olo[c]);
          n[0] = n[1] = n[2] = 0.0;
          n[a] = side ? 1.0 : -1.0;
          W[q] = gw[i] * gw[j] * (ohi[b] - olo[b]) * (ohi[c] - olo[c]);
          q++;
        }
  }
  return q;
}

/* G2: the Green surrogate of a cluster, nr x 2Q row-major: row r is test
 * triangle rows[r]; column nu < Q holds W_nu int_T g(x, z_nu) dx and column
 * Q + nu holds W_nu int_T dg/dn_z(x, z_nu) dx, dg/dn_z = n.(x - z) /
 * (4 pi |x - z|^3) (the two families of Green's representation formula),
 * both integrals by the collapsed Gauss rule with qt nodes per direction
 * (R5), vertices in mesh order. */
static void gca_surrogate(const orh2 *h, const int32_t *rows, int nr, const double *Z, const double *N,
                          const double *W, int Q, int qt, double *M) {
  double gx[32], gw[32];
  or_gauss01(qt, gx, gw);
  for (int r = 0; r < nr; ++r) {
    int64_t t = rows[r];
    const double *A = h->vert + 3 * (int64_t)h->tri[3 * t + 0];
    const double *B = h->vert + 3 * (int64_t)h->tri[3 * t + 1];
    const double *C = h->vert + 3 * (int64_t)h->tri[3 * t + 2];
    double jac = 2.0 * h->area[t];
    for (int nu = 0; nu < Q; ++nu) {
      double s1 = 0.0, s2 = 0.0;
      for (int a = 0; a < qt; ++a)
        for (int b = 0; b < qt; ++b) {
          double x[3];
          ref_map(A, B, C, gx[a], gx[a] * gx[b], x);
          double w = jac * gw[a] * gw[b] * gx[a];
          double e0 = x[0] - Z[3 * nu], e1 = x[1] - Z[3 * nu + 1], e2 = x[2] - Z[3 * nu + 2];
          double rr = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
          s1 += w / (4.0 * OR_PI * rr);
          s2 += w * (N[3 * nu] * e0 + N[3 * nu + 1] * e1 + N[3 * nu + 2] * e2) / (4.0 * OR_PI * rr * rr * rr);
        }
      M[(int64_t)r * 2 * Q + nu] = W[nu] * s1;
      M[(int64_t)r * 2 * Q + Q + nu] = W[nu] * s2;
    }
  }
}

/* G3-G5: cross approximation of M (nr x nc, row-major) with complete
 * pivoting.  Step k takes the largest modulus of the residual R_k (R_0 = M);
 * it stops when that is at most eps times the largest modulus of M, or
 * after min(nr, nc, kmax) steps (kmax <= 0: no cap).  The pivot is the first entry in row-major
 * order whose modulus is at least (1 - 2^-30) times the largest (ties,
 * which symmetric meshes produce, go to the lowest index).  Update:
 * R <- R - R[:, j] R[i, :] / R[i, j], then row i and column j of R are set
 * to zero.  Output: the rank k, the row and column pivots I, J (in pivot
 * order) and Vhat = M[:, J] M[I, J]^{-1} (nr x k, row-major), solved by
 * Gaussian elimination with partial pivoting, with the rows I set to the
 * unit vectors (their exact values).  Vhat capacity: nr x min(nr, nc). */
int or_gca_aca(const double *M, int nr, int nc, double eps, int kcap, int *I, int *J, double *Vhat) {
  int kmax = nr < nc ? nr : nc;
  if (kcap > 0 && kcap < kmax) kmax = kcap;
  double *R = (double *)malloc((size_t)nr * nc * sizeof(double));
  memcpy(R, M, (size_t)nr * nc * sizeof(double));
  double mx0 = 0.0;
  for (int64_t e = 0; e < (int64_t)nr * nc; ++e) if (fabs(M[e]) > mx0) mx0 = fabs(M[e]);
  int k = 0;
  while (k < kmax) {
    double mx = 0.0;
    for (int64_t e = 0; e < (int64_t)nr * nc; ++e) if (fabs(R[e]) > mx) mx = fabs(R[e]);
    if (mx == 0.0 || mx <= eps * mx0) break;
    double thr = mx * (1.0 - ldexp(1.0, -30));
    int64_t pe = 0;
    while (fabs(R[pe]) < thr) pe++;
    int i = (int)(pe / nc), j = (int)(pe % nc);
    I[k] = i;
    J[k] = j;
    k++;
    double piv = R[pe];
    for (int r = 0; r < nr; ++r) {
      if (r == i) continue;
      double f = R[(int64_t)r * nc + j] / piv;
      for (int c = 0; c < nc; ++c)
        if (c != j) R[(int64_t)r * nc + c] -= f * R[(int64_t)i * nc + c];
    }
    for (int c = 0; c < nc; ++c) R[(int64_t)i * nc + c] = 0.0;
    for (int r = 0; r < nr; ++r) R[(int64_t)r * nc + j] = 0.0;
  }
  free(R);
  if (k == 0) return 0;
  /* Vhat A = B with A = M[I, J], B = M[:, J]: solve A^T v = b per row */
  double *At = (double *)malloc((size_t)k * k * sizeof(double));
  int *perm = (int *)malloc(k * sizeof(int));
  for (int a = 0; a < k; ++a)
    for (int b = 0; b < k; ++b) At[a * k + b] = M[(int64_t)I[b] * nc + J[a]];   /* At[a][b] = A[b][a] */
  for (int a = 0; a < k; ++a) perm[a] = a;
  for (int col = 0; col < k; ++col) {          /* LU with partial pivoting, in place */
    int p = col;
    for (int r = col + 1; r < k; ++r) if (fabs(At[r * k + col]) > fabs(At[p * k + col])) p = r;
    if (p != col) {
      for (int c = 0; c < k; ++c) { double t = At[col * k + c]; At[col * k + c] = At[p * k + c]; At[p * k + c] = t; }
      int t = perm[col]; perm[col] = perm[p]; perm[p] = t;
    }
    for (int r = col + 1; r < k; ++r) {
      double f = At[r * k + col] / At[col * k + col];
      At[r * k + col] = f;
      for (int c = col + 1; c < k; ++c) At[r * k + c] -= f * At[col * k + c];
    }
  }
  double *b = (double *)malloc(k * sizeof(double));
  for (int r = 0; r < nr; ++r) {
    for (int a = 0; a < k; ++a) b[a] = M[(int64_t)r * nc + J[perm[a]]];
    for (int a = 0; a < k; ++a)
      for (int c = 0; c < a; ++c) b[a] -= At[a * k + c] * b[c];
    for (int a = k - 1; a >= 0; --a) {
      for (int c = a + 1; c < k; ++c) b[a] -= At[a * k + c] * b[c];
      b[a] /= At[a * k + a];
    }
    for (int a = 0; a < k; ++a) Vhat[(int64_t)r * k + a] = b[a];
  }
  for (int a = 0; a < k; ++a)
    for (int c = 0; c < k; ++c) Vhat[(int64_t)I[a] * k + c] = a == c ? 1.0 : 0.0;
  free(At); free(perm); free(b);
  return k;
}

typedef struct {
  orh2 *h;          /* trees, blocks, nearfield */
  int qg, qt, kcap;
  double eps, gamma;
  int *rank;        /* per cluster */
  int32_t **piv;    /* per cluster: pivot triangles (caller's indices), pivot order */
  double **V;       /* leaves: size x rank, rows in cluster order */
  double **E;       /* non-root clusters: rank x rank(parent) */
  int64_t *soff;    /* per block: offset into S (admissible), or -1 */
  double *S;        /* admissible blocks: rank(t) x rank(s), row-major */
} orgca;

/* cluster c of the tree: its pivots, leaf basis or its sons' transfer
 * matrices (G6: the candidate rows of a parent are the pivots of son 1
 * followed by those of son 2) */
static void gca_cluster(orgca *g, int64_t c) {
  orh2 *h = g->h;
  int Q = 6 * g->qg * g->qg, nc = 2 * Q;
  int nr;
  int32_t *rows;
  int64_t leaf0 = ((int64_t)1 << h->depth) - 1;
  if (c >= leaf0) {
    nr = (int)h->size[c];
    rows = (int32_t *)malloc((nr > 0 ? nr : 1) * sizeof(int32_t));
    for (int r = 0; r < nr; ++r) rows[r] = (int32_t)h->idx[h->first[c] + r];
  } else {
    int k1 = g->rank[2 * c + 1], k2 = g->rank[2 * c + 2];
    nr = k1 + k2;
    rows = (int32_t *)malloc((nr > 0 ? nr : 1) * sizeof(int32_t));
    memcpy(rows, g->piv[2 * c + 1], k1 * sizeof(int32_t));
    memcpy(rows + k1, g->piv[2 * c + 2], k2 * sizeof(int32_t));
  }
  double *Z = (double *)malloc(Q * 3 * sizeof(double)), *N = (double *)malloc(Q * 3 * sizeof(double));
  double *W = (double *)malloc(Q * sizeof(double));
  or_gca_green_rule(h->lo + 3 * c, h->hi + 3 * c, g->gamma, g->qg, Z, N, W);
  double *M = (double *)malloc((size_t)(nr > 0 ? nr : 1) * nc * sizeof(double));
  gca_surrogate(h, rows, nr, Z, N, W, Q, g->qt, M);
  int kcap = nr < nc ? nr : nc;
  int *I = (int *)malloc((kcap > 0 ? kcap : 1) * sizeof(int)), *J = (int *)malloc((kcap > 0 ? kcap : 1) * sizeof(int));
  double *Vh = (double *)malloc((size_t)(nr > 0 ? nr : 1) * (kcap > 0 ? kcap : 1) * sizeof(double));
  int k = nr > 0 ? or_gca_aca(M, nr, nc, g->eps, g->kcap, I, J, Vh) : 0;
  g->rank[c] = k;
  g->piv[c] = (int32_t *)malloc((k > 0 ? k : 1) * sizeof(int32_t));
  for (int a = 0; a < k; ++a) g->piv[c][a] = rows[I[a]];
  if (c >= leaf0) {
    g->V[c] = (double *)malloc((size_t)(nr > 0 ? nr : 1) * (k > 0 ? k : 1) * sizeof(double));
    memcpy(g->V[c], Vh, (size_t)nr * k * sizeof(double));
  } else {
    int k1 = g->rank[2 * c + 1], k2 = g->rank[2 * c + 2];
    g->E[2 * c + 1] = (double *)malloc((size_t)(k1 > 0 ? k1 : 1) * (k > 0 ? k : 1) * sizeof(double));
    g->E[2 * c + 2] = (double *)malloc((size_t)(k2 > 0 ? k2 : 1) * (k > 0 ? k : 1) * sizeof(double));
    memcpy(g->E[2 * c + 1], Vh, (size_t)k1 * k * sizeof(double));
    memcpy(g->E[2 * c + 2], Vh + (size_t)k1 * k, (size_t)k2 * k * sizeof(double));
  }
  free(rows); free(Z); free(N); free(W); free(M); free(I); free(J); free(Vh);
}

void or_gca_free(orgca *g) {
  if (!g) return;
  if (g->h) {
    for (int64_t c = 0; c < g->h->nclu; ++c) {
      if (g->piv) free(g->piv[c]);
      if (g->V) free(g->V[c]);
      if (g->E) free(g->E[c]);
    }
    or_free(g->h);
  }
  free(g->rank); free(g->piv); free(g->V); free(g->E); free(g->soff); free(g->S);
  free(g);
}

/* Build the GCA-H^2 matrix of the Laplace single-layer operator: trees and
 * blocks as for or_build (R2, R3), nearfield with quadrature order q (R7),
 * Green quadrature order qg, enlargement gamma, triangle rule qt,
 * cross-approximation accuracy eps, at most kcap pivots per cluster (<= 0:
 * no cap).  store_S: keep the coupling matrices (else they are evaluated
 * when used).  NULL on invalid arguments. */
orgca *or_gca_build(const double *vert, int64_t nv, const int32_t *tri, int64_t nt, int leaf, double eta, int qg,
                    double eps, double gamma, int qt, int kcap, int q, int store_near, int store_S) {
  if (qg < 1 || qg > 32 || qt < 1 || qt > 30 || !(eps >= 0.0) || !(gamma > 0.0)) return NULL;
  orh2 *h = or_build(vert, nv, tri, nt, leaf, eta, 1, q, 0, 0.0, store_near, 0);
  if (!h) return NULL;
  orgca *g = (orgca *)calloc(1, sizeof(orgca));
  g->h = h; g->qg = qg; g->qt = qt; g->eps = eps; g->gamma = gamma; g->kcap = kcap;
  g->rank = (int *)calloc(h->nclu, sizeof(int));
  g->piv = (int32_t **)calloc(h->nclu, sizeof(int32_t *));
  g->V = (double **)calloc(h->nclu, sizeof(double *));
  g->E = (double **)calloc(h->nclu, sizeof(double *));
  for (int l = h->depth; l >= 0; --l) {
    int64_t c0 = ((int64_t)1 << l) - 1, c1 = ((int64_t)2 << l) - 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = c0; c < c1; ++c) gca_cluster(g, c);
  }
  g->soff = (int64_t *)malloc((h->nblk > 0 ? h->nblk : 1) * sizeof(int64_t));
  int64_t tot = 0;
  for (int64_t b = 0; b < h->nblk; ++b) {
    g->soff[b] = -1;
    if (h->badm[b]) { g->soff[b] = tot; tot += (int64_t)g->rank[h->bt[b]] * g->rank[h->bs[b]]; }
  }
  if (store_S) {
    g->S = (double *)calloc(tot > 0 ? tot : 1, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < h->nblk; ++b) {
      if (!h->badm[b]) continue;
      int64_t t = h->bt[b], s = h->bs[b];
      for (int a = 0; a < g->rank[t]; ++a)
        for (int c = 0; c < g->rank[s]; ++c)
          g->S[g->soff[b] + (int64_t)a * g->rank[s] + c] = galerkin_entry_q(h, g->piv[t][a], g->piv[s][c], h->q);
    }
  }
  return g;
}

const orh2 *or_gca_h2(const orgca *g) { return g->h; }
void or_gca_ranks(const orgca *g, int32_t *out) {
  for (int64_t c = 0; c < g->h->nclu; ++c) out[c] = g->rank[c];
}
void or_gca_pivots(const orgca *g, int64_t c, int32_t *out) { memcpy(out, g->piv[c], g->rank[c] * sizeof(int32_t)); }
void or_gca_V(const orgca *g, int64_t c, double *out) {
  memcpy(out, g->V[c], (size_t)g->h->size[c] * g->rank[c] * sizeof(double));
}
void or_gca_E(const orgca *g, int64_t c, double *out) {
  memcpy(out, g->E[c], (size_t)g->rank[c] * g->rank[(c - 1) / 2] * sizeof(double));
}
/* S_{t,s} = G|_{t_0 x s_0} (rank(t) x rank(s), row-major) */
void or_gca_S(const orgca *g, int64_t t, int64_t s, double *out) {
  for (int a = 0; a < g->rank[t]; ++a)
    for (int c = 0; c < g->rank[s]; ++c)
      out[(int64_t)a * g->rank[s] + c] = galerkin_entry_q(g->h, g->piv[t][a], g->piv[s][c], g->h->q);
}

static const double *gca_block_S(const orgca *g, int64_t b, double *tmp) {
  if (g->S) return g->S + g->soff[b];
  or_gca_S(g, g->h->bt[b], g->h->bs[b], tmp);
  return tmp;
}

/* Algorithm 1 with the GCA bases: xh[c] (rank x nrhs) */
static void gca_forward(const orgca *g, int64_t c, int lev, const double *x, int nrhs, double **xh) {
  const orh2 *h = g->h;
  int k = g->rank[c];
  double *xc = xh[c];
  for (int i = 0; i < k * nrhs; ++i) xc[i] = 0.0;
  if (lev == h->depth) {
    for (int nu = 0; nu < k; ++nu)
      for (int r = 0; r < nrhs; ++r) {
        double acc = 0.0;
        for (int64_t p = 0; p < h->size[c]; ++p) acc += g->V[c][p * k + nu] * x[h->idx[h->first[c] + p] + r * h->nt];
        xc[nu * nrhs + r] = acc;
      }
    return;
  }
  for (int a = 1; a <= 2; ++a) {
    int64_t ch = 2 * c + a;
    gca_forward(g, ch, lev + 1, x, nrhs, xh);
    int kc = g->rank[ch];
    for (int nu = 0; nu < k; ++nu)
      for (int r = 0; r < nrhs; ++r) {
        double acc = 0.0;
        for (int nup = 0; nup < kc; ++nup) acc += g->E[ch][nup * k + nu] * xh[ch][nup * nrhs + r];
        xc[nu * nrhs + r] += acc;
      }
  }
}

/* Algorithm 2 with the GCA bases */
static void gca_backward(const orgca *g, int64_t c, int lev, double **yh, int nrhs, double *y) {
  const orh2 *h = g->h;
  int k = g->rank[c];
  if (lev == h->depth) {
    for (int64_t p = 0; p < h->size[c]; ++p)
      for (int r = 0; r < nrhs; ++r) {
        double acc = 0.0;
        for (int nu = 0; nu < k; ++nu) acc += g->V[c][p * k + nu] * yh[c][nu * nrhs + r];
        y[h->idx[h->first[c] + p] + r * h->nt] += acc;
      }
    return;
  }
  for (int a = 1; a <= 2; ++a) {
    int64_t ch = 2 * c + a;
    int kc = g->rank[ch];
    for (int nup = 0; nup < kc; ++nup)
      for (int r = 0; r < nrhs; ++r) {
        double acc = 0.0;
        for (int nu = 0; nu < k; ++nu) acc += g->E[ch][nup * k + nu] * yh[c][nu * nrhs + r];
        yh[ch][nup * nrhs + r] += acc;
      }
    gca_backward(g, ch, lev + 1, yh, nrhs, y);
  }
}

static int gca_maxrank(const orgca *g) {
  int km = 1;
  for (int64_t c = 0; c < g->h->nclu; ++c) if (g->rank[c] > km) km = g->rank[c];
  return km;
}

/* y = G~ x (Algorithms 1-3) with the GCA-H^2 matrix; layout as or_matvec */
int or_gca_matvec(const orgca *g, const double *x, double *y, int nrhs) {
  const orh2 *h = g->h;
  double **xh = (double **)malloc(h->nclu * sizeof(double *)), **yh = (double **)malloc(h->nclu * sizeof(double *));
  for (int64_t c = 0; c < h->nclu; ++c) {
    xh[c] = (double *)calloc((size_t)(g->rank[c] > 0 ? g->rank[c] : 1) * nrhs, sizeof(double));
    yh[c] = (double *)calloc((size_t)(g->rank[c] > 0 ? g->rank[c] : 1) * nrhs, sizeof(double));
  }
  gca_forward(g, 0, 0, x, nrhs, xh);
  memset(y, 0, (size_t)h->nt * nrhs * sizeof(double));
  int km = gca_maxrank(g);
#pragma omp parallel
  {
    double *tmp = (double *)malloc((size_t)km * km * sizeof(double));
#pragma omp for schedule(dynamic, 4)
    for (int64_t t = 0; t < h->nclu; ++t) {
      for (int64_t e = h->rowptr[t]; e < h->rowptr[t + 1]; ++e) {
        int64_t b = h->rowblk[e], s = h->bs[b];
        if (h->badm[b]) {
          const double *S = gca_block_S(g, b, tmp);
          int kt = g->rank[t], ks = g->rank[s];
          for (int nu = 0; nu < kt; ++nu)
            for (int r = 0; r < nrhs; ++r) {
              double acc = 0.0;
              for (int mu = 0; mu < ks; ++mu) acc += S[nu * ks + mu] * xh[s][mu * nrhs + r];
              yh[t][nu * nrhs + r] += acc;
            }
        } else {
          for (int64_t i = 0; i < h->size[t]; ++i)
            for (int r = 0; r < nrhs; ++r) {
              double acc = 0.0;
              for (int64_t j = 0; j < h->size[s]; ++j) {
                double gv = h->store_near ? h->nval[h->noff[b] + i * h->size[s] + j]
                                          : galerkin_entry_q(h, h->idx[h->first[t] + i], h->idx[h->first[s] + j], h->q);
                acc += gv * x[h->idx[h->first[s] + j] + r * h->nt];
              }
              y[h->idx[h->first[t] + i] + r * h->nt] += acc;
            }
        }
      }
    }
    free(tmp);
  }
  gca_backward(g, 0, 0, yh, nrhs, y);
  for (int64_t c = 0; c < h->nclu; ++c) { free(xh[c]); free(yh[c]); }
  free(xh); free(yh);
  return 0;
}

/* Rows of y = G~ x one by one (as or_matvec_rows): the forward phase over
 * the whole tree, then per row the blocks of the clusters on the path from
 * the root to the row's leaf, the coefficients pushed down by E. */
int or_gca_matvec_rows(const orgca *g, const double *x, int nrhs, const int64_t *rows, int64_t nrows, double *yrows) {
  const orh2 *h = g->h;
  double **xh = (double **)malloc(h->nclu * sizeof(double *));
  for (int64_t c = 0; c < h->nclu; ++c)
    xh[c] = (double *)calloc((size_t)(g->rank[c] > 0 ? g->rank[c] : 1) * nrhs, sizeof(double));
  gca_forward(g, 0, 0, x, nrhs, xh);
  int64_t *pos = (int64_t *)malloc(h->nt * sizeof(int64_t));
  for (int64_t p = 0; p < h->nt; ++p) pos[h->idx[p]] = p;
  int64_t leaf0 = ((int64_t)1 << h->depth) - 1;
  int km = gca_maxrank(g);
#pragma omp parallel
  {
    double *tmp = (double *)malloc((size_t)km * km * sizeof(double));
    double *acc = (double *)malloc((size_t)km * nrhs * sizeof(double));
    double *nxt = (double *)malloc((size_t)km * nrhs * sizeof(double));
    int64_t path[64];
#pragma omp for schedule(dynamic, 1)
    for (int64_t ri = 0; ri < nrows; ++ri) {
      int64_t i = rows[ri], p = pos[i];
      int64_t leaf = leaf0;
      while (!(p >= h->first[leaf] && p < h->first[leaf] + h->size[leaf])) leaf++;
      int np = 0;
      for (int64_t c = leaf;; c = (c - 1) / 2) {
        path[np++] = c;
        if (c == 0) break;
      }
      for (int r = 0; r < nrhs; ++r) yrows[ri + r * nrows] = 0.0;
      for (int64_t e = h->rowptr[leaf]; e < h->rowptr[leaf + 1]; ++e) {
        int64_t b = h->rowblk[e], s = h->bs[b];
        if (h->badm[b]) continue;
        for (int64_t j = 0; j < h->size[s]; ++j) {
          int64_t tj = h->idx[h->first[s] + j];
          double gv = galerkin_entry_q(h, i, tj, h->q);
          for (int r = 0; r < nrhs; ++r) yrows[ri + r * nrows] += gv * x[tj + r * h->nt];
        }
      }
      int kprev = 0;
      for (int a = np - 1; a >= 0; --a) {
        int64_t t = path[a];
        int kt = g->rank[t];
        if (a == np - 1) {
          for (int q = 0; q < kt * nrhs; ++q) acc[q] = 0.0;
        } else {
          for (int nup = 0; nup < kt; ++nup)
            for (int r = 0; r < nrhs; ++r) {
              double s_ = 0.0;
              for (int nu = 0; nu < kprev; ++nu) s_ += g->E[t][nup * kprev + nu] * acc[nu * nrhs + r];
              nxt[nup * nrhs + r] = s_;
            }
          memcpy(acc, nxt, (size_t)kt * nrhs * sizeof(double));
        }
        for (int64_t e = h->rowptr[t]; e < h->rowptr[t + 1]; ++e) {
          int64_t b = h->rowblk[e], s = h->bs[b];
          if (!h->badm[b]) continue;
          const double *S = gca_block_S(g, b, tmp);
          int ks = g->rank[s];
          for (int nu = 0; nu < kt; ++nu)
            for (int r = 0; r < nrhs; ++r) {
              double s_ = 0.0;
              for (int mu = 0; mu < ks; ++mu) s_ += S[nu * ks + mu] * xh[s][mu * nrhs + r];
              acc[nu * nrhs + r] += s_;
            }
        }
        kprev = kt;
      }
      int kl = g->rank[leaf];
      int64_t pl = p - h->first[leaf];
      for (int r = 0; r < nrhs; ++r) {
        double s_ = 0.0;
        for (int nu = 0; nu < kl; ++nu) s_ += g->V[leaf][pl * kl + nu] * acc[nu * nrhs + r];
        yrows[ri + r * nrows] += s_;
      }
    }
    free(tmp); free(acc); free(nxt);
  }
  free(pos);
  for (int64_t c = 0; c < h->nclu; ++c) free(xh[c]);
  free(xh);
  return 0;
}

/* ---------------- restarted GMRES (Saad, Alg. 6.9) ---------------- */
static double dot_(const double *a, const double *b, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Solves G~ z = b column by column, x0 = 0.  Stops a column when the true
 * residual |b - G~ z| / |b| <= rtol (checked at the end of every cycle and
 * whenever the Givens estimate falls below rtol) or after maxit
 * iterations.  iters[c], relres[c] report the iterations and the true
 * relative residual.  Returns the number of columns that did not converge. */
int or_gmres(const orh2 *h, const double *b, double *z, int nrhs, double rtol, int restart, int maxit,
             int *iters, double *relres) {
  int64_t n = h->nt;
  int mr = restart;
  double *Vk = (double *)malloc((size_t)(mr + 1) * n * sizeof(double));
  double *H = (double *)calloc((size_t)(mr + 1) * mr, sizeof(double));
  double *cs = (double *)malloc(mr * sizeof(double)), *sn = (double *)malloc(mr * sizeof(double));
  double *g = (double *)malloc((mr + 1) * sizeof(double)), *yv = (double *)malloc(mr * sizeof(double));
  double *w = (double *)malloc(n * sizeof(double)), *r = (double *)malloc(n * sizeof(double));
  int fails = 0;
  for (int col = 0; col < nrhs; ++col) {
    const double *bc = b + (size_t)col * n;
    double *zc = z + (size_t)col * n;
    for (int64_t i = 0; i < n; ++i) zc[i] = 0.0;
    double bn = sqrt(dot_(bc, bc, n));
    int it = 0, done = 0;
    double rel = 1.0;
    if (bn == 0.0) { iters[col] = 0; relres[col] = 0.0; continue; }
    while (!done) {
      or_matvec(h, zc, w, 1, NULL, NULL);
      for (int64_t i = 0; i < n; ++i) r[i] = bc[i] - w[i];
      double beta = sqrt(dot_(r, r, n));
      rel = beta / bn;
      if (rel <= rtol || it >= maxit) { done = 1; break; }
      for (int64_t i = 0; i < n; ++i) Vk[i] = r[i] / beta;
      for (int i = 0; i <= mr; ++i) g[i] = 0.0;
      g[0] = beta;
      int j;
      for (j = 0; j < mr && it < maxit; ++j) {
        it++;
        or_matvec(h, Vk + (size_t)j * n, w, 1, NULL, NULL);
        for (int i = 0; i <= j; ++i) {
          double hij = dot_(w, Vk + (size_t)i * n, n);
          H[i * mr + j] = hij;
          for (int64_t l = 0; l < n; ++l) w[l] -= hij * Vk[(size_t)i * n + l];
        }
        double hn = sqrt(dot_(w, w, n));
        H[(j + 1) * mr + j] = hn;
        if (hn > 0.0)
          for (int64_t l = 0; l < n; ++l) Vk[(size_t)(j + 1) * n + l] = w[l] / hn;
        for (int i = 0; i < j; ++i) {
          double a = H[i * mr + j], c = H[(i + 1) * mr + j];
          H[i * mr + j] = cs[i] * a + sn[i] * c;
          H[(i + 1) * mr + j] = -sn[i] * a + cs[i] * c;
        }
        double a = H[j * mr + j], c = H[(j + 1) * mr + j];
        double den = sqrt(a * a + c * c);
        cs[j] = den > 0.0 ? a / den : 1.0;
        sn[j] = den > 0.0 ? c / den : 0.0;
        H[j * mr + j] = cs[j] * a + sn[j] * c;
        H[(j + 1) * mr + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        if (fabs(g[j + 1]) <= rtol * bn || hn == 0.0) { j++; break; }
      }
      /* back substitution and update */
      for (int i = j - 1; i >= 0; --i) {
        double s = g[i];
        for (int l = i + 1; l < j; ++l) s -= H[i * mr + l] * yv[l];
        yv[i] = s / H[i * mr + i];
      }
      for (int i = 0; i < j; ++i)
        for (int64_t l = 0; l < n; ++l) zc[l] += yv[i] * Vk[(size_t)i * n + l];
    }
    iters[col] = it;
    relres[col] = rel;
    if (rel > rtol) fails++;
  }
  free(Vk); free(H); free(cs); free(sn); free(g); free(yv); free(w); free(r);
  return fails;
}
