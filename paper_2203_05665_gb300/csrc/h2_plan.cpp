// Host planning of the H^2 matrix: cluster tree, block tree, interpolation
// points, leaf bases and transfer factors (Boerm, Section 2).
//
// Compiled with -ffp-contract=off: centroids, boxes and the admissibility
// test are evaluated without fused multiply-adds so that the trees are the
// same on every host architecture.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <thread>

#include "h2_internal.hpp"

namespace h2 {

static constexpr double kPi = 3.141592653589793238462643383279502884;

void gauss_legendre01(int q, std::vector<double> &x, std::vector<double> &w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  // roots of P_q by Newton from the Chebyshev-like first guess; the
  // derivative from (1 - t^2) P_q'(t) = q (P_{q-1}(t) - t P_q(t)).
  for (int i = 0; i < q; ++i) {
    double t = std::cos(kPi * (4.0 * i + 3.0) / (4.0 * q + 2.0));
    double pq = 0, pqm1 = 0;
    auto legendre = [&](double s) {
      double a = 1.0, b = s;  // P_0, P_1
      if (q == 0) { pq = 1; pqm1 = 0; return; }
      for (int j = 1; j < q; ++j) {
        double c = ((2 * j + 1) * s * b - j * a) / (j + 1);
        a = b;
        b = c;
      }
      pq = b;
      pqm1 = a;
    };
    for (int it = 0; it < 64; ++it) {
      legendre(t);
      double d = q * (pqm1 - t * pq) / (1.0 - t * t);
      double step = pq / d;
      t -= step;
      if (std::fabs(step) <= 1e-17) break;
    }
    legendre(t);
    double d = q * (pqm1 - t * pq) / (1.0 - t * t);
    // on [-1,1]: w = 2 / ((1 - t^2) P_q'(t)^2); mapped to [0,1] halves it
    x[i] = 0.5 * (t + 1.0);
    w[i] = 1.0 / ((1.0 - t * t) * d * d);
  }
}

namespace {

struct Box {
  double lo[3], hi[3];
};

bool admissible_pair(const Plan &p, int64_t a, int64_t b, double eta) {
  const double *la = &p.lo[3 * a], *ha = &p.hi[3 * a];
  const double *lb = &p.lo[3 * b], *hb = &p.hi[3 * b];
  double da = std::sqrt((ha[0] - la[0]) * (ha[0] - la[0]) + (ha[1] - la[1]) * (ha[1] - la[1]) +
                        (ha[2] - la[2]) * (ha[2] - la[2]));
  double db = std::sqrt((hb[0] - lb[0]) * (hb[0] - lb[0]) + (hb[1] - lb[1]) * (hb[1] - lb[1]) +
                        (hb[2] - lb[2]) * (hb[2] - lb[2]));
  double gap[3];
  for (int d = 0; d < 3; ++d) gap[d] = std::max(0.0, std::max(la[d] - hb[d], lb[d] - ha[d]));
  double dist = std::sqrt(gap[0] * gap[0] + gap[1] * gap[1] + gap[2] * gap[2]);
  return std::max(da, db) <= (2.0 * eta) * dist;
}

// 1-D Lagrange polynomial j on the node set z[0..m-1] at t
double lag1(const double *z, int m, int j, double t) {
  double v = 1.0;
  for (int i = 0; i < m; ++i)
    if (i != j) v *= (t - z[i]) / (z[j] - z[i]);
  return v;
}

template <class F>
void parallel_for(int64_t n, F f) {
  unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  if (n < 256 || nt == 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      for (int64_t i = t; i < n; i += nt) f(i);
    });
  for (auto &x : th) x.join();
}

}  // namespace

int make_plan(const double *vert, int64_t nv, const int32_t *tri, int64_t nt, int leaf_size, double eta, int order,
              bool with_bases, Plan &p) {
  if (!vert || !tri) return fail(H2_EINVAL, "vert and tri must not be NULL");
  if (nt < 1 || nv < 3) return fail(H2_EINVAL, "need at least one triangle and three vertices");
  if (nt > (int64_t)1 << 30) return fail(H2_EINVAL, "too many triangles");
  if (leaf_size < 2) return fail(H2_EINVAL, "leaf_size must be >= 2");
  if (!(eta > 0.0) || !std::isfinite(eta)) return fail(H2_EINVAL, "eta must be positive");
  if (order < 1 || order > 5) return fail(H2_EINVAL, "order must be in [1, 5]");
  for (int64_t i = 0; i < 3 * nt; ++i)
    if (tri[i] < 0 || tri[i] >= nv) return fail(H2_EINVAL, "triangle vertex index out of range");
  for (int64_t i = 0; i < 3 * nv; ++i)
    if (!std::isfinite(vert[i])) return fail(H2_EINVAL, "non-finite vertex coordinate");

  p = Plan();
  p.n = nt;
  p.nv = nv;
  p.vert.assign(vert, vert + 3 * nv);
  p.tri.assign(tri, tri + 3 * nt);
  p.leaf = leaf_size;
  p.m = order;
  p.k = order * order * order;
  p.eta = eta;

  // centroids (characteristic points) and areas
  p.cen.resize(3 * nt);
  p.area.resize(nt);
  for (int64_t t = 0; t < nt; ++t) {
    const double *a = &vert[3 * tri[3 * t]], *b = &vert[3 * tri[3 * t + 1]], *c = &vert[3 * tri[3 * t + 2]];
    for (int d = 0; d < 3; ++d) p.cen[3 * t + d] = (a[d] + b[d] + c[d]) / 3.0;
    double u[3], v[3];
    for (int d = 0; d < 3; ++d) { u[d] = b[d] - a[d]; v[d] = c[d] - a[d]; }
    double nx = u[1] * v[2] - u[2] * v[1], ny = u[2] * v[0] - u[0] * v[2], nz = u[0] * v[1] - u[1] * v[0];
    p.area[t] = 0.5 * std::sqrt(nx * nx + ny * ny + nz * nz);
  }

  // depth: every cluster above it is bisected; leaves hold <= leaf_size
  int D = 0;
  while (((nt + ((int64_t)1 << D) - 1) >> D) > leaf_size) ++D;
  p.depth = D;
  p.nclu = ((int64_t)2 << D) - 1;
  p.nleaf = (int64_t)1 << D;
  p.leaf0 = p.nleaf - 1;
  p.perm.resize(nt);
  std::iota(p.perm.begin(), p.perm.end(), 0);
  p.first.assign(p.nclu, 0);
  p.size.assign(p.nclu, 0);
  p.lo.assign(3 * p.nclu, 0.0);
  p.hi.assign(3 * p.nclu, 0.0);
  p.size[0] = nt;

  // level-by-level bisection of the characteristic points
  for (int l = 0; l <= D; ++l) {
    int64_t c0 = ((int64_t)1 << l) - 1, c1 = ((int64_t)2 << l) - 1;
    for (int64_t c = c0; c < c1; ++c) {
      int64_t *beg = p.perm.data() + p.first[c], *end = beg + p.size[c];
      Box bx{{INFINITY, INFINITY, INFINITY}, {-INFINITY, -INFINITY, -INFINITY}};
      for (int64_t *q = beg; q != end; ++q)
        for (int v = 0; v < 3; ++v) {
          const double *x = &vert[3 * tri[3 * *q + v]];
          for (int d = 0; d < 3; ++d) {
            bx.lo[d] = std::min(bx.lo[d], x[d]);
            bx.hi[d] = std::max(bx.hi[d], x[d]);
          }
        }
      for (int d = 0; d < 3; ++d) { p.lo[3 * c + d] = bx.lo[d]; p.hi[3 * c + d] = bx.hi[d]; }
      if (l == D) continue;
      double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (int64_t *q = beg; q != end; ++q)
        for (int d = 0; d < 3; ++d) {
          clo[d] = std::min(clo[d], p.cen[3 * *q + d]);
          chi[d] = std::max(chi[d], p.cen[3 * *q + d]);
        }
      int axis = 0;
      for (int d = 1; d < 3; ++d)
        if (chi[d] - clo[d] > chi[axis] - clo[axis]) axis = d;
      const double *cen = p.cen.data();
      std::sort(beg, end, [cen, axis](int64_t a, int64_t b) {
        double ka = cen[3 * a + axis], kb = cen[3 * b + axis];
        return ka < kb || (ka == kb && a < b);
      });
      int64_t h0 = p.size[c] / 2;
      p.first[2 * c + 1] = p.first[c];
      p.size[2 * c + 1] = h0;
      p.first[2 * c + 2] = p.first[c] + h0;
      p.size[2 * c + 2] = p.size[c] - h0;
    }
  }
  p.lmax = 0;
  for (int64_t j = 0; j < p.nleaf; ++j) p.lmax = std::max(p.lmax, p.size[p.leaf0 + j]);

  // Chebyshev nodes of the first kind per cluster and axis; a flat axis is
  // widened for interpolation only
  int m = p.m;
  p.cheb.assign(p.nclu * 3 * m, 0.0);
  p.icen.assign(p.nclu * 3, 0.0);
  p.ihalf.assign(p.nclu * 3, 0.0);
  for (int64_t c = 0; c < p.nclu; ++c) {
    double ext[3], emax = 0;
    for (int d = 0; d < 3; ++d) { ext[d] = p.hi[3 * c + d] - p.lo[3 * c + d]; emax = std::max(emax, ext[d]); }
    for (int d = 0; d < 3; ++d) {
      double mid = 0.5 * (p.lo[3 * c + d] + p.hi[3 * c + d]);
      double hw = (ext[d] <= 1e-12 * emax) ? 1e-6 * emax : 0.5 * ext[d];
      p.icen[3 * c + d] = mid;
      p.ihalf[3 * c + d] = hw;
      for (int j = 0; j < m; ++j) p.cheb[(3 * c + d) * m + j] = mid + hw * std::cos((2 * j + 1) * kPi / (2.0 * m));
    }
  }

  // block tree, level by level: admissible pairs become far-field leaves,
  // other pairs are split into chil x chil until the leaf level
  std::vector<std::pair<int32_t, int32_t>> cur{{0, 0}}, nxt, adm, near;
  p.first_adm_level = D + 1;
  for (int l = 0; l <= D; ++l) {
    nxt.clear();
    for (auto &b : cur) {
      if (admissible_pair(p, b.first, b.second, eta)) {
        adm.push_back(b);
        p.first_adm_level = std::min(p.first_adm_level, l);
      } else if (l < D) {
        for (int i = 1; i <= 2; ++i)
          for (int j = 1; j <= 2; ++j) nxt.push_back({2 * b.first + i, 2 * b.second + j});
      } else {
        near.push_back(b);
      }
    }
    cur.swap(nxt);
  }
  std::sort(adm.begin(), adm.end());
  std::sort(near.begin(), near.end());
  p.adm_ptr.assign(p.nclu + 1, 0);
  p.adm_col.resize(adm.size());
  for (size_t i = 0; i < adm.size(); ++i) {
    p.adm_ptr[adm[i].first + 1]++;
    p.adm_col[i] = adm[i].second;
  }
  for (int64_t c = 0; c < p.nclu; ++c) p.adm_ptr[c + 1] += p.adm_ptr[c];
  p.near_ptr.assign(p.nleaf + 1, 0);
  p.near_col.resize(near.size());
  p.near_entries = 0;
  for (size_t i = 0; i < near.size(); ++i) {
    p.near_ptr[near[i].first - p.leaf0 + 1]++;
    p.near_col[i] = (int32_t)(near[i].second - p.leaf0);
    p.near_entries += p.size[near[i].first] * p.size[near[i].second];
  }
  for (int64_t j = 0; j < p.nleaf; ++j) p.near_ptr[j + 1] += p.near_ptr[j];

  if (!with_bases) return H2_OK;

  // leaf bases v_{i,nu} = int_{T_i} ell_nu, exact: collapsed Gauss rule with
  // enough points for total degree 3(m-1)
  int qv = (3 * (m - 1) + 3) / 2 + 1;
  std::vector<double> gx, gw;
  gauss_legendre01(qv, gx, gw);
  p.V.assign(nt * p.k, 0.0);
  const int k = p.k;
  parallel_for(p.nleaf, [&](int64_t j) {
    int64_t c = p.leaf0 + j;
    const double *zx = &p.cheb[(3 * c + 0) * m], *zy = &p.cheb[(3 * c + 1) * m], *zz = &p.cheb[(3 * c + 2) * m];
    std::vector<double> lx(m), ly(m), lz(m);
    for (int64_t r = p.first[c]; r < p.first[c] + p.size[c]; ++r) {
      int64_t t = p.perm[r];
      const double *A = &vert[3 * tri[3 * t]], *B = &vert[3 * tri[3 * t + 1]], *C = &vert[3 * tri[3 * t + 2]];
      double *row = &p.V[r * k];
      for (int a = 0; a < qv; ++a)
        for (int b = 0; b < qv; ++b) {
          double s = gx[a], tt = gx[a] * gx[b], wgt = 2.0 * p.area[t] * gw[a] * gw[b] * gx[a];
          double x[3];
          for (int d = 0; d < 3; ++d) x[d] = A[d] + s * (B[d] - A[d]) + tt * (C[d] - B[d]);
          for (int i = 0; i < m; ++i) {
            lx[i] = lag1(zx, m, i, x[0]);
            ly[i] = lag1(zy, m, i, x[1]);
            lz[i] = lag1(zz, m, i, x[2]);
          }
          for (int iz = 0; iz < m; ++iz)
            for (int iy = 0; iy < m; ++iy)
              for (int ix = 0; ix < m; ++ix) row[ix + m * (iy + m * iz)] += wgt * lx[ix] * ly[iy] * lz[iz];
        }
    }
  });

  // transfer factors: E_c = Ex (x) Ey (x) Ez with Ed[j'][j] = ell_{parent,d,j}(xi_{c,d,j'})
  p.Ef.assign(p.nclu * 3 * m * m, 0.0);
  for (int64_t c = 1; c < p.nclu; ++c) {
    int64_t par = (c - 1) / 2;
    for (int d = 0; d < 3; ++d)
      for (int jp = 0; jp < m; ++jp)
        for (int j = 0; j < m; ++j)
          p.Ef[((c * 3 + d) * m + jp) * m + j] = lag1(&p.cheb[(3 * par + d) * m], m, j, p.cheb[(3 * c + d) * m + jp]);
  }
  return H2_OK;
}

}  // namespace h2
