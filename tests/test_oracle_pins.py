"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: library
routines (numpy Gauss-Legendre, LAPACK), closed forms, invariants stated in
the paper (Definition 1, the partition of I x J, Eq. (10)), exactness on
polynomial kernels, brute-force assembly on tiny meshes and an independent
closed-form potential of a flat triangle.
"""
import numpy as np
import pytest

from oracle import KIND_POLY, Oracle, gauss01, pair_quad
from paper_2203_05665_gb300 import inputs as I


def _areas(v, f):
    return 0.5 * np.linalg.norm(np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]]), axis=1)


def _collapsed_rule(q):
    """Reference-triangle rule {0<=t<=s<=1}: (s, t) = (u, u v), weight u (numpy nodes)."""
    x, w = np.polynomial.legendre.leggauss(q)
    x = (x + 1) / 2
    w = w / 2
    s = np.repeat(x, q)
    t = s * np.tile(x, q)
    ww = np.repeat(w, q) * np.tile(w, q) * s
    return s, t, ww


def _ref_points(T, s, t):
    A, B, C = T
    return A[None, :] + s[:, None] * (B - A)[None, :] + t[:, None] * (C - B)[None, :]


@pytest.fixture(scope="module")
def l3():
    v, f = I.icosphere(3)
    return v, f, Oracle(v, f, leaf_size=32, eta=2.0, order=3)


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("n", [1, 2, 3, 6, 10, 20])
def test_gauss_matches_numpy(n):
    x, w = gauss01(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    o = np.argsort(x)
    assert np.allclose(x[o], (xr + 1) / 2, atol=1e-15, rtol=0)
    assert np.allclose(w[o], wr / 2, atol=1e-15, rtol=0)


TRI = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.3, 0.9, 0.0]])
TRI_EDGE = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.4, -0.8, 0.3]])   # shares (0,1) with TRI
TRI_VERT = np.array([[0.0, 0.0, 0.0], [-0.7, 0.2, 0.1], [-0.2, -0.9, 0.4]])  # shares vertex 0


@pytest.mark.parametrize("mode,T2", [(1, TRI), (2, TRI_EDGE), (3, TRI_VERT)])
def test_singular_maps_cover_product_domain(mode, T2):
    """For a smooth kernel the Sauter-Schwab maps must reproduce the plain
    tensor integral over T1 x T2: this checks region coverage and Jacobians."""
    m = 3
    exact = pair_quad(TRI, T2, 0, 8, KIND_POLY, m)   # exact: integrand polynomial
    # the transformed integrand is a polynomial of degree <= 19 per coordinate
    for q in (10, 12):
        assert abs(pair_quad(TRI, T2, mode, q, KIND_POLY, m) - exact) < 1e-13 * abs(exact)


@pytest.mark.parametrize("mode,T2", [(1, TRI), (2, TRI_EDGE), (3, TRI_VERT)])
def test_singular_quadrature_converges_exponentially(mode, T2):
    ref = pair_quad(TRI, T2, mode, 16)
    errs = [abs(pair_quad(TRI, T2, mode, q) - ref) for q in (2, 3, 4, 6, 8, 10)]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-11 * ref
    assert errs[1] < 2e-3 * ref           # the order-3 rule used in the matrix


def _triangle_potential(x, T):
    """int_T 1/|x-y| dy for a flat triangle, closed form (Wilton et al., IEEE TAP 1984)."""
    a, b, c = T
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n)
    d = float(np.dot(x - a, n))
    rho = x - d * n
    tot = 0.0
    for p, q in ((a, b), (b, c), (c, a)):
        l = (q - p) / np.linalg.norm(q - p)
        u = np.cross(l, n)
        lp, lm = np.dot(q - rho, l), np.dot(p - rho, l)
        t0 = np.dot(p - rho, u)
        Rp, Rm = np.linalg.norm(x - q), np.linalg.norm(x - p)
        if abs(t0) > 0:
            tot += t0 * np.log((Rp + lp) / (Rm + lm))
        if abs(d) > 0:
            r0 = t0 * t0 + d * d
            tot -= abs(d) * (np.arctan(t0 * lp / (r0 + abs(d) * Rp)) - np.arctan(t0 * lm / (r0 + abs(d) * Rm)))
    return tot


def _outer_integral(T1, T2, q, nsub):
    """int_{T1} potential_{T2}(x) dx with T1 refined nsub times, collapsed Gauss on each piece."""
    tris = [np.asarray(T1, float)]
    for _ in range(nsub):
        nxt = []
        for A, B, C in tris:
            ab, bc, ca = (A + B) / 2, (B + C) / 2, (C + A) / 2
            nxt += [np.array(t) for t in ((A, ab, ca), (B, bc, ab), (C, ca, bc), (ab, bc, ca))]
        tris = nxt
    s, t, w = _collapsed_rule(q)
    tot = 0.0
    for T in tris:
        ar = 0.5 * np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0]))
        pts = _ref_points(T, s, t)
        tot += 2 * ar * sum(wi * _triangle_potential(p, T2) for wi, p in zip(w, pts))
    return tot / (4 * np.pi)


def test_triangle_potential_closed_form_far_point():
    x = np.array([0.2, 0.5, 1.5])
    s, t, w = _collapsed_rule(20)
    pts = _ref_points(TRI, s, t)
    ar = 0.5 * np.linalg.norm(np.cross(TRI[1] - TRI[0], TRI[2] - TRI[0]))
    brute = 2 * ar * np.sum(w / np.linalg.norm(pts - x, axis=1))
    assert abs(_triangle_potential(x, TRI) - brute) < 1e-13


@pytest.mark.parametrize("mode,T2", [(1, TRI), (2, TRI_EDGE), (3, TRI_VERT)])
def test_singular_entries_match_closed_form_potential(mode, T2):
    """g_ij by Sauter-Schwab (q=12) against an outer rule over the closed-form
    inner potential; Richardson extrapolation in the refinement level."""
    ar = lambda T: 0.5 * np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0]))
    # pair_quad integrates 1/(4 pi r) over the reference domains; 4|T1||T2| is the Jacobian
    ss = 4 * ar(TRI) * ar(T2) * pair_quad(TRI, T2, mode, 12)
    a2 = _outer_integral(TRI, T2, 8, 2)
    a3 = _outer_integral(TRI, T2, 8, 3)
    extrap = a3 + (a3 - a2) / 3.0      # the outer rule converges like h^2 near the shared set
    assert abs(a3 - ss) < 2e-6 * ss
    assert abs(extrap - ss) < 1e-7 * ss


def _mesh_pairs(f, i):
    """Partners of triangle i by the number of shared vertex ids: (3: i itself, 2: the
    edge neighbours, 1: the vertex neighbours)."""
    sets = [set(t) for t in f.tolist()]
    out = {3: [i], 2: [], 1: []}
    for j, sj in enumerate(sets):
        k = len(sets[i] & sj)
        if j != i and k in (1, 2):
            out[k].append(j)
    return out


@pytest.mark.parametrize("i", [0, 77, 203])
def test_mesh_pair_classifier_against_closed_form(i):
    """The oracle classifies every pair of mesh triangles as identical, common edge,
    common vertex or regular from shared global vertex ids and reorders their
    vertices before the Sauter-Schwab maps.  Here oracle.entry(i, j) for real
    icosphere pairs of every kind, every local position of the shared edge or
    vertex and both index orders, is checked against the outer rule over the
    closed-form inner potential of the triangles as the mesh stores them, which
    involves neither the classification nor the reordering."""
    v, f = I.icosphere(2)
    o = Oracle(v, f, leaf_size=8, eta=2.0, order=2, store_near=False)
    part = _mesh_pairs(f, i)
    assert len(part[2]) == 3 and len(part[1]) >= 6
    # all three edges, and vertex neighbours around every corner of triangle i
    corners = {}
    for j in part[1]:
        shared = (set(f[i].tolist()) & set(f[j].tolist())).pop()
        corners.setdefault(int(np.where(f[i] == shared)[0][0]), j)
    assert len(corners) == 3
    pairs = [(i, i)] + [(i, j) for j in part[2]] + [(i, j) for j in corners.values()]
    pairs += [(j, i) for j in part[2][:1]] + [(j, i) for j in list(corners.values())[:1]]
    for a, b in pairs:
        g = o.entry(int(a), int(b), 12)
        Ta, Tb = v[f[a]], v[f[b]]
        a2 = _outer_integral(Ta, Tb, 8, 2)
        a3 = _outer_integral(Ta, Tb, 8, 3)
        extrap = a3 + (a3 - a2) / 3.0
        assert abs(extrap - g) < 2e-7 * g, (a, b, g, extrap)
    # a regular pair next to i (no shared vertex) takes the plain rule: same check
    near = np.argsort(np.linalg.norm(v[f].mean(axis=1) - v[f[i]].mean(axis=0), axis=1))
    j = next(int(j) for j in near if not set(f[j].tolist()) & set(f[i].tolist()))
    g = o.entry(int(i), j, 12)
    assert abs(_outer_integral(v[f[i]], v[f[j]], 8, 1) - g) < 1e-9 * g


# ---------------------------------------------------------------- trees
def test_cluster_tree_definition_1(l3):
    v, f, o = l3
    tr = o.tree()
    n = f.shape[0]
    D = o.depth
    assert sorted(tr["idx"]) == list(range(n))
    assert tr["first"][0] == 0 and tr["size"][0] == n           # root holds I
    for c in range(o.nclu):
        sl = tr["idx"][tr["first"][c]:tr["first"][c] + tr["size"][c]]
        pv = v[f[sl].reshape(-1)]
        assert np.all(pv >= tr["lo"][c]) and np.all(pv <= tr["hi"][c])   # supports inside the box
        assert np.allclose(pv.min(axis=0), tr["lo"][c]) and np.allclose(pv.max(axis=0), tr["hi"][c])
        lev = int(np.floor(np.log2(c + 1)))
        if lev < D:
            c0, c1 = 2 * c + 1, 2 * c + 2
            assert tr["first"][c0] == tr["first"][c]
            assert tr["first"][c1] == tr["first"][c0] + tr["size"][c0]
            assert tr["size"][c0] + tr["size"][c1] == tr["size"][c]          # disjoint union
            assert abs(tr["size"][c0] - tr["size"][c1]) <= 1
            assert np.all(tr["lo"][c0] >= tr["lo"][c]) and np.all(tr["hi"][c0] <= tr["hi"][c])
    assert D == int(np.ceil(np.log2(n / 32)))
    assert np.all(tr["size"][2 ** D - 1:] <= 32)


def _assemble_cover(o, n, tr):
    cover = np.zeros((n, n), dtype=np.int32)
    t, s, adm = o.blocks()
    for tt, ss in zip(t, s):
        rows = tr["idx"][tr["first"][tt]:tr["first"][tt] + tr["size"][tt]]
        cols = tr["idx"][tr["first"][ss]:tr["first"][ss] + tr["size"][ss]]
        cover[np.ix_(rows, cols)] += 1
    return cover, t, s, adm


@pytest.mark.parametrize("L,leaf,eta", [(2, 8, 2.0), (3, 32, 2.0), (3, 16, 1.0)])
def test_block_tree_partitions_index_pairs(L, leaf, eta):
    v, f = I.icosphere(L)
    o = Oracle(v, f, leaf_size=leaf, eta=eta, order=2, store_near=False, with_bases=False)
    tr = o.tree()
    cover, t, s, adm = _assemble_cover(o, f.shape[0], tr)
    assert np.all(cover == 1)                           # every (i,j) in exactly one leaf block
    blocks = {(a, b): c for a, b, c in zip(t, s, adm)}
    assert all(blocks.get((b, a)) == c for (a, b), c in blocks.items())    # symmetric
    lev = lambda c: int(np.floor(np.log2(c + 1)))
    assert all(lev(a) == lev(b) for a, b in blocks)
    # admissible blocks satisfy Eq. (8); inadmissible ones are leaf x leaf
    for (a, b), c in blocks.items():
        da = np.linalg.norm(tr["hi"][a] - tr["lo"][a])
        db = np.linalg.norm(tr["hi"][b] - tr["lo"][b])
        gap = np.maximum(0, np.maximum(tr["lo"][a] - tr["hi"][b], tr["lo"][b] - tr["hi"][a]))
        if c:
            assert max(da, db) <= 2 * eta * np.linalg.norm(gap)
        else:
            assert lev(a) == o.depth and not max(da, db) <= 2 * eta * np.linalg.norm(gap)


# ---------------------------------------------------------------- interpolation, V, E, S
def test_lagrange_partition_of_unity_and_nodal(l3):
    _, _, o = l3
    tr = o.tree()
    rng = np.random.default_rng(3)
    for c in (0, 5, o.nclu - 1):
        x = tr["lo"][c] + rng.uniform(size=(40, 3)) * (tr["hi"][c] - tr["lo"][c])
        tot = sum(o.lagrange(c, nu, x) for nu in range(o.k))
        assert np.allclose(tot, 1.0, atol=1e-13)
        m = o.m
        for nu in range(o.k):
            xi = np.array([[tr["pts"][c, 0, mu % m], tr["pts"][c, 1, (mu // m) % m], tr["pts"][c, 2, mu // (m * m)]]
                           for mu in range(o.k)])
            assert np.allclose(o.lagrange(c, nu, xi), np.eye(o.k)[nu], atol=1e-12)
        # Chebyshev nodes of the first kind on the box
        j = np.arange(m)
        ref = (tr["lo"][c][:, None] + tr["hi"][c][:, None]) / 2 + \
              (tr["hi"][c][:, None] - tr["lo"][c][:, None]) / 2 * np.cos((2 * j + 1) * np.pi / (2 * m))[None, :]
        assert np.allclose(tr["pts"][c], ref, atol=1e-15)


def _direct_V(o, c, v, f, tr, q=8):
    """V_c by a numpy quadrature of the oracle's Lagrange polynomials, Eq. (6a)."""
    rows = tr["idx"][tr["first"][c]:tr["first"][c] + tr["size"][c]]
    s, t, w = _collapsed_rule(q)
    out = np.zeros((rows.size, o.k))
    for r, tri in enumerate(rows):
        T = v[f[tri]]
        ar = 0.5 * np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0]))
        pts = _ref_points(T, s, t)
        for nu in range(o.k):
            out[r, nu] = 2 * ar * np.sum(w * o.lagrange(c, nu, pts))
    return out


def test_leaf_basis_rows_sum_to_area_and_nested_identity(l3):
    v, f, o = l3
    tr = o.tree()
    V = o.V()
    areas = _areas(v, f)[tr["idx"]]
    assert np.allclose(V.sum(axis=1), areas, rtol=1e-13)              # sum_nu ell_nu = 1
    leaf0 = 2 ** o.depth - 1
    # leaf rows match a direct quadrature with more points (exactness of q_V)
    for c in (leaf0, leaf0 + 17):
        assert np.allclose(V[tr["first"][c]:tr["first"][c] + tr["size"][c]], _direct_V(o, c, v, f, tr),
                           rtol=0, atol=1e-15)
    # Eq. (10): V_parent restricted to a child's rows equals V_child E_child
    for c in (leaf0 + 3, leaf0 + 8):
        par = (c - 1) // 2
        Vp = _direct_V(o, par, v, f, tr)
        off = tr["first"][c] - tr["first"][par]
        Vc = V[tr["first"][c]:tr["first"][c] + tr["size"][c]]
        assert np.allclose(Vp[off:off + tr["size"][c]], Vc @ o.E(c), rtol=0, atol=1e-14)
    # and one level higher, through two transfer matrices
    c = leaf0 + 5
    par, gp = (c - 1) // 2, (((c - 1) // 2) - 1) // 2
    Vg = _direct_V(o, gp, v, f, tr)
    off = tr["first"][c] - tr["first"][gp]
    Vc = V[tr["first"][c]:tr["first"][c] + tr["size"][c]]
    assert np.allclose(Vg[off:off + tr["size"][c]], Vc @ o.E(c) @ o.E(par), rtol=0, atol=1e-14)


def test_transfer_rows_sum_to_one(l3):
    _, _, o = l3
    for c in (1, 2, 9, o.nclu - 1):
        assert np.allclose(o.E(c).sum(axis=1), 1.0, atol=1e-13)


def test_coupling_symmetry_and_kernel(l3):
    _, _, o = l3
    t, s, adm = o.blocks()
    tr = o.tree()
    b = np.flatnonzero(adm)[7]
    S1 = o.S(t[b], s[b])
    S2 = o.S(s[b], t[b])
    assert np.array_equal(S1, S2.T)
    m = o.m
    pt = lambda c, nu: np.array([tr["pts"][c, 0, nu % m], tr["pts"][c, 1, (nu // m) % m], tr["pts"][c, 2, nu // m // m]])
    assert np.isclose(S1[4, 11], 1 / (4 * np.pi * np.linalg.norm(pt(t[b], 4) - pt(s[b], 11))), rtol=1e-15)


# ---------------------------------------------------------------- the Galerkin matrix
@pytest.fixture(scope="module")
def dense_l3(l3):
    _, _, o = l3
    return o.dense()


def test_dense_galerkin_symmetric_positive_definite(dense_l3):
    G = dense_l3
    assert np.array_equal(G, G.T)
    np.linalg.cholesky(G)                    # single layer is coercive in 3-D


def test_constant_density_on_unit_sphere():
    """The single-layer potential of unit density on the unit sphere is 1, so
    (G 1)_i -> area_i with an O(h^2)-decreasing error on the icosphere."""
    errs = []
    for L in (1, 2, 3):
        v, f = I.icosphere(L)
        o = Oracle(v, f, leaf_size=16, eta=2.0, order=4)
        a = _areas(v, f)
        y = o.matvec(np.ones((f.shape[0], 1)))[:, 0]
        errs.append(np.linalg.norm(y - a) / np.linalg.norm(a))
    assert errs[0] < 0.05 and errs[-1] < 3e-3
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3


def test_h2_error_falls_with_order(l3, dense_l3):
    v, f, _ = l3
    x = I.uniform_rhs(f.shape[0], 2, 5)
    yd = dense_l3 @ x
    errs = []
    for m in (1, 2, 3, 4, 5):
        o = Oracle(v, f, leaf_size=16, eta=2.0, order=m)
        errs.append(np.linalg.norm(o.matvec(x) - yd) / np.linalg.norm(yd))
    assert all(b < a / 2.5 for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 5e-4


@pytest.mark.parametrize("m,L,leaf", [(2, 3, 16), (3, 3, 16), (4, 2, 8)])
def test_h2_exact_for_polynomial_kernel(m, L, leaf):
    """A kernel of per-axis degree <= m-1 is reproduced exactly by order-m
    interpolation (Eq. (4)), so G~ x must equal G x to round-off: this pins
    V, E, S, the block tree and Algorithms 1-3 together."""
    v, f = I.icosphere(L)
    o = Oracle(v, f, leaf_size=leaf, eta=1.0, order=m, kind=KIND_POLY)
    assert o.nadm > 1000
    x = I.uniform_rhs(f.shape[0], 3, 11)
    yd = o.dense() @ x
    assert np.linalg.norm(o.matvec(x) - yd) <= 1e-13 * np.linalg.norm(yd)


@pytest.mark.parametrize("L,leaf,eta,m", [(1, 4, 1.0, 2), (1, 6, 3.0, 3), (2, 8, 2.0, 2)])
def test_h2_matvec_equals_blockwise_assembly(L, leaf, eta, m):
    """Brute force on tiny meshes: form G~ block by block from Eq. (7) with
    directly computed V_tau (no transfer matrices) and nearfield entries,
    then compare with the oracle's recursive Algorithms 1-3 column by column."""
    v, f = I.icosphere(L)
    n = f.shape[0]
    o = Oracle(v, f, leaf_size=leaf, eta=eta, order=m)
    tr = o.tree()
    G = o.dense()
    Gt = np.zeros((n, n))
    t, s, adm = o.blocks()
    Vd = {}
    for tt, ss, a in zip(t, s, adm):
        rows = tr["idx"][tr["first"][tt]:tr["first"][tt] + tr["size"][tt]]
        cols = tr["idx"][tr["first"][ss]:tr["first"][ss] + tr["size"][ss]]
        if a:
            for c in (tt, ss):
                if c not in Vd:
                    Vd[c] = _direct_V(o, c, v, f, tr)
            Gt[np.ix_(rows, cols)] = Vd[tt] @ o.S(tt, ss) @ Vd[ss].T
        else:
            Gt[np.ix_(rows, cols)] = G[np.ix_(rows, cols)]
    assert adm.any() and (~adm).any()
    cols = o.matvec(np.eye(n))
    assert np.allclose(cols, Gt, rtol=0, atol=1e-13 * np.abs(Gt).max())


def test_matvec_rows_agree_with_full_matvec(l3):
    _, f, o = l3
    x = I.uniform_rhs(f.shape[0], 3, 2)
    y = o.matvec(x)
    rows = np.array([0, 7, 100, 555, f.shape[0] - 1])
    assert np.allclose(o.matvec_rows(x, rows), y[rows], rtol=0, atol=1e-14 * np.abs(y).max())


def test_coefficients_are_nested_forward_transform(l3):
    """x^_c after Algorithm 1 equals V_c^T x|c computed directly (Eq. (10))."""
    v, f, o = l3
    tr = o.tree()
    x = I.uniform_rhs(f.shape[0], 2, 4)
    _, xh, _ = o.matvec(x, coeffs=True)
    for c in (0, 3, 20):
        rows = tr["idx"][tr["first"][c]:tr["first"][c] + tr["size"][c]]
        assert np.allclose(xh[c], _direct_V(o, c, v, f, tr).T @ x[rows], rtol=0, atol=1e-13)


# ---------------------------------------------------------------- GMRES
def test_gmres_matches_dense_solve_of_h2_matrix():
    v, f = I.icosphere(2)
    n = f.shape[0]
    o = Oracle(v, f, leaf_size=16, eta=2.0, order=3)
    Gt = o.matvec(np.eye(n))
    b = I.uniform_rhs(n, 2, 9)
    z, it, rel = o.gmres(b, rtol=1e-10, restart=30, maxit=2000)
    zs = np.linalg.solve(Gt, b)
    kappa = np.linalg.cond(Gt)
    assert np.all(rel <= 1e-10)
    assert np.all(np.linalg.norm(Gt @ z - b, axis=0) / np.linalg.norm(b, axis=0) <= 1e-10)
    assert np.linalg.norm(z - zs) <= kappa * 1e-10 * np.linalg.norm(zs)
    assert np.all(it > 0)


def test_gmres_constant_density_solution_is_one():
    v, f = I.icosphere(3)
    o = Oracle(v, f, leaf_size=32, eta=2.0, order=3)
    b = _areas(v, f)[:, None]
    z, it, rel = o.gmres(b, rtol=1e-8)
    assert rel[0] <= 1e-8
    # z -> 1 as h -> 0; at level 3 the discretisation error is a few percent
    assert abs(np.dot(b[:, 0], z[:, 0]) / b.sum() - 1.0) < 1e-2
    assert np.abs(z[:, 0] - 1.0).max() < 0.1
