"""Pins of the oracle's GCA-H^2 matrix (Section 3's GCA-H^2 example: pivot
elements per cluster, nested through the sons' pivots, the coupling
S_{tau sigma} = G on the pivot pairs), against things other than the oracle
itself:

* the boundary quadrature of the auxiliary box: its total weight is the
  box's surface area, the weighted normals cancel, the flux of a point source
  is -1 inside and 0 outside (Gauss's law), and Green's representation
  formula reproduces g(x, y) (closed forms of potential theory);
* the cross approximation: a rank-r matrix is recovered with exactly r
  pivots, the first pivot is the largest modulus, ties go to the first entry
  in row-major order, the interpolation rows are unit vectors, and the
  stopping rule holds (numpy recomputes the residual from the pivots);
* the whole matrix: with eps = 0 every admissible block of a small mesh has
  full rank and the product equals the dense Galerkin matrix; a brute-force
  numpy assembly of near + V_t S V_s^T from the exported pivots, bases and
  transfer matrices equals the oracle's product (Algorithms 1-3); the error
  against the dense Galerkin matrix follows eps; structural invariants."""
import numpy as np
import pytest

import oracle
from paper_2203_05665_gb300 import inputs as I


def _g(x, z):
    return 1.0 / (4 * np.pi * np.linalg.norm(x - z, axis=-1))


def _dn(x, z, n):
    d = x - z
    return np.sum(n * d, axis=-1) / (4 * np.pi * np.linalg.norm(d, axis=-1) ** 3)


LO, HI = np.array([0.1, -0.3, 0.2]), np.array([0.6, 0.1, 0.35])


def test_green_rule_area_and_normals():
    for gamma in (0.5, 1.0):
        Z, N, W = oracle.green_rule(LO, HI, gamma, 3)
        rho = 0.5 * np.linalg.norm(HI - LO)
        a, b, c = HI - LO + 2 * gamma * rho
        assert W.shape == (54,)
        assert abs(W.sum() - 2 * (a * b + b * c + c * a)) < 1e-13
        assert np.abs((W[:, None] * N).sum(axis=0)).max() < 1e-14
        assert np.all(np.abs(N).sum(axis=1) == 1.0)
        # every point lies on the face its normal names
        olo, ohi = LO - gamma * rho, HI + gamma * rho
        ax = np.abs(N).argmax(axis=1)
        side = np.where(N[np.arange(len(N)), ax] > 0, ohi[ax], olo[ax])
        assert np.allclose(Z[np.arange(len(Z)), ax], side, atol=0, rtol=0)
        assert np.all(Z >= olo - 1e-15) and np.all(Z <= ohi + 1e-15)


def test_green_rule_gauss_law():
    Z, N, W = oracle.green_rule(LO, HI, 1.0, 16)
    inside = np.array([0.3, -0.1, 0.3])
    outside = np.array([3.0, 2.0, -1.0])
    assert abs(np.sum(W * _dn(inside, Z, N)) + 1.0) < 1e-6
    assert abs(np.sum(W * _dn(outside, Z, N))) < 1e-10


@pytest.mark.parametrize("gamma", [0.5, 1.0])
def test_green_representation_formula(gamma):
    """g(x, y) = int [g(x, z) dg(z, y)/dn - dg(x, z)/dn_z g(z, y)] dz for x in
    the box and y outside the auxiliary box; the rule converges."""
    x = np.array([0.35, -0.05, 0.28])
    y = np.array([4.0, -2.0, 3.0])
    errs = []
    for qg in (2, 4, 8, 12, 16, 20):
        Z, N, W = oracle.green_rule(LO, HI, gamma, qg)
        val = np.sum(W * (_g(x, Z) * _dn(y, Z, N) - _dn(x, Z, N) * _g(Z, y)))
        errs.append(abs(val - _g(x, y)) / _g(x, y))
    assert errs[-1] < 1e-9
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_aca_recovers_low_rank_exactly():
    rng = np.random.default_rng(3)
    M = rng.standard_normal((30, 3)) @ rng.standard_normal((3, 50))
    Ii, J, Vh = oracle.aca(M, 1e-13)
    assert len(Ii) == 3 and len(set(Ii)) == 3 and len(set(J)) == 3
    assert np.abs(M - Vh @ M[Ii, :]).max() < 1e-12 * np.abs(M).max()
    # complete pivoting: the first pivot is the largest modulus
    i0, j0 = np.unravel_index(np.argmax(np.abs(M)), M.shape)
    assert (Ii[0], J[0]) == (i0, j0)
    assert np.array_equal(Vh[Ii], np.eye(3))
    # the rank cap stops the approximation early
    Ii2, J2, Vh2 = oracle.aca(M, 1e-13, max_rank=2)
    assert len(Ii2) == 2 and np.array_equal(Ii2, Ii[:2]) and np.array_equal(J2, J[:2])


def test_aca_ties_and_stopping_rule():
    M = np.array([[1.0, 2.0, -2.0], [2.0, 0.5, 1.0]])
    Ii, J, Vh = oracle.aca(M, 0.0)
    assert (Ii[0], J[0]) == (0, 1)          # |2| three times: the first in row-major order wins
    # a smooth kernel matrix: singular values decay, the rank follows eps
    xs, ys = np.linspace(0, 1, 40), np.linspace(3, 4, 60)
    K = 1.0 / np.abs(xs[:, None] - ys[None, :])
    for eps in (1e-2, 1e-5, 1e-9):
        Ii, J, Vh = oracle.aca(K, eps)
        k = len(Ii)
        R = K - Vh @ K[Ii, :]
        assert np.abs(R).max() <= eps * np.abs(K).max() * (1 + 1e-6)
        # one pivot fewer leaves a residual above the threshold
        Ik, Jk = Ii[:k - 1], J[:k - 1]
        Rk = K - K[:, Jk] @ np.linalg.solve(K[np.ix_(Ik, Jk)], K[Ik, :]) if k > 1 else K
        assert np.abs(Rk).max() > eps * np.abs(K).max()
        assert np.array_equal(Vh[Ii], np.eye(k))
        ref = np.linalg.solve(K[np.ix_(Ii, J)].T, K[:, J].T).T
        assert np.abs(Vh - ref).max() < 1e-6 * max(1.0, np.abs(ref).max())


def _assemble(g):
    """Dense G~ from the exported pivots, leaf bases, transfer matrices and
    coupling matrices (full bases built recursively), the nearfield taken
    from the dense Galerkin matrix."""
    tr = g.tree()
    idx, first, size = tr["idx"], tr["first"], tr["size"]
    n, D = g.n, g.depth
    leaf0 = (1 << D) - 1
    G = g.dense()
    basis = {}

    def full(c):
        if c not in basis:
            if c >= leaf0:
                B = np.zeros((n, g.rank[c]))
                B[idx[first[c]:first[c] + size[c]], :] = g.V(c, int(size[c]))
            else:
                B = full(2 * c + 1) @ g.E(2 * c + 1) + full(2 * c + 2) @ g.E(2 * c + 2)
            basis[c] = B
        return basis[c]

    Gt = np.zeros((n, n))
    t, s, a = g.blocks()
    for bt, bs, adm in zip(t, s, a):
        it, js = idx[first[bt]:first[bt] + size[bt]], idx[first[bs]:first[bs] + size[bs]]
        if adm:
            Gt[np.ix_(it, js)] = full(bt)[it] @ g.S(bt, bs) @ full(bs)[js].T
        else:
            Gt[np.ix_(it, js)] = G[np.ix_(it, js)]
    return Gt, G


def test_eps_zero_is_the_galerkin_matrix():
    v, f = I.icosphere(2)
    g = oracle.GcaOracle(v, f, leaf_size=32, eps=0.0, max_rank=0)
    t, s, a = g.blocks()
    tr = g.tree()
    for bt in set(t[a]):
        assert g.rank[bt] == tr["size"][bt]       # full rank in every admissible block
    x = I.uniform_rhs(g.n, 3, 11)
    G = g.dense()
    assert np.linalg.norm(g.matvec(x) - G @ x) / np.linalg.norm(G @ x) < 1e-13


@pytest.mark.parametrize("mesh", ["ico3", "cube4"])
def test_product_equals_brute_force_assembly(mesh):
    v, f = I.icosphere(3) if mesh == "ico3" else I.cube(4)
    g = oracle.GcaOracle(v, f, leaf_size=16, eps=1e-4)
    Gt, G = _assemble(g)
    x = I.uniform_rhs(g.n, 2, 12)
    y = g.matvec(x)
    assert np.linalg.norm(y - Gt @ x) / np.linalg.norm(Gt @ x) < 1e-13
    rows = np.array([0, 5, g.n // 2, g.n - 1])
    assert np.abs(g.matvec_rows(x, rows) - y[rows]).max() < 1e-14 * np.abs(y).max()


def test_error_follows_eps():
    v, f = I.icosphere(3)
    errs = []
    G = None
    x = I.uniform_rhs(f.shape[0], 2, 13)
    for eps in (1e-2, 1e-3, 1e-4, 1e-5):
        g = oracle.GcaOracle(v, f, leaf_size=16, eps=eps)
        if G is None:
            G = g.dense()
        err = np.linalg.norm(g.matvec(x) - G @ x) / np.linalg.norm(G @ x)
        assert err < 2.0 * eps
        errs.append(err)
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_structure():
    v, f = I.cube(5)
    g = oracle.GcaOracle(v, f, leaf_size=16, eps=1e-4)
    tr = g.tree()
    idx, first, size = tr["idx"], tr["first"], tr["size"]
    leaf0 = (1 << g.depth) - 1
    for c in range(g.nclu):
        p = g.pivots(c)
        assert len(set(p)) == len(p) == g.rank[c] >= 1
        assert set(p) <= set(idx[first[c]:first[c] + size[c]])
        if c < leaf0:
            cand = list(g.pivots(2 * c + 1)) + list(g.pivots(2 * c + 2))
            assert set(p) <= set(cand)
            assert g.rank[c] <= min(len(cand), 2 * 6 * 4 * 4)
            # the sons' transfer rows at pivots the parent kept are unit vectors
            for son in (2 * c + 1, 2 * c + 2):
                Es = g.E(son)
                for r, tri in enumerate(g.pivots(son)):
                    if tri in p:
                        e = np.zeros(g.rank[c])
                        e[list(p).index(tri)] = 1.0
                        assert np.array_equal(Es[r], e)
        else:
            Vc = g.V(c, int(size[c]))
            rows = list(idx[first[c]:first[c] + size[c]])
            for a_, tri in enumerate(p):
                e = np.zeros(g.rank[c])
                e[a_] = 1.0
                assert np.array_equal(Vc[rows.index(tri)], e)
    t, s, a = g.blocks()
    for bt, bs in list(zip(t[a], s[a]))[:50]:
        assert np.array_equal(g.S(bt, bs), g.S(bs, bt).T)
        assert g.S(bt, bs)[0, 0] == g.entry(g.pivots(bt)[0], g.pivots(bs)[0])
