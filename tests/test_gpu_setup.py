"""The device set-up entry by entry: the nearfield blocks (Eq. (3), Sauter-Schwab
quadrature), the coupling matrices (Eq. (6c)), the leaf bases (Eq. (6a)) and the
transfer factors (Eq. (9)) that h2_build stores on the GPU, read back through
h2_export and compared with the oracle element by element."""
import numpy as np
import pytest

import oracle
from paper_2203_05665_gb300 import H2Matrix, Plan, inputs as I

pytestmark = pytest.mark.gpu

CASES = {
    "ico3_m4": (lambda: I.icosphere(3), 32, 2.0, 4),
    "cube7_m2": (lambda: I.cube(7), 16, 2.0, 2),        # ragged leaves, flat boxes
    "ell3_m3": (lambda: I.ellipsoid(3, (2.0, 1.0, 0.5)), 24, 1.5, 3),
}
_cache = {}


def _setup(name):
    if name not in _cache:
        make, leaf, eta, m = CASES[name]
        v, f = make()
        o = oracle.Oracle(v, f, leaf_size=leaf, eta=eta, order=m)
        p = Plan(v, f, leaf_size=leaf, eta=eta, order=m)
        _cache[name] = (v, f, o, p, o.dense())
    return _cache[name]


def _leaf_rows(tree, c, L):
    """Triangle of every leaf-local row of cluster c (-1 for padding)."""
    rows = -np.ones(L, dtype=np.int64)
    sz = tree["size"][c]
    rows[:sz] = tree["perm"][tree["first"][c]:tree["first"][c] + sz]
    return rows


# relative tolerance per stored entry: FP64 storage and double-float (48 bits) well
# below 1e-13; rounded storage: the unit roundoff of the format (2^-24, 2^-8, 2^-11) (with room for the 1e-15
# by which the two FP64 quadratures differ before rounding)
ENTRY_TOL = {"f64n": 1e-13, "f64": 1e-13, "f32": 2 ** -24 * 1.001, "bf16": 2 ** -8 * 1.001, "f16": 2 ** -11 * 1.001}


@pytest.mark.parametrize("prec", ["f64n", "f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_every_nearfield_entry(require_gpu, name, prec):
    make, leaf, eta, m = CASES[name]
    v, f, o, p, G = _setup(name)
    h = H2Matrix(v, f, leaf_size=leaf, eta=eta, order=m, prec=prec)
    L = h.stats["leaf_max"]
    near = h.export("near")
    tr = p.tree()
    _, (nt, ns) = p.blocks()
    assert near.shape[0] == len(nt) == o.nnear
    worst = 0.0
    for b in range(len(nt)):
        rt, rs = _leaf_rows(tr, nt[b], L), _leaf_rows(tr, ns[b], L)
        ref = np.zeros((L, L))
        vt, vs = rt >= 0, rs >= 0
        ref[np.ix_(vt, vs)] = G[np.ix_(rt[vt], rs[vs])]
        # padding stays zero; every real entry within its storage precision
        assert np.all(near[b][~vt, :] == 0) and np.all(near[b][:, ~vs] == 0)
        tol = ENTRY_TOL[prec]
        if prec == "bf16" and nt[b] == ns[b]:
            tol = 2 ** -24 * 1.001    # the self blocks of bfloat16 handles are held in FP32
        err = np.abs(near[b] - ref)[np.ix_(vt, vs)] / np.abs(ref[np.ix_(vt, vs)])
        worst = max(worst, err.max())
        assert err.max() <= tol, (b, err.max())
    h.close()


@pytest.mark.parametrize("prec", ["f64n", "f64", "f32"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_coupling_bases_and_transfer(require_gpu, name, prec):
    make, leaf, eta, m = CASES[name]
    v, f, o, p, _ = _setup(name)
    h = H2Matrix(v, f, leaf_size=leaf, eta=eta, order=m, prec=prec, coupling="stored")
    k, L = m ** 3, h.stats["leaf_max"]
    tol = {"f64n": 1e-13, "f64": 1e-13, "f32": 2 ** -24}[prec]
    (at, as_), _ = p.blocks()
    rng = np.random.default_rng(12)
    pick = np.unique(np.concatenate([[0, len(at) - 1], rng.choice(len(at), min(64, len(at)), replace=False)]))
    for b in pick:
        S = h.export("coupling", int(b), 1)[0]
        ref = o.S(int(at[b]), int(as_[b]))
        assert np.abs(S - ref).max() <= tol * np.abs(ref).max() * 2, (b,)
    # leaf bases in padded cluster order against the oracle's V (rows by triangle)
    Vd = h.export("V")
    tr = p.tree()
    Vo = o.V()
    depth = h.stats["depth"]
    for j in range(2 ** depth):
        rows = _leaf_rows(tr, 2 ** depth - 1 + j, L)
        blk = Vd[j * L:(j + 1) * L]
        assert np.all(blk[rows < 0] == 0)
        real = rows >= 0
        # the oracle's V is in cluster order as well (row p = DoF p of its tree)
        first = tr["first"][2 ** depth - 1 + j]
        ref = Vo[first:first + real.sum()]
        assert np.abs(blk[real] - ref).max() <= tol * np.abs(Vo).max() * 4
    # transfer factors: E_c = E_x (x) E_y (x) E_z against the oracle's explicit k x k
    E = h.export("E")
    for c in (1, 2, h.stats["clusters"] // 2, h.stats["clusters"] - 1):
        Ek = np.kron(E[c, 2], np.kron(E[c, 1], E[c, 0]))
        assert np.abs(Ek - o.E(c)).max() <= tol * 8
    h.close()


def test_full_size_nearfield_and_coupling_samples(require_gpu):
    """Icosphere level 7 (327,680 triangles), m = 4, as the benchmark builds it:
    sampled nearfield blocks against oracle.entry one by one, sampled coupling
    matrices against oracle.S."""
    v, f = I.icosphere(7)
    h = H2Matrix(v, f, leaf_size=32, eta=2.0, order=4, prec="f64n")
    p = Plan(v, f, leaf_size=32, eta=2.0, order=4)
    o = oracle.Oracle(v, f, leaf_size=32, eta=2.0, order=4, store_near=False, with_bases=False)
    tr = p.tree()
    (at, as_), (nt, ns) = p.blocks()
    L = h.stats["leaf_max"]
    rng = np.random.default_rng(13)
    for b in rng.choice(len(nt), 24, replace=False):
        blk = h.export("near", int(b), 1)[0]
        rt, rs = _leaf_rows(tr, nt[b], L), _leaf_rows(tr, ns[b], L)
        for t in range(L):
            for c in range(L):
                if rt[t] >= 0 and rs[c] >= 0:
                    g = o.entry(int(rt[t]), int(rs[c]))
                    assert abs(blk[t, c] - g) <= 1e-13 * abs(g), (b, t, c)
    for b in rng.choice(len(at), 24, replace=False):
        S = h.export("coupling", int(b), 1)[0]
        ref = o.S(int(at[b]), int(as_[b]))
        assert np.abs(S - ref).max() <= 1e-13 * np.abs(ref).max()
    h.close()
