"""Host-side checks of libh2 that need no GPU: exported symbols, argument
validation and the planning step (trees, blocks, V, transfer factors)
against the oracle, which is an independent implementation."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2203_05665_gb300 as pkg
from oracle import Oracle
from paper_2203_05665_gb300 import Plan, inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session", autouse=True)
def built():
    pkg.build_library()
    pkg.load()


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "h2.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    declared = set(re.findall(r"\b(h2_[a-z_0-9]+)\s*\(", hdr))
    assert declared == set(pkg.EXPORTED)
    lib = C.CDLL(pkg.library_path())
    for name in declared:
        assert hasattr(lib, name), name


MESHES = {
    "ico3": (lambda: I.icosphere(3), 32, 2.0, 3),
    "ico4": (lambda: I.icosphere(4), 32, 2.0, 3),
    "cube7": (lambda: I.cube(7), 16, 2.0, 2),            # 588 triangles: ragged leaves (18/19)
    "ell3": (lambda: I.ellipsoid(3, (2.0, 1.0, 0.5)), 24, 1.5, 4),
    "cube5_flat": (lambda: I.cube(5), 8, 2.0, 3),        # flat leaf boxes on the faces
}


@pytest.mark.parametrize("name", sorted(MESHES))
def test_plan_matches_oracle(name):
    make, leaf, eta, m = MESHES[name]
    v, f = make()
    p = Plan(v, f, leaf_size=leaf, eta=eta, order=m)
    o = Oracle(v, f, leaf_size=leaf, eta=eta, order=m, store_near=False)
    assert (p.depth, p.nclu, p.nadm, p.nnear, p.near_entries) == (o.depth, o.nclu, o.nadm, o.nnear, o.near_entries)
    tp, to = p.tree(), o.tree()
    assert np.array_equal(tp["perm"], to["idx"])                 # bit-exact index work
    assert np.array_equal(tp["first"], to["first"]) and np.array_equal(tp["size"], to["size"])
    assert np.array_equal(tp["lo"], to["lo"]) and np.array_equal(tp["hi"], to["hi"])
    (at, as_), (nt, ns) = p.blocks()
    t, s, adm = o.blocks()
    assert set(zip(at.tolist(), as_.tolist())) == set(zip(t[adm].tolist(), s[adm].tolist()))
    assert set(zip(nt.tolist(), ns.tolist())) == set(zip(t[~adm].tolist(), s[~adm].tolist()))
    assert p.leaf_max == int(to["size"][2 ** o.depth - 1:].max())
    lev = [int(np.floor(np.log2(c + 1))) for c in t[adm]]
    assert p.first_adm_level == (min(lev) if lev else o.depth + 1)
    V, E = p.bases()
    Vo = o.V()
    assert np.abs(V - Vo).max() <= 1e-14 * np.abs(Vo).max()
    for c in (1, 2, o.nclu // 2, o.nclu - 1):
        Ek = np.kron(E[c, 2], np.kron(E[c, 1], E[c, 0]))
        assert np.abs(Ek - o.E(c)).max() <= 1e-13


@pytest.mark.parametrize("args,msg", [
    (dict(leaf_size=1), "leaf_size"),
    (dict(order=0), "order"),
    (dict(order=6), "order"),
    (dict(eta=0.0), "eta"),
    (dict(eta=float("nan")), "eta"),
])
def test_plan_rejects_bad_arguments(args, msg):
    v, f = I.icosphere(1)
    kw = dict(leaf_size=8, eta=2.0, order=3)
    kw.update(args)
    with pytest.raises(pkg.H2Error, match=msg) as e:
        Plan(v, f, **kw)
    assert e.value.status == 1


def test_plan_rejects_bad_mesh():
    v, f = I.icosphere(1)
    bad = f.copy()
    bad[3, 1] = v.shape[0]
    with pytest.raises(pkg.H2Error, match="out of range"):
        Plan(v, bad)
    vv = v.copy()
    vv[2, 0] = np.inf
    with pytest.raises(pkg.H2Error, match="non-finite"):
        Plan(vv, f)


def test_single_leaf_mesh_has_no_far_field():
    v, f = I.icosphere(0)                       # 20 triangles, one leaf at leaf_size 32
    p = Plan(v, f, leaf_size=32, eta=2.0, order=3)
    assert p.depth == 0 and p.nadm == 0 and p.nnear == 1 and p.first_adm_level == 1


@pytest.mark.parametrize("prec,basis", [("f64", "f32"), ("f32", "bf16"), ("bf16", "f64n"), ("f16", "bf16")])
def test_build_rejects_bad_basis_precision(prec, basis):
    """basis_prec is checked before any device call: only H2_BF16 / H2_F16 handles
    take it, with H2_F32 or their own 16-bit type."""
    v, f = I.icosphere(1)
    with pytest.raises(pkg.H2Error, match="basis_prec") as e:
        pkg.H2Matrix(v, f, leaf_size=8, order=3, prec=prec, basis=basis)
    assert e.value.status == 1
