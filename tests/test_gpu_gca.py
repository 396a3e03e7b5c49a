"""GPU parity of the GCA-H^2 matrix (Section 3's GCA-H^2 example) through the
C ABI (h2_build_gca, h2_gca_pivots, h2_export, h2_matvec, h2_solve) against
the oracle's GCA-H^2 matrix on the same seeded meshes:

* pivots and ranks of every cluster from the leaves to the first admissible
  level equal the oracle's (bit for bit: integers);
* the stored coupling matrices agree entry by entry (FP64 to 1e-13 relative
  to each block's largest entry, FP32 to the unit roundoff); the leaf bases
  and transfer matrices, whose rounding grows with the condition of the
  pivot blocks, to 1e-11 (FP32: twice the unit roundoff);
* products (y = G~ x, y += G~ x, host buffers, graph replay, no-alloc) agree
  with the oracle's product (FP64 1e-12, FP32 1e-6) for 1 to 32 right-hand
  sides; too many right-hand sides for one tile are refused before any launch;
* GMRES and GMRES-IR reach 1e-8 in the true residual (the oracle's product),
  also through the serving engine;
* sampled rows at 327,680 triangles (the product's launch configuration)."""
import numpy as np
import pytest

import oracle
from paper_2203_05665_gb300 import GcaMatrix, H2Error, colmajor, inputs as I

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f64n": 1e-12, "f32": 1e-6}
CASES = {
    # name: (mesh, leaf, eta, eps)
    "ico3": (lambda: I.icosphere(3), 16, 2.0, 1e-4),
    "ico4": (lambda: I.icosphere(4), 32, 2.0, 1e-4),
    "cube6": (lambda: I.cube(6), 16, 2.0, 1e-3),                   # ragged leaves, flat boxes
    "ell4": (lambda: I.ellipsoid(4, (2.0, 1.0, 0.5)), 24, 1.5, 1e-5),
}
_or = {}


def _oracle(name):
    if name not in _or:
        make, leaf, eta, eps = CASES[name]
        v, f = make()
        _or[name] = (v, f, oracle.GcaOracle(v, f, leaf_size=leaf, eta=eta, eps=eps))
    return _or[name]


def _gca(name, prec="f64"):
    make, leaf, eta, eps = CASES[name]
    v, f, _ = _oracle(name)
    return GcaMatrix(v, f, leaf_size=leaf, eta=eta, eps=eps, prec=prec)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", sorted(CASES))
def test_pivots_equal_oracle(require_gpu, name):
    v, f, o = _oracle(name)
    h = _gca(name)
    try:
        rank, piv = h.gca_pivots()
        lmin, D = h.stats["first_adm_level"], h.stats["depth"]
        assert h.stats["gca"] == 1
        for c in range((1 << lmin) - 1, (2 << D) - 1):
            assert rank[c] == o.rank[c], c
            assert np.array_equal(piv[c, :rank[c]], o.pivots(c)), c
        assert np.all(rank[:(1 << lmin) - 1] == 0)
    finally:
        h.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name", ["ico3", "cube6"])
def test_stored_bases_and_coupling_match_oracle(require_gpu, name, prec):
    v, f, o = _oracle(name)
    h = _gca(name, prec)
    # S: Galerkin entries, plain quadrature; V and E: the interpolation
    # operator M[:, J] M[I, J]^{-1}, whose rounding grows with the condition
    # of the pivot block (the library forms it by a triangular solve, the
    # oracle by an LU solve)
    tol, tol_ve = (1e-13, 1e-11) if prec == "f64" else (2.0 ** -23, 2.0 ** -22)
    try:
        st = h.stats
        D, lmin = st["depth"], st["first_adm_level"]
        tr = o.tree()
        leaf0 = (1 << D) - 1
        Vg = h.export_gca("V")
        for j in range(1 << D):
            c = leaf0 + j
            ref = o.V(c, int(tr["size"][c]))
            got = Vg[j, :ref.shape[0], :ref.shape[1]]
            assert np.abs(got - ref).max() <= tol_ve * max(1.0, np.abs(ref).max()), c
            assert not Vg[j, :, ref.shape[1]:].any() and not Vg[j, ref.shape[0]:, :].any()
        Eg = h.export_gca("E")
        for c in range((2 << lmin) - 1, (2 << D) - 1):
            ref = o.E(c)
            got = Eg[c, :ref.shape[0], :ref.shape[1]]
            assert np.abs(got - ref).max() <= tol_ve * max(1.0, np.abs(ref).max()), c
        t, s, a = o.blocks()
        adm = sorted(zip(t[a], s[a]))
        Sg = h.export_gca("S")
        assert Sg.shape[0] == len(adm)
        for i in range(0, len(adm), max(1, len(adm) // 200)):
            bt, bs = adm[i]
            ref = o.S(bt, bs)
            got = Sg[i, :ref.shape[0], :ref.shape[1]]
            assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (bt, bs)
    finally:
        h.close()


@pytest.mark.parametrize("prec", ["f64", "f64n", "f32"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_matvec_matches_oracle(require_gpu, name, prec):
    import torch
    v, f, o = _oracle(name)
    h = _gca(name, prec)
    try:
        vn, es = (4, 4) if prec == "f32" else (2, 8)
        lp = -(-h.stats["leaf_max"] // 4) * 4
        for nrhs in (1, 5, 16, 32):
            x = I.uniform_rhs(f.shape[0], nrhs, 3000 + nrhs)
            dt = torch.float32 if prec == "f32" else torch.float64
            xd = colmajor(torch.from_numpy(x).to(device="cuda", dtype=dt))
            yd = colmajor(torch.empty_like(xd))
            rp = -(-nrhs * es // 16) * 16 // es
            if (max(h.stats["rank"], lp) // 4) * (rp // vn) > 256:
                with pytest.raises(H2Error):       # the output tile does not fit one CTA
                    h.matvec(xd, yd)
                continue
            h.matvec(xd, yd)
            assert _rel(yd.double().cpu().numpy(), o.matvec(x)) < TOL[prec], nrhs
    finally:
        h.close()


def test_product_variants_agree(require_gpu):
    """y += G~ x, host buffers, graph replay and the no-alloc entry point give
    the launched product's result (bit for bit where the path is the same)."""
    import torch
    v, f, o = _oracle("ico4")
    h = _gca("ico4")
    try:
        x = I.uniform_rhs(f.shape[0], 4, 3100)
        xd = colmajor(torch.from_numpy(x).cuda())
        yd = colmajor(torch.empty_like(xd))
        h.matvec(xd, yd)
        y = yd.cpu().numpy()
        assert _rel(y, o.matvec(x)) < 1e-12
        y0 = I.uniform_rhs(f.shape[0], 4, 3101)
        ya = colmajor(torch.from_numpy(y0).cuda())
        h.matvec_acc(xd, ya)
        assert np.abs(ya.cpu().numpy() - (y0 + y)).max() < 1e-13 * np.abs(y0 + y).max()
        assert np.array_equal(h.matvec_host(x), y)
        yg = colmajor(torch.empty_like(xd))
        g = h.graph(xd, yg)
        g.launch()
        torch.cuda.synchronize()
        assert np.array_equal(yg.cpu().numpy(), y)
        yn = colmajor(torch.full_like(xd, float("nan")))
        h.matvec_noalloc(xd, yn)
        torch.cuda.synchronize()
        assert np.array_equal(yn.cpu().numpy(), y)
    finally:
        h.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_gmres_reaches_1e8(require_gpu, prec):
    v, f, o = _oracle("ico4")
    h = _gca("ico4", "f64")
    lo = _gca("ico4", "f32") if prec == "f32" else None
    try:
        b = I.uniform_rhs(f.shape[0], 3, 3200)
        if lo is None:
            z, it, rel, st = h.solve(b, rtol=1e-8)
        else:
            z, it, rel, st = h.solve_ir(lo, b, rtol=1e-8)
        assert st == 0 and np.all(rel <= 1e-8)
        r = b - o.matvec(z)
        assert np.all(np.linalg.norm(r, axis=0) / np.linalg.norm(b, axis=0) <= 1.5e-8)
    finally:
        h.close()
        if lo is not None:
            lo.close()


def test_rejects_oversized_tiles(require_gpu):
    """64 double-float columns with a padded rank above 32 do not fit one
    output tile: H2_EINVAL before any launch, and the handle still works."""
    import torch
    v, f, o = _oracle("ico4")
    h = _gca("ico4")
    try:
        assert h.stats["rank"] > 32
        x = colmajor(torch.from_numpy(I.uniform_rhs(f.shape[0], 64, 3300)).cuda())
        y = colmajor(torch.empty_like(x))
        with pytest.raises(H2Error):
            h.matvec(x, y)
        x1 = I.uniform_rhs(f.shape[0], 2, 3301)
        assert _rel(h.matvec_host(x1), o.matvec(x1)) < 1e-12
    finally:
        h.close()


def test_serving_engine_with_gca_handles(require_gpu):
    """A GCA-H^2 pair (FP64-accurate residuals, FP32 inner solves) registered
    with the serving engine: requests reach their tolerance in the oracle's
    true residual."""
    from paper_2203_05665_gb300 import Server
    v, f, o = _oracle("ico4")
    hi, lo = _gca("ico4", "f64"), _gca("ico4", "f32")
    srv = Server()
    try:
        srv.register(hi, lo, slots=8)
        reqs = [(I.uniform_rhs(f.shape[0], nr, 3400 + nr), rt) for nr, rt in ((1, 1e-8), (3, 1e-6), (2, 1e-8))]
        tickets = [srv.submit(hi, b, rt) for b, rt in reqs]
        for (b, rt), (t, shape) in zip(reqs, tickets):
            assert srv.wait(t, 120)
            z, it, rel, st = srv.poll(t, shape)
            assert st == 0 and np.all(rel <= rt)
            r = b - o.matvec(z)
            assert np.all(np.linalg.norm(r, axis=0) / np.linalg.norm(b, axis=0) <= 1.5 * rt)
    finally:
        srv.close()
        hi.close()
        lo.close()


def test_rejects_bad_options(require_gpu):
    v, f = I.icosphere(2)
    for kw in (dict(prec="bf16"), dict(eps=-1.0), dict(green_order=9), dict(max_rank=200), dict(gamma=0.0)):
        with pytest.raises(H2Error):
            GcaMatrix(v, f, leaf_size=16, **kw)


def test_full_size_sampled_rows(require_gpu):
    """327,680 triangles (icosphere L7, leaf 32, eta 2, eps 1e-4, 16 RHS, the
    benchmark's configuration): sampled rows of the GPU product against the
    oracle's rows (its GCA-H^2 matrix built without stored S and nearfield)."""
    import torch
    v, f = I.icosphere(7)
    n = f.shape[0]
    h = GcaMatrix(v, f, leaf_size=32, eta=2.0, eps=1e-4, prec="f64")
    try:
        x = I.uniform_rhs(n, 16, 1002)
        xd = colmajor(torch.from_numpy(x).cuda())
        yd = colmajor(torch.empty_like(xd))
        h.matvec(xd, yd)
        y = yd.cpu().numpy()
        o = oracle.GcaOracle(v, f, leaf_size=32, eta=2.0, eps=1e-4, store_near=False, store_S=False)
        rank, piv = h.gca_pivots()
        lmin = h.stats["first_adm_level"]
        assert np.array_equal(rank[(1 << lmin) - 1:], o.rank[(1 << lmin) - 1:])
        rows = np.random.default_rng(5).choice(n, 24, replace=False)
        ref = o.matvec_rows(x, rows)
        assert np.abs(y[rows] - ref).max() <= 1e-12 * np.abs(ref).max()
    finally:
        h.close()
