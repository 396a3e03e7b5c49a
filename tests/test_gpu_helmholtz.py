"""GPU parity of the Helmholtz single-layer matrix (Section 1's kernel
e^{i kappa r} / (4 pi r)): the complex product and the GMRES solve through the
C ABI (h2_zbuild, h2_zmatvec, h2_zsolve) against the oracle's complex
matrix G_c + i G_s on the same seeded inputs."""
import numpy as np
import pytest

import oracle
from paper_2203_05665_gb300 import H2Matrix, HelmholtzMatrix, colmajor, inputs as I

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f64n": 1e-12, "f32": 1e-6}

CASES = {
    # name: (mesh, leaf, eta, m, kappa)
    "ico3_m4": (lambda: I.icosphere(3), 32, 2.0, 4, 2.0),      # tensor-core coupling and nearfield (f64)
    "ico4_m3": (lambda: I.icosphere(4), 32, 2.0, 3, 2.5),
    "cube7_m2": (lambda: I.cube(7), 16, 2.0, 2, 1.0),          # ragged leaves, flat boxes
    "ell3_m4": (lambda: I.ellipsoid(3, (2.0, 1.0, 0.5)), 24, 1.5, 4, 1.5),
}
_or = {}


def _oracle(name):
    if name not in _or:
        make, leaf, eta, m, kappa = CASES[name]
        v, f = make()
        _or[name] = (v, f, oracle.HelmholtzOracle(v, f, kappa, leaf_size=leaf, eta=eta, order=m))
    return _or[name]


def _crhs(n, nrhs, seed):
    return I.uniform_rhs(n, nrhs, seed) + 1j * I.uniform_rhs(n, nrhs, seed + 500)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["f64", "f64n", "f32"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_zmatvec_matches_oracle(require_gpu, name, prec):
    v, f, o = _oracle(name)
    make, leaf, eta, m, kappa = CASES[name]
    h = HelmholtzMatrix(v, f, kappa, leaf_size=leaf, eta=eta, order=m, prec=prec)
    n = f.shape[0]
    for nrhs in (1, 3, 8):
        x = _crhs(n, nrhs, 5100 + nrhs)
        ref = o.matvec(x)
        y = h.matvec_host(x)
        assert _rel(y, ref) <= TOL[prec], (name, prec, nrhs, _rel(y, ref))
    h.close()


def test_zmatvec_device_pointers_and_determinism(require_gpu):
    import torch
    v, f, o = _oracle("ico3_m4")
    h = HelmholtzMatrix(v, f, 2.0, leaf_size=32, eta=2.0, order=4, prec="f64")
    x = _crhs(f.shape[0], 5, 5200)
    xd = colmajor(torch.from_numpy(x).cuda())
    y1 = colmajor(torch.empty_like(xd))
    y2 = colmajor(torch.full_like(xd, complex("nan")))
    h.matvec(xd, y1)
    h.matvec(xd, y2)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    assert _rel(y1.cpu().numpy(), o.matvec(x)) <= 1e-12
    assert np.array_equal(h.matvec_host(x), y1.cpu().numpy())
    h.close()


def test_kappa_zero_is_the_laplace_matrix(require_gpu):
    """At kappa = 0 the real part's kernel is the Laplace kernel (cos 0 = 1) and
    the imaginary part's vanishes: the complex product equals the Laplace
    product of the real and imaginary parts, bit for bit (same widths)."""
    v, f = I.icosphere(3)
    n = f.shape[0]
    for prec in ("f64", "f32"):
        hz = HelmholtzMatrix(v, f, 0.0, leaf_size=32, eta=2.0, order=4, prec=prec)
        hl = H2Matrix(v, f, leaf_size=32, eta=2.0, order=4, prec=prec)
        x = _crhs(n, 3, 5300)
        y = hz.matvec_host(x)
        side = np.empty((n, 6))
        side[:, 0::2], side[:, 1::2] = x.real, x.imag      # the real and imaginary columns side by side
        yl = hl.matvec_host(side)
        assert np.array_equal(y.real, yl[:, 0::2]) and np.array_equal(y.imag, yl[:, 1::2]), prec
        hz.close()
        hl.close()


def test_constant_density_on_unit_sphere(require_gpu):
    """G 1 approaches area_i e^{i kappa} sin(kappa) / kappa on the unit sphere."""
    kappa = 1.5
    lam = np.exp(1j * kappa) * np.sin(kappa) / kappa
    errs = []
    for L in (3, 4, 5):
        v, f = I.icosphere(L)
        h = HelmholtzMatrix(v, f, kappa, leaf_size=32, eta=2.0, order=4, prec="f64")
        area = 0.5 * np.linalg.norm(np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]]), axis=1)
        y = h.matvec_host(np.ones((f.shape[0], 1), dtype=np.complex128))[:, 0]
        errs.append(_rel(y, lam * area))
        h.close()
    assert errs[0] > errs[1] > errs[2] and errs[2] < 5e-3, errs


@pytest.mark.parametrize("prec", ["f64", "f64n"])
def test_zsolve_reaches_1e8(require_gpu, prec):
    """GMRES(30) on the real form: the true complex residual with the oracle's
    matrix below 1e-8, and the solution against a dense complex solve of the
    oracle's H^2 matrix (formed column by column) within kappa_hat * rtol."""
    v, f, o = _oracle("ico4_m3")
    make, leaf, eta, m, kappa = CASES["ico4_m3"]
    h = HelmholtzMatrix(v, f, kappa, leaf_size=leaf, eta=eta, order=m, prec=prec)
    n = f.shape[0]
    b = _crhs(n, 2, 5400)
    z, it, rel, st = h.solve(b, rtol=1e-8, restart=30, maxit=5000)
    assert st == 0 and np.all(rel <= 1e-8) and np.all(it > 0)
    r = b - o.matvec(z)
    assert np.all(np.linalg.norm(r, axis=0) / np.linalg.norm(b, axis=0) <= 1.5e-8)
    if "dense" not in _or:
        _or["dense"] = o.matvec(np.eye(n, dtype=np.complex128))
    zs = np.linalg.solve(_or["dense"], b)
    assert _rel(z, zs) <= 1e-5
    h.close()


def test_full_size_sampled_rows(require_gpu):
    """Icosphere level 6 (81,920 triangles), m = 4, kappa = 2, 8 complex RHS
    (16 real columns: the tensor-core path): sampled rows against the oracle."""
    v, f = I.icosphere(6)
    kappa = 2.0
    h = HelmholtzMatrix(v, f, kappa, leaf_size=32, eta=2.0, order=4, prec="f64")
    assert h.stats["tensor"] == 1 and h.stats["tensor_near"] == 1
    n = f.shape[0]
    x = _crhs(n, 8, 5500)
    y = h.matvec_host(x)
    h.close()
    o = oracle.HelmholtzOracle(v, f, kappa, leaf_size=32, eta=2.0, order=4, store_near=False)
    rows = np.concatenate([np.random.default_rng(55).choice(n, 40, replace=False), [0, n - 1]])
    assert _rel(y[rows], o.matvec_rows(x, rows)) <= 1e-12
