"""The single-launch product (h2_options.fused = 1) of small FP64-accurate
matrices: one cooperative launch runs Algorithms 1-3 with grid-wide
barriers between the steps.  Checked against the oracle (1e-12) and against
the launch-per-phase product of the same mesh (1e-13), with the accumulate
form, CUDA-graph replay, the allocation-free entry point, a column outside
the double-float range (range guard), a mesh without admissible blocks, ragged leaves, order 4 (whose
handles also keep the tensor-core digits) and GMRES."""
import numpy as np
import pytest

import oracle
from paper_2203_05665_gb300 import H2Matrix, colmajor, inputs as I

pytestmark = pytest.mark.gpu

CASES = {
    # name: (mesh, leaf, eta, m)
    "ico4_m3": (lambda: I.icosphere(4), 32, 2.0, 3),    # the 5,120-triangle latency configuration
    "ico3_m4": (lambda: I.icosphere(3), 32, 2.0, 4),
    "cube6_m2": (lambda: I.cube(6), 16, 2.0, 2),        # ragged leaves (padding rows)
    "ell3_m3": (lambda: I.ellipsoid(3, (2.0, 1.0, 0.5)), 24, 1.5, 3),
    "ico1_near": (lambda: I.icosphere(1), 32, 2.0, 3),  # 80 triangles: no admissible block
}
_or = {}


def _case(name):
    if name not in _or:
        make, leaf, eta, m = CASES[name]
        v, f = make()
        _or[name] = (v, f, oracle.Oracle(v, f, leaf_size=leaf, eta=eta, order=m))
    return _or[name]


def _mats(name):
    make, leaf, eta, m = CASES[name]
    v, f, o = _case(name)
    fz = H2Matrix(v, f, leaf_size=leaf, eta=eta, order=m, prec="f64", fused=True)
    st = H2Matrix(v, f, leaf_size=leaf, eta=eta, order=m, prec="f64")
    return v, f, o, fz, st


def _dev(a):
    import torch
    return colmajor(torch.from_numpy(np.asfortranarray(a)).cuda())


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", sorted(CASES))
def test_fused_matches_oracle_and_phase_product(require_gpu, name):
    import torch
    v, f, o, fz, st = _mats(name)
    try:
        for nrhs in (1, 3, 16):
            x = I.uniform_rhs(f.shape[0], nrhs, 4000 + nrhs)
            xd = _dev(x)
            y1, y2 = colmajor(torch.empty_like(xd)), colmajor(torch.empty_like(xd))
            fz.matvec(xd, y1)
            st.matvec(xd, y2)
            a, b = y1.cpu().numpy(), y2.cpu().numpy()
            assert _rel(a, o.matvec(x)) < 1e-12, nrhs
            assert _rel(a, b) < 1e-13, nrhs
            # a second call on the same buffers gives the same bits
            fz.matvec(xd, y1)
            assert np.array_equal(y1.cpu().numpy(), a)
    finally:
        fz.close()
        st.close()


def test_fused_accumulate_graph_and_range_guard(require_gpu):
    import torch
    v, f, o, fz, st = _mats("ico4_m3")
    try:
        n = f.shape[0]
        x = I.uniform_rhs(n, 4, 4100)
        x[:, 1] *= 1e-20      # below the double-float range: scaled on the way in and out
        x[:, 2] *= 1e20
        xd = _dev(x)
        y = colmajor(torch.empty_like(xd))
        fz.matvec(xd, y)
        ref = o.matvec(x)
        got = y.cpu().numpy()
        for c in range(4):
            assert _rel(got[:, c], ref[:, c]) < 1e-12, c
        y0 = I.uniform_rhs(n, 4, 4101)
        ya = _dev(y0)
        fz.matvec_acc(xd, ya)
        assert np.abs(ya.cpu().numpy() - (y0 + got)).max() <= 1e-13 * np.abs(y0 + got).max()
        yg = colmajor(torch.empty_like(xd))
        g = fz.graph(xd, yg)
        for _ in range(2):
            g.launch()
            torch.cuda.synchronize()
            assert np.array_equal(yg.cpu().numpy(), got)
        assert np.array_equal(fz.matvec_host(x), got)
        # through the allocation-free entry point (the fused kernel's work vectors in its fixed array)
        yn = colmajor(torch.full_like(xd, float("nan")))
        fz.matvec_noalloc(xd, yn)
        torch.cuda.synchronize()
        assert np.array_equal(yn.cpu().numpy(), got)
    finally:
        fz.close()
        st.close()


def test_fused_gmres(require_gpu):
    v, f, o, fz, st = _mats("ico4_m3")
    try:
        b = I.uniform_rhs(f.shape[0], 2, 4200)
        z, it, rel, s = fz.solve(b, rtol=1e-8)
        assert s == 0 and np.all(rel <= 1e-8)
        r = b - o.matvec(z)
        assert np.all(np.linalg.norm(r, axis=0) / np.linalg.norm(b, axis=0) <= 1.5e-8)
    finally:
        fz.close()
        st.close()
