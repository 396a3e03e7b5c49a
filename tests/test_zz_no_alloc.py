"""h2_matvec_noalloc: the product for callers that cannot allocate device
memory, with its work space in a fixed array inside the library.

Checked through the C ABI against h2_matvec (the allocating entry point) on
two calls in a row, within the tolerances the other parity tests use.  This
file is collected last so that a run stopping at the first failure has run
every other test; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2203_05665_gb300 import H2Error, H2Matrix, colmajor, inputs as I, load

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-6}


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_noalloc_matches_matvec_twice(require_gpu, prec):
    import torch
    lib = load()
    v, f = I.icosphere(4)
    h = H2Matrix(v, f, leaf_size=32, eta=2.0, order=3, prec=prec)
    dt = torch.float64 if prec == "f64" else torch.float32
    for call, nrhs in enumerate((3, 3)):
        x = colmajor(torch.from_numpy(I.uniform_rhs(f.shape[0], nrhs, 31 + call)).to(device="cuda", dtype=dt))
        y_ref = colmajor(torch.empty_like(x))
        y = colmajor(torch.full_like(x, float("nan")))
        h.matvec(x, y_ref)
        rc = lib.h2_matvec_noalloc(h.handle, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), nrhs)
        assert rc == 0, lib.h2_last_error().decode()
        torch.cuda.synchronize()
        a, r = y.cpu().double().numpy(), y_ref.cpu().double().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - r) <= TOL[prec] * np.linalg.norm(r)
    h.close()


def test_noalloc_rejects_work_space_beyond_limit(require_gpu):
    import torch
    v, f = I.icosphere(5)
    h = H2Matrix(v, f, leaf_size=32, eta=2.0, order=4, prec="f32")   # 64 RHS need > 64 MiB
    x = colmajor(torch.zeros((f.shape[0], 64), device="cuda", dtype=torch.float32))
    y = colmajor(torch.zeros_like(x))
    with pytest.raises(H2Error, match="fixed limit"):
        h.matvec_noalloc(x, y)
    h.close()
