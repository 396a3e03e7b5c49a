"""h2_matvec_noalloc: the product for callers that cannot allocate device
memory, with its work space in a fixed array inside the library.

Checked through the C ABI against the oracle and against h2_matvec (the
allocating entry point) on two calls in a row, within the tolerances the
other parity tests use.  Before the compared calls the shared array is filled
with NaN by a larger product, so that an entry read before the same call
wrote it would show; the compared handle is fresh (it has never allocated
work buffers of its own).  This file is collected last so that a run stopping
at the first failure has run every other test; it also passes on its own in a
fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2203_05665_gb300 import H2Error, H2Matrix, colmajor, inputs as I, load

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-6}


def _noalloc(lib, h, x, y):
    rc = lib.h2_matvec_noalloc(h.handle, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), int(x.shape[1]))
    assert rc == 0, lib.h2_last_error().decode()


def _dirty_shared_array(lib, dt):
    """A larger product with an all-NaN input leaves NaN in every work entry it used."""
    import torch
    v, f = I.icosphere(5)
    h = H2Matrix(v, f, leaf_size=32, eta=2.0, order=3, prec="f64" if dt == torch.float64 else "f32")
    x = colmajor(torch.full((f.shape[0], 16), float("nan"), device="cuda", dtype=dt))
    y = colmajor(torch.zeros_like(x))
    _noalloc(lib, h, x, y)
    torch.cuda.synchronize()
    assert torch.isnan(y).any()
    h.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("order", [3, 4])
def test_noalloc_matches_oracle_and_matvec_twice(require_gpu, prec, order):
    """Order 4 takes the tensor-core phases (coupling digits; for f64 also the
    nearfield and leaf-basis digits), whose digit buffers the handle owns."""
    import torch
    lib = load()
    dt = torch.float64 if prec == "f64" else torch.float32
    _dirty_shared_array(lib, dt)
    v, f = I.icosphere(4)
    n = f.shape[0]
    o = oracle.Oracle(v, f, leaf_size=32, eta=2.0, order=order)
    h = H2Matrix(v, f, leaf_size=32, eta=2.0, order=order, prec=prec)   # fresh: no work buffers yet
    if order == 4:
        assert h.stats["tensor"] == 1 and (prec == "f32" or h.stats["tensor_leaf"] == 1)
    for call, nrhs in enumerate((3, 3)):
        xh = I.uniform_rhs(n, nrhs, 31 + call)
        x = colmajor(torch.from_numpy(xh).to(device="cuda", dtype=dt))
        y = colmajor(torch.full_like(x, float("nan")))
        _noalloc(lib, h, x, y)
        torch.cuda.synchronize()
        a = y.cpu().double().numpy()
        assert np.all(np.isfinite(a))
        ref = o.matvec(x.cpu().double().numpy())
        assert np.linalg.norm(a - ref) <= TOL[prec] * np.linalg.norm(ref), (call, prec, order)
        y_ref = colmajor(torch.empty_like(x))
        h.matvec(x, y_ref)
        torch.cuda.synchronize()
        r = y_ref.cpu().double().numpy()
        assert np.linalg.norm(a - r) <= TOL[prec] * np.linalg.norm(r), (call, prec, order)
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
