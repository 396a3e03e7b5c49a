"""h2_matvec_host_stream: a sequence of products from host blocks, the
copies of neighbouring blocks overlapped with each product.  Every block's
result must equal the one-call h2_matvec_host result bit for bit (the same
kernels on the same inputs), for FP64-accurate and FP32 handles, for one
block and for several, and the result must match the oracle."""
import numpy as np
import pytest

import oracle
from paper_2203_05665_gb300 import H2Error, H2Matrix, inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("count", [1, 2, 5])
def test_stream_equals_single_calls(require_gpu, prec, count):
    import torch
    v, f = I.icosphere(4)
    n, nrhs = f.shape[0], 3
    h = H2Matrix(v, f, leaf_size=32, eta=2.0, order=3, prec=prec)
    try:
        xs = torch.empty((count, nrhs, n), dtype=torch.float64).pin_memory()
        ys = torch.full((count, nrhs, n), float("nan"), dtype=torch.float64).pin_memory()
        blocks = [I.uniform_rhs(n, nrhs, 5000 + i) for i in range(count)]
        for i, b in enumerate(blocks):
            xs[i] = torch.from_numpy(np.ascontiguousarray(b.T))
        h.matvec_host_stream(xs, ys)
        for i, b in enumerate(blocks):
            assert np.array_equal(ys[i].numpy().T, h.matvec_host(b)), i
        if prec == "f64":
            o = oracle.Oracle(v, f, leaf_size=32, eta=2.0, order=3)
            ref = o.matvec(blocks[-1])
            assert np.linalg.norm(ys[-1].numpy().T - ref) / np.linalg.norm(ref) < 1e-12
        with pytest.raises(H2Error):
            h.matvec_host_stream(xs[:0], ys[:0])      # count 0: refused
    finally:
        h.close()
