"""h2_graph_*: one H² product captured as a CUDA graph and replayed.

A replay runs the same kernels with the same launch shapes as h2_matvec on the
same buffers, so its output must equal h2_matvec's bit for bit; new values
written into the captured input buffer must be picked up by the next replay;
and a graph whose handle reallocated its work space must be refused, not run
on freed memory.  One case per coupling path (double-float FP64, tensor-core
FP64, FP32 stored, tensor-core FP32, FP32 regenerated) is also checked
against the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2203_05665_gb300 import H2Error, H2Matrix, colmajor, inputs as I

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-6}

CASES = [
    # (mesh level, order, precision, coupling, nrhs)
    (4, 3, "f64", "stored", 1),     # the 5,120-triangle configuration, one right-hand side
    (3, 4, "f64", "stored", 5),     # the coupling on the tensor cores
    (4, 3, "f32", "stored", 2),
    (3, 4, "f32", "stored", 4),     # FP32 coupling on the tensor cores
    (3, 4, "f32", "regen", 3),
]


@pytest.mark.parametrize("level,order,prec,coupling,nrhs", CASES)
def test_graph_replay_matches_matvec_and_oracle(require_gpu, level, order, prec, coupling, nrhs):
    import torch
    v, f = I.icosphere(level)
    n = f.shape[0]
    h = H2Matrix(v, f, leaf_size=32, eta=2.0, order=order, prec=prec, coupling=coupling)
    if order == 4 and coupling == "stored":
        assert h.stats["tensor"] == 1
    dt = torch.float64 if prec == "f64" else torch.float32
    x = colmajor(torch.zeros((n, nrhs), dtype=dt, device="cuda"))
    y = colmajor(torch.full_like(x, float("nan")))
    g = h.graph(x, y)
    o = oracle.Oracle(v, f, leaf_size=32, eta=2.0, order=order)
    for rep in range(3):
        xs = I.uniform_rhs(n, nrhs, 700 + rep)
        x.copy_(torch.from_numpy(xs).to(dt))          # new values in the captured buffer
        y.fill_(float("nan"))
        g.launch()
        torch.cuda.synchronize()
        yg = y.cpu().double().numpy()
        y_ref = colmajor(torch.empty_like(x))
        h.matvec(x, y_ref)
        torch.cuda.synchronize()
        assert np.array_equal(yg, y_ref.cpu().double().numpy()), "graph replay differs from h2_matvec"
        if rep == 0:
            ref = o.matvec(xs)
            assert np.linalg.norm(yg - ref) <= TOL[prec] * np.linalg.norm(ref)
    g.close()
    h.close()


def test_graph_refused_after_work_space_grows(require_gpu):
    import torch
    v, f = I.icosphere(3)
    n = f.shape[0]
    h = H2Matrix(v, f, leaf_size=32, eta=2.0, order=3, prec="f64")
    x = colmajor(torch.from_numpy(I.uniform_rhs(n, 1, 5)).cuda())
    y = colmajor(torch.empty_like(x))
    g = h.graph(x, y)
    g.launch()
    torch.cuda.synchronize()
    # more right-hand sides than the work space holds: it is reallocated
    x16 = colmajor(torch.from_numpy(I.uniform_rhs(n, 16, 6)).cuda())
    h.matvec(x16, colmajor(torch.empty_like(x16)))
    torch.cuda.synchronize()
    with pytest.raises(H2Error, match="reallocated"):
        g.launch()
    # a new capture works again
    g2 = h.graph(x, y)
    g2.launch()
    torch.cuda.synchronize()
    assert np.all(np.isfinite(y.cpu().numpy()))
    h.close()     # closes the graphs of the handle first
    assert g2._g is None and g._g is None
