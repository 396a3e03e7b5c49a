"""Serving with continuous batching: results alone and in a mix agree bit for bit.

An engine runs every batched operation (products, residuals, norms, the GMRES
cycle) at its full slot width with the free slots held at zero, and every
kernel treats each column with the same instruction sequence whatever its
slot, so a column's arithmetic does not depend on the other requests in the
batch: the results of a request submitted alone and in a mix of interleaved
arrivals from two threads must be identical, for the plain FP64-accurate
engine and for the GMRES-IR engine (FP32 inner cycles)."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2203_05665_gb300 import H2Matrix, Server, inputs as I

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def geoms():
    out = []
    for make, leaf, m in ((lambda: I.icosphere(3), 32, 3), (lambda: I.cube(6), 16, 3)):
        v, f = make()
        hi = H2Matrix(v, f, leaf_size=leaf, eta=2.0, order=m, prec="f64")
        lo = H2Matrix(v, f, leaf_size=leaf, eta=2.0, order=m, prec="f32")
        out.append((v, f, hi, lo, oracle.Oracle(v, f, leaf_size=leaf, eta=2.0, order=m)))
    yield out
    for g in out:
        g[2].close()
        g[3].close()


@pytest.mark.parametrize("mixed", [False, True])
def test_serve_mix_equals_alone(require_gpu, geoms, mixed):
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(10):
        g = i % 2
        nrhs = int(rng.integers(1, 5))
        reqs.append((g, I.uniform_rhs(geoms[g][1].shape[0], nrhs, 2000 + i), [1e-8, 1e-6][i % 3 == 0]))
    # alone: one request at a time on a fresh server
    alone, alone_it = [], []
    srv = Server()
    for v, f, hi, lo, o in geoms:
        srv.register(hi, lo if mixed else None, slots=16)
    for g, b, rtol in reqs:
        t, shape = srv.submit(geoms[g][2], b, rtol)
        assert srv.wait(t, 60)
        z, it, rel, st = srv.poll(t, shape)
        assert st == 0 and np.all(rel <= rtol)
        alone.append(z)
        alone_it.append(it)
    srv.close()
    # in the mix: all requests submitted from two threads at once, interleaved arrivals
    srv = Server()
    for v, f, hi, lo, o in geoms:
        srv.register(hi, lo if mixed else None, slots=16)
    tickets = [None] * len(reqs)

    def submit(idx):
        for i in idx:
            g, b, rtol = reqs[i]
            tickets[i] = srv.submit(geoms[g][2], b, rtol)
            time.sleep(0.002)

    th = [threading.Thread(target=submit, args=(list(range(k, len(reqs), 2)),)) for k in (0, 1)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for i, (g, b, rtol) in enumerate(reqs):
        t, shape = tickets[i]
        assert srv.wait(t, 120)
        z, it, rel, st = srv.poll(t, shape)
        assert st == 0 and np.all(rel <= rtol)
        # true residual against the FP64 oracle, and agreement with the lone run
        o = geoms[g][4]
        r = b - o.matvec(z)
        assert np.all(np.linalg.norm(r, axis=0) / np.linalg.norm(b, axis=0) <= 1.5 * rtol)
        assert np.array_equal(z, alone[i]), (i, _rel(z, alone[i]))
        assert np.array_equal(it, alone_it[i])
    st = srv.stats()
    assert st["queued"] == 0 and st["running_columns"] == 0 and st["completed"] == len(reqs)
    srv.close()


def test_serve_rejects_bad_requests(require_gpu, geoms):
    from paper_2203_05665_gb300 import H2Error
    srv = Server()
    v, f, hi, lo, o = geoms[0]
    with pytest.raises(H2Error):
        srv.submit(hi, np.ones((f.shape[0], 1)))        # not registered
    srv.register(hi, None, slots=4)
    with pytest.raises(H2Error):
        srv.submit(hi, np.ones((f.shape[0], 5)))        # more columns than slots
    with pytest.raises(H2Error):
        srv.register(hi, None)                          # registered twice
    t, shape = srv.submit(hi, np.zeros((f.shape[0], 2)))   # b = 0 -> z = 0 at once
    assert srv.wait(t, 30)
    z, it, rel, st = srv.poll(t, shape)
    assert st == 0 and not z.any()
    srv.close()
