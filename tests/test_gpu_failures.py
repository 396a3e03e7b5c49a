"""Failure paths, made to happen on the host or inside a bounded wait (never
as a GPU fault): an injected allocation failure in every allocating entry
point, a bounded device wait that runs out, GMRES stopping at maxit, and
serving admission refused beyond the memory budget.  After each failure the
library must report the status the header promises, release what it held
and keep working."""
import ctypes as C
import time

import numpy as np
import pytest

import oracle
from paper_2203_05665_gb300 import H2Error, H2Matrix, colmajor, inputs as I, load
from paper_2203_05665_gb300._lib import H2_ENOCONV, H2_ENOMEM, H2_ETIMEOUT, H2_OK, Server

pytestmark = pytest.mark.gpu


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.fixture
def lib():
    lb = load()
    yield lb
    lb.h2_inject_alloc_failure(-1)


def test_build_fails_cleanly_at_every_allocation(require_gpu, lib):
    """h2_build with the k-th device allocation failing, for every k: H2_ENOMEM,
    nothing leaked; the next build works."""
    v, f = I.icosphere(3)
    H2Matrix(v, f, leaf_size=32, eta=2.0, order=4, prec="f64").close()   # warm the context
    free0 = _free_bytes()
    k = 0
    while True:
        assert lib.h2_inject_alloc_failure(k) == H2_OK
        try:
            h = H2Matrix(v, f, leaf_size=32, eta=2.0, order=4, prec="f64")
        except H2Error as e:
            assert e.status == H2_ENOMEM, (k, str(e))
            assert abs(_free_bytes() - free0) < (4 << 20), k
            k += 1
            assert k < 200
            continue
        break
    # the injection was not consumed: the build makes k allocations
    lib.h2_inject_alloc_failure(-1)
    assert k >= 10
    x = I.uniform_rhs(f.shape[0], 2, 7)
    ref = oracle.Oracle(v, f, leaf_size=32, eta=2.0, order=4).matvec(x)
    y = h.matvec_host(x)
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)
    h.close()


def test_work_buffers_and_solver_fail_cleanly(require_gpu, lib):
    v, f = I.icosphere(3)
    n = f.shape[0]
    o = oracle.Oracle(v, f, leaf_size=32, eta=2.0, order=3)
    h = H2Matrix(v, f, leaf_size=32, eta=2.0, order=3, prec="f64")
    x = I.uniform_rhs(n, 3, 8)
    lib.h2_inject_alloc_failure(0)            # the product's work buffers
    with pytest.raises(H2Error) as e:
        h.matvec_host(x)
    assert e.value.status == H2_ENOMEM
    y = h.matvec_host(x)                       # allocates now and works
    assert np.linalg.norm(y - o.matvec(x)) <= 1e-12 * np.linalg.norm(o.matvec(x))
    for k in range(0, 40):                     # staging and GMRES work space: each allocation in turn
        lib.h2_inject_alloc_failure(k)
        try:
            z, it, rel, st = h.solve(x[:, :1], rtol=1e-8)
        except H2Error as e:
            assert e.status == H2_ENOMEM, (k, str(e))
            continue
        finally:
            lib.h2_inject_alloc_failure(-1)
        assert st == H2_OK and k > 2
        break
    else:
        pytest.fail("GMRES kept failing")
    assert rel[0] <= 1e-8
    h.close()


def test_bounded_wait_runs_out_and_handle_stays_usable(require_gpu, lib):
    v, f = I.icosphere(3)
    n = f.shape[0]
    o = oracle.Oracle(v, f, leaf_size=32, eta=2.0, order=4)
    h = H2Matrix(v, f, leaf_size=32, eta=2.0, order=4, prec="f64")
    seen = C.c_int(-1)
    assert lib.h2_wait_selftest(h.handle, 0, 0, C.byref(seen)) == H2_OK and seen.value == 4
    for limit in (1, 1000, 100000):
        seen.value = -1
        t0 = time.time()
        rc = lib.h2_wait_selftest(h.handle, 1, limit, C.byref(seen))
        assert rc == H2_ETIMEOUT, (limit, rc, lib.h2_last_error().decode())
        # a tiny limit may run out before an earlier stage has landed too
        assert 0 <= seen.value <= 3 and time.time() - t0 < 30
        if limit >= 100000:
            assert seen.value == 3
    # the error was read and cleared: products and the untouched self-test work again
    x = I.uniform_rhs(n, 4, 9)
    ref = o.matvec(x)
    assert np.linalg.norm(h.matvec_host(x) - ref) <= 1e-12 * np.linalg.norm(ref)
    assert lib.h2_wait_selftest(h.handle, 0, 0, None) == H2_OK
    h.close()


def test_gmres_stops_at_maxit_with_its_best_iterate(require_gpu):
    """H2_ENOCONV: the returned z is the last iterate, whose true residual is
    reported; restarted GMRES never increases the residual, so it is also the
    best one, and more iterations give a smaller residual."""
    v, f = I.icosphere(3)
    n = f.shape[0]
    o = oracle.Oracle(v, f, leaf_size=32, eta=2.0, order=3)
    h = H2Matrix(v, f, leaf_size=32, eta=2.0, order=3, prec="f64")
    b = I.uniform_rhs(n, 2, 10)
    last = np.ones(2)
    for maxit in (2, 5, 11, 23):
        z, it, rel, st = h.solve(b, rtol=1e-14, restart=4, maxit=maxit)
        assert st == H2_ENOCONV and np.all(it == maxit)
        true = np.linalg.norm(b - o.matvec(z), axis=0) / np.linalg.norm(b, axis=0)
        assert np.allclose(rel, true, rtol=1e-6, atol=0)
        assert np.all(rel <= last * (1 + 1e-12)) and np.all(rel < 1)
        last = rel
    h.close()


def test_serve_admission_by_memory_budget(require_gpu):
    """An engine larger than the budget is refused at registration (H2_ENOMEM);
    two engines that fit only one at a time both finish their requests, and the
    memory in use never exceeds the budget."""
    v, f = I.icosphere(3)
    n = f.shape[0]
    ha = H2Matrix(v, f, leaf_size=32, eta=2.0, order=3, prec="f64")
    hb = H2Matrix(v, f, leaf_size=32, eta=2.0, order=3, prec="f64")
    one = 8 * n * 8 * (30 + 1 + 3 + 5) + 8 * 8 * (4 * 30 + 16)   # work space of an 8-slot engine
    s = Server(0, hbm_budget=one // 2)
    with pytest.raises(H2Error) as e:
        s.register(ha, slots=8)
    assert e.value.status == H2_ENOMEM
    s.close()
    s = Server(0, hbm_budget=int(1.5 * one))
    s.register(ha, slots=8)
    s.register(hb, slots=8)
    b = I.uniform_rhs(n, 4, 11)
    reqs = {s.submit(ha, b[:, :2], 1e-8): b[:, :2], s.submit(ha, b[:, 2:], 1e-8): b[:, 2:],
            s.submit(hb, b, 1e-8): b}
    deadline = time.time() + 120
    results = {}
    while len(results) < len(reqs) and time.time() < deadline:
        st = s.stats()
        assert st["engine_bytes"] <= st["budget"]
        for (t, shape), cols in reqs.items():
            if t not in results:
                r = s.poll(t, shape)
                if r is not None:
                    results[t] = (r, cols)
        time.sleep(0.005)
    assert len(results) == len(reqs)
    o = oracle.Oracle(v, f, leaf_size=32, eta=2.0, order=3)
    for t, ((z, iters, relres, status), cols) in results.items():
        assert status == H2_OK and np.all(relres <= 1e-8)
        r = np.linalg.norm(cols - o.matvec(z), axis=0) / np.linalg.norm(cols, axis=0)
        assert np.all(r <= 1.5e-8)
    s.close()
    ha.close()
    hb.close()
