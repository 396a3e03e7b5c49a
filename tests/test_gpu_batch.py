"""GPU parity of the batched product (h2_batch_*): uneven FP32 problems in
one launch per block-row phase against the FP64 oracle, problem by problem.

Tolerance: 1e-6 relative 2-norm per problem, as for the single FP32 product
(every stored entry is rounded once to FP32 and sums run in FP32).
"""
import numpy as np
import pytest

import oracle
from paper_2203_05665_gb300 import Batch, H2Matrix, H2Error, inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-6

# (mesh, leaf, order, nrhs): ragged leaves, flat boxes, every rank and a nearfield-only problem
SMALL = [
    (lambda: I.icosphere(3), 16, 3, 1),
    (lambda: I.cube(6), 32, 4, 3),
    (lambda: I.ellipsoid(3, (2.0, 1.0, 0.5)), 64, 4, 8),
    (lambda: I.icosphere(0), 32, 3, 2),
    (lambda: I.icosphere(2), 8, 2, 5),
    (lambda: I.cube(9), 16, 3, 16),
    (lambda: I.ellipsoid(2, (0.7, 1.3, 1.9)), 24, 4, 12),
    # a cube whose clusters reach 138 admissible and 140 nearfield blocks per row:
    # those rows are cut in chunks and their partial sums added in order
    (lambda: I.cube(30), 16, 3, 4),
    (lambda: I.cube(30), 32, 4, 2),
]

_cache = {}


def _small():
    if "p" not in _cache:
        probs = []
        for i, (make, leaf, m, nrhs) in enumerate(SMALL):
            v, f = make()
            o = oracle.Oracle(v, f, leaf_size=leaf, eta=2.0, order=m)
            x = I.uniform_rhs(f.shape[0], nrhs, 4100 + i)
            probs.append(dict(v=v, f=f, leaf=leaf, m=m, nrhs=nrhs, x=x, ref=o.matvec(x)))
        _cache["p"] = probs
    return _cache["p"]


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _mats(probs):
    return [H2Matrix(p["v"], p["f"], leaf_size=p["leaf"], eta=2.0, order=p["m"], prec="f32", coupling="stored")
            for p in probs]


def _pack(b, probs):
    import torch
    x = torch.zeros(b.length, dtype=torch.float32, device="cuda")
    for p, xv in zip(probs, b.split(x)):
        xv.copy_(torch.from_numpy(p["x"]).to(torch.float32))
    return x


def test_batch_matches_oracle_every_shape(require_gpu):
    import torch
    probs = _small()
    mats = _mats(probs)
    b = Batch(mats, [p["nrhs"] for p in probs])
    x = _pack(b, probs)
    y = torch.empty_like(x)
    nshape = 8
    for s in range(nshape):
        b.set_shapes([s, s, s, s])
        y.fill_(float("nan"))
        b.matvec(x, y)
        b.sync()
        for i, (p, yv) in enumerate(zip(probs, b.split(y))):
            err = _rel(yv.double().cpu().numpy(), p["ref"])
            assert err <= TOL, (s, i, err)
    b.close()
    for m in mats:
        m.close()


def test_batch_equals_single_products_and_is_deterministic(require_gpu):
    import torch
    probs = _small()
    mats = _mats(probs)
    b = Batch(mats, [p["nrhs"] for p in probs])
    x = _pack(b, probs)
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    b.matvec(x, y1)
    b.matvec(x, y2)   # graph replay
    b.sync()
    assert torch.equal(y1, y2)
    for p, m, yv in zip(probs, mats, b.split(y1)):
        ys = m.matvec_host(p["x"])
        assert _rel(yv.double().cpu().numpy(), ys) <= 1e-6
    # new inputs in the same buffer: the replayed graph reads them
    for i, xv in enumerate(b.split(x)):
        xv.mul_(-2.0)
    b.matvec(x, y2)
    b.sync()
    assert torch.allclose(y2, -2.0 * y1, rtol=1e-5, atol=1e-6 * float(y1.abs().max()))
    # the same matrix twice in one batch (separate work vectors)
    b2 = Batch([mats[1], mats[1]], [probs[1]["nrhs"], 2])
    x2 = torch.zeros(b2.length, dtype=torch.float32, device="cuda")
    v0, v1 = b2.split(x2)
    v0.copy_(torch.from_numpy(probs[1]["x"]).float())
    v1.copy_(torch.from_numpy(probs[1]["x"][:, :2]).float())
    y3 = torch.empty_like(x2)
    b2.matvec(x2, y3)
    b2.sync()
    w0, w1 = b2.split(y3)
    assert _rel(w0.double().cpu().numpy(), probs[1]["ref"]) <= TOL
    assert _rel(w1.double().cpu().numpy(), probs[1]["ref"][:, :2]) <= TOL
    b2.close()
    b.close()
    for m in mats:
        m.close()


def test_batch_tune_profile_and_launch_count(require_gpu):
    import torch
    probs = _small()
    mats = _mats(probs)
    b = Batch(mats, [p["nrhs"] for p in probs])
    x = _pack(b, probs)
    y = torch.empty_like(x)
    b.matvec(x, y)
    ch = b.tune(2)
    assert len(ch) == 4 and all(0 <= c < 8 for c in ch)
    b.profile(True)
    for _ in range(3):
        b.matvec(x, y)
    ph, n = b.phase_times()
    assert n == 3 and all(v[0] >= 0 for v in ph.values())
    # one launch per block-row phase, one per transfer level step, two permutations, and
    # one reduction each for the coupling and nearfield rows cut in chunks (the cube)
    assert ph["leaf_forward"][1] == 1 and ph["coupling"][1] == 2 and ph["leaf_near"][1] == 3
    info = b.info()
    assert info["launches"] == sum(v[1] for v in ph.values())
    for p, yv in zip(probs, b.split(y)):
        assert _rel(yv.double().cpu().numpy(), p["ref"]) <= TOL
    b.close()
    for m in mats:
        m.close()


def test_batch_rejects_unsupported(require_gpu):
    v, f = I.icosphere(2)
    good = H2Matrix(v, f, leaf_size=16, order=3, prec="f32", coupling="stored")
    f64 = H2Matrix(v, f, leaf_size=16, order=3, prec="f64")
    regen = H2Matrix(v, f, leaf_size=16, order=3, prec="f32", coupling="regen")
    big = H2Matrix(v, f, leaf_size=16, order=5, prec="f32", coupling="stored")
    for mats, nrhs in (([f64], [1]), ([regen], [1]), ([big], [1]), ([good], [17]), ([good], [0]),
                       ([good, f64], [1, 1])):
        with pytest.raises(H2Error):
            Batch(mats, nrhs)
    for m in (good, f64, regen, big):
        m.close()


def test_batch_full_size_sampled_rows(require_gpu):
    """Three problems of the uneven batch recipe at full size (leaf 16, 32, 64):
    sampled output rows against the oracle, row by row."""
    import torch
    specs = I.batch_problems(64, 1004)
    pick = [(specs[6], 16), (specs[7], 32), (specs[2], 64)]
    mats, xs = [], []
    for spec, leaf in pick:
        v, f = I.problem_mesh(spec)
        mats.append(H2Matrix(v, f, leaf_size=leaf, eta=2.0, order=spec["order"], prec="f32", coupling="stored"))
        xs.append(I.uniform_rhs(f.shape[0], spec["nrhs"], 4200 + spec["index"]))
    b = Batch(mats, [s["nrhs"] for s, _ in pick])
    x = torch.zeros(b.length, dtype=torch.float32, device="cuda")
    for xv, xh in zip(b.split(x), xs):
        xv.copy_(torch.from_numpy(xh).float())
    b.tune(2)
    y = torch.empty_like(x)
    b.matvec(x, y)
    b.sync()
    rng = np.random.default_rng(6)
    for (spec, leaf), yv, xh in zip(pick, b.split(y), xs):
        v, f = I.problem_mesh(spec)
        o = oracle.Oracle(v, f, leaf_size=leaf, eta=2.0, order=spec["order"], store_near=False)
        n = f.shape[0]
        rows = np.concatenate([rng.choice(n, 24, replace=False), [0, n - 1]])
        ref = o.matvec_rows(xh, rows)
        yy = yv.double().cpu().numpy()
        assert np.all(np.isfinite(yy))
        assert _rel(yy[rows], ref) <= TOL, (spec["index"], leaf)
    b.close()
    for m in mats:
        m.close()
