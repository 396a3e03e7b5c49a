"""Host logic of the batched path: the uneven-batch recipe and the leaf-size
autotuner's choices (with stand-in timings; no GPU)."""
import numpy as np
import pytest

from paper_2203_05665_gb300 import inputs as I
from paper_2203_05665_gb300 import tune


def test_batch_recipe():
    specs = I.batch_problems(64, 1004)
    assert len(specs) == 64
    assert specs == I.batch_problems(64, 1004)          # seeded
    assert specs != I.batch_problems(64, 1005)
    for p, s in enumerate(specs):
        assert s["index"] == p
        assert s["order"] in (3, 4) and 1 <= s["nrhs"] <= 8
        if p % 2 == 0:
            assert s["kind"] == "ellipsoid" and s["level"] in (5, 6, 7)
            assert all(0.5 <= a <= 2.0 for a in s["axes"])
            assert s["n"] == 20 * 4 ** s["level"]
        else:
            assert s["kind"] == "cube" and 41 <= s["s"] <= 182 and s["n"] == 12 * s["s"] ** 2
    n = np.array([s["n"] for s in specs])
    assert n.min() >= 20_000 and n.max() <= 400_000
    # both orders and a spread of right-hand sides occur
    assert {s["order"] for s in specs} == {3, 4}
    assert len({s["nrhs"] for s in specs}) >= 6


def test_problem_mesh_counts():
    s = dict(kind="cube", s=5, n=300)
    v, f = I.problem_mesh(s)
    assert f.shape == (300, 3)
    e = dict(kind="ellipsoid", level=2, axes=[1.5, 1.0, 0.7], n=320)
    v, f = I.problem_mesh(e)
    assert f.shape == (320, 3)
    assert np.allclose(np.abs(v).max(axis=0), [1.5, 1.0, 0.7], rtol=0.05)
    with pytest.raises(ValueError):
        I.problem_mesh(dict(kind="torus"))


def test_representative_sizes():
    assert tune.representative(dict(kind="cube", s=150, n=270000))["n"] == 12 * 82 * 82
    assert tune.representative(dict(kind="ellipsoid", level=7, n=327680, axes=[1, 1, 1]))["level"] == 6


def test_choose_leaf_takes_the_fastest_per_group():
    specs = I.batch_problems(16, 1004)
    calls = []

    def measure(spec, leaf):
        calls.append((tune.group_key(spec), leaf))
        # order 3 prefers small leaves, order 4 large ones; cubes shifted
        best = 16 if spec["order"] == 3 else 64
        if spec["kind"] == "cube" and spec["order"] == 3:
            best = 32
        return 1.0 + abs(np.log2(leaf) - np.log2(best))

    leaf, timings = tune.choose_leaf(specs, measure=measure)
    groups = {tune.group_key(s) for s in specs}
    assert len(calls) == 3 * len(groups)                 # one representative per group and candidate
    for s in specs:
        want = 16 if s["order"] == 3 else 64
        if s["kind"] == "cube" and s["order"] == 3:
            want = 32
        assert leaf[s["index"]] == want
    assert set(timings) == groups


def test_fit_budget_moves_to_smaller_memory():
    specs = [dict(kind="cube", s=10, n=1200, order=4, nrhs=4, index=0),
             dict(kind="ellipsoid", level=3, axes=[1, 1, 1], n=1280, order=3, nrhs=4, index=1)]
    # bytes fall with the leaf size in this stand-in; timings rank 16 first
    mem = {16: 300, 32: 200, 64: 150}
    ranking = {tune.group_key(s): [16, 32, 64] for s in specs}
    leaf = {0: 16, 1: 16}
    out = tune.fit_budget(specs, leaf, ranking, 400, plan_bytes=lambda s, lf: mem[lf])
    assert sum(mem[out[i]] for i in (0, 1)) <= 400
    assert tune.fit_budget(specs, leaf, ranking, 10_000, plan_bytes=lambda s, lf: mem[lf]) == leaf
    with pytest.raises(MemoryError):
        tune.fit_budget(specs, leaf, ranking, 100, plan_bytes=lambda s, lf: mem[lf])


def test_stored_bytes_from_plan():
    from paper_2203_05665_gb300 import Plan
    v, f = I.icosphere(3)
    p = Plan(v, f, leaf_size=16, eta=2.0, order=3)
    b = tune.stored_bytes(p, 4)
    k, kp = 27, 28
    assert b >= 4 * p.nadm * k * kp + 4 * p.near_entries
