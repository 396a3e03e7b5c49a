"""Leaf-size autotuner for batched products.

The leaf size trades the nearfield (dense leaf x leaf blocks, which grow with
the leaf) against the far field (coupling matrices and transfer work, which
grow with the number of clusters).  Which side wins depends on the order m,
the number of right-hand sides and the surface, so the tuner measures it:
problems are grouped by (surface kind, order, padded right-hand sides); for
each group one representative mesh of moderate size is built at every
candidate leaf size and its batched product is timed on the device (launch
shapes tuned too); the group takes the fastest candidate that fits the memory
budget.  All timing runs in libh2; this module only chooses.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs
from ._lib import Batch, H2Matrix, Plan

CANDIDATES = (16, 32, 64)


def group_key(spec):
    """Problems of one group share surface kind, order and padded right-hand sides."""
    return (spec["kind"], int(spec["order"]), (int(spec["nrhs"]) + 3) // 4 * 4)


def representative(spec, target_n=80_000):
    """A mesh of the same kind as spec with about target_n triangles."""
    r = dict(spec)
    if spec["kind"] == "cube":
        s = max(4, int(round((target_n / 12) ** 0.5)))
        r.update(s=s, n=12 * s * s)
    else:
        level = max(1, int(round(np.log(target_n / 20) / np.log(4))))
        r.update(level=level, n=20 * 4 ** level)
    return r


def stored_bytes(plan: Plan, nrhs: int, esize: int = 4):
    """Device bytes of a stored-coupling matrix and its work vectors (from the plan's counts)."""
    k, L = plan.k, plan.leaf_max
    kp = (k + 3) // 4 * 4
    lp = (L + 3) // 4 * 4
    rp = (nrhs + 3) // 4 * 4
    nleaf = (plan.nclu + 1) // 2
    s = plan.nadm * k * kp
    near = plan.nnear * L * lp
    v = 2 * nleaf * L * kp
    vec = 2 * nleaf * L * rp + 2 * plan.nclu * k * rp
    return esize * (s + near + v + vec)


def time_product(mat, nrhs, reps=10, tune_reps=3, seed=7):
    """Median device time (ms) of the batched product of one matrix, launch shapes tuned."""
    import torch
    b = Batch([mat], [nrhs])
    try:
        x = torch.empty(b.length, dtype=torch.float32, device="cuda").uniform_(-1, 1,
                                                                            generator=torch.Generator("cuda").manual_seed(seed))
        y = torch.empty_like(x)
        b.matvec(x, y)
        b.sync()
        b.tune(tune_reps)
        b.profile(True)
        for _ in range(reps):
            b.matvec(x, y)
        ph, n = b.phase_times()
        return sum(v[0] for v in ph.values()) / max(n, 1)
    finally:
        b.close()


def choose_leaf(specs, candidates=CANDIDATES, measure=None, budget_bytes=None, target_n=80_000, log=None):
    """Leaf size per problem index.

    measure(spec, leaf) -> ms of one product (default: build the matrix on the
    GPU and time it); budget_bytes bounds the stored bytes of the whole batch
    (the fastest assignment that fits is kept, growing the leaf of the largest
    groups first when needed).  Returns ({index: leaf}, {group: {leaf: ms}}).
    """
    if measure is None:
        def measure(spec, leaf):
            v, t = inputs.problem_mesh(spec)
            m = H2Matrix(v, t, leaf_size=leaf, eta=2.0, order=spec["order"], prec="f32", coupling="stored")
            try:
                return time_product(m, spec["nrhs"])
            finally:
                m.close()
    groups = {}
    for s in specs:
        groups.setdefault(group_key(s), []).append(s)
    timings, choice = {}, {}
    for key in sorted(groups):
        members = groups[key]
        rep = representative(members[0], target_n)
        rep["nrhs"] = max(s["nrhs"] for s in members)
        t0 = time.perf_counter()
        timings[key] = {leaf: float(measure(rep, leaf)) for leaf in candidates}
        # per-DoF time of the representative ranks the candidates
        order = sorted(candidates, key=lambda lf: timings[key][lf])
        choice[key] = order
        if log:
            log(f"tune {key}: " + ", ".join(f"leaf {lf}: {timings[key][lf]:.3f} ms" for lf in candidates)
                + f" -> {order[0]} ({time.perf_counter() - t0:.1f} s)")
    leaf = {s["index"]: choice[group_key(s)][0] for s in specs}
    if budget_bytes is not None:
        leaf = fit_budget(specs, leaf, choice, budget_bytes)
    return leaf, timings


def fit_budget(specs, leaf, ranking, budget_bytes, plan_bytes=None):
    """Move groups to slower-ranked leaf sizes that need fewer bytes until the batch fits."""
    if plan_bytes is None:
        per_tri = {}

        def plan_bytes(spec, lf):
            # bytes per triangle of a representative mesh of the group, times n
            key = (group_key(spec), lf)
            if key not in per_tri:
                rep = representative(spec)
                v, t = inputs.problem_mesh(rep)
                per_tri[key] = stored_bytes(Plan(v, t, leaf_size=lf, eta=2.0, order=spec["order"]),
                                            key[0][2]) / rep["n"]
            return per_tri[key] * spec["n"]
    cache = {}

    def bytes_of(spec, lf):
        k = (spec["index"], lf)
        if k not in cache:
            cache[k] = plan_bytes(spec, lf)
        return cache[k]

    leaf = dict(leaf)
    while True:
        total = sum(bytes_of(s, leaf[s["index"]]) for s in specs)
        if total <= budget_bytes:
            return leaf
        # among all groups and their slower-ranked candidates, take the switch that saves the most bytes
        best, save = None, 0
        for key, order in ranking.items():
            members = [s for s in specs if group_key(s) == key]
            cur = leaf[members[0]["index"]]
            for nxt in order[order.index(cur) + 1:]:
                d = sum(bytes_of(s, cur) - bytes_of(s, nxt) for s in members)
                if d > save:
                    best, save = (key, nxt), d
        if best is None:
            raise MemoryError(f"the batch needs {total} bytes at the smallest-memory leaf sizes; budget {budget_bytes}")
        for s in specs:
            if group_key(s) == best[0]:
                leaf[s["index"]] = best[1]
