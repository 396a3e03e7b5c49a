"""Seeded synthetic inputs shared by the oracle and the GPU path.

This module holds no arithmetic of the H²-matrix method: it only produces
the surface meshes and right-hand sides both sides consume.

* ``icosphere(L)``: polyhedral approximation of the unit sphere (the paper's
  test surface, Section 3 experiments) obtained by ``L`` regular refinements of
  the icosahedron, midpoints projected to the sphere.
* ``ellipsoid(L, axes)``: the icosphere with coordinates scaled per axis.
* ``cube(s)``: the surface of [-1, 1]^3 with s x s squares per face, each
  square split into two triangles along one diagonal.
* ``uniform_rhs(n, nrhs, seed)``: entries uniform in [-1, 1].
* ``batch_problems(nprob, seed)``: the uneven batch of independent problems
  (random ellipsoids and subdivided cubes of 20k to 400k triangles, order 3
  or 4, 1 to 8 right-hand sides); ``problem_mesh(spec)`` builds one mesh.

Triangles are returned as int32 (nt, 3) vertex indices oriented so that the
normal (b - a) x (c - a) points out of the enclosed volume; vertices are
float64 (nv, 3).
"""
from __future__ import annotations

import numpy as np

GOLDEN = (1.0 + 5.0 ** 0.5) / 2.0


def _icosahedron():
    raw = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            raw.append((0.0, s1, s2 * GOLDEN))
            raw.append((s1, s2 * GOLDEN, 0.0))
            raw.append((s2 * GOLDEN, 0.0, s1))
    v = np.array(raw, dtype=np.float64)
    # faces: triples of mutually adjacent vertices (edge length 2 before scaling)
    nv = len(v)
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=2)
    adj = np.abs(d - 2.0) < 1e-9
    faces = []
    for a in range(nv):
        for b in range(a + 1, nv):
            if not adj[a, b]:
                continue
            for c in range(b + 1, nv):
                if adj[a, c] and adj[b, c]:
                    faces.append((a, b, c))
    assert len(faces) == 20
    v = v / np.linalg.norm(v, axis=1, keepdims=True)
    out = []
    for a, b, c in faces:
        n = np.cross(v[b] - v[a], v[c] - v[a])
        if np.dot(n, v[a] + v[b] + v[c]) < 0.0:
            b, c = c, b
        out.append((a, b, c))
    return v, np.array(out, dtype=np.int64)


def icosphere(level: int):
    """Icosahedron refined ``level`` times: 20*4^level triangles on the unit sphere."""
    if level < 0:
        raise ValueError("level must be >= 0")
    v, f = _icosahedron()
    verts = [tuple(p) for p in v]
    for _ in range(level):
        edge_mid = {}
        newf = []

        def mid(i, j):
            key = (i, j) if i < j else (j, i)
            idx = edge_mid.get(key)
            if idx is None:
                p = np.array(verts[i]) + np.array(verts[j])
                p = p / np.sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2])
                idx = len(verts)
                verts.append(tuple(p))
                edge_mid[key] = idx
            return idx

        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            newf.extend([(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)])
        f = np.array(newf, dtype=np.int64)
    return np.array(verts, dtype=np.float64), f.astype(np.int32)


def ellipsoid(level: int, axes):
    """Icosphere of the given level with x, y, z scaled by ``axes``."""
    v, f = icosphere(level)
    return v * np.asarray(axes, dtype=np.float64)[None, :], f


def cube(s: int):
    """Surface of [-1,1]^3, s x s squares per face, 12 s^2 outward triangles."""
    if s < 1:
        raise ValueError("s must be >= 1")
    index = {}
    verts = []

    def vid(p):
        k = index.get(p)
        if k is None:
            k = len(verts)
            index[p] = k
            verts.append(p)
        return k

    tris = []
    for axis in range(3):
        u_ax, v_ax = (axis + 1) % 3, (axis + 2) % 3
        for side in (0, s):
            for i in range(s):
                for j in range(s):
                    def P(a, b):
                        p = [0, 0, 0]
                        p[axis] = side
                        p[u_ax] = a
                        p[v_ax] = b
                        return vid(tuple(p))
                    p00, p10, p11, p01 = P(i, j), P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)
                    # (u, v, axis) is right-handed, so (p00, p10, p11) has normal +axis
                    if side == s:
                        tris.append((p00, p10, p11))
                        tris.append((p00, p11, p01))
                    else:
                        tris.append((p00, p11, p10))
                        tris.append((p00, p01, p11))
    v = np.array(verts, dtype=np.float64) * (2.0 / s) - 1.0
    return v, np.array(tris, dtype=np.int32)


def uniform_rhs(n: int, nrhs: int, seed: int):
    """n x nrhs right-hand sides, entries uniform in [-1, 1], Fortran (column-major) order."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.uniform(-1.0, 1.0, (n, nrhs)))


def batch_problems(nprob: int = 64, seed: int = 1004):
    """Specifications of an uneven batch, drawn in problem order from one generator.

    Even index: ellipsoid = icosphere of level 5, 6 or 7 (20,480 / 81,920 /
    327,680 triangles) with semi-axes uniform in [0.5, 2].  Odd index: cube
    with s uniform in {41, ..., 182} (12 s^2 = 20,172 ... 397,488 triangles).
    Then the interpolation order m in {3, 4} and nrhs uniform in {1, ..., 8}.
    The leaf size is not drawn: an autotuner chooses it.
    """
    rng = np.random.default_rng(seed)
    specs = []
    for p in range(nprob):
        if p % 2 == 0:
            level = int(rng.integers(5, 8))
            axes = [float(a) for a in rng.uniform(0.5, 2.0, 3)]
            spec = dict(kind="ellipsoid", level=level, axes=axes, n=20 * 4 ** level)
        else:
            s = int(rng.integers(41, 183))
            spec = dict(kind="cube", s=s, n=12 * s * s)
        spec["order"] = int(rng.integers(3, 5))
        spec["nrhs"] = int(rng.integers(1, 9))
        spec["index"] = p
        specs.append(spec)
    return specs


def problem_mesh(spec):
    """(vert, tri) of a batch_problems specification."""
    if spec["kind"] == "ellipsoid":
        return ellipsoid(spec["level"], spec["axes"])
    if spec["kind"] == "cube":
        return cube(spec["s"])
    if spec["kind"] == "icosphere":
        return icosphere(spec["level"])
    raise ValueError(f"unknown mesh kind {spec['kind']!r}")
