"""Seeded input meshes: counts, topology and orientation."""
import numpy as np
import pytest

from paper_2203_05665_gb300 import inputs as I


def _areas(v, f):
    return 0.5 * np.linalg.norm(np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]]), axis=1)


def _signed_volume(v, f):
    return np.einsum("ij,ij->i", v[f[:, 0]], np.cross(v[f[:, 1]], v[f[:, 2]])).sum() / 6.0


@pytest.mark.parametrize("L", [0, 1, 2, 3, 4])
def test_icosphere_counts_and_geometry(L):
    v, f = I.icosphere(L)
    nv, nt = v.shape[0], f.shape[0]
    edges = {tuple(sorted(e)) for t in f for e in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0]))}
    assert nv == 10 * 4 ** L + 2
    assert nt == 20 * 4 ** L
    assert len(edges) == 30 * 4 ** L
    assert nv - len(edges) + nt == 2                      # Euler characteristic of the sphere
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-15)
    # every edge is shared by exactly two triangles, traversed in opposite directions
    directed = {(t[a], t[(a + 1) % 3]) for t in f for a in range(3)}
    assert len(directed) == 3 * nt
    assert all((b, a) in directed for a, b in directed)
    assert _signed_volume(v, f) > 0                       # outward orientation
    assert _areas(v, f).sum() < 4 * np.pi


def test_icosphere_area_increases_to_sphere():
    s = [_areas(*I.icosphere(L)).sum() for L in range(6)]
    assert all(a < b for a, b in zip(s, s[1:])) and s[-1] < 4 * np.pi and 4 * np.pi - s[-1] < 1e-2


@pytest.mark.parametrize("s", [1, 2, 5])
def test_cube(s):
    v, f = I.cube(s)
    assert f.shape[0] == 12 * s * s
    assert v.shape[0] == 6 * s * s + 2
    assert abs(_signed_volume(v, f) - 8.0) < 1e-12
    assert abs(_areas(v, f).sum() - 24.0) < 1e-12
    n = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    c = v[f].mean(axis=1)
    assert np.all(np.einsum("ij,ij->i", n, c) > 0)       # each normal points away from the centre


def test_ellipsoid_and_rhs():
    v, f = I.ellipsoid(2, (2.0, 1.0, 0.5))
    assert np.allclose(((v / np.array([2.0, 1.0, 0.5])) ** 2).sum(axis=1), 1.0)
    b1 = I.uniform_rhs(100, 3, 7)
    b2 = I.uniform_rhs(100, 3, 7)
    assert b1.flags.f_contiguous and np.array_equal(b1, b2)
    assert b1.min() >= -1 and b1.max() <= 1
