"""ctypes wrapper of the C oracle (test infrastructure only)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "h2oracle.c")
_SO = os.path.join(_HERE, "libh2oracle.so")
_lock = threading.Lock()
_lib = None

KIND_LAPLACE = 0
KIND_POLY = 1
KIND_HELM_COS = 2   # real part of the Helmholtz kernel (Section 1): cos(kappa r) / (4 pi r)
KIND_HELM_SIN = 3   # imaginary part: sin(kappa r) / (4 pi r)


def build_library(force: bool = False) -> str:
    """Compile h2oracle.c with gcc (FP64, OpenMP, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            tmp = _SO + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                   _SRC, "-o", tmp, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build_library()
    lib = C.CDLL(_SO)
    dp = C.POINTER(C.c_double)
    ip64 = C.POINTER(C.c_int64)
    ip32 = C.POINTER(C.c_int32)
    u8p = C.POINTER(C.c_uint8)
    lib.or_build.restype = C.c_void_p
    lib.or_build.argtypes = [dp, C.c_int64, ip32, C.c_int64, C.c_int, C.c_double, C.c_int, C.c_int,
                             C.c_int, C.c_double, C.c_int, C.c_int]
    lib.or_free.argtypes = [C.c_void_p]
    lib.or_info.argtypes = [C.c_void_p, ip64]
    lib.or_tree.argtypes = [C.c_void_p, ip64, ip64, ip64, dp, dp, dp]
    lib.or_blocks.argtypes = [C.c_void_p, ip32, ip32, u8p]
    lib.or_V.argtypes = [C.c_void_p, dp]
    lib.or_E.argtypes = [C.c_void_p, C.c_int64, dp]
    lib.or_S.argtypes = [C.c_void_p, C.c_int64, C.c_int64, dp]
    lib.or_lagrange.argtypes = [C.c_void_p, C.c_int64, C.c_int, dp, C.c_int64, dp]
    lib.or_entry.restype = C.c_double
    lib.or_entry.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int]
    lib.or_pair_quad.restype = C.c_double
    lib.or_pair_quad.argtypes = [dp, dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double]
    lib.or_dense.argtypes = [C.c_void_p, dp]
    lib.or_matvec.restype = C.c_int
    lib.or_matvec.argtypes = [C.c_void_p, dp, dp, C.c_int, dp, dp]
    lib.or_matvec_rows.restype = C.c_int
    lib.or_matvec_rows.argtypes = [C.c_void_p, dp, C.c_int, ip64, C.c_int64, dp]
    lib.or_gmres.restype = C.c_int
    lib.or_gmres.argtypes = [C.c_void_p, dp, dp, C.c_int, C.c_double, C.c_int, C.c_int,
                             C.POINTER(C.c_int), dp]
    lib.or_gauss01.argtypes = [C.c_int, dp, dp]
    lib.or_threads.restype = C.c_int
    lib.or_gca_build.restype = C.c_void_p
    lib.or_gca_build.argtypes = [dp, C.c_int64, ip32, C.c_int64, C.c_int, C.c_double, C.c_int, C.c_double,
                                 C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
    lib.or_gca_free.argtypes = [C.c_void_p]
    lib.or_gca_h2.restype = C.c_void_p
    lib.or_gca_h2.argtypes = [C.c_void_p]
    lib.or_gca_ranks.argtypes = [C.c_void_p, ip32]
    lib.or_gca_pivots.argtypes = [C.c_void_p, C.c_int64, ip32]
    lib.or_gca_V.argtypes = [C.c_void_p, C.c_int64, dp]
    lib.or_gca_E.argtypes = [C.c_void_p, C.c_int64, dp]
    lib.or_gca_S.argtypes = [C.c_void_p, C.c_int64, C.c_int64, dp]
    lib.or_gca_matvec.restype = C.c_int
    lib.or_gca_matvec.argtypes = [C.c_void_p, dp, dp, C.c_int]
    lib.or_gca_matvec_rows.restype = C.c_int
    lib.or_gca_matvec_rows.argtypes = [C.c_void_p, dp, C.c_int, ip64, C.c_int64, dp]
    lib.or_gca_green_rule.restype = C.c_int
    lib.or_gca_green_rule.argtypes = [dp, dp, C.c_double, C.c_int, dp, dp, dp]
    lib.or_gca_aca.restype = C.c_int
    lib.or_gca_aca.argtypes = [dp, C.c_int, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                               dp]
    lib.or_set_threads.argtypes = [C.c_int]
    _lib = lib
    return lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def gauss01(n: int):
    """Gauss-Legendre nodes and weights on [0, 1] from the oracle."""
    lib = _load()
    x = np.zeros(n)
    w = np.zeros(n)
    lib.or_gauss01(n, _p(x, C.c_double), _p(w, C.c_double))
    return x, w


def pair_quad(T1, T2, mode: int, q: int, kind: int = KIND_LAPLACE, m: int = 1, kappa: float = 0.0) -> float:
    """Reference-domain integral of the kernel over T1 x T2 (no 4|T1||T2| factor).

    mode 0 regular, 1 identical (T1 only), 2 common edge T1[0]T1[1] = T2[0]T2[1],
    3 common vertex T1[0] = T2[0]."""
    lib = _load()
    a = np.ascontiguousarray(T1, dtype=np.float64).reshape(9)
    b = np.ascontiguousarray(T2, dtype=np.float64).reshape(9)
    return lib.or_pair_quad(_p(a, C.c_double), _p(b, C.c_double), mode, q, kind, m, float(kappa))


def threads() -> int:
    return _load().or_threads()


def set_threads(n: int) -> None:
    _load().or_set_threads(n)


class Oracle:
    """The oracle's H² approximation of one mesh (Section 2 of the paper)."""

    def __init__(self, vert, tri, leaf_size=32, eta=2.0, order=3, quad_order=3,
                 kind=KIND_LAPLACE, store_near=True, with_bases=True, kappa=0.0):
        lib = _load()
        self._lib = lib
        self.vert = np.ascontiguousarray(vert, dtype=np.float64)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        self.n = int(self.tri.shape[0])
        self.m = int(order)
        self.k = self.m ** 3
        h = lib.or_build(_p(self.vert, C.c_double), self.vert.shape[0], _p(self.tri, C.c_int32), self.n,
                         int(leaf_size), float(eta), self.m, int(quad_order), int(kind), float(kappa),
                         int(store_near),
                         int(with_bases))
        if not h:
            raise ValueError("oracle: invalid arguments")
        self._h = C.c_void_p(h)
        info = np.zeros(7, dtype=np.int64)
        lib.or_info(self._h, _p(info, C.c_int64))
        (self.depth, self.nclu, self.nblk, self.nadm, self.nnear, self.near_entries, _) = (int(v) for v in info)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.or_free(h)
            self._h = None

    # ---- structure ----
    def tree(self):
        nc = self.nclu
        idx = np.zeros(self.n, dtype=np.int64)
        first = np.zeros(nc, dtype=np.int64)
        size = np.zeros(nc, dtype=np.int64)
        lo = np.zeros((nc, 3))
        hi = np.zeros((nc, 3))
        pts = np.zeros((nc, 3, self.m))
        self._lib.or_tree(self._h, _p(idx, C.c_int64), _p(first, C.c_int64), _p(size, C.c_int64),
                          _p(lo, C.c_double), _p(hi, C.c_double), _p(pts, C.c_double))
        return dict(idx=idx, first=first, size=size, lo=lo, hi=hi, pts=pts)

    def blocks(self):
        t = np.zeros(self.nblk, dtype=np.int32)
        s = np.zeros(self.nblk, dtype=np.int32)
        a = np.zeros(self.nblk, dtype=np.uint8)
        self._lib.or_blocks(self._h, _p(t, C.c_int32), _p(s, C.c_int32), _p(a, C.c_uint8))
        return t, s, a.astype(bool)

    def V(self):
        v = np.zeros((self.n, self.k))
        self._lib.or_V(self._h, _p(v, C.c_double))
        return v

    def E(self, c: int):
        e = np.zeros((self.k, self.k))
        self._lib.or_E(self._h, int(c), _p(e, C.c_double))
        return e

    def S(self, t: int, s: int):
        out = np.zeros((self.k, self.k))
        self._lib.or_S(self._h, int(t), int(s), _p(out, C.c_double))
        return out

    def lagrange(self, c: int, nu: int, x):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        out = np.zeros(x.shape[0])
        self._lib.or_lagrange(self._h, int(c), int(nu), _p(x, C.c_double), x.shape[0], _p(out, C.c_double))
        return out

    def entry(self, i: int, j: int, q: int | None = None) -> float:
        return self._lib.or_entry(self._h, int(i), int(j), int(q if q is not None else 3))

    def dense(self):
        g = np.zeros((self.n, self.n), order="F")
        self._lib.or_dense(self._h, _p(g, C.c_double))
        return g

    # ---- products and solves ----
    def matvec(self, x, coeffs: bool = False):
        x = np.asfortranarray(np.asarray(x, dtype=np.float64).reshape(self.n, -1))
        nrhs = x.shape[1]
        y = np.zeros((self.n, nrhs), order="F")
        if coeffs:
            xh = np.zeros((self.nclu, self.k, nrhs))
            yh = np.zeros((self.nclu, self.k, nrhs))
            rc = self._lib.or_matvec(self._h, _p(x, C.c_double), _p(y, C.c_double), nrhs,
                                     _p(xh, C.c_double), _p(yh, C.c_double))
        else:
            rc = self._lib.or_matvec(self._h, _p(x, C.c_double), _p(y, C.c_double), nrhs, None, None)
        if rc:
            raise RuntimeError("oracle built without bases")
        return (y, xh, yh) if coeffs else y

    def matvec_rows(self, x, rows):
        x = np.asfortranarray(np.asarray(x, dtype=np.float64).reshape(self.n, -1))
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        nrhs = x.shape[1]
        out = np.zeros((rows.shape[0], nrhs), order="F")
        rc = self._lib.or_matvec_rows(self._h, _p(x, C.c_double), nrhs, _p(rows, C.c_int64), rows.shape[0],
                                      _p(out, C.c_double))
        if rc:
            raise RuntimeError("oracle built without bases")
        return out

    def gmres(self, b, rtol=1e-8, restart=30, maxit=1000):
        b = np.asfortranarray(np.asarray(b, dtype=np.float64).reshape(self.n, -1))
        nrhs = b.shape[1]
        z = np.zeros((self.n, nrhs), order="F")
        iters = np.zeros(nrhs, dtype=np.int32)
        rel = np.zeros(nrhs)
        self._lib.or_gmres(self._h, _p(b, C.c_double), _p(z, C.c_double), nrhs, float(rtol), int(restart),
                           int(maxit), iters.ctypes.data_as(C.POINTER(C.c_int)), _p(rel, C.c_double))
        return z, iters, rel


class HelmholtzOracle:
    """The Helmholtz single-layer matrix of Section 1, G = G_c + i G_s, as two
    oracle H^2 matrices of the same mesh and trees with the real kernels
    cos(kappa r) / (4 pi r) and sin(kappa r) / (4 pi r); complex vectors are
    numpy complex128 arrays (n, nrhs)."""

    def __init__(self, vert, tri, kappa, leaf_size=32, eta=2.0, order=3, quad_order=3, store_near=True,
                 with_bases=True):
        kw = dict(leaf_size=leaf_size, eta=eta, order=order, quad_order=quad_order, store_near=store_near,
                  with_bases=with_bases, kappa=kappa)
        self.c = Oracle(vert, tri, kind=KIND_HELM_COS, **kw)
        self.s = Oracle(vert, tri, kind=KIND_HELM_SIN, **kw)
        self.n = self.c.n
        self.kappa = float(kappa)

    def matvec(self, x):
        x = np.asarray(x, dtype=np.complex128).reshape(self.n, -1)
        xr, xi = np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)
        return (self.c.matvec(xr) - self.s.matvec(xi)) + 1j * (self.c.matvec(xi) + self.s.matvec(xr))

    def matvec_rows(self, x, rows):
        x = np.asarray(x, dtype=np.complex128).reshape(self.n, -1)
        xr, xi = np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)
        c, s = self.c.matvec_rows, self.s.matvec_rows
        return (c(xr, rows) - s(xi, rows)) + 1j * (c(xi, rows) + s(xr, rows))

    def dense(self):
        return self.c.dense() + 1j * self.s.dense()

    def entry(self, i, j, q=None):
        return self.c.entry(i, j, q) + 1j * self.s.entry(i, j, q)


def green_rule(lo, hi, gamma: float, qg: int):
    """The oracle's quadrature on the boundary of the box [lo - gamma rho,
    hi + gamma rho] (rho = half diagonal): points (Q, 3), outward normals
    (Q, 3), weights (Q,)."""
    lib = _load()
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    q = 6 * qg * qg
    Z, N, W = np.zeros((q, 3)), np.zeros((q, 3)), np.zeros(q)
    lib.or_gca_green_rule(_p(lo, C.c_double), _p(hi, C.c_double), float(gamma), int(qg), _p(Z, C.c_double),
                          _p(N, C.c_double), _p(W, C.c_double))
    return Z, N, W


def aca(M, eps: float, max_rank: int = 0):
    """The oracle's cross approximation with complete pivoting of M (nr, nc),
    at most max_rank pivots (0: no cap): row pivots I, column pivots J and
    V^ = M[:, J] M[I, J]^{-1} (nr, k)."""
    lib = _load()
    M = np.ascontiguousarray(M, dtype=np.float64)
    nr, nc = M.shape
    kc = min(nr, nc)
    I = np.zeros(kc, dtype=np.int32)
    J = np.zeros(kc, dtype=np.int32)
    Vh = np.zeros(nr * kc)
    k = lib.or_gca_aca(_p(M, C.c_double), nr, nc, float(eps), int(max_rank), I.ctypes.data_as(C.POINTER(C.c_int)),
                       J.ctypes.data_as(C.POINTER(C.c_int)), _p(Vh, C.c_double))
    return I[:k].copy(), J[:k].copy(), Vh[:nr * k].reshape(nr, k).copy()


class GcaOracle:
    """The oracle's GCA-H^2 matrix of one mesh (Section 3's GCA-H^2 example:
    pivot elements per cluster, nested through the sons' pivots, and the
    coupling S = G on the pivot pairs), Laplace kernel."""

    def __init__(self, vert, tri, leaf_size=32, eta=2.0, green_order=4, eps=1e-4, gamma=1.0, tri_order=3,
                 max_rank=128, quad_order=3, store_near=True, store_S=True):
        lib = _load()
        self._lib = lib
        self.vert = np.ascontiguousarray(vert, dtype=np.float64)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        self.n = int(self.tri.shape[0])
        g = lib.or_gca_build(_p(self.vert, C.c_double), self.vert.shape[0], _p(self.tri, C.c_int32), self.n,
                             int(leaf_size), float(eta), int(green_order), float(eps), float(gamma), int(tri_order),
                             int(max_rank), int(quad_order), int(store_near), int(store_S))
        if not g:
            raise ValueError("oracle: invalid arguments")
        self._g = C.c_void_p(g)
        self._h = C.c_void_p(lib.or_gca_h2(self._g))
        info = np.zeros(7, dtype=np.int64)
        lib.or_info(self._h, _p(info, C.c_int64))
        (self.depth, self.nclu, self.nblk, self.nadm, self.nnear, self.near_entries, _) = (int(v) for v in info)
        self.rank = np.zeros(self.nclu, dtype=np.int32)
        lib.or_gca_ranks(self._g, _p(self.rank, C.c_int32))

    def __del__(self):
        g = getattr(self, "_g", None)
        if g is not None and g.value:
            self._lib.or_gca_free(g)
            self._g = None

    def tree(self):
        nc = self.nclu
        idx = np.zeros(self.n, dtype=np.int64)
        first = np.zeros(nc, dtype=np.int64)
        size = np.zeros(nc, dtype=np.int64)
        lo = np.zeros((nc, 3))
        hi = np.zeros((nc, 3))
        pts = np.zeros((nc, 3, 1))
        self._lib.or_tree(self._h, _p(idx, C.c_int64), _p(first, C.c_int64), _p(size, C.c_int64),
                          _p(lo, C.c_double), _p(hi, C.c_double), _p(pts, C.c_double))
        return dict(idx=idx, first=first, size=size, lo=lo, hi=hi)

    def blocks(self):
        t = np.zeros(self.nblk, dtype=np.int32)
        s = np.zeros(self.nblk, dtype=np.int32)
        a = np.zeros(self.nblk, dtype=np.uint8)
        self._lib.or_blocks(self._h, _p(t, C.c_int32), _p(s, C.c_int32), _p(a, C.c_uint8))
        return t, s, a.astype(bool)

    def pivots(self, c: int):
        out = np.zeros(int(self.rank[c]), dtype=np.int32)
        self._lib.or_gca_pivots(self._g, int(c), _p(out, C.c_int32))
        return out

    def V(self, c: int, size: int):
        out = np.zeros((size, int(self.rank[c])))
        self._lib.or_gca_V(self._g, int(c), _p(out, C.c_double))
        return out

    def E(self, c: int):
        out = np.zeros((int(self.rank[c]), int(self.rank[(c - 1) // 2])))
        self._lib.or_gca_E(self._g, int(c), _p(out, C.c_double))
        return out

    def S(self, t: int, s: int):
        out = np.zeros((int(self.rank[t]), int(self.rank[s])))
        self._lib.or_gca_S(self._g, int(t), int(s), _p(out, C.c_double))
        return out

    def entry(self, i: int, j: int, q: int | None = None) -> float:
        return self._lib.or_entry(self._h, int(i), int(j), int(q if q is not None else 3))

    def dense(self):
        """The Galerkin matrix itself (every pair by the nearfield rule)."""
        g = np.zeros((self.n, self.n), order="F")
        self._lib.or_dense(self._h, _p(g, C.c_double))
        return g

    def matvec(self, x):
        x = np.asfortranarray(np.asarray(x, dtype=np.float64).reshape(self.n, -1))
        y = np.zeros(x.shape, order="F")
        self._lib.or_gca_matvec(self._g, _p(x, C.c_double), _p(y, C.c_double), x.shape[1])
        return y

    def matvec_rows(self, x, rows):
        x = np.asfortranarray(np.asarray(x, dtype=np.float64).reshape(self.n, -1))
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.zeros((rows.shape[0], x.shape[1]), order="F")
        self._lib.or_gca_matvec_rows(self._g, _p(x, C.c_double), x.shape[1], _p(rows, C.c_int64), rows.shape[0],
                                     _p(out, C.c_double))
        return out
