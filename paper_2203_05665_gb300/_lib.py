"""ctypes binding of libh2 (include/h2.h): argument marshalling only.

Every computation runs in the compiled library; if libh2.so is missing the
calls raise instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
import weakref

import numpy as np

from . import _build

H2_OK, H2_EINVAL, H2_ENOMEM, H2_ECUDA, H2_ENOCONV, H2_ETIMEOUT, H2_PENDING, H2_EBUSY = range(8)
H2_F64, H2_F32, H2_F64_NATIVE, H2_BF16, H2_F16 = 0, 1, 2, 3, 4
PREC = {"f64": H2_F64, "f32": H2_F32, "f64n": H2_F64_NATIVE, "bf16": H2_BF16, "f16": H2_F16}
COUPLING = {"auto": 0, "stored": 1, "regen": 2}

_lock = threading.Lock()
_lib = None


class H2Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libh2 status {status}: {msg}")
        self.status = status


class Options(C.Structure):
    _fields_ = [("prec", C.c_int), ("quad_order", C.c_int), ("device", C.c_int), ("stream", C.c_void_p),
                ("coupling", C.c_int), ("tensor", C.c_int), ("basis_prec", C.c_int), ("fused", C.c_int),
                ("reserved", C.c_int * 4)]


class Stats(C.Structure):
    _fields_ = [(name, C.c_int64) for name in
                ("n", "depth", "clusters", "leaf_max", "order", "rank", "adm_blocks", "near_blocks",
                 "near_entries", "first_adm_level", "device_bytes", "prec", "coupling", "tensor",
                 "tensor_near", "basis_prec", "gca", "coupling_entries", "tensor_leaf")]


class GcaOptions(C.Structure):
    _fields_ = [("eps", C.c_double), ("gamma", C.c_double), ("green_order", C.c_int), ("tri_order", C.c_int),
                ("max_rank", C.c_int), ("reserved", C.c_int * 5)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("relres", C.c_double)]


EXPORTED = ["h2_options_default", "h2_plan_create", "h2_plan_destroy", "h2_plan_counts", "h2_plan_tree",
            "h2_plan_blocks", "h2_plan_bases", "h2_build", "h2_destroy", "h2_info", "h2_matvec", "h2_matvec_acc",
            "h2_matvec_noalloc", "h2_matvec_host", "h2_matvec_host_stream", "h2_coefficients", "h2_solve", "h2_solve_ir", "h2_profile", "h2_phase_times",
            "h2_serve_create", "h2_serve_register", "h2_serve_submit", "h2_serve_poll", "h2_serve_wait",
            "h2_serve_stats", "h2_serve_destroy", "h2_batch_create", "h2_batch_offsets", "h2_batch_matvec",
            "h2_batch_tune", "h2_batch_set_shapes", "h2_batch_profile", "h2_batch_phase_times", "h2_batch_info",
            "h2_batch_sync", "h2_batch_destroy", "h2_graph_create", "h2_graph_launch", "h2_graph_destroy",
            "h2_inject_alloc_failure", "h2_wait_selftest", "h2_export", "h2_build_times",
            "h2_gca_options_default", "h2_build_gca", "h2_gca_pivots", "h2_zbuild", "h2_zdestroy", "h2_zpart", "h2_zinfo", "h2_zmatvec", "h2_zmatvec_host", "h2_zsolve", "h2_last_error"]
PHASES = ["permute_in", "leaf_forward", "upward", "coupling", "downward", "leaf_near", "permute_out"]


def library_path() -> str:
    return _build.LIB


def load():
    """Load libh2.so (built by ``__graft_entry__.build()`` / ``_build.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libh2.so not found at {_build.LIB}: run __graft_entry__.build() first")
        lib = C.CDLL(_build.LIB)
        vp, dp, i64p, i32p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int32)
        sig = {
            "h2_options_default": (C.c_int, [C.POINTER(Options)]),
            "h2_plan_create": (C.c_int, [dp, C.c_int64, i32p, C.c_int64, C.c_int, C.c_double, C.c_int,
                                         C.POINTER(vp)]),
            "h2_plan_destroy": (C.c_int, [vp]),
            "h2_plan_counts": (C.c_int, [vp, i64p]),
            "h2_plan_tree": (C.c_int, [vp, i64p, i64p, i64p, dp, dp]),
            "h2_plan_blocks": (C.c_int, [vp, i32p, i32p, i32p, i32p]),
            "h2_plan_bases": (C.c_int, [vp, dp, dp]),
            "h2_build": (C.c_int, [dp, C.c_int64, i32p, C.c_int64, C.c_int, C.c_double, C.c_int,
                                   C.POINTER(Options), C.POINTER(vp)]),
            "h2_destroy": (C.c_int, [vp]),
            "h2_info": (C.c_int, [vp, C.POINTER(Stats)]),
            "h2_matvec": (C.c_int, [vp, vp, vp, C.c_int]),
            "h2_matvec_acc": (C.c_int, [vp, vp, vp, C.c_int]),
            "h2_matvec_noalloc": (C.c_int, [vp, vp, vp, C.c_int]),
            "h2_matvec_host": (C.c_int, [vp, dp, dp, C.c_int]),
            "h2_matvec_host_stream": (C.c_int, [vp, dp, dp, C.c_int, C.c_int]),
            "h2_coefficients": (C.c_int, [vp, C.c_int, dp]),
            "h2_solve": (C.c_int, [vp, vp, vp, C.c_int, C.c_double, C.c_int, C.c_int, C.POINTER(SolveInfo)]),
            "h2_solve_ir": (C.c_int, [vp, vp, vp, vp, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
                                      C.POINTER(SolveInfo)]),
            "h2_profile": (C.c_int, [vp, C.c_int]),
            "h2_phase_times": (C.c_int, [vp, dp, i64p, i64p]),
            "h2_serve_create": (C.c_int, [C.c_int, C.c_size_t, C.POINTER(vp)]),
            "h2_serve_register": (C.c_int, [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_double]),
            "h2_serve_submit": (C.c_int, [vp, vp, dp, C.c_int, C.c_double, C.POINTER(C.c_uint64)]),
            "h2_serve_poll": (C.c_int, [vp, C.c_uint64, dp, C.POINTER(SolveInfo)]),
            "h2_serve_wait": (C.c_int, [vp, C.c_uint64, C.c_double]),
            "h2_serve_stats": (C.c_int, [vp, i64p]),
            "h2_serve_destroy": (C.c_int, [vp]),
            "h2_batch_create": (C.c_int, [C.POINTER(vp), C.c_int, C.POINTER(C.c_int), vp, C.POINTER(vp)]),
            "h2_batch_offsets": (C.c_int, [vp, i64p]),
            "h2_batch_matvec": (C.c_int, [vp, vp, vp]),
            "h2_batch_tune": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int)]),
            "h2_batch_set_shapes": (C.c_int, [vp, C.POINTER(C.c_int)]),
            "h2_batch_profile": (C.c_int, [vp, C.c_int]),
            "h2_batch_phase_times": (C.c_int, [vp, dp, i64p, i64p]),
            "h2_batch_info": (C.c_int, [vp, i64p]),
            "h2_batch_sync": (C.c_int, [vp]),
            "h2_batch_destroy": (C.c_int, [vp]),
            "h2_graph_create": (C.c_int, [vp, vp, vp, C.c_int, C.POINTER(vp)]),
            "h2_graph_launch": (C.c_int, [vp]),
            "h2_graph_destroy": (C.c_int, [vp]),
            "h2_inject_alloc_failure": (C.c_int, [C.c_int64]),
            "h2_export": (C.c_int, [vp, C.c_int, C.c_int64, C.c_int64, dp]),
            "h2_build_times": (C.c_int, [vp, dp]),
            "h2_zbuild": (C.c_int, [dp, C.c_int64, i32p, C.c_int64, C.c_int, C.c_double, C.c_int, C.c_double,
                                    C.POINTER(Options), C.POINTER(vp)]),
            "h2_zdestroy": (C.c_int, [vp]),
            "h2_zpart": (C.c_int, [vp, C.c_int, C.POINTER(vp)]),
            "h2_zinfo": (C.c_int, [vp, C.POINTER(Stats)]),
            "h2_zmatvec": (C.c_int, [vp, vp, vp, C.c_int]),
            "h2_zmatvec_host": (C.c_int, [vp, dp, dp, C.c_int]),
            "h2_zsolve": (C.c_int, [vp, vp, vp, C.c_int, C.c_double, C.c_int, C.c_int, C.POINTER(SolveInfo)]),
            "h2_wait_selftest": (C.c_int, [vp, C.c_int, C.c_uint32, C.POINTER(C.c_int)]),
            "h2_gca_options_default": (C.c_int, [C.POINTER(GcaOptions)]),
            "h2_build_gca": (C.c_int, [dp, C.c_int64, i32p, C.c_int64, C.c_int, C.c_double, C.POINTER(GcaOptions),
                                       C.POINTER(Options), C.POINTER(vp)]),
            "h2_gca_pivots": (C.c_int, [vp, i32p, i32p, C.c_int64]),
            "h2_last_error": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(status):
    if status != H2_OK:
        raise H2Error(status, load().h2_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _mesh(vert, tri):
    v = np.ascontiguousarray(vert, dtype=np.float64)
    t = np.ascontiguousarray(tri, dtype=np.int32)
    if v.ndim != 2 or v.shape[1] != 3 or t.ndim != 2 or t.shape[1] != 3:
        raise ValueError("vert must be (nv, 3) and tri (nt, 3)")
    return v, t


class Plan:
    """Host-only planning (trees, blocks, V, transfer factors); needs no GPU."""

    def __init__(self, vert, tri, leaf_size=32, eta=2.0, order=3):
        lib = load()
        v, t = _mesh(vert, tri)
        h = C.c_void_p()
        _check(lib.h2_plan_create(_dp(v), v.shape[0], t.ctypes.data_as(C.POINTER(C.c_int32)), t.shape[0],
                                  int(leaf_size), float(eta), int(order), C.byref(h)))
        self._h = h
        self._lib = lib
        self.m = int(order)
        self.k = self.m ** 3
        cnt = np.zeros(8, dtype=np.int64)
        _check(lib.h2_plan_counts(h, cnt.ctypes.data_as(C.POINTER(C.c_int64))))
        (self.n, self.depth, self.nclu, self.leaf_max, self.nadm, self.nnear, self.near_entries,
         self.first_adm_level) = (int(x) for x in cnt)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.h2_plan_destroy(h)
            self._h = None

    def tree(self):
        i64 = lambda n: np.zeros(n, dtype=np.int64)
        perm, first, size = i64(self.n), i64(self.nclu), i64(self.nclu)
        lo, hi = np.zeros((self.nclu, 3)), np.zeros((self.nclu, 3))
        p64 = lambda a: a.ctypes.data_as(C.POINTER(C.c_int64))
        _check(self._lib.h2_plan_tree(self._h, p64(perm), p64(first), p64(size), _dp(lo), _dp(hi)))
        return dict(perm=perm, first=first, size=size, lo=lo, hi=hi)

    def blocks(self):
        i32 = lambda n: np.zeros(n, dtype=np.int32)
        at, as_, nt, ns = i32(self.nadm), i32(self.nadm), i32(self.nnear), i32(self.nnear)
        p32 = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
        _check(self._lib.h2_plan_blocks(self._h, p32(at), p32(as_), p32(nt), p32(ns)))
        return (at, as_), (nt, ns)

    def bases(self):
        V = np.zeros((self.n, self.k))
        E = np.zeros((self.nclu, 3, self.m, self.m))
        _check(self._lib.h2_plan_bases(self._h, _dp(V), _dp(E)))
        return V, E


def colmajor(t):
    """A column-major (n, nrhs) view of a torch tensor (copies if needed)."""
    if t.dim() == 1:
        t = t[:, None]
    if t.stride(0) == 1 and (t.shape[1] == 1 or t.stride(1) == t.shape[0]):
        return t
    return t.t().contiguous().t()


class H2Matrix:
    """An H² matrix of one mesh on one GPU (see include/h2.h)."""

    def __init__(self, vert, tri, leaf_size=32, eta=2.0, order=3, prec="f64", quad_order=3, device=0,
                 stream=None, coupling="auto", tensor="auto", basis=None, gca=None, fused=False):
        lib = load()
        v, t = _mesh(vert, tri)
        opt = Options()
        _check(lib.h2_options_default(C.byref(opt)))
        opt.prec = PREC[prec]
        opt.quad_order = int(quad_order)
        opt.device = int(device)
        opt.stream = stream
        opt.coupling = COUPLING[coupling]
        opt.tensor = {"auto": 0, "off": 1}[tensor]
        opt.basis_prec = 0 if basis is None else PREC[basis]
        opt.fused = 1 if fused else 0
        h = C.c_void_p()
        if gca is None:
            _check(lib.h2_build(_dp(v), v.shape[0], t.ctypes.data_as(C.POINTER(C.c_int32)), t.shape[0],
                                int(leaf_size), float(eta), int(order), C.byref(opt), C.byref(h)))
        else:
            g = GcaOptions()
            _check(lib.h2_gca_options_default(C.byref(g)))
            for key, val in gca.items():
                setattr(g, key, val)
            _check(lib.h2_build_gca(_dp(v), v.shape[0], t.ctypes.data_as(C.POINTER(C.c_int32)), t.shape[0],
                                    int(leaf_size), float(eta), C.byref(g), C.byref(opt), C.byref(h)))
        self._h = h
        self._lib = lib
        self.prec = prec
        self.n = int(t.shape[0])
        self.device = int(device)
        st = Stats()
        _check(lib.h2_info(h, C.byref(st)))
        self.stats = {f: int(getattr(st, f)) for f, _ in Stats._fields_}

    def close(self):
        for g in list(getattr(self, "_graphs", ())):
            g.close()   # a graph refers to the handle: destroy it first
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.h2_destroy(h)
            self._h = None

    def __del__(self):
        self.close()

    @property
    def handle(self):
        return self._h

    def matvec(self, x, y):
        """y = G~ x on the device; x, y column-major CUDA tensors (n, nrhs) of the handle's dtype."""
        if x.shape != y.shape or x.shape[0] != self.n:
            raise ValueError("x and y must both be (n, nrhs)")
        if x.stride(0) != 1 or y.stride(0) != 1:
            raise ValueError("x and y must be column-major (use colmajor())")
        _check(self._lib.h2_matvec(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), int(x.shape[1])))
        return y

    def matvec_acc(self, x, y):
        """y <- y + G~ x on the device (h2_matvec_acc); x, y as for matvec."""
        if x.shape != y.shape or x.shape[0] != self.n:
            raise ValueError("x and y must both be (n, nrhs)")
        if x.stride(0) != 1 or y.stride(0) != 1:
            raise ValueError("x and y must be column-major (use colmajor())")
        _check(self._lib.h2_matvec_acc(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                       int(x.shape[1])))
        return y

    def matvec_noalloc(self, x, y):
        """As matvec, through h2_matvec_noalloc: no device allocation, fixed 64 MiB work space."""
        if x.shape != y.shape or x.shape[0] != self.n:
            raise ValueError("x and y must both be (n, nrhs)")
        if x.stride(0) != 1 or y.stride(0) != 1:
            raise ValueError("x and y must be column-major (use colmajor())")
        _check(self._lib.h2_matvec_noalloc(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                           int(x.shape[1])))
        return y

    def graph(self, x, y):
        """The product y = G~ x for these fixed device buffers, captured once as a CUDA graph.

        Returns a ProductGraph whose launch() replays it on the handle's stream;
        x and y must stay alive (and in place) while the graph is used.
        """
        if x.shape != y.shape or x.shape[0] != self.n:
            raise ValueError("x and y must both be (n, nrhs)")
        if x.stride(0) != 1 or y.stride(0) != 1:
            raise ValueError("x and y must be column-major (use colmajor())")
        g = C.c_void_p()
        _check(self._lib.h2_graph_create(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                         int(x.shape[1]), C.byref(g)))
        pg = ProductGraph(self, g, (x, y))
        if not hasattr(self, "_graphs"):
            self._graphs = weakref.WeakSet()
        self._graphs.add(pg)
        return pg

    def profile(self, enable=True):
        """Start (or stop) per-phase CUDA-event timing on the handle's stream."""
        _check(self._lib.h2_profile(self._h, 1 if enable else 0))

    def phase_times(self):
        """{phase: (ms total, kernel launches)} since profile(True), and the products timed."""
        ms = np.zeros(len(PHASES))
        ln = np.zeros(len(PHASES), dtype=np.int64)
        pr = np.zeros(1, dtype=np.int64)
        _check(self._lib.h2_phase_times(self._h, _dp(ms), ln.ctypes.data_as(C.POINTER(C.c_int64)),
                                        pr.ctypes.data_as(C.POINTER(C.c_int64))))
        return {p: (float(a), int(b)) for p, a, b in zip(PHASES, ms, ln)}, int(pr[0])

    def matvec_host(self, x):
        """y = G~ x from host FP64 arrays (numpy, or pinned torch CPU tensors given as (x, y))."""
        if isinstance(x, tuple):
            xt, yt = x
            _check(self._lib.h2_matvec_host(self._h, C.cast(C.c_void_p(xt.data_ptr()), C.POINTER(C.c_double)),
                                            C.cast(C.c_void_p(yt.data_ptr()), C.POINTER(C.c_double)),
                                            int(xt.shape[1])))
            return yt
        x = np.asfortranarray(np.asarray(x, dtype=np.float64).reshape(self.n, -1))
        y = np.zeros_like(x, order="F")
        _check(self._lib.h2_matvec_host(self._h, _dp(x), _dp(y), int(x.shape[1])))
        return y

    def matvec_host_stream(self, x, y):
        """A sequence of products from host FP64 blocks (h2_matvec_host_stream):
        x and y pinned torch CPU tensors of shape (count, nrhs, n), each block
        column-major (n x nrhs), copies overlapped with the products."""
        count, nrhs = int(x.shape[0]), int(x.shape[1])
        if tuple(y.shape) != tuple(x.shape) or x.shape[2] != self.n:
            raise ValueError("x and y must both be (count, nrhs, n)")
        _check(self._lib.h2_matvec_host_stream(self._h, C.cast(C.c_void_p(x.data_ptr()), C.POINTER(C.c_double)),
                                               C.cast(C.c_void_p(y.data_ptr()), C.POINTER(C.c_double)), nrhs, count))
        return y

    def build_times(self):
        """Wall-clock ms of the build phases (h2_build_times)."""
        ms = np.zeros(5)
        _check(self._lib.h2_build_times(self._h, _dp(ms)))
        return dict(zip(["plan", "bases", "coupling", "near", "total"], (float(v) for v in ms)))

    def export(self, what, first=0, count=None):
        """The stored representation as built on the device (h2_export), as float64:
        what = "near" (count, lmax, lmax), "coupling" (count, k, k), "V" (count, k)
        over padded DoFs, "E" (count, 3, m, m)."""
        st = self.stats
        L, k, m = st["leaf_max"], st["rank"], st["order"]
        item, total, shape = {"near": (0, st["near_blocks"], (L, L)), "coupling": (1, st["adm_blocks"], (k, k)),
                              "V": (2, (2 ** st["depth"]) * L, (k,)), "E": (3, st["clusters"], (3, m, m))}[what]
        count = total - first if count is None else count
        out = np.zeros((count,) + shape)
        _check(self._lib.h2_export(self._h, item, int(first), int(count), _dp(out)))
        return out

    def export_gca(self, what, first=0, count=None):
        """GCA-H^2 items of h2_export as float64 (K = stats["rank"], zero padded):
        what = "S" (count, K, K) over admissible blocks, "V" (count, lmax, K)
        over leaves, "E" (count, K, K) over clusters."""
        st = self.stats
        L, K = st["leaf_max"], st["rank"]
        item, total, shape = {"S": (4, st["adm_blocks"], (K, K)), "V": (5, 2 ** st["depth"], (L, K)),
                              "E": (6, st["clusters"], (K, K))}[what]
        count = total - first if count is None else count
        out = np.zeros((count,) + shape)
        _check(self._lib.h2_export(self._h, item, int(first), int(count), _dp(out)))
        return out

    def gca_pivots(self):
        """(rank[clusters], pivots[clusters][K]) of a GCA-H^2 handle, -1 beyond the rank."""
        nc, K = self.stats["clusters"], self.stats["rank"]
        rank = np.zeros(nc, dtype=np.int32)
        piv = np.zeros((nc, K), dtype=np.int32)
        _check(self._lib.h2_gca_pivots(self._h, rank.ctypes.data_as(C.POINTER(C.c_int32)),
                                       piv.ctypes.data_as(C.POINTER(C.c_int32)), int(K)))
        return rank, piv

    def coefficients(self, which, nrhs):
        out = np.zeros((self.stats["clusters"], self.stats["rank"], nrhs))
        _check(self._lib.h2_coefficients(self._h, int(which), _dp(out)))
        return out

    def solve(self, b, rtol=1e-8, restart=30, maxit=1000):
        """GMRES(restart) solve; b numpy (host) or column-major CUDA tensor (device)."""
        nrhs = b.shape[1] if b.ndim == 2 else 1
        info = (SolveInfo * nrhs)()
        if isinstance(b, np.ndarray):
            bb = np.asfortranarray(np.asarray(b, dtype=np.float64).reshape(self.n, -1))
            z = np.zeros_like(bb, order="F")
            st = self._lib.h2_solve(self._h, bb.ctypes.data_as(C.c_void_p), z.ctypes.data_as(C.c_void_p), nrhs,
                                    float(rtol), int(restart), int(maxit), info)
        else:
            import torch
            bb = colmajor(b)
            z = colmajor(torch.zeros_like(bb))
            st = self._lib.h2_solve(self._h, C.c_void_p(bb.data_ptr()), C.c_void_p(z.data_ptr()), nrhs,
                                    float(rtol), int(restart), int(maxit), info)
        if st not in (H2_OK, H2_ENOCONV):
            _check(st)
        it = np.array([i.iters for i in info])
        rel = np.array([i.relres for i in info])
        return z, it, rel, st

    def solve_ir(self, lo, b, rtol=1e-8, inner_rtol=1e-4, restart=30, maxit_inner=1000, maxit_outer=50):
        """GMRES-IR: residuals with this handle, inner GMRES with handle lo (numpy b, host)."""
        nrhs = b.shape[1] if b.ndim == 2 else 1
        info = (SolveInfo * nrhs)()
        bb = np.asfortranarray(np.asarray(b, dtype=np.float64).reshape(self.n, -1))
        z = np.zeros_like(bb, order="F")
        st = self._lib.h2_solve_ir(self._h, lo._h, bb.ctypes.data_as(C.c_void_p), z.ctypes.data_as(C.c_void_p),
                                   nrhs, float(rtol), float(inner_rtol), int(restart), int(maxit_inner),
                                   int(maxit_outer), info)
        if st not in (H2_OK, H2_ENOCONV):
            _check(st)
        return z, np.array([i.iters for i in info]), np.array([i.relres for i in info]), st


class HelmholtzMatrix:
    """The Helmholtz single-layer matrix G = G_c + i G_s of one mesh on one GPU
    (h2_zbuild); complex vectors are complex128 (numpy on the host, torch on
    the device), column-major (n, nrhs)."""

    def __init__(self, vert, tri, kappa, leaf_size=32, eta=2.0, order=3, prec="f64", quad_order=3, device=0,
                 stream=None, tensor="auto"):
        lib = load()
        v, t = _mesh(vert, tri)
        opt = Options()
        _check(lib.h2_options_default(C.byref(opt)))
        opt.prec = PREC[prec]
        opt.quad_order = int(quad_order)
        opt.device = int(device)
        opt.stream = stream
        opt.coupling = COUPLING["stored"]
        opt.tensor = {"auto": 0, "off": 1}[tensor]
        h = C.c_void_p()
        _check(lib.h2_zbuild(_dp(v), v.shape[0], t.ctypes.data_as(C.POINTER(C.c_int32)), t.shape[0],
                             int(leaf_size), float(eta), int(order), float(kappa), C.byref(opt), C.byref(h)))
        self._h = h
        self._lib = lib
        self.n = int(t.shape[0])
        self.kappa = float(kappa)
        st = Stats()
        _check(lib.h2_zinfo(h, C.byref(st)))
        self.stats = {f: int(getattr(st, f)) for f, _ in Stats._fields_}

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.h2_zdestroy(h)
            self._h = None

    def __del__(self):
        self.close()

    @property
    def handle(self):
        return self._h

    def export(self, which, what, first=0, count=None):
        """h2_export of part `which` (0 real, 1 imaginary); see H2Matrix.export."""
        p = C.c_void_p()
        _check(self._lib.h2_zpart(self._h, int(which), C.byref(p)))
        st = self.stats
        L, k, m = st["leaf_max"], st["rank"], st["order"]
        item, total, shape = {"near": (0, st["near_blocks"], (L, L)), "coupling": (1, st["adm_blocks"], (k, k)),
                              "V": (2, (2 ** st["depth"]) * L, (k,)), "E": (3, st["clusters"], (3, m, m))}[what]
        count = total - first if count is None else count
        out = np.zeros((count,) + shape)
        _check(self._lib.h2_export(p, item, int(first), int(count), _dp(out)))
        return out

    def matvec(self, x, y):
        """y = G~ x on the device; x, y complex128 CUDA tensors (n, nrhs), column-major."""
        if x.shape != y.shape or x.shape[0] != self.n:
            raise ValueError("x and y must both be (n, nrhs)")
        if x.stride(0) != 1 or y.stride(0) != 1:
            raise ValueError("x and y must be column-major (use colmajor())")
        _check(self._lib.h2_zmatvec(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), int(x.shape[1])))
        return y

    def matvec_host(self, x):
        x = np.asfortranarray(np.asarray(x, dtype=np.complex128).reshape(self.n, -1))
        y = np.zeros_like(x, order="F")
        _check(self._lib.h2_zmatvec_host(self._h, x.ctypes.data_as(C.POINTER(C.c_double)),
                                         y.ctypes.data_as(C.POINTER(C.c_double)), int(x.shape[1])))
        return y

    def solve(self, b, rtol=1e-8, restart=30, maxit=2000):
        """GMRES(restart) on the real form; b numpy complex (host)."""
        bb = np.asfortranarray(np.asarray(b, dtype=np.complex128).reshape(self.n, -1))
        nrhs = bb.shape[1]
        z = np.zeros_like(bb, order="F")
        info = (SolveInfo * nrhs)()
        st = self._lib.h2_zsolve(self._h, bb.ctypes.data_as(C.c_void_p), z.ctypes.data_as(C.c_void_p), nrhs,
                                 float(rtol), int(restart), int(maxit), info)
        if st not in (H2_OK, H2_ENOCONV):
            _check(st)
        return z, np.array([i.iters for i in info]), np.array([i.relres for i in info]), st


class Server:
    """Continuous-batching solve server (h2_serve_*): a native worker thread on one GPU."""

    def __init__(self, device=0, hbm_budget=0):
        self._lib = load()
        h = C.c_void_p()
        _check(self._lib.h2_serve_create(int(device), int(hbm_budget), C.byref(h)))
        self._h = h
        self._n = {}

    def register(self, hi, lo=None, slots=32, restart=30, maxit=5000, inner_rtol=1e-4):
        _check(self._lib.h2_serve_register(self._h, hi.handle, lo.handle if lo is not None else None, int(slots),
                                           int(restart), int(maxit), float(inner_rtol)))
        self._n[hi.handle.value] = hi.n

    def submit(self, hi, b, rtol=1e-8):
        bb = np.asfortranarray(np.asarray(b, dtype=np.float64).reshape(hi.n, -1))
        t = C.c_uint64()
        _check(self._lib.h2_serve_submit(self._h, hi.handle, _dp(bb), int(bb.shape[1]), float(rtol), C.byref(t)))
        return int(t.value), bb.shape

    def poll(self, ticket, shape):
        """None while pending, else (z, iters, relres, status)."""
        z = np.zeros(shape, order="F")
        info = (SolveInfo * shape[1])()
        st = self._lib.h2_serve_poll(self._h, C.c_uint64(ticket), _dp(z), info)
        if st == H2_PENDING:
            return None
        if st not in (H2_OK, H2_ENOCONV):
            _check(st)
        return z, np.array([i.iters for i in info]), np.array([i.relres for i in info]), st

    def wait(self, ticket, timeout=60.0):
        st = self._lib.h2_serve_wait(self._h, C.c_uint64(ticket), float(timeout))
        if st not in (H2_OK, H2_PENDING):
            _check(st)
        return st == H2_OK

    def stats(self):
        out = np.zeros(6, dtype=np.int64)
        _check(self._lib.h2_serve_stats(self._h, out.ctypes.data_as(C.POINTER(C.c_int64))))
        return dict(zip(["queued", "running_columns", "completed", "steps", "engine_bytes", "budget"],
                        (int(v) for v in out)))

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.h2_serve_destroy(h)
            self._h = None

    def __del__(self):
        self.close()


class ProductGraph:
    """One H² product captured as a CUDA graph (h2_graph_*); holds its matrix and buffers alive."""

    def __init__(self, mat, g, bufs):
        self._lib = mat._lib
        self._mat = mat
        self._g = g
        self._bufs = bufs

    def launch(self):
        _check(self._lib.h2_graph_launch(self._g))

    def close(self):
        g = getattr(self, "_g", None)
        if g is not None and g.value:
            self._lib.h2_graph_destroy(g)
            self._g = None

    def __del__(self):
        self.close()


class Batch:
    """Batched products over independent FP32 H² matrices (h2_batch_*).

    Vectors are packed: problem p occupies elements offsets[p] .. offsets[p+1]
    of one float32 CUDA tensor, as a column-major (n_p, nrhs_p) block.
    The matrices must outlive the batch (it keeps references to them).
    """

    def __init__(self, mats, nrhs, stream=None):
        self._lib = load()
        if len(mats) != len(nrhs):
            raise ValueError("one nrhs per matrix")
        self._mats = list(mats)   # keep the handles alive
        hs = (C.c_void_p * len(mats))(*[m.handle.value for m in mats])
        nr = (C.c_int * len(mats))(*[int(v) for v in nrhs])
        h = C.c_void_p()
        _check(self._lib.h2_batch_create(hs, len(mats), nr, stream, C.byref(h)))
        self._h = h
        self.nrhs = [int(v) for v in nrhs]
        off = np.zeros(len(mats) + 1, dtype=np.int64)
        _check(self._lib.h2_batch_offsets(h, off.ctypes.data_as(C.POINTER(C.c_int64))))
        self.offsets = off

    @property
    def length(self):
        return int(self.offsets[-1])

    def matvec(self, x, y):
        """y = G~_p x_p for every problem; x, y float32 CUDA tensors of `length` elements."""
        if x.numel() != self.length or y.numel() != self.length:
            raise ValueError("x and y must hold the packed vectors of all problems")
        _check(self._lib.h2_batch_matvec(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr())))
        return y

    def split(self, v):
        """The (n_p, nrhs_p) column-major views of a packed vector."""
        out = []
        for p, m in enumerate(self._mats):
            a, b = int(self.offsets[p]), int(self.offsets[p + 1])
            out.append(v[a:b].view(self.nrhs[p], m.n).t())
        return out

    def tune(self, reps=5):
        ch = (C.c_int * 4)()
        _check(self._lib.h2_batch_tune(self._h, int(reps), ch))
        return list(ch)

    def set_shapes(self, choice):
        ch = (C.c_int * 4)(*[int(c) for c in choice])
        _check(self._lib.h2_batch_set_shapes(self._h, ch))

    def profile(self, enable=True):
        _check(self._lib.h2_batch_profile(self._h, 1 if enable else 0))

    def phase_times(self):
        ms = np.zeros(len(PHASES))
        ln = np.zeros(len(PHASES), dtype=np.int64)
        pr = np.zeros(1, dtype=np.int64)
        _check(self._lib.h2_batch_phase_times(self._h, _dp(ms), ln.ctypes.data_as(C.POINTER(C.c_int64)),
                                              pr.ctypes.data_as(C.POINTER(C.c_int64))))
        return {p: (float(a), int(b)) for p, a, b in zip(PHASES, ms, ln)}, int(pr[0])

    def info(self):
        out = np.zeros(9, dtype=np.int64)
        _check(self._lib.h2_batch_info(self._h, out.ctypes.data_as(C.POINTER(C.c_int64))))
        keys = ["problems", "packed", "dofs", "work_bytes", "launches", "shape_forward", "shape_coupling",
                "shape_backward", "shape_near"]
        return dict(zip(keys, (int(v) for v in out)))

    def sync(self):
        _check(self._lib.h2_batch_sync(self._h))

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.h2_batch_destroy(h)
            self._h = None

    def __del__(self):
        self.close()


class GcaMatrix(H2Matrix):
    """A GCA-H^2 matrix (Section 3's GCA-H^2 example; h2_build_gca): pivot
    bases from cross approximation of a Green-quadrature surrogate, coupling
    S = G on the pivot pairs.  Products, solves and graphs as for H2Matrix."""

    def __init__(self, vert, tri, leaf_size=32, eta=2.0, eps=1e-4, green_order=4, gamma=1.0, tri_order=3,
                 max_rank=128, prec="f64", quad_order=3, device=0, stream=None, tensor="auto"):
        super().__init__(vert, tri, leaf_size=leaf_size, eta=eta, order=1, prec=prec, quad_order=quad_order,
                         device=device, stream=stream, coupling="auto", tensor=tensor,
                         gca=dict(eps=float(eps), gamma=float(gamma), green_order=int(green_order),
                                  tri_order=int(tri_order), max_rank=int(max_rank)))
