"""CPU checker (float64) for the improved-BVH ray tracer -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference leg may import this package.  The product path (the
CUDA library and its Python binding) never imports, links or runs it.

The computation lives in ``oracle.cpp`` (plain C++17, float64, built with
``-ffp-contract=off``); this module only builds it with g++ and marshals numpy
arrays through ctypes.  See the header of ``oracle.cpp`` for which part of the
paper each function follows.

Pinning status: every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, brute force written another way, invariants and
special cases.  The alpha < 1 split choice is pinned on a hand-derived Eq. 2
example (raw and scale-free distance term), and the recursive tree cost at
alpha = 0.5 on the same example; the paper prints no tree, so no full-size
alpha < 1 tree is compared with a published one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.cpp")
_lock = threading.Lock()
_lib = None

_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (portable flags; x86_64 and aarch64)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-pthread", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.orc_version.restype = ctypes.c_int
            L.orc_tri_hit.argtypes = [_f32p, _f32p, _f64p, _f64p, _f64p]
            L.orc_closest_brute.argtypes = [_f32p, ctypes.c_int64, _f32p, ctypes.c_int64, _i32p,
                                            _f64p, _i32p, _f64p, _f64p, _f64p, ctypes.c_int]
            L.orc_any_brute.argtypes = [_f32p, ctypes.c_int64, _f32p, ctypes.c_int64, _i32p, _u8p,
                                        ctypes.c_int]
            L.orc_bvh_build.restype = ctypes.c_void_p
            L.orc_bvh_build.argtypes = [_f32p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, _f64p, ctypes.c_int, ctypes.c_int]
            L.orc_bvh_free.argtypes = [ctypes.c_void_p]
            L.orc_bvh_info.argtypes = [ctypes.c_void_p, _i64p]
            L.orc_bvh_export.argtypes = [ctypes.c_void_p, _i32p, _i64p, _i64p, _i32p]
            L.orc_bvh_closest.argtypes = [ctypes.c_void_p, _f32p, ctypes.c_int64, _i32p, _f64p,
                                          _i32p, _f64p, _f64p, _f64p, ctypes.c_int]
            L.orc_bvh_any.argtypes = [ctypes.c_void_p, _f32p, ctypes.c_int64, _i32p, _u8p,
                                      ctypes.c_int]
            L.orc_eq2_cost.restype = ctypes.c_double
            L.orc_eq2_cost.argtypes = [_f64p, ctypes.c_double, _f64p, ctypes.c_double, _f64p,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, _f64p,
                                       ctypes.c_int]
            L.orc_tree_cost.restype = ctypes.c_double
            L.orc_tree_cost.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int64, _i32p, _i64p, _i64p,
                                        ctypes.c_int64, _i32p, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, _f64p, ctypes.c_int]
            L.orc_reflect.argtypes = [_f32p, _f32p, _i32p, _f64p, ctypes.c_int64, _f64p]
            L.orc_fibonacci.argtypes = [ctypes.c_int64, _f64p]
            L.orc_icosphere.restype = ctypes.c_int64
            L.orc_icosphere.argtypes = [ctypes.c_int, _f64p]
            L.orc_receive.restype = ctypes.c_int64
            L.orc_receive.argtypes = [_f32p, _f32p, ctypes.c_int64, _f32p, ctypes.c_int64,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double, _i32p,
                                      _f64p, ctypes.c_int64]
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _tris(tris):
    t = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
    return t


def _rays(rays):
    return np.ascontiguousarray(rays, dtype=np.float32).reshape(-1, 8)


def _skip(skip, n):
    if skip is None:
        return None
    s = np.ascontiguousarray(skip, dtype=np.int32)
    assert s.shape == (n,)
    return s


class Hits:
    """Closest-hit results: t (inf on miss), id (-1), u, v, t2 (second-nearest t)."""

    def __init__(self, n):
        self.t = np.empty(n, np.float64)
        self.id = np.empty(n, np.int32)
        self.u = np.empty(n, np.float64)
        self.v = np.empty(n, np.float64)
        self.t2 = np.empty(n, np.float64)


def tri_hit(tri, ray):
    """One triangle (3x3 float32) vs one ray (8 float32); (hit, t, u, v), t unrestricted."""
    t, u, v = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    tr = _tris(tri)
    ry = _rays(ray)
    h = lib().orc_tri_hit(_p(tr, _f32p), _p(ry, _f32p), ctypes.byref(t), ctypes.byref(u),
                          ctypes.byref(v))
    return bool(h), t.value, u.value, v.value


def closest_brute(tris, rays, skip=None, threads=0) -> Hits:
    tr, ry = _tris(tris), _rays(rays)
    n = ry.shape[0]
    h = Hits(n)
    sk = _skip(skip, n)
    lib().orc_closest_brute(_p(tr, _f32p), tr.shape[0], _p(ry, _f32p), n, _p(sk, _i32p),
                            _p(h.t, _f64p), _p(h.id, _i32p), _p(h.u, _f64p), _p(h.v, _f64p),
                            _p(h.t2, _f64p), threads)
    return h


def any_brute(tris, rays, skip=None, threads=0) -> np.ndarray:
    tr, ry = _tris(tris), _rays(rays)
    n = ry.shape[0]
    out = np.empty(n, np.uint8)
    sk = _skip(skip, n)
    lib().orc_any_brute(_p(tr, _f32p), tr.shape[0], _p(ry, _f32p), n, _p(sk, _i32p),
                        _p(out, _u8p), threads)
    return out


class Bvh:
    """CPU BVH built with the exact-sweep Eq. 2 split (Sec. II.C)."""

    def __init__(self, tris, alpha=1.0, source=(0.0, 0.0, 0.0), max_leaf=4, t_i=1.0,
                 t_trav=1.0, dist_norm=0):
        self.tris = _tris(tris)          # kept alive: the C side holds a pointer
        self.params = dict(alpha=alpha, source=tuple(float(s) for s in source), max_leaf=max_leaf,
                           t_i=t_i, t_trav=t_trav, dist_norm=dist_norm)
        src = np.asarray(source, dtype=np.float64)
        self._h = lib().orc_bvh_build(_p(self.tris, _f32p), self.tris.shape[0], alpha, t_i,
                                      t_trav, _p(src, _f64p), int(max_leaf), int(dist_norm))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_bvh_free(h)
            self._h = None

    def info(self) -> dict:
        a = np.zeros(6, np.int64)
        lib().orc_bvh_info(self._h, _p(a, _i64p))
        return dict(nodes=int(a[0]), leaves=int(a[1]), depth=int(a[2]), largest_leaf=int(a[3]),
                    smallest_leaf=int(a[4]), prims=int(a[5]))

    def export(self):
        """Binary tree in the neutral form understood by tree_cost()."""
        inf = self.info()
        n_int = inf["nodes"] - inf["leaves"]
        child = np.zeros(2 * max(n_int, 1), np.int32)
        lf = np.zeros(inf["leaves"], np.int64)
        lc = np.zeros(inf["leaves"], np.int64)
        prims = np.zeros(inf["prims"], np.int32)
        lib().orc_bvh_export(self._h, _p(child, _i32p), _p(lf, _i64p), _p(lc, _i64p),
                             _p(prims, _i32p))
        return dict(child=child[: 2 * n_int].reshape(-1, 2), leaf_first=lf, leaf_count=lc,
                    prims=prims)

    def closest(self, rays, skip=None, threads=0) -> Hits:
        ry = _rays(rays)
        n = ry.shape[0]
        h = Hits(n)
        sk = _skip(skip, n)
        lib().orc_bvh_closest(self._h, _p(ry, _f32p), n, _p(sk, _i32p), _p(h.t, _f64p),
                              _p(h.id, _i32p), _p(h.u, _f64p), _p(h.v, _f64p), _p(h.t2, _f64p),
                              threads)
        return h

    def any(self, rays, skip=None, threads=0) -> np.ndarray:
        ry = _rays(rays)
        n = ry.shape[0]
        out = np.empty(n, np.uint8)
        sk = _skip(skip, n)
        lib().orc_bvh_any(self._h, _p(ry, _f32p), n, _p(sk, _i32p), _p(out, _u8p), threads)
        return out

    def cost(self) -> float:
        e = self.export()
        p = self.params
        return tree_cost(self.tris, e["child"], e["leaf_first"], e["leaf_count"], e["prims"],
                         p["alpha"], p["source"], t_i=p["t_i"], t_trav=p["t_trav"],
                         dist_norm=p["dist_norm"])


def eq2_cost(box_a, k_a, box_b, k_b, box_c, alpha, source, t_i=1.0, t_trav=1.0, dist_norm=0):
    """Eq. 2 for explicit boxes [lo(3), hi(3)] and triangle counts."""
    a = np.asarray(box_a, np.float64).reshape(6)
    b = np.asarray(box_b, np.float64).reshape(6)
    c = np.asarray(box_c, np.float64).reshape(6)
    s = np.asarray(source, np.float64).reshape(3)
    return lib().orc_eq2_cost(_p(a, _f64p), float(k_a), _p(b, _f64p), float(k_b), _p(c, _f64p),
                              alpha, t_i, t_trav, _p(s, _f64p), int(dist_norm))


def tree_cost(tris, child, leaf_first, leaf_count, prims, alpha, source, t_i=1.0, t_trav=1.0,
              dist_norm=0) -> float:
    """Eq. 2 applied recursively to a binary tree (neutral form, see Bvh.export)."""
    tr = _tris(tris)
    ch = np.ascontiguousarray(child, dtype=np.int32).reshape(-1)
    lf = np.ascontiguousarray(leaf_first, dtype=np.int64)
    lc = np.ascontiguousarray(leaf_count, dtype=np.int64)
    pr = np.ascontiguousarray(prims, dtype=np.int32)
    s = np.asarray(source, np.float64).reshape(3)
    return lib().orc_tree_cost(_p(tr, _f32p), tr.shape[0], ch.size // 2, _p(ch, _i32p),
                               _p(lf, _i64p), _p(lc, _i64p), lf.size, _p(pr, _i32p), alpha, t_i,
                               t_trav, _p(s, _f64p), int(dist_norm))


def reflect(tris, rays, hit_id, hit_t) -> np.ndarray:
    """float64 [n, 8] reflected rays (o + t d, 0, d - 2 (d.n) n, tmax - t)."""
    tr, ry = _tris(tris), _rays(rays)
    n = ry.shape[0]
    hid = np.ascontiguousarray(hit_id, dtype=np.int32)
    ht = np.ascontiguousarray(hit_t, dtype=np.float64)
    out = np.empty((n, 8), np.float64)
    lib().orc_reflect(_p(tr, _f32p), _p(ry, _f32p), _p(hid, _i32p), _p(ht, _f64p), n,
                      _p(out, _f64p))
    return out


def fibonacci(n) -> np.ndarray:
    out = np.empty((n, 3), np.float64)
    lib().orc_fibonacci(n, _p(out, _f64p))
    return out


def icosphere(level) -> np.ndarray:
    n = lib().orc_icosphere(level, None)
    out = np.empty((n, 3), np.float64)
    m = lib().orc_icosphere(level, _p(out, _f64p))
    assert m == n
    return out


def receive(rays, hit_t, rx, delta, range0, tol=0.0):
    """Receiving-sphere test of Sec. III.C (Eq. 4), every segment against every receiver.

    Returns (pairs int32 [k, 3] = (ray, rx, class), vals float64 [k, 3] = (l, distance,
    radius)); class 1 = received with more than `tol` to spare, class 2 = within `tol` of
    the sphere or of a segment end (either answer is right at float32 precision)."""
    ry = _rays(rays)
    n = ry.shape[0]
    ht = np.ascontiguousarray(hit_t, dtype=np.float32).reshape(n)
    p = np.ascontiguousarray(rx, dtype=np.float32).reshape(-1, 3)
    cap = 1 << 16
    while True:
        oi = np.empty((cap, 3), np.int32)
        od = np.empty((cap, 3), np.float64)
        k = lib().orc_receive(_p(ry, _f32p), _p(ht, _f32p), n, _p(p, _f32p), p.shape[0],
                              float(delta), float(range0), float(tol), _p(oi, _i32p),
                              _p(od, _f64p), cap)
        if k <= cap:
            return oi[:k].copy(), od[:k].copy()
        cap = int(k)
