"""Python binding of librtbvh (include/rtbvh.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch
tensors / numpy arrays to pointers and sizes, passes the current CUDA stream
and turns error codes into exceptions.  There is no CPU fallback: if the
library cannot be built or loaded, every call raises.

Tensor conventions
  tris  float32 [T, 3, 3]  (numpy on the host or a CUDA tensor)
  rays  float32 [R, 8]     CUDA tensor, 16-byte aligned: (o, tmin, d, tmax)
  hits  float32 [R, 4]     CUDA tensor: (t, tri id as int32 bits, u, v);
                           hits.view(torch.int32)[:, 1] gives the ids
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build_ext

RT_NO_FP64_RETEST = 1
RT_COUNT_STATS = 2
RT_QUANTIZED_NODES = 4
RT_RAYS_FIBONACCI = 0
RT_RAYS_ICOSPHERE = 1

_lock = threading.Lock()
_lib = None

ERRORS = {-1: "RT_EINVAL", -2: "RT_ENOMEM", -3: "RT_ENOTBUILT", -4: "RT_ETIMEOUT", -5: "RT_ECUDA",
          -6: "RT_EBUSY", -7: "RT_EINTERNAL"}

# Every symbol the header declares (checked by the ABI test).
EXPORTS = ["rt_version", "rt_launch_count", "rt_last_error", "rt_scene_upload", "rt_scene_destroy", "rt_scene_update",
           "rt_bvh_build", "rt_bvh_info", "rt_bvh_export", "rt_trace_closest", "rt_trace_any",
           "rt_trace_closest_host", "rt_trace_closest_noalloc", "rt_ray_count", "rt_launch_index", "rt_gen_rays",
           "rt_reflect", "rt_batch_create", "rt_batch_run", "rt_batch_stats_get", "rt_batch_order",
           "rt_batch_visibility", "rt_batch_destroy", "rt_session_create", "rt_session_add_scene",
           "rt_session_submit", "rt_session_poll", "rt_session_wait", "rt_session_release", "rt_session_stats_get",
           "rt_session_destroy", "rt_scene_set_split_events", "rt_autotune", "rt_debug_inject",
           "rt_rxset_create", "rt_rxset_destroy", "rt_receive", "rt_batch_received", "rt_abi_struct_sizes", "rt_probe_l2_read"]

# test hooks (rt_debug_inject)
RT_DEBUG_SPIN_LIMIT, RT_DEBUG_PHANTOM_TASK, RT_DEBUG_PHANTOM_ITEM, RT_DEBUG_FAIL_ALLOC = 1, 2, 3, 4


class RtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class BuildParams(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_float), ("t_i", ctypes.c_float), ("t_trav", ctypes.c_float),
                ("source", ctypes.c_float * 3), ("max_leaf", ctypes.c_int32),
                ("bins", ctypes.c_int32), ("width", ctypes.c_int32), ("dist_norm", ctypes.c_int32),
                ("range", ctypes.c_float), ("quantize", ctypes.c_int32)]


class TraceParams(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("skip_tri_dev", ctypes.c_void_p),
                ("stats_dev", ctypes.c_void_p), ("n_flagged_dev", ctypes.c_void_p), ("block", ctypes.c_int32),
                ("stack", ctypes.c_int32)]


class ReceiveParams(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_float), ("range0", ctypes.c_float), ("max_records", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("stats_dev", ctypes.c_void_p), ("delta_ray_dev", ctypes.c_void_p)]


class TuneResult(ctypes.Structure):
    _fields_ = [("max_leaf", ctypes.c_int32), ("bins", ctypes.c_int32), ("block", ctypes.c_int32),
                ("n_tried", ctypes.c_int32), ("build_ms", ctypes.c_float), ("trace_ms", ctypes.c_float),
                ("score_ms", ctypes.c_float), ("default_score_ms", ctypes.c_float), ("width", ctypes.c_int32),
                ("stack", ctypes.c_int32)]


class BvhInfo(ctypes.Structure):
    _fields_ = [("n_tri", ctypes.c_int64), ("n_bvh2_internal", ctypes.c_int64),
                ("n_leaves", ctypes.c_int64), ("n_wide", ctypes.c_int64), ("depth2", ctypes.c_int32),
                ("depth_wide", ctypes.c_int32), ("max_leaf_size", ctypes.c_int32),
                ("status", ctypes.c_int32), ("build_ms", ctypes.c_double), ("n_built", ctypes.c_int64)]


RT_BATCH_MAX_ORDER = 8


class BatchDesc(ctypes.Structure):
    _fields_ = [("n_tx", ctypes.c_int32), ("tx_pos", ctypes.c_void_p), ("tx_param", ctypes.c_void_p),
                ("dir_kind", ctypes.c_int32), ("max_order", ctypes.c_int32), ("tmax", ctypes.c_float),
                ("n_rx", ctypes.c_int32), ("rx_pos", ctypes.c_void_p), ("use_graph", ctypes.c_int32),
                ("ray_tile", ctypes.c_int32), ("receive", ctypes.c_int32), ("max_rx_records", ctypes.c_int32),
                ("rx_delta", ctypes.c_void_p)]


class BatchStats(ctypes.Structure):
    _fields_ = [("n_orders", ctypes.c_int32), ("rays", ctypes.c_int64 * (RT_BATCH_MAX_ORDER + 1)),
                ("segments", ctypes.c_int64), ("total_rays", ctypes.c_int64), ("visible", ctypes.c_int64),
                ("flagged", ctypes.c_int32), ("received", ctypes.c_int64 * (RT_BATCH_MAX_ORDER + 1))]


class Request(ctypes.Structure):
    _fields_ = [("scene_id", ctypes.c_int32), ("tx", ctypes.c_float * 3), ("dir_kind", ctypes.c_int32),
                ("param", ctypes.c_int64), ("max_order", ctypes.c_int32), ("tmax", ctypes.c_float),
                ("hits_host", ctypes.c_void_p), ("order_counts_host", ctypes.c_void_p),
                ("order_hits_host", ctypes.c_void_p), ("order_src_host", ctypes.c_void_p)]


class SessionStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("running", ctypes.c_int64), ("peak_running", ctypes.c_int64),
                ("rays", ctypes.c_int64), ("pool_bytes", ctypes.c_int64), ("peak_pool_bytes", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("span_s", ctypes.c_double), ("wait_p50_ms", ctypes.c_double), ("wait_p99_ms", ctypes.c_double),
                ("run_p50_ms", ctypes.c_double), ("run_p99_ms", ctypes.c_double)]


def lib_path() -> str:
    return build_ext.LIB


def lib(build: bool = True):
    """Load librtbvh.so (building it first if sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = build_ext.build() if build else build_ext.LIB
            if not os.path.exists(path):
                raise RuntimeError("librtbvh.so is missing at %s; run __graft_entry__.build()" % path)
            L = ctypes.CDLL(path)
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            L.rt_version.restype = i32
            L.rt_launch_count.restype = ctypes.c_uint64
            L.rt_last_error.restype = ctypes.c_char_p
            L.rt_scene_upload.argtypes = [vp, i64, i32, vp, ctypes.POINTER(vp)]
            L.rt_scene_update.argtypes = [vp, vp, i64, i32, vp]
            L.rt_scene_destroy.argtypes = [vp]
            L.rt_bvh_build.argtypes = [vp, ctypes.POINTER(BuildParams), vp]
            L.rt_bvh_info.argtypes = [vp, vp, ctypes.POINTER(BvhInfo)]
            L.rt_scene_set_split_events.argtypes = [vp, vp, vp]
            L.rt_debug_inject.argtypes = [i32, i64]
            L.rt_autotune.argtypes = [vp, ctypes.POINTER(BuildParams), vp, i64, ctypes.c_float,
                                      ctypes.POINTER(TuneResult), vp]
            L.rt_bvh_export.argtypes = [vp, vp, vp, vp, vp, vp, vp]
            L.rt_trace_closest.argtypes = [vp, vp, i64, vp, ctypes.POINTER(TraceParams), vp]
            L.rt_trace_any.argtypes = [vp, vp, i64, vp, ctypes.POINTER(TraceParams), vp]
            L.rt_trace_closest_host.argtypes = [vp, vp, i64, vp, ctypes.POINTER(TraceParams), vp]
            L.rt_trace_closest_noalloc.argtypes = [vp, vp, i64, vp, ctypes.POINTER(TraceParams), vp]
            L.rt_ray_count.restype = i64
            L.rt_ray_count.argtypes = [i32, i64]
            L.rt_launch_index.restype = i64
            L.rt_launch_index.argtypes = [i32, i64, i64]
            L.rt_gen_rays.argtypes = [i32, ctypes.POINTER(ctypes.c_float), i64, ctypes.c_float, ctypes.c_float,
                                      vp, i64, vp]
            L.rt_reflect.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp, vp]
            L.rt_batch_create.argtypes = [vp, ctypes.POINTER(BatchDesc), ctypes.POINTER(vp)]
            L.rt_batch_run.argtypes = [vp, vp]
            L.rt_batch_stats_get.argtypes = [vp, vp, ctypes.POINTER(BatchStats)]
            L.rt_batch_order.argtypes = [vp, i32, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                         ctypes.POINTER(vp)]
            L.rt_batch_visibility.argtypes = [vp, ctypes.POINTER(vp)]
            L.rt_batch_received.argtypes = [vp, i32, ctypes.POINTER(vp), ctypes.POINTER(vp)]
            L.rt_abi_struct_sizes.argtypes = [ctypes.POINTER(ctypes.c_int64), i32]
            L.rt_probe_l2_read.argtypes = [vp, i64, i32, vp, vp]
            L.rt_batch_destroy.argtypes = [vp]
            L.rt_session_create.argtypes = [ctypes.c_size_t, i32, ctypes.POINTER(vp)]
            L.rt_session_add_scene.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int32)]
            L.rt_session_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
            L.rt_session_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]
            L.rt_session_wait.argtypes = [vp, ctypes.c_uint64, i64]
            L.rt_session_release.argtypes = [vp, ctypes.c_uint64]
            L.rt_session_stats_get.argtypes = [vp, ctypes.POINTER(SessionStats)]
            L.rt_session_destroy.argtypes = [vp]
            L.rt_rxset_create.argtypes = [vp, i32, ctypes.c_float, ctypes.POINTER(vp)]
            L.rt_rxset_destroy.argtypes = [vp]
            L.rt_receive.argtypes = [vp, vp, vp, i64, vp, ctypes.POINTER(ReceiveParams), vp, vp, vp]
            _lib = L
    return _lib


def _check(code):
    if code != 0:
        raise RtError(code, lib().rt_last_error().decode(errors="replace"))


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, dtype, cols=None, name="tensor", rows=0):
    """Raw pointer of a contiguous CUDA tensor: [>= rows, cols] when cols is
    given, else at least `rows` elements (the library writes that many)."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError("%s must be contiguous %s" % (name, dtype))
    if cols is not None and (t.dim() != 2 or t.shape[1] != cols):
        raise TypeError("%s must have shape [n, %d]" % (name, cols))
    if (t.shape[0] if cols is not None else t.numel()) < rows:
        raise TypeError("%s holds fewer than %d %s" % (name, rows, "rows" if cols is not None else "elements"))
    return ctypes.c_void_p(t.data_ptr())


class Scene:
    """Owns one rt_scene handle."""

    def __init__(self, handle, n_tri):
        self._h = handle
        self.n_tri = n_tri

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("scene destroyed")
        return self._h

    def destroy(self):
        if self._h:
            _check(lib().rt_scene_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def rt_version() -> int:
    return lib().rt_version()


def rt_launch_count() -> int:
    return int(lib().rt_launch_count())


def rt_scene_upload(tris, stream=None) -> Scene:
    import torch
    h = ctypes.c_void_p()
    if isinstance(tris, torch.Tensor) and tris.is_cuda:
        t = tris.reshape(-1, 9)
        _dev_ptr(t, torch.float32, 9, "tris")
        n = t.shape[0]
        _check(lib().rt_scene_upload(ctypes.c_void_p(t.data_ptr()), n, 1, _stream(stream), ctypes.byref(h)))
    else:
        a = np.ascontiguousarray(np.asarray(tris, dtype=np.float32).reshape(-1, 9))
        n = a.shape[0]
        _check(lib().rt_scene_upload(a.ctypes.data_as(ctypes.c_void_p), n, 0, _stream(stream), ctypes.byref(h)))
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    return Scene(h.value, n)


def rt_scene_update(scene: Scene, tris, stream=None):
    """Replace the scene's triangles: a CUDA tensor, a host tensor (pinned: the
    copy is asynchronous on `stream`; keep the tensor until the stream has
    reached the call) or any array-like (copied, then waited for)."""
    import torch
    if isinstance(tris, torch.Tensor) and tris.is_cuda:
        t = tris.reshape(-1, 9)
        _dev_ptr(t, torch.float32, 9, "tris")
        _check(lib().rt_scene_update(scene.handle, ctypes.c_void_p(t.data_ptr()), t.shape[0], 1, _stream(stream)))
        scene.n_tri = t.shape[0]
    elif isinstance(tris, torch.Tensor):
        if tris.dtype != torch.float32 or not tris.is_contiguous() or tris.numel() % 9:
            raise TypeError("host tris must be a contiguous float32 tensor of [n, 3, 3] or [n, 9]")
        n = tris.numel() // 9
        _check(lib().rt_scene_update(scene.handle, ctypes.c_void_p(tris.data_ptr()), n, 0, _stream(stream)))
        scene.n_tri = n
    else:
        a = np.ascontiguousarray(np.asarray(tris, dtype=np.float32).reshape(-1, 9))
        _check(lib().rt_scene_update(scene.handle, a.ctypes.data_as(ctypes.c_void_p), a.shape[0], 0, _stream(stream)))
        scene.n_tri = a.shape[0]
        (torch.cuda.current_stream() if stream is None else stream).synchronize()


def build_params(alpha=1.0, source=(0.0, 0.0, 0.0), max_leaf=4, bins=16, width=4, dist_norm=0,
                 t_i=1.0, t_trav=1.0, range=0.0, quantize=0) -> BuildParams:
    p = BuildParams()
    p.alpha, p.t_i, p.t_trav = alpha, t_i, t_trav
    p.source[0], p.source[1], p.source[2] = float(source[0]), float(source[1]), float(source[2])
    p.max_leaf, p.bins, p.width, p.dist_norm = int(max_leaf), int(bins), int(width), int(dist_norm)
    p.range = float(range)
    p.quantize = int(quantize)
    return p


def rt_bvh_build(scene: Scene, stream=None, **kw):
    p = build_params(**kw)
    _check(lib().rt_bvh_build(scene.handle, ctypes.byref(p), _stream(stream)))


def rt_scene_set_split_events(scene: Scene, ev_begin=None, ev_end=None):
    """Record two torch.cuda.Event (timing enabled) around the split kernel of
    every later build of `scene`; no arguments stops it."""
    for e in (ev_begin, ev_end):
        if e is not None and not e.cuda_event:
            e.record()  # torch creates its event on the first record
    h = [ctypes.c_void_p(e.cuda_event) if e is not None else None for e in (ev_begin, ev_end)]
    _check(lib().rt_scene_set_split_events(scene.handle, h[0], h[1]))


def rt_debug_inject(hook: int, value: int):
    """Test hooks (see rtbvh.h): spin limit, phantom work, failing allocations."""
    _check(lib().rt_debug_inject(int(hook), int(value)))


def rt_autotune(scene: Scene, rays, build_weight=1.0, stream=None, **base) -> dict:
    """Time build + walk of `rays` over max_leaf x bins x ray tile and leave the
    scene built with the fastest; returns the choice and its timings."""
    import torch
    rp = _dev_ptr(rays, torch.float32, 8, "rays")
    p = build_params(**base)
    r = TuneResult()
    _check(lib().rt_autotune(scene.handle, ctypes.byref(p), rp, rays.shape[0], float(build_weight),
                             ctypes.byref(r), _stream(stream)))
    return {f: getattr(r, f) for f, _ in TuneResult._fields_}


def rt_bvh_info(scene: Scene, stream=None) -> dict:
    info = BvhInfo()
    code = lib().rt_bvh_info(scene.handle, _stream(stream), ctypes.byref(info))
    d = {f: getattr(info, f) for f, _ in BvhInfo._fields_}
    if code != 0:
        raise RtError(code, lib().rt_last_error().decode() + " info=%r" % d)
    return d


def rt_bvh_export(scene: Scene, stream=None) -> dict:
    info = rt_bvh_info(scene, stream)
    ni, nl, n = info["n_bvh2_internal"], info["n_leaves"], info["n_tri"]
    child = np.zeros(2 * max(ni, 1), np.int32)
    lf = np.zeros(max(nl, 1), np.int64)
    lc = np.zeros(max(nl, 1), np.int64)
    prims = np.zeros(max(n, 1), np.int32)
    boxes = np.zeros(12 * max(ni, 1), np.float32)
    _check(lib().rt_bvh_export(scene.handle, _stream(stream), child.ctypes.data_as(ctypes.c_void_p),
                               lf.ctypes.data_as(ctypes.c_void_p), lc.ctypes.data_as(ctypes.c_void_p),
                               prims.ctypes.data_as(ctypes.c_void_p), boxes.ctypes.data_as(ctypes.c_void_p)))
    return dict(child=child[: 2 * ni].reshape(-1, 2), leaf_first=lf[:nl], leaf_count=lc[:nl],
                prims=prims[:n], boxes=boxes[: 12 * ni].reshape(-1, 12), info=info)


def _trace_params(flags, skip, stats, n_flagged, n, block=0, stack=0):
    import torch
    tp = TraceParams()
    tp.flags = int(flags)
    tp.block = int(block)
    tp.stack = int(stack)
    tp.stack = int(stack)
    if skip is not None:
        if skip.shape != (n,):
            raise TypeError("skip must have shape [n]")
        tp.skip_tri_dev = _dev_ptr(skip, torch.int32, None, "skip").value
    if stats is not None:
        if stats.shape != (n, 2):
            raise TypeError("stats must have shape [n, 2]")
        tp.stats_dev = _dev_ptr(stats, torch.int32, 2, "stats").value
        tp.flags |= RT_COUNT_STATS
    if n_flagged is not None:
        tp.n_flagged_dev = _dev_ptr(n_flagged, torch.int32, None, "n_flagged", 1).value
    return tp


def rt_trace_closest(scene: Scene, rays, hits=None, skip=None, flags=0, stats=None, n_flagged=None,
                     stream=None, block=0, stack=0):
    """Closest hit of every ray; returns hits float32 [n, 4] (see module doc)."""
    import torch
    rp = _dev_ptr(rays, torch.float32, 8, "rays")
    n = rays.shape[0]
    if hits is None:
        hits = torch.empty((n, 4), dtype=torch.float32, device=rays.device)
    hp = _dev_ptr(hits, torch.float32, 4, "hits", n)
    tp = _trace_params(flags, skip, stats, n_flagged, n, block, stack)
    _check(lib().rt_trace_closest(scene.handle, rp, n, hp, ctypes.byref(tp), _stream(stream)))
    return hits


def rt_trace_closest_noalloc(scene: Scene, rays, hits, flags=0, stream=None):
    """Closest hit without device allocation (n <= RT_NOALLOC_MAX_RAYS); hits is caller-provided."""
    import torch
    rp = _dev_ptr(rays, torch.float32, 8, "rays")
    hp = _dev_ptr(hits, torch.float32, 4, "hits", rays.shape[0])
    tp = TraceParams()
    tp.flags = int(flags)
    _check(lib().rt_trace_closest_noalloc(scene.handle, rp, rays.shape[0], hp, ctypes.byref(tp),
                                          _stream(stream)))
    return hits


RT_NOALLOC_MAX_RAYS = 262144


def rt_trace_any(scene: Scene, rays, occluded=None, skip=None, flags=0, stats=None, n_flagged=None,
                 stream=None, block=0, stack=0):
    """Any hit of every ray; returns uint8 [n] (1 = some triangle within (tmin, tmax))."""
    import torch
    rp = _dev_ptr(rays, torch.float32, 8, "rays")
    n = rays.shape[0]
    if occluded is None:
        occluded = torch.empty((n,), dtype=torch.uint8, device=rays.device)
    op = _dev_ptr(occluded, torch.uint8, None, "occluded", n)
    tp = _trace_params(flags, skip, stats, n_flagged, n, block, stack)
    _check(lib().rt_trace_any(scene.handle, rp, n, op, ctypes.byref(tp), _stream(stream)))
    return occluded


def rt_trace_closest_host(scene: Scene, rays_host, hits_host=None, flags=0, stream=None, block=0, stack=0):
    """Closest hit with host buffers (pinned torch tensors or numpy arrays)."""
    import torch
    if isinstance(rays_host, torch.Tensor):
        if rays_host.is_cuda or rays_host.dtype != torch.float32 or not rays_host.is_contiguous() \
                or rays_host.dim() != 2 or rays_host.shape[1] != 8:
            raise TypeError("rays_host must be a contiguous host float32 tensor [n, 8]")
        n = rays_host.shape[0]
        rp = ctypes.c_void_p(rays_host.data_ptr())
        if hits_host is None:
            hits_host = torch.empty((n, 4), dtype=torch.float32, pin_memory=True)
        if not isinstance(hits_host, torch.Tensor) or hits_host.is_cuda or hits_host.dtype != torch.float32 \
                or not hits_host.is_contiguous() or hits_host.numel() < 4 * n:
            raise TypeError("hits_host must be a contiguous host float32 tensor of at least [n, 4]")
        hp = ctypes.c_void_p(hits_host.data_ptr())
    else:
        a = np.ascontiguousarray(rays_host, dtype=np.float32)
        if a.ndim != 2 or a.shape[1] != 8:
            raise TypeError("rays_host must be [n, 8] (o.xyz, tmin, d.xyz, tmax)")
        n = a.shape[0]
        rp = a.ctypes.data_as(ctypes.c_void_p)
        if hits_host is None:
            hits_host = np.empty((n, 4), np.float32)
        if not isinstance(hits_host, np.ndarray) or hits_host.dtype != np.float32 \
                or not hits_host.flags.c_contiguous or hits_host.size < 4 * n:
            raise TypeError("hits_host must be a C-contiguous float32 array of at least [n, 4]")
        hp = hits_host.ctypes.data_as(ctypes.c_void_p)
    tp = TraceParams()
    tp.flags = int(flags)
    tp.block = int(block)
    tp.stack = int(stack)
    _check(lib().rt_trace_closest_host(scene.handle, rp, n, hp, ctypes.byref(tp), _stream(stream)))
    return hits_host


def hit_ids(hits):
    """int32 triangle ids of a hits tensor/array [n, 4]."""
    import torch
    if isinstance(hits, torch.Tensor):
        return hits.view(torch.int32)[:, 1]
    return np.ascontiguousarray(hits).view(np.int32)[:, 1]


def rt_ray_count(kind: int, param: int) -> int:
    return int(lib().rt_ray_count(int(kind), int(param)))


def rt_launch_index(kind: int, param: int, slot: int) -> int:
    """Direction index (RT_RAYS_* order) that a launch writes to `slot`; -1 if invalid."""
    return int(lib().rt_launch_index(int(kind), int(param), int(slot)))


def rt_gen_rays(kind: int, origin, param: int, tmin: float = 0.0, tmax: float = float("inf"), rays=None,
                stream=None):
    """Launch rays of Sec. III.A on the device; returns float32 [n, 8] CUDA tensor.

    Slot s holds direction rt_launch_index(kind, param, s) (Fibonacci rays in
    band order: neighbouring slots are neighbouring directions)."""
    import torch
    n = rt_ray_count(kind, param)
    if n < 0:
        raise RtError(-1, "bad launch kind or param")
    if rays is None:
        rays = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    rp = _dev_ptr(rays, torch.float32, 8, "rays")
    o = (ctypes.c_float * 3)(*[float(x) for x in origin])
    _check(lib().rt_gen_rays(int(kind), o, int(param), float(tmin), float(tmax), rp, rays.shape[0],
                             _stream(stream)))
    return rays


def rt_reflect(scene: Scene, rays, hits, out_rays=None, out_skip=None, out_src=None, out_count=None,
               stream=None):
    """Specular bounce + compaction; returns (out_rays, out_skip, out_src, out_count) device tensors."""
    import torch
    n = rays.shape[0]
    dev = rays.device
    if out_rays is None:
        out_rays = torch.empty((n, 8), dtype=torch.float32, device=dev)
    if out_skip is None:
        out_skip = torch.empty((n,), dtype=torch.int32, device=dev)
    if out_src is None:
        out_src = torch.empty((n,), dtype=torch.int32, device=dev)
    if out_count is None:
        out_count = torch.zeros((1,), dtype=torch.int32, device=dev)
    _check(lib().rt_reflect(scene.handle, _dev_ptr(rays, torch.float32, 8, "rays"),
                            _dev_ptr(hits, torch.float32, 4, "hits", n), n,
                            _dev_ptr(out_rays, torch.float32, 8, "out_rays", n),
                            _dev_ptr(out_skip, torch.int32, None, "out_skip", n),
                            _dev_ptr(out_src, torch.int32, None, "out_src", n),
                            _dev_ptr(out_count, torch.int32, None, "out_count", 1), _stream(stream)))
    return out_rays, out_skip, out_src, out_count


class _DevArray:
    """Zero-copy view of library-owned device memory (__cuda_array_interface__)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 3, "strides": None}


def _view(ptr, shape, typestr):
    import torch
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device="cuda")


class Batch:
    """Owns one rt_batch handle (multi-transmitter, multi-bounce pipeline)."""

    def __init__(self, scene, tx_pos, tx_param, kind=RT_RAYS_FIBONACCI, max_order=3, tmax=1000.0, rx_pos=None,
                 use_graph=True, ray_tile=0, receive=False, max_rx_records=1 << 16, rx_delta=None):
        self.scene = scene          # keeps the scene alive
        self.tx = np.ascontiguousarray(tx_pos, dtype=np.float32).reshape(-1, 3)
        self.param = np.ascontiguousarray(tx_param, dtype=np.int64).reshape(-1)
        self.rx = None if rx_pos is None else np.ascontiguousarray(rx_pos, dtype=np.float32).reshape(-1, 3)
        d = BatchDesc()
        d.n_tx = len(self.tx)
        d.tx_pos = self.tx.ctypes.data
        d.tx_param = self.param.ctypes.data
        d.dir_kind, d.max_order, d.tmax = int(kind), int(max_order), float(tmax)
        d.n_rx = 0 if self.rx is None else len(self.rx)
        d.rx_pos = None if self.rx is None else self.rx.ctypes.data
        d.use_graph = 1 if use_graph else 0
        d.ray_tile = int(ray_tile)
        d.receive = 1 if receive else 0
        d.max_rx_records = int(max_rx_records)
        self.rx_delta = None if rx_delta is None else np.ascontiguousarray(rx_delta, dtype=np.float32).reshape(-1)
        d.rx_delta = None if self.rx_delta is None else self.rx_delta.ctypes.data
        self.max_rx_records = int(max_rx_records)
        h = ctypes.c_void_p()
        _check(lib().rt_batch_create(scene.handle, ctypes.byref(d), ctypes.byref(h)))
        self._h = h.value
        self.max_order = int(max_order)
        self.n0 = int(sum(rt_ray_count(kind, p) for p in self.param))
        self.n_seg = d.n_tx * d.n_rx

    def run(self, stream=None):
        _check(lib().rt_batch_run(self._h, _stream(stream)))

    def stats(self, stream=None) -> dict:
        st = BatchStats()
        _check(lib().rt_batch_stats_get(self._h, _stream(stream), ctypes.byref(st)))
        return dict(rays=list(st.rays)[: st.n_orders], segments=st.segments, total_rays=st.total_rays,
                    visible=st.visible, flagged=st.flagged, received=list(st.received)[: st.n_orders])

    def received(self, k):
        """(records int32 [count, 4] view (ray in order k, rx, l bits, dist bits), count) of order k."""
        r, c = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().rt_batch_received(self._h, int(k), ctypes.byref(r), ctypes.byref(c)))
        n = int(_view(c.value, (1,), "<i4").item())
        return _view(r.value, (min(n, self.max_rx_records), 4), "<i4"), n

    def order(self, k):
        """(rays [n,8], hits [n,4], src [n] or None, count) for order k (views; count is a python int)."""
        r, h, s, c = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().rt_batch_order(self._h, int(k), ctypes.byref(r), ctypes.byref(h), ctypes.byref(s),
                                    ctypes.byref(c)))
        n = self.n0
        if k > 0:
            n = int(_view(c.value, (1,), "<i4").item())
        rays = _view(r.value, (n, 8), "<f4")
        hits = _view(h.value, (n, 4), "<f4")
        src = _view(s.value, (n,), "<i4") if k > 0 else None
        return rays, hits, src, n

    def visibility(self):
        p = ctypes.c_void_p()
        _check(lib().rt_batch_visibility(self._h, ctypes.byref(p)))
        return _view(p.value, (self.n_seg,), "|u1")

    def destroy(self):
        if getattr(self, "_h", None):
            _check(lib().rt_batch_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Session:
    """Owns one rt_session (resident scenes, memory-admitted requests)."""

    def __init__(self, pool_bytes, max_slots=4):
        h = ctypes.c_void_p()
        _check(lib().rt_session_create(int(pool_bytes), int(max_slots), ctypes.byref(h)))
        self._h = h.value
        self._keep = {}        # ticket -> host buffers kept alive until completion
        self._scenes = []

    def add_scene(self, scene) -> int:
        sid = ctypes.c_int32()
        _check(lib().rt_session_add_scene(self._h, scene.handle, ctypes.byref(sid)))
        self._scenes.append(scene)
        return sid.value

    def submit(self, scene_id, tx, kind, param, max_order=0, tmax=1000.0, want_hits=True, want_orders=False):
        """Returns a ticket; results via result(ticket) after wait().  want_orders:
        also the hits and parent indices of every reflection order (orders(ticket))."""
        n = rt_ray_count(kind, param)
        hits = np.empty((n, 4), np.float32) if want_hits else None
        counts = np.zeros(RT_BATCH_MAX_ORDER + 1, np.int64)
        r = Request()
        r.scene_id, r.dir_kind, r.param, r.max_order, r.tmax = int(scene_id), int(kind), int(param), \
            int(max_order), float(tmax)
        for k in range(3):
            r.tx[k] = float(tx[k])
        r.hits_host = hits.ctypes.data if hits is not None else None
        r.order_counts_host = counts.ctypes.data
        orders = None
        if want_orders and max_order > 0:
            oh = [None] + [np.empty((n, 4), np.float32) for _ in range(max_order)]
            osrc = [None] + [np.empty(n, np.int32) for _ in range(max_order)]
            ph = (ctypes.c_void_p * (max_order + 1))(*([None] + [a.ctypes.data for a in oh[1:]]))
            ps = (ctypes.c_void_p * (max_order + 1))(*([None] + [a.ctypes.data for a in osrc[1:]]))
            r.order_hits_host = ctypes.cast(ph, ctypes.c_void_p)
            r.order_src_host = ctypes.cast(ps, ctypes.c_void_p)
            orders = (oh, osrc, ph, ps)
        t = ctypes.c_uint64()
        _check(lib().rt_session_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        self._keep[t.value] = (hits, counts, int(max_order), orders)
        return t.value

    def poll(self, ticket) -> bool:
        d = ctypes.c_int()
        _check(lib().rt_session_poll(self._h, ticket, ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket, timeout_s=None):
        ns = -1 if timeout_s is None else int(timeout_s * 1e9)
        _check(lib().rt_session_wait(self._h, ticket, ns))

    def result(self, ticket):
        hits, counts, mo, _ = self._keep[ticket]
        return hits, counts[: mo + 1]

    def orders(self, ticket):
        """[(hits [c_k, 4], parent index [c_k]) for k = 1 .. max_order] of a request
        submitted with want_orders."""
        _, counts, mo, orders = self._keep[ticket]
        if orders is None:
            return []
        oh, osrc = orders[0], orders[1]
        return [(oh[k][: counts[k]], osrc[k][: counts[k]]) for k in range(1, mo + 1)]

    def release(self, ticket):
        """Forget a finished request (rt_session_release); returns its results."""
        _check(lib().rt_session_release(self._h, ticket))
        hits, counts, mo, _ = self._keep.pop(ticket)
        return hits, counts[: mo + 1]

    def stats(self) -> dict:
        st = SessionStats()
        _check(lib().rt_session_stats_get(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in SessionStats._fields_}

    def destroy(self):
        if getattr(self, "_h", None):
            _check(lib().rt_session_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ---- reception (Sec. III.C, Eq. 4) -----------------------------------------
class RxSet:
    """Owns one rt_rxset (receivers in a device grid)."""

    def __init__(self, handle, m, r_max):
        self._h = handle
        self.m = m
        self.r_max = r_max

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("receiver set destroyed")
        return self._h

    def destroy(self):
        if self._h:
            _check(lib().rt_rxset_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def rt_rxset_create(rx, r_max):
    """Receivers rx (host [m, 3]) for receiving spheres up to radius r_max."""
    a = np.ascontiguousarray(rx, dtype=np.float32).reshape(-1, 3)
    h = ctypes.c_void_p()
    _check(lib().rt_rxset_create(a.ctypes.data_as(ctypes.c_void_p), a.shape[0], float(r_max), ctypes.byref(h)))
    return RxSet(h.value, a.shape[0], float(r_max))


def rt_receive(rs: RxSet, rays, hits, delta, range0, out=None, count=None, n_dev=None, max_records=None,
               stats=None, stream=None):
    """Receiving-sphere test (Eq. 4) of every ray's segment against the receivers.

    Returns (records int32 [max_records, 4] = (ray, rx, l bits, dist bits), count int32 [1]),
    both on the device; records[:count] are valid (view columns 2-3 as float32 for l, dist).
    stats (optional int64 [2] device tensor): cells visited and receiver entries tested are
    added to it."""
    import torch
    rp = _dev_ptr(rays, torch.float32, 8, "rays")
    n = rays.shape[0]
    hp = _dev_ptr(hits, torch.float32, 4, "hits", n)
    if out is None:
        out = torch.empty((max_records if max_records is not None else max(1024, n // 4), 4), dtype=torch.int32,
                          device=rays.device)
    op = _dev_ptr(out, torch.int32, 4, "out")
    if count is None:
        count = torch.zeros(1, dtype=torch.int32, device=rays.device)
    cp = _dev_ptr(count, torch.int32, None, "count", 1)
    nd = None if n_dev is None else _dev_ptr(n_dev, torch.int32, None, "n_dev", 1)
    sp = None if stats is None else _dev_ptr(stats, torch.int64, None, "stats", 2).value
    p = ReceiveParams(float(delta), float(range0), int(out.shape[0]), 0, sp, None)
    _check(lib().rt_receive(rs.handle, rp, hp, n, nd, ctypes.byref(p), op, cp, _stream(stream)))
    return out, count


def rt_probe_l2_read(buf, reps, stream=None):
    """One launch reading the device tensor `buf` (fits in L2) `reps` times; time it with events."""
    import torch
    if not (isinstance(buf, torch.Tensor) and buf.is_cuda and buf.is_contiguous()):
        raise TypeError("buf must be a contiguous CUDA tensor")
    nbytes = buf.numel() * buf.element_size()
    _check(lib().rt_probe_l2_read(ctypes.c_void_p(buf.data_ptr()), nbytes, int(reps), None, _stream(stream)))
