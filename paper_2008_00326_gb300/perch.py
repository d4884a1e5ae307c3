"""Thin ctypes binding of libperch (include/perch.h), same names as the C ABI.

Argument marshalling only: every step of the scoring path runs in the CUDA
library.  Host-pointer (synchronous) calls take numpy arrays; device-pointer
(asynchronous) calls take torch CUDA tensors plus a stream, and PyTorch is used
for nothing but that device memory and the stream handle.  The module fails
loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

PERCH_OK = 0
STATUS = {0: "PERCH_OK", -1: "PERCH_E_INVALID", -2: "PERCH_E_NOMEM", -3: "PERCH_E_BUDGET",
          -4: "PERCH_E_NOTFOUND", -5: "PERCH_E_CUDA", -6: "PERCH_E_TIMEOUT", -7: "PERCH_E_BUSY"}

# every function that include/perch.h declares
EXPORTS = ("perch_default_params", "perch_create", "perch_destroy", "perch_last_error",
           "perch_hbm_used", "perch_load_mesh", "perch_release_mesh", "perch_set_observation",
           "perch_release_scene", "perch_score_hypotheses", "perch_best", "perch_set_launch_config",
           "perch_debug_render_keys", "perch_best_noalloc", "perch_score_batch",
           "perch_batch_graph_create", "perch_batch_graph_launch", "perch_batch_graph_destroy",
           "perch_autotune", "perch_server_start", "perch_submit", "perch_poll", "perch_wait",
           "perch_ticket_times", "perch_server_stop", "perch_pose_proposals",
           "perch_default_gicp_params", "perch_refine_hypotheses", "perch_tree_search",
           "perch_measure_smem_atomics", "perch_add_s", "perch_add_s_auc", "perch_sync",
           "perch_ticket_release", "perch_server_tickets", "perch_best_key", "perch_set_raster_bins")


class PerchError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class perch_work_item(C.Structure):
    _fields_ = [("scene_id", C.c_int32), ("mesh_id", C.c_int32), ("label", C.c_int32),
                ("roi", C.c_int32 * 4), ("pose_offset", C.c_int64), ("n", C.c_int64)]


def work_items(specs):
    """ctypes array of perch_work_item from (scene_id, mesh_id, label, roi|None, offset, n)."""
    arr = (perch_work_item * max(1, len(specs)))()
    for i, (sid, mid, label, roi, off, n) in enumerate(specs):
        arr[i].scene_id, arr[i].mesh_id, arr[i].label = sid, mid, label
        r = roi if roi is not None else (0, 0, 0, 0)
        for k in range(4):
            arr[i].roi[k] = int(r[k])
        arr[i].pose_offset, arr[i].n = int(off), int(n)
    return arr


class perch_server_config(C.Structure):
    _fields_ = [("slots", C.c_int32), ("max_batch_hypotheses", C.c_int64), ("max_wait_us", C.c_int32)]


class perch_request(C.Structure):
    _fields_ = [("scene_id", C.c_int32), ("mesh_id", C.c_int32), ("label", C.c_int32),
                ("roi", C.c_int32 * 4), ("poses", C.c_void_p), ("n", C.c_int64), ("costs", C.c_void_p)]


class Server:
    """A continuous-batching server on a Context (perch_server_* calls).

    submit() copies the poses and returns (ticket, costs array); the costs are
    valid once wait(ticket) returns."""

    def __init__(self, ctx, slots=2, max_batch_hypotheses=1 << 17, max_wait_us=0):
        self.ctx = ctx
        cfg = perch_server_config(slots, max_batch_hypotheses, max_wait_us)
        self.h = C.c_void_p()
        st = load().perch_server_start(ctx.ctx, C.byref(cfg), C.byref(self.h))
        if st != PERCH_OK:
            raise PerchError(st, perch_last_error(ctx.ctx))
        self._keep = {}

    def submit(self, scene_id, mesh_id, label, roi, poses):
        p = np.ascontiguousarray(poses, np.float32)
        n = p.size // 12
        costs = np.zeros((n, 2), np.int32)
        r = perch_request()
        r.scene_id, r.mesh_id, r.label = scene_id, mesh_id, label
        rr = roi if roi is not None else (0, 0, 0, 0)
        for k in range(4):
            r.roi[k] = int(rr[k])
        r.poses, r.n, r.costs = p.ctypes.data, n, costs.ctypes.data
        t = C.c_uint64()
        st = load().perch_submit(self.h, C.byref(r), C.byref(t))
        if st != PERCH_OK:
            raise PerchError(st, "perch_submit")
        self._keep[t.value] = costs
        return t.value, costs

    def poll(self, ticket):
        return load().perch_poll(self.h, ticket)

    def wait(self, ticket, timeout_us=-1):
        st = load().perch_wait(self.h, ticket, timeout_us)
        if st != PERCH_OK:
            raise PerchError(st, "perch_wait")
        return self._keep.pop(ticket)

    def release(self, ticket):
        """Forget a finished ticket (perch_ticket_release)."""
        st = load().perch_ticket_release(self.h, ticket)
        if st != PERCH_OK:
            raise PerchError(st, "perch_ticket_release")

    def held(self):
        """Tickets the server holds (perch_server_tickets)."""
        n = C.c_int64()
        st = load().perch_server_tickets(self.h, C.byref(n))
        if st != PERCH_OK:
            raise PerchError(st, "perch_server_tickets")
        return n.value

    def times(self, ticket):
        a = C.c_int64()
        b = C.c_int64()
        st = load().perch_ticket_times(self.h, ticket, C.byref(a), C.byref(b))
        if st != PERCH_OK:
            raise PerchError(st, "perch_ticket_times")
        return a.value, b.value

    def stop(self):
        if self.h is not None and self.h.value:
            load().perch_server_stop(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.stop()


class perch_params(C.Structure):
    _fields_ = [("delta_m", C.c_float), ("tau_c", C.c_float), ("color_check", C.c_int32),
                ("stride", C.c_int32), ("occ_margin_units", C.c_int32), ("z_near_m", C.c_float),
                ("jo_mode", C.c_int32)]


class perch_gicp_params(C.Structure):
    _fields_ = [("max_iterations", C.c_int32), ("epsilon", C.c_float),
                ("normal_max_jump_units", C.c_int32), ("min_correspondences", C.c_int32),
                ("stop_rotation_rad", C.c_float), ("stop_translation_m", C.c_float),
                ("max_source_points", C.c_int32)]


class perch_tree_object(C.Structure):
    _fields_ = [("mesh_id", C.c_int32), ("label", C.c_int32), ("roi", C.c_int32 * 4),
                ("poses", C.c_void_p), ("n", C.c_int32)]


_lib = None


def load(path: str | None = None):
    """Load libperch.so (in-tree; PERCH_LIB=checks in the environment loads
    the debug build libperch_checks.so instead).  Raises if it is missing:
    build it first."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or (_build.LIB_CHECKS if os.environ.get("PERCH_LIB") == "checks" else LIB_PATH)
    if not os.path.exists(path):
        raise RuntimeError(f"libperch.so not found at {path}; run __graft_entry__.build() "
                           "(the scoring path has no CPU fallback)")
    L = C.CDLL(path)
    P, I32, I64, U64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    sig = {
        "perch_default_params": ([P], I32),
        "perch_create": ([P, I32, U64], I32),
        "perch_destroy": ([P], I32),
        "perch_last_error": ([P], C.c_char_p),
        "perch_hbm_used": ([P], U64),
        "perch_load_mesh": ([P, P, P, I32, P, I32, C.c_float, C.c_float, P], I32),
        "perch_release_mesh": ([P, I32], I32),
        "perch_set_observation": ([P, P, P, P, I32, I32, C.c_float, C.c_float, C.c_float,
                                   C.c_float, P, P], I32),
        "perch_release_scene": ([P, I32], I32),
        "perch_score_hypotheses": ([P, I32, I32, I32, P, P, I64, P, P], I32),
        "perch_best": ([P, P, P, I64, P, P, P], I32),
        "perch_set_launch_config": ([P, I32, I32, I32], I32),
        "perch_debug_render_keys": ([P, I32, I32, P, P, P], I32),
        "perch_best_noalloc": ([P, P, I64, P, P, P], I32),
        "perch_score_batch": ([P, P, I32, P, P, P], I32),
        "perch_batch_graph_create": ([P, P, I32, P, P, P], I32),
        "perch_batch_graph_launch": ([P, P], I32),
        "perch_batch_graph_destroy": ([P], I32),
        "perch_autotune": ([P, P, I32, P, P, P, P, P], I32),
        "perch_set_raster_bins": ([P, I32], I32),
        "perch_server_start": ([P, P, P], I32),
        "perch_submit": ([P, P, P], I32),
        "perch_poll": ([P, U64], I32),
        "perch_wait": ([P, U64, I64], I32),
        "perch_ticket_times": ([P, U64, P, P], I32),
        "perch_server_stop": ([P], I32),
        "perch_pose_proposals": ([P, I32, I32, I32, P, I32, I32, I32, P, P, P], I32),
        "perch_default_gicp_params": ([P], I32),
        "perch_refine_hypotheses": ([P, I32, I32, I32, P, P, I64, P, P, P, P], I32),
        "perch_tree_search": ([P, I32, P, I32, I32, P, P, P, P], I32),
        "perch_measure_smem_atomics": ([I32, P, P], I32),
        "perch_add_s": ([P, I32, P, P, I64, I32, P, P], I32),
        "perch_add_s_auc": ([P, I64, C.c_double, P], I32),
        "perch_sync": ([P, P], I32),
        "perch_best_key": ([P, P, P, I64, P, P], I32),
        "perch_ticket_release": ([P, U64], I32),
        "perch_server_tickets": ([P, P], I32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(ctx, st):
    if st != PERCH_OK:
        msg = load().perch_last_error(ctx)
        raise PerchError(st, msg.decode() if msg else "")


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype)
    return a, a.ctypes.data


def _ptr_of(x):
    """Device pointer of a torch CUDA tensor, or host pointer of a numpy array."""
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def perch_default_params(**over) -> perch_params:
    p = perch_params()
    load().perch_default_params(C.byref(p))
    for k, v in over.items():
        setattr(p, k, v)
    return p


def perch_create(device: int = 0, hbm_budget_bytes: int = 0):
    ctx = C.c_void_p()
    st = load().perch_create(C.byref(ctx), device, hbm_budget_bytes)
    if st != PERCH_OK:
        raise PerchError(st, "perch_create failed")
    return ctx


def perch_destroy(ctx):
    _check(ctx, load().perch_destroy(ctx))


def perch_last_error(ctx) -> str:
    m = load().perch_last_error(ctx)
    return m.decode() if m else ""


def perch_hbm_used(ctx) -> int:
    return int(load().perch_hbm_used(ctx))


def perch_load_mesh(ctx, verts, rgb, tris, vol_radius_m, vol_height_m) -> int:
    v, pv = _host(verts, np.float32)
    c, pc = _host(rgb, np.uint8)
    t, pt = _host(tris, np.int32)
    mid = C.c_int32()
    _check(ctx, load().perch_load_mesh(ctx, pv, pc, v.shape[0], pt, t.shape[0], vol_radius_m,
                                        vol_height_m, C.byref(mid)))
    return mid.value


def perch_release_mesh(ctx, mesh_id):
    _check(ctx, load().perch_release_mesh(ctx, mesh_id))


def perch_set_observation(ctx, depth, rgb, labels, fx, fy, cx, cy, params: perch_params) -> int:
    d, pd = _host(depth, np.uint16)
    c, pc = _host(rgb, np.uint8)
    lab, pl = (None, None) if labels is None else _host(labels, np.int32)
    H, W = d.shape
    sid = C.c_int32()
    _check(ctx, load().perch_set_observation(ctx, pd, pc, pl, W, H, fx, fy, cx, cy,
                                              C.byref(params), C.byref(sid)))
    return sid.value


def perch_release_scene(ctx, scene_id):
    _check(ctx, load().perch_release_scene(ctx, scene_id))


def _roi(roi):
    if roi is None:
        return None, None
    r = (C.c_int32 * 4)(*[int(x) for x in roi])
    return r, C.cast(r, C.c_void_p)


def perch_score_hypotheses(ctx, scene_id, mesh_id, label, roi, poses, costs=None, stream=None):
    """Host mode (stream None): poses numpy (n,12) -> returns costs (n,2) int32.
    Device mode: poses and costs torch CUDA tensors, stream a torch.cuda.Stream or
    raw handle; enqueues and returns costs."""
    keep, proi = _roi(roi)
    if stream is None:
        p, pp = _host(poses, np.float32)
        n = p.size // 12
        out = np.empty((n, 2), np.int32) if costs is None else costs
        _check(ctx, load().perch_score_hypotheses(ctx, scene_id, mesh_id, label, proi, pp, n,
                                                   out.ctypes.data, None))
        return out
    n = poses.numel() // 12
    handle = getattr(stream, "cuda_stream", stream)
    _check(ctx, load().perch_score_hypotheses(ctx, scene_id, mesh_id, label, proi,
                                               _ptr_of(poses), n, _ptr_of(costs), handle))
    return costs


def perch_best(ctx, costs, ids=None, stream=None, out_index=None, out_cost=None):
    """Host mode: costs numpy (n,2) -> (best_index, best_cost).  Device mode:
    costs/ids/out_index/out_cost torch CUDA tensors, result written on `stream`."""
    if stream is None:
        c, pc = _host(costs, np.int32)
        n = c.size // 2
        pi = None
        if ids is not None:
            ids_a, pi = _host(ids, np.uint64)
        bi = C.c_int64()
        bc = C.c_int32()
        _check(ctx, load().perch_best(ctx, pc, pi, n, C.byref(bi), C.byref(bc), None))
        return bi.value, bc.value
    n = costs.numel() // 2
    handle = getattr(stream, "cuda_stream", stream)
    _check(ctx, load().perch_best(ctx, _ptr_of(costs), None if ids is None else _ptr_of(ids), n,
                                   _ptr_of(out_index), _ptr_of(out_cost), handle))


def _require_cuda(name, t, dtypes, min_numel=1):
    """t must be a contiguous torch CUDA tensor on the current device with one
    of `dtypes` and at least min_numel elements (the kernel would otherwise be
    handed a host pointer or read past the end)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a torch CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on {t.device}, not the current device")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.dtype not in dtypes:
        raise TypeError(f"{name} has dtype {t.dtype}; expected one of {dtypes}")
    if t.numel() < min_numel:
        raise ValueError(f"{name} needs at least {min_numel} elements")


def perch_best_key(ctx, costs, key, ids=None, stream=None):
    """The winner of costs as the packed key (J << 32) | id, written to the
    one-element int64 CUDA tensor `key` on `stream` (device mode only)."""
    n = costs.numel() // 2
    _check(ctx, load().perch_best_key(ctx, _ptr_of(costs), None if ids is None else _ptr_of(ids), n,
                                       _ptr_of(key), getattr(stream, "cuda_stream", stream)))


def perch_best_noalloc(costs, ids, out_index, out_cost, stream=None):
    """Argmin without a context or any allocation: contiguous torch CUDA tensors
    on the current device -- costs int32 (n, 2), ids int64 (n,) or None,
    out_index int64 and out_cost int32 with at least one element each."""
    import torch
    _require_cuda("costs", costs, (torch.int32,))
    if costs.dim() != 2 or costs.shape[1] != 2:
        raise ValueError("costs must have shape (n, 2)")
    n = costs.shape[0]
    if ids is not None:
        _require_cuda("ids", ids, (torch.int64,), n)
    _require_cuda("out_index", out_index, (torch.int64,))
    _require_cuda("out_cost", out_cost, (torch.int32,))
    handle = getattr(stream, "cuda_stream", stream)
    st = load().perch_best_noalloc(_ptr_of(costs), None if ids is None else _ptr_of(ids), n,
                                   _ptr_of(out_index), _ptr_of(out_cost), handle)
    if st != PERCH_OK:
        raise PerchError(st, "perch_best_noalloc failed")


def perch_score_batch(ctx, items, poses, costs=None, stream=None):
    """items: ctypes array from work_items().  Host mode: poses numpy (N,12) ->
    costs (N,2).  Device mode: poses/costs torch CUDA tensors and a stream."""
    n_items = len(items)
    if stream is None:
        p, pp = _host(poses, np.float32)
        out = np.zeros((p.size // 12, 2), np.int32) if costs is None else costs
        _check(ctx, load().perch_score_batch(ctx, items, n_items, pp, out.ctypes.data, None))
        return out
    handle = getattr(stream, "cuda_stream", stream)
    _check(ctx, load().perch_score_batch(ctx, items, n_items, _ptr_of(poses), _ptr_of(costs), handle))
    return costs


def perch_batch_graph_create(ctx, items, poses, costs):
    g = C.c_void_p()
    _check(ctx, load().perch_batch_graph_create(ctx, items, len(items), _ptr_of(poses), _ptr_of(costs),
                                                 C.byref(g)))
    return g


def perch_batch_graph_launch(ctx, graph, stream):
    _check(ctx, load().perch_batch_graph_launch(graph, getattr(stream, "cuda_stream", stream)))


def perch_batch_graph_destroy(graph):
    load().perch_batch_graph_destroy(graph)


def perch_autotune(ctx, items, poses, costs):
    """(threads, z-buffer words, tile-bin capacity) chosen for this batch's class."""
    t = C.c_int32()
    z = C.c_int32()
    b = C.c_int32()
    _check(ctx, load().perch_autotune(ctx, items, len(items), _ptr_of(poses), _ptr_of(costs),
                                       C.byref(t), C.byref(z), C.byref(b)))
    return t.value, z.value, b.value


def perch_pose_proposals(ctx, scene_id, mesh_id, label, bbox, M, N, K, poses=None, z_range=None,
                         stream=None):
    """Host mode: returns (poses (M*N*K,12) float32, (z_min, z_max)).  Device
    mode: poses/z_range torch CUDA tensors filled on `stream`."""
    keep, pbox = _roi(bbox)
    if stream is None:
        out = np.empty((M * N * K, 12), np.float32)
        zr = np.zeros(2, np.int32)
        _check(ctx, load().perch_pose_proposals(ctx, scene_id, mesh_id, label, pbox, M, N, K,
                                                 out.ctypes.data, zr.ctypes.data, None))
        return out, (int(zr[0]), int(zr[1]))
    _check(ctx, load().perch_pose_proposals(ctx, scene_id, mesh_id, label, pbox, M, N, K, _ptr_of(poses),
                                             None if z_range is None else _ptr_of(z_range),
                                             getattr(stream, "cuda_stream", stream)))
    return poses


def perch_default_gicp_params(**over) -> perch_gicp_params:
    p = perch_gicp_params()
    st = load().perch_default_gicp_params(C.byref(p))
    if st != PERCH_OK:
        raise PerchError(st, "perch_default_gicp_params")
    for k, v in over.items():
        setattr(p, k, v)
    return p


def perch_refine_hypotheses(ctx, scene_id, mesh_id, label, roi, poses, params=None, poses_out=None,
                            info=None, stream=None):
    """M2M GICP refinement.  Host mode (stream None): poses numpy (n,12) ->
    (refined poses (n,12) float32, info (n,2) int32).  Device mode: poses,
    poses_out (and info, or None) torch CUDA tensors; enqueued on `stream`."""
    keep, proi = _roi(roi)
    gp = params if params is not None else perch_default_gicp_params()
    if stream is None:
        p, pp = _host(poses, np.float32)
        n = p.size // 12
        out = np.empty((n, 12), np.float32) if poses_out is None else poses_out
        inf = np.empty((n, 2), np.int32) if info is None else info
        _check(ctx, load().perch_refine_hypotheses(ctx, scene_id, mesh_id, label, proi, pp, n, C.byref(gp),
                                                    out.ctypes.data, inf.ctypes.data, None))
        return out, inf
    n = poses.numel() // 12
    _check(ctx, load().perch_refine_hypotheses(ctx, scene_id, mesh_id, label, proi, _ptr_of(poses), n,
                                                C.byref(gp), _ptr_of(poses_out),
                                                None if info is None else _ptr_of(info),
                                                getattr(stream, "cuda_stream", stream)))
    return poses_out


def perch_tree_search(ctx, scene_id, objects, beam_width):
    """Monotone Scene Generation tree search.  objects: list of (mesh_id, label,
    roi or None, poses (n,12)).  Returns (order, pose_index, level_cost, edges)."""
    K = len(objects)
    arr = (perch_tree_object * K)()
    keep = []
    for k, (mid, label, roi, poses) in enumerate(objects):
        p = np.ascontiguousarray(poses, np.float32).reshape(-1, 12)
        keep.append(p)
        arr[k].mesh_id = mid
        arr[k].label = label
        for i, x in enumerate(roi if roi is not None else (0, 0, 0, 0)):
            arr[k].roi[i] = int(x)
        arr[k].poses = p.ctypes.data
        arr[k].n = p.shape[0]
    order = np.zeros(K, np.int32)
    pidx = np.zeros(K, np.int32)
    lc = np.zeros(K, np.int64)
    edges = C.c_int64()
    _check(ctx, load().perch_tree_search(ctx, scene_id, arr, K, beam_width, order.ctypes.data,
                                          pidx.ctypes.data, lc.ctypes.data, C.byref(edges)))
    return order.tolist(), pidx.tolist(), lc.tolist(), edges.value


def perch_add_s(ctx, mesh_id, poses, poses_true, symmetric=True, out=None, stream=None):
    """ADD-S (symmetric) or ADD per pose pair.  Host mode: numpy in, float64 (n,) out."""
    if stream is None:
        p, pp = _host(poses, np.float32)
        t, pt = _host(poses_true, np.float32)
        n = p.size // 12
        res = np.empty(n, np.float64)
        _check(ctx, load().perch_add_s(ctx, mesh_id, pp, pt, n, int(bool(symmetric)), res.ctypes.data, None))
        return res
    n = poses.numel() // 12
    _check(ctx, load().perch_add_s(ctx, mesh_id, _ptr_of(poses), _ptr_of(poses_true), n, int(bool(symmetric)),
                                    _ptr_of(out), getattr(stream, "cuda_stream", stream)))
    return out


def perch_add_s_auc(add, max_threshold=0.1):
    a, pa = _host(add, np.float64)
    out = C.c_double()
    st = load().perch_add_s_auc(pa, a.size, max_threshold, C.byref(out))
    if st != PERCH_OK:
        raise PerchError(st, "perch_add_s_auc")
    return out.value


def perch_measure_smem_atomics(device=0):
    """(u32, u64) shared-memory atomicMin operations per second."""
    a, b = C.c_double(), C.c_double()
    st = load().perch_measure_smem_atomics(device, C.byref(a), C.byref(b))
    if st != PERCH_OK:
        raise PerchError(st, "perch_measure_smem_atomics")
    return a.value, b.value


def perch_sync(ctx, stream=None):
    """Wait for `stream` (None: the context's stream) and raise if the kernels
    of earlier asynchronous calls reported an error."""
    _check(ctx, load().perch_sync(ctx, getattr(stream, "cuda_stream", stream)))


def perch_set_launch_config(ctx, threads, zbuf_words, mark_bits=0):
    _check(ctx, load().perch_set_launch_config(ctx, threads, zbuf_words, mark_bits))


def perch_set_raster_bins(ctx, bin_cap):
    _check(ctx, load().perch_set_raster_bins(ctx, bin_cap))


def perch_debug_render_keys(ctx, scene_id, mesh_id, roi, pose, W, H):
    keep, proi = _roi(roi)
    p, pp = _host(pose, np.float32)
    keys = np.empty((H, W), np.uint64)
    _check(ctx, load().perch_debug_render_keys(ctx, scene_id, mesh_id, proi, pp, keys.ctypes.data))
    return keys


class Context:
    """Owning wrapper: a perch context plus the meshes and scenes loaded into it."""

    def __init__(self, device=0, hbm_budget_bytes=0):
        self.ctx = perch_create(device, hbm_budget_bytes)

    def close(self):
        if self.ctx is not None:
            perch_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_mesh(self, mesh):
        return perch_load_mesh(self.ctx, mesh.verts, mesh.rgb, mesh.tris, mesh.vol_radius,
                               mesh.vol_height)

    def set_observation(self, scene, **over):
        p = scene.params
        params = perch_default_params(delta_m=p.delta_m, tau_c=p.tau_c, color_check=p.color_check,
                                      stride=p.stride, occ_margin_units=p.occ_margin_units,
                                      z_near_m=p.z_near_m, jo_mode=p.jo_mode)
        for k, v in over.items():
            setattr(params, k, v)
        return perch_set_observation(self.ctx, scene.depth, scene.rgb, scene.labels, scene.fx,
                                     scene.fy, scene.cx, scene.cy, params)

    def score(self, scene_id, mesh_id, label, roi, poses, costs=None, stream=None):
        return perch_score_hypotheses(self.ctx, scene_id, mesh_id, label, roi, poses, costs, stream)

    def best(self, costs, ids=None, **kw):
        return perch_best(self.ctx, costs, ids, **kw)

    def refine(self, scene_id, mesh_id, label, roi, poses, params=None, **kw):
        return perch_refine_hypotheses(self.ctx, scene_id, mesh_id, label, roi, poses, params, **kw)

    def set_launch_config(self, threads, zbuf_words, mark_bits=0, bin_cap=0):
        perch_set_launch_config(self.ctx, threads, zbuf_words, mark_bits)
        perch_set_raster_bins(self.ctx, bin_cap)

    def render_keys(self, scene_id, mesh_id, roi, pose, W, H):
        return perch_debug_render_keys(self.ctx, scene_id, mesh_id, roi, pose, W, H)

    @property
    def hbm_used(self):
        return perch_hbm_used(self.ctx)

    def last_error(self):
        return perch_last_error(self.ctx)
