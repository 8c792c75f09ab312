"""Thin ctypes binding of include/orca_gb300.h.

Each ``orca_*`` function here has the name and argument order of the C entry point and
only marshals arguments: numpy arrays become host pointers (ORCA_HOST), CUDA torch
tensors become device pointers (ORCA_DEVICE), and ``stream=None`` means torch's current
stream.  All work runs in liborca_gb300.so; if the library is missing this module raises
instead of falling back to anything.

``OrcaSim`` bundles a context with a torch-owned device workspace.
"""
from __future__ import annotations

import contextlib
import ctypes
import os

import numpy as np

from . import build as _build

ORCA_OK = 0
ORCA_ERR_ARG = -1
ORCA_ERR_NOMEM = -2
ORCA_ERR_CUDA = -3
ORCA_ERR_STATE = -4
ORCA_ERR_NUMERIC = -5
ORCA_ERR_TIMEOUT = -6
ORCA_ERR_CAPACITY = -7
ORCA_ERR_BOUNDS = -8
ORCA_HOST = 0
ORCA_DEVICE = 1
ORCA_FLAG_RECORD = 1
ORCA_FLAG_NO_GRAPH = 2

LIB_PATH = _build.LIB
HEADER = os.path.join(_build.ROOT, "include", "orca_gb300.h")


class OrcaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class orca_params(ctypes.Structure):
    _fields_ = [("max_agents", ctypes.c_int32), ("max_neighbors", ctypes.c_int32),
                ("max_cells", ctypes.c_int32), ("neighbor_dist", ctypes.c_float),
                ("dt", ctypes.c_float), ("cell_size", ctypes.c_float),
                ("flags", ctypes.c_uint32), ("max_scenes", ctypes.c_int32)]


class orca_scene(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("max_neighbors", ctypes.c_int32),
                ("neighbor_dist", ctypes.c_float), ("dt", ctypes.c_float),
                ("cell_size", ctypes.c_float), ("reserved", ctypes.c_int32)]


_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load liborca_gb300.so (built by ``build.build()``).  Raises if it is absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OrcaError(ORCA_ERR_STATE, f"{p} is missing: run paper_1908_10107_gb300.build.build()")
    lib = ctypes.CDLL(p)
    c = ctypes
    vp, i32, sz = c.c_void_p, c.c_int32, c.c_size_t
    P = c.POINTER(orca_params)
    sigs = {
        "orca_workspace_size": ([P, c.POINTER(sz)], c.c_int),
        "orca_create": ([P, vp, sz, c.POINTER(vp)], c.c_int),
        "orca_destroy": ([vp], c.c_int),
        "orca_set_agents": ([vp, i32] + [vp] * 7 + [c.c_int, vp], c.c_int),
        "orca_update_state": ([vp, vp, vp, c.c_int, vp], c.c_int),
        "orca_step_host": ([vp, vp, vp, i32, vp, vp, vp], c.c_int),
        "orca_set_scenes": ([vp, i32, vp] + [vp] * 7 + [c.c_int, vp], c.c_int),
        "orca_get_scene_grids": ([vp, vp, vp, vp], c.c_int),
        "orca_step": ([vp, i32, vp], c.c_int),
        "orca_get_state": ([vp, vp, vp, c.c_int, vp], c.c_int),
        "orca_get_neighbors": ([vp, vp, c.c_int, vp], c.c_int),
        "orca_get_cells": ([vp, vp, vp, vp, c.c_int, vp], c.c_int),
        "orca_get_counters": ([vp, vp, vp], c.c_int),
        "orca_count_ops": ([vp, i32], c.c_int),
        "orca_remove_arrived": ([vp, c.POINTER(i32), vp, c.c_int, vp], c.c_int),
        "orca_spawn_agents": ([vp, i32] + [vp] * 6 + [c.c_float, c.c_int, vp, c.POINTER(i32), vp], c.c_int),
        "orca_set_obstacles": ([vp, i32, vp, c.c_float, i32, c.c_int, vp], c.c_int),
        "orca_get_obstacle_neighbors": ([vp, vp, c.c_int, vp], c.c_int),
        "orca_get_op_counters": ([vp, vp, vp], c.c_int),
        "orca_get_search_counters": ([vp, vp, vp], c.c_int),
        "orca_sync": ([vp, vp], c.c_int),
        "orca_profile": ([vp, c.c_int], c.c_int),
        "orca_profile_read": ([vp, vp], c.c_int),
        "orca_launches_per_step": ([vp, c.POINTER(i32)], c.c_int),
        "orca_set_cell_size": ([vp, c.c_float], c.c_int),
        "orca_rollout_workspace_size": ([vp, i32, i32, c.POINTER(sz)], c.c_int),
        "orca_rollout_forward": ([vp, i32, i32, vp, vp, sz, vp], c.c_int),
        "orca_rollout_backward": ([vp, vp, vp, vp, vp, vp, vp, vp, sz, vp], c.c_int),
        "orca_set_launch": ([vp, i32, i32], c.c_int),
        "orca_step_static": ([i32] + [vp] * 7 + [c.c_float, i32, c.c_float, c.c_float, vp, vp, vp],
                             c.c_int),
        "orca_fma_bench": ([i32, i32, vp, c.POINTER(c.c_int64), vp], c.c_int),
        "orca_validate_rollout_fp64": ([i32, i32, c.c_float, c.c_double, i32] + [vp] * 14, c.c_int),
        "orca_num_agents": ([vp, c.POINTER(i32)], c.c_int),
        "orca_last_error": ([vp], c.c_char_p),
        "orca_status_string": ([c.c_int], c.c_char_p),
    }
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    if path is None:
        _lib = lib
    return lib


@contextlib.contextmanager
def use_library(path: str):
    """Route every binding call through another build of the library -- the ORCA_CHECKS
    build, say -- inside the with-block.  Contexts created inside must be closed inside."""
    global _lib
    saved = _lib
    _lib = load_library(path)
    try:
        yield _lib
    finally:
        _lib = saved


def _check(status: int, ctx=None):
    if status != ORCA_OK:
        lib = load_library()
        msg = lib.orca_last_error(ctx).decode() or lib.orca_status_string(status).decode()
        raise OrcaError(status, msg)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(a, dtype):
    """(pointer, where) for a numpy array or a CUDA torch tensor; None -> (None, None)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected C-contiguous {np.dtype(dtype)} array")
        return ctypes.c_void_p(a.ctypes.data), ORCA_HOST
    import torch
    if isinstance(a, torch.Tensor):
        tdt = {np.float32: torch.float32, np.int32: torch.int32, np.uint32: torch.int32}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            raise TypeError(f"expected contiguous {tdt} tensor")
        return ctypes.c_void_p(a.data_ptr()), (ORCA_DEVICE if a.is_cuda else ORCA_HOST)
    raise TypeError(f"unsupported array type {type(a)}")


def make_params(max_agents: int, max_neighbors: int, neighbor_dist: float, dt: float,
                cell_size: float = 0.0, max_cells: int = 0, flags: int = 0,
                max_scenes: int = 0) -> orca_params:
    return orca_params(int(max_agents), int(max_neighbors), int(max_cells), float(neighbor_dist),
                       float(dt), float(cell_size), int(flags), int(max_scenes))


def orca_workspace_size(params: orca_params) -> int:
    n = ctypes.c_size_t(0)
    _check(load_library().orca_workspace_size(ctypes.byref(params), ctypes.byref(n)))
    return int(n.value)


def orca_create(params: orca_params, workspace=None, workspace_bytes: int = 0):
    """workspace: a CUDA torch tensor (caller-owned) or None (library-owned cudaMalloc)."""
    ctx = ctypes.c_void_p()
    wp = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None else None
    nbytes = workspace_bytes or (workspace.numel() * workspace.element_size() if workspace is not None else 0)
    _check(load_library().orca_create(ctypes.byref(params), wp, nbytes, ctypes.byref(ctx)))
    return ctx


def orca_destroy(ctx):
    _check(load_library().orca_destroy(ctx), ctx)


def orca_set_agents(ctx, n, pos_xy, vel_xy, goal_xy, radius, max_speed, pref_speed,
                    time_horizon, where=None, stream=None):
    ptrs = [_ptr(a, np.float32) for a in (pos_xy, vel_xy, goal_xy, radius, max_speed,
                                           pref_speed, time_horizon)]
    w = where if where is not None else ptrs[0][1]
    _check(load_library().orca_set_agents(ctx, int(n), *[p for p, _ in ptrs], int(w),
                                          _stream(stream) if w == ORCA_DEVICE or stream is not None else None),
           ctx)


def orca_update_state(ctx, pos_xy=None, vel_xy=None, where=None, stream=None):
    """New positions and/or velocities for the current agents (agent order); parameters,
    memory order and search-radius predictions are kept."""
    (pp, pw), (vp_, vw) = _ptr(pos_xy, np.float32), _ptr(vel_xy, np.float32)
    w = where if where is not None else (pw if pw is not None else (vw if vw is not None else ORCA_HOST))
    _check(load_library().orca_update_state(ctx, pp, vp_, int(w),
                                            _stream(stream) if w == ORCA_DEVICE or stream is not None else None),
           ctx)


def orca_step_host(ctx, pos_in=None, vel_in=None, nsteps=1, pos_out=None, vel_out=None,
                   stream=None):
    """Write a host state, advance nsteps, read the new state back: one call, one
    synchronisation.  All arrays are host memory (numpy or CPU tensors); None skips one."""
    ptrs = [_ptr(a, np.float32) for a in (pos_in, vel_in, pos_out, vel_out)]
    if any(w == ORCA_DEVICE for _, w in ptrs):
        raise TypeError("orca_step_host takes host arrays")
    _check(load_library().orca_step_host(ctx, ptrs[0][0], ptrs[1][0], int(nsteps), ptrs[2][0],
                                         ptrs[3][0], _stream(stream)), ctx)


def orca_set_scenes(ctx, scenes, pos_xy, vel_xy, goal_xy, radius, max_speed, pref_speed,
                    time_horizon, where=None, stream=None):
    """scenes: sequence of (count, max_neighbors, neighbor_dist, dt, cell_size)."""
    arr = (orca_scene * len(scenes))(*[orca_scene(int(c), int(k), float(nd), float(dt), float(cs), 0)
                                       for c, k, nd, dt, cs in scenes])
    ptrs = [_ptr(a, np.float32) for a in (pos_xy, vel_xy, goal_xy, radius, max_speed,
                                           pref_speed, time_horizon)]
    w = where if where is not None else ptrs[0][1]
    _check(load_library().orca_set_scenes(ctx, len(scenes), ctypes.cast(arr, ctypes.c_void_p),
                                          *[p for p, _ in ptrs], int(w),
                                          _stream(stream) if w == ORCA_DEVICE or stream is not None else None),
           ctx)


def orca_get_scene_grids(ctx, n_scenes: int, stream=None):
    gf = np.zeros(4 * n_scenes, np.float32)
    gi = np.zeros(3 * n_scenes, np.int32)
    _check(load_library().orca_get_scene_grids(ctx, ctypes.c_void_p(gf.ctypes.data),
                                               ctypes.c_void_p(gi.ctypes.data), _stream(stream)), ctx)
    return gf.reshape(n_scenes, 4), gi.reshape(n_scenes, 3)


def orca_step(ctx, nsteps: int = 1, stream=None):
    _check(load_library().orca_step(ctx, int(nsteps), _stream(stream)), ctx)


def orca_get_state(ctx, pos_xy, vel_xy, where=None, stream=None):
    pp, w1 = _ptr(pos_xy, np.float32)
    vp, w2 = _ptr(vel_xy, np.float32)
    w = where if where is not None else (w1 if w1 is not None else w2)
    _check(load_library().orca_get_state(ctx, pp, vp, int(w), _stream(stream)), ctx)


def orca_get_neighbors(ctx, nbr, where=None, stream=None):
    p, w = _ptr(nbr, np.int32)
    _check(load_library().orca_get_neighbors(ctx, p, int(where if where is not None else w),
                                             _stream(stream)), ctx)


def orca_get_cells(ctx, cell, grid_f=None, grid_i=None, where=None, stream=None):
    p, w = _ptr(cell, np.uint32)
    gf = ctypes.c_void_p(grid_f.ctypes.data) if grid_f is not None else None
    gi = ctypes.c_void_p(grid_i.ctypes.data) if grid_i is not None else None
    _check(load_library().orca_get_cells(ctx, p, gf, gi, int(where if where is not None else w),
                                         _stream(stream)), ctx)


def orca_get_counters(ctx, stream=None) -> np.ndarray:
    out = np.zeros(4, np.int64)
    _check(load_library().orca_get_counters(ctx, ctypes.c_void_p(out.ctypes.data),
                                            _stream(stream)), ctx)
    return out


def orca_remove_arrived(ctx, kept_ids=None, stream=None) -> int:
    """Remove the agents at their goal; returns the new count.  kept_ids: None, a host
    int32 array or a device tensor of at least the old count (receives old indices)."""
    m = ctypes.c_int32(0)
    ptr, where = _ptr(kept_ids, np.int32)
    _check(load_library().orca_remove_arrived(ctx, ctypes.byref(m), ptr,
                                              int(ORCA_HOST if where is None else where),
                                              _stream(stream)), ctx)
    return int(m.value)


MAX_OBSTACLE_NEIGHBORS = 4


def orca_set_obstacles(ctx, segments, time_horizon: float = 2.0, max_obstacle_neighbors: int = 4,
                       stream=None):
    """Static obstacle segments (float32[m, 4]: x1, y1, x2, y2; None or empty clears)."""
    if segments is None or len(segments) == 0:
        _check(load_library().orca_set_obstacles(ctx, 0, None, float(time_horizon), 1, ORCA_HOST,
                                                 _stream(stream)), ctx)
        return
    if isinstance(segments, np.ndarray):
        segments = np.ascontiguousarray(segments, np.float32).reshape(-1, 4)
    p, w = _ptr(segments, np.float32)
    m = segments.shape[0]
    _check(load_library().orca_set_obstacles(ctx, int(m), p, float(time_horizon),
                                             int(max_obstacle_neighbors), int(w), _stream(stream)), ctx)


def orca_get_obstacle_neighbors(ctx, out, where=None, stream=None):
    p, w = _ptr(out, np.int32)
    _check(load_library().orca_get_obstacle_neighbors(ctx, p, int(where if where is not None else w),
                                                      _stream(stream)), ctx)


def orca_spawn_agents(ctx, cand_pos, goal_xy, radius, max_speed, pref_speed, time_horizon,
                      window: float, accepted=None, stream=None) -> int:
    """Spawn candidates (arrays of m or 2m float32, host or CUDA) that overlap nobody within
    ``window`` seconds; returns the new agent count; ``accepted`` (int32[m], same memory
    kind) receives 1/0 per candidate."""
    arrays = (cand_pos, goal_xy, radius, max_speed, pref_speed, time_horizon)
    m = int(np.asarray(radius.shape)[0]) if hasattr(radius, "shape") else len(radius)
    ptrs, where = [], None
    for a, k in zip(arrays, (2, 2, 1, 1, 1, 1)):
        p, w = _ptr(a, np.float32)
        if where is not None and w != where:
            raise TypeError("orca_spawn_agents: all arrays host or all device")
        size = a.size if isinstance(a, np.ndarray) else a.numel()
        if size != k * m:
            raise ValueError("orca_spawn_agents: arrays of m or 2m elements")
        where = w
        ptrs.append(p)
    acc = None
    if accepted is not None:
        acc, w = _ptr(accepted, np.int32)
        if w != where:
            raise TypeError("accepted must live where the candidates do")
    n_after = ctypes.c_int32(0)
    _check(load_library().orca_spawn_agents(ctx, m, *ptrs, float(window), where, acc,
                                            ctypes.byref(n_after), _stream(stream)), ctx)
    return int(n_after.value)


def orca_count_ops(ctx, on: bool):
    _check(load_library().orca_count_ops(ctx, int(bool(on))), ctx)


def orca_get_op_counters(ctx, stream=None) -> np.ndarray:
    out = np.zeros(4, np.int64)
    _check(load_library().orca_get_op_counters(ctx, ctypes.c_void_p(out.ctypes.data),
                                               _stream(stream)), ctx)
    return out


def orca_get_search_counters(ctx, stream=None) -> np.ndarray:
    out = np.zeros(4, np.int64)
    _check(load_library().orca_get_search_counters(ctx, ctypes.c_void_p(out.ctypes.data),
                                                   _stream(stream)), ctx)
    return out


def orca_sync(ctx, stream=None):
    _check(load_library().orca_sync(ctx, _stream(stream)), ctx)


def orca_profile(ctx, enable: bool):
    _check(load_library().orca_profile(ctx, int(bool(enable))), ctx)


def orca_profile_read(ctx) -> np.ndarray:
    out = np.zeros(3, np.float32)
    _check(load_library().orca_profile_read(ctx, ctypes.c_void_p(out.ctypes.data)), ctx)
    return out


def orca_rollout_workspace_size(ctx, T: int, ckpt_every: int) -> int:
    n = ctypes.c_size_t(0)
    _check(load_library().orca_rollout_workspace_size(ctx, int(T), int(ckpt_every), ctypes.byref(n)), ctx)
    return int(n.value)


def _dptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def orca_rollout_forward(ctx, T, ckpt_every, traj_pos, workspace, stream=None):
    """traj_pos: CUDA tensor [T, n, 2] or None; workspace: CUDA uint8 tensor (256-B aligned)."""
    _check(load_library().orca_rollout_forward(ctx, int(T), int(ckpt_every), _dptr(traj_pos),
                                               _dptr(workspace), workspace.numel(), _stream(stream)), ctx)


def orca_rollout_backward(ctx, dL_dpos, g_pref_speed, g_radius, g_time_horizon, g_pos0, g_vel0,
                          workspace, stream=None):
    _check(load_library().orca_rollout_backward(ctx, _dptr(dL_dpos), _dptr(g_pref_speed),
                                                _dptr(g_radius), _dptr(g_time_horizon),
                                                _dptr(g_pos0), _dptr(g_vel0), _dptr(workspace),
                                                workspace.numel(), _stream(stream)), ctx)


def orca_set_cell_size(ctx, cell_size: float):
    _check(load_library().orca_set_cell_size(ctx, float(cell_size)), ctx)


def orca_set_launch(ctx, threads_per_block: int = 128, lp3_lanes: int = 0):
    _check(load_library().orca_set_launch(ctx, int(threads_per_block), int(lp3_lanes)), ctx)


def orca_launches_per_step(ctx) -> int:
    n = ctypes.c_int32(0)
    _check(load_library().orca_launches_per_step(ctx, ctypes.byref(n)), ctx)
    return int(n.value)


def orca_step_static(n, pos_xy, vel_xy, goal_xy, radius, max_speed, pref_speed, time_horizon,
                     neighbor_dist, max_neighbors, dt, cell_size, pos_out_xy, vel_out_xy,
                     stream=None):
    """One step with no allocation (library-internal fixed scratch); device tensors only.

    The library launches on the current CUDA device and reads 2n / n floats from each
    input, so every tensor must live on one device, which becomes current for the call,
    and hold at least that many elements; anything else is refused before any launch."""
    import torch
    n = int(n)
    if n < 0:
        raise ValueError("orca_step_static: n < 0")
    arrays = (pos_xy, vel_xy, goal_xy, radius, max_speed, pref_speed, time_horizon, pos_out_xy,
              vel_out_xy)
    per_agent = (2, 2, 2, 1, 1, 1, 1, 2, 2)
    ptrs, devices = [], set()
    for a, m in zip(arrays, per_agent):
        if not isinstance(a, torch.Tensor) or not a.is_cuda:
            raise TypeError("orca_step_static takes CUDA tensors")
        if a.numel() < m * n:
            raise ValueError(f"orca_step_static: a tensor of {a.numel()} elements, "
                             f"{m * n} needed for {n} agents")
        p, _ = _ptr(a, np.float32)
        ptrs.append(p)
        devices.add(a.device)
    if len(devices) != 1:
        raise ValueError("orca_step_static: tensors on more than one device")
    with torch.cuda.device(devices.pop()):
        _check(load_library().orca_step_static(n, *ptrs[:7], float(neighbor_dist),
                                               int(max_neighbors), float(dt), float(cell_size),
                                               ptrs[7], ptrs[8], _stream(stream)))


def orca_fma_bench(blocks: int, iters: int, out, stream=None) -> int:
    """Enqueue the FP32 FMA microbenchmark (``out``: CUDA float32 tensor of >= blocks, or
    of >= 8 x SMs elements when blocks <= 0); returns the FP32 operations enqueued."""
    p, w = _ptr(out, np.float32)
    if w != ORCA_DEVICE:
        raise TypeError("orca_fma_bench takes a CUDA tensor")
    flops = ctypes.c_int64(0)
    _check(load_library().orca_fma_bench(int(blocks), int(iters), p, ctypes.byref(flops),
                                         _stream(stream)))
    return int(flops.value)


def orca_validate_rollout_fp64(pos0, vel0, goal, radius, max_speed, pref_speed, time_horizon,
                               neighbor_dist, max_neighbors, dt, T, dL_dpos=None, stream=None):
    """FP64 rollout of T steps and, with ``dL_dpos`` ([T, n, 2]), the FP64 adjoint (validation
    only).  Takes CUDA float64 tensors in agent order; returns a dict with ``traj`` [T, n, 2]
    and, with dL_dpos, the gradients ``pref``, ``radius``, ``tau`` [n], ``pos0``, ``vel0``
    [n, 2] (CUDA float64 tensors)."""
    import torch
    arrays = [pos0, vel0, goal, radius, max_speed, pref_speed, time_horizon]
    n = int(radius.numel())
    dev = pos0.device
    for a, m in zip(arrays, (2, 2, 2, 1, 1, 1, 1)):
        if not isinstance(a, torch.Tensor) or not a.is_cuda or a.dtype != torch.float64 \
                or not a.is_contiguous() or a.numel() != m * n or a.device != dev:
            raise TypeError("orca_validate_rollout_fp64 takes contiguous CUDA float64 tensors "
                            "of n or 2n elements on one device")
    T = int(T)
    traj = torch.empty((T, n, 2), dtype=torch.float64, device=dev)
    out = {"traj": traj}
    gp = []
    if dL_dpos is not None:
        if dL_dpos.dtype != torch.float64 or dL_dpos.numel() != T * n * 2 or dL_dpos.device != dev:
            raise TypeError("dL_dpos: CUDA float64 [T, n, 2]")
        dL_dpos = dL_dpos.contiguous()
        out.update(pref=torch.empty(n, dtype=torch.float64, device=dev),
                   radius=torch.empty(n, dtype=torch.float64, device=dev),
                   tau=torch.empty(n, dtype=torch.float64, device=dev),
                   pos0=torch.empty((n, 2), dtype=torch.float64, device=dev),
                   vel0=torch.empty((n, 2), dtype=torch.float64, device=dev))
        gp = [out[k] for k in ("pref", "radius", "tau", "pos0", "vel0")]
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    with torch.cuda.device(dev):
        _check(load_library().orca_validate_rollout_fp64(
            n, int(max_neighbors), float(neighbor_dist), float(dt), T, *[ptr(a) for a in arrays],
            ptr(dL_dpos), ptr(traj), *(ptr(g) for g in gp) if gp else (None,) * 5,
            _stream(stream)))
    return out


def orca_num_agents(ctx) -> int:
    n = ctypes.c_int32(0)
    _check(load_library().orca_num_agents(ctx, ctypes.byref(n)), ctx)
    return int(n.value)


def orca_last_error(ctx) -> str:
    return load_library().orca_last_error(ctx).decode()


def orca_status_string(status: int) -> str:
    return load_library().orca_status_string(int(status)).decode()


class OrcaSim:
    """A context plus its torch-owned device workspace.

    >>> sim = OrcaSim(max_agents=n, max_neighbors=10, neighbor_dist=10.0, dt=1/60)
    >>> sim.set_scene(scene); sim.step(100); pos, vel = sim.get_state()
    """

    def __init__(self, max_agents: int, max_neighbors: int, neighbor_dist: float, dt: float,
                 cell_size: float = 0.0, max_cells: int = 0, flags: int = 0, device=None,
                 max_scenes: int = 0):
        import torch
        self.params = make_params(max_agents, max_neighbors, neighbor_dist, dt, cell_size,
                                  max_cells, flags, max_scenes)
        self.n_scenes = 0
        self.device = torch.device(device or "cuda")
        nbytes = orca_workspace_size(self.params)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            off = (-self.workspace.data_ptr()) % 256
            self._ws = self.workspace[off: off + nbytes]
            self.ctx = orca_create(self.params, self._ws, nbytes)
        self.k = int(max_neighbors)

    @classmethod
    def for_batch(cls, batch, **kw):
        return cls(max_agents=max(batch.n, 1), max_neighbors=batch.max_neighbors,
                   neighbor_dist=batch.scenes[0].neighbor_dist, dt=batch.scenes[0].dt,
                   max_scenes=len(batch.scenes), **kw)

    @classmethod
    def for_scene(cls, scene, **kw):
        return cls(max_agents=max(scene.n, 1), max_neighbors=scene.max_neighbors,
                   neighbor_dist=scene.neighbor_dist, dt=scene.dt, **kw)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            orca_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n(self) -> int:
        return orca_num_agents(self.ctx)

    def set_agents(self, pos, vel, goal, radius, max_speed, pref_speed, time_horizon, stream=None):
        n = (pos.shape[0] if pos.ndim == 2 else pos.shape[0] // 2)
        orca_set_agents(self.ctx, n, pos, vel, goal, radius, max_speed, pref_speed,
                        time_horizon, stream=stream)

    def set_scene(self, scene, stream=None):
        """Load a ``scenarios.Scene``: its agents and its static obstacles (none clears them)."""
        obs = getattr(scene, "obstacles", None)
        if obs is not None or getattr(self, "_has_obstacles", False):
            orca_set_obstacles(self.ctx, obs, getattr(scene, "obstacle_time_horizon", 2.0),
                               getattr(scene, "max_obstacle_neighbors", 4), stream)
            self._has_obstacles = obs is not None and len(obs) > 0
        self.set_agents(*scene.arrays(), stream=stream)

    def get_obstacle_neighbors(self, stream=None) -> np.ndarray:
        out = np.empty((self.n, MAX_OBSTACLE_NEIGHBORS), np.int32)
        orca_get_obstacle_neighbors(self.ctx, out, stream=stream)
        return out

    def set_batch(self, batch, cell_size: float = 0.0, stream=None):
        """Load a ``scenarios.Batch`` (needs max_scenes >= its scene count)."""
        self.n_scenes = len(batch.scenes)
        orca_set_scenes(self.ctx, batch.scene_params(cell_size), *batch.arrays(), stream=stream)

    def get_scene_grids(self, stream=None):
        return orca_get_scene_grids(self.ctx, self.n_scenes, stream)

    def update_state(self, pos=None, vel=None, stream=None):
        """Replace positions and/or velocities; parameters and predictions are kept."""
        orca_update_state(self.ctx, pos, vel, stream=stream)

    def step_host(self, pos_in=None, vel_in=None, nsteps: int = 1, pos_out=None, vel_out=None,
                  stream=None):
        """Host state in, nsteps, host state out (one synchronisation)."""
        orca_step_host(self.ctx, pos_in, vel_in, nsteps, pos_out, vel_out, stream=stream)

    def step(self, nsteps: int = 1, stream=None):
        orca_step(self.ctx, nsteps, stream)

    def get_state(self, device: bool = False, stream=None):
        n = self.n
        if device:
            import torch
            pos = torch.empty((n, 2), dtype=torch.float32, device=self.device)
            vel = torch.empty((n, 2), dtype=torch.float32, device=self.device)
        else:
            pos = np.empty((n, 2), np.float32)
            vel = np.empty((n, 2), np.float32)
        orca_get_state(self.ctx, pos, vel, stream=stream)
        return pos, vel

    def get_neighbors(self, stream=None) -> np.ndarray:
        out = np.empty((self.n, self.k), np.int32)
        orca_get_neighbors(self.ctx, out, stream=stream)
        return out

    def get_cells(self, stream=None):
        cell = np.empty(self.n, np.uint32)
        gf = np.zeros(4, np.float32)
        gi = np.zeros(2, np.int32)
        orca_get_cells(self.ctx, cell, gf, gi, stream=stream)
        return cell, gf, gi

    def counters(self, stream=None) -> dict:
        c = orca_get_counters(self.ctx, stream)
        return dict(zip(("agent_steps", "lp3_agent_steps", "candidates", "lines"), map(int, c)))

    def remove_arrived(self, stream=None):
        """Remove the agents that have reached their goal; returns (count, kept old
        indices as int32[count])."""
        kept = np.zeros(max(self.n, 1), np.int32)
        m = orca_remove_arrived(self.ctx, kept, stream)
        return m, kept[:m].copy()

    def search_counters(self, stream=None) -> dict:
        c = orca_get_search_counters(self.ctx, stream)
        return dict(zip(("extra_passes", "unpredicted", "rows", "lp3_problem_lines"), map(int, c)))

    def spawn(self, cand_pos, goal, radius, max_speed, pref_speed, time_horizon, window, stream=None):
        """Spawn the candidates that overlap nobody within ``window`` s; returns accepted
        flags (bool[m]).  The entrants get agent indices n, n+1, ... in candidate order."""
        f = lambda a: np.ascontiguousarray(np.asarray(a, np.float32))  # noqa: E731
        acc = np.zeros(max(len(radius), 1), np.int32)
        orca_spawn_agents(self.ctx, f(cand_pos).reshape(-1, 2), f(goal).reshape(-1, 2), f(radius),
                          f(max_speed), f(pref_speed), f(time_horizon), window, acc[:len(radius)], stream)
        return acc[:len(radius)].astype(bool)

    def op_counters(self, stream=None) -> dict:
        c = orca_get_op_counters(self.ctx, stream)
        return dict(zip(("lp1_calls", "lp1_bounds", "lp_checks", "bisectors"), map(int, c)))

    def sync(self, stream=None):
        orca_sync(self.ctx, stream)
