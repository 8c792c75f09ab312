"""FP64 CPU oracle for one ORCA step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The GPU library never imports, links or calls it.

The arithmetic lives in ``orca_oracle.c`` (plain C, FP64, neighbour decisions in FP32);
this module compiles it with gcc and marshals numpy arrays through ctypes.  Every
function cites the passage of "Fast Simulation of Crowd Collision Avoidance" (or of the
ORCA method it defers to) that it follows; see the C file's header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orca_oracle.c")
_LIB = os.path.join(_HERE, "liborca_oracle.so")
_lock = threading.Lock()
_lib = None

_F32P = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_F64P = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_U32P = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_I64P = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def compile_source(src: str, out: str) -> str:
    """gcc -O2, FP contraction off (FP32 decisions must round once per operation)."""
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", src, "-o", out + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(out + ".tmp", out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available).  Returns the library path."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        return compile_source(_SRC, _LIB)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def _bind(lib):
    c = ctypes
    lib.oracle_grid.argtypes = [_F32P, c.c_int, c.c_float, c.c_longlong, _F32P, _I32P]
    lib.oracle_grid.restype = c.c_int
    lib.oracle_cells.argtypes = [_F32P, c.c_int, _F32P, _I32P, _U32P]
    lib.oracle_cells.restype = None
    lib.oracle_knn.argtypes = [_F32P, c.c_int, c.c_float, c.c_int, c.c_int, c.c_void_p,
                               c.c_void_p, _I32P, _F32P]
    lib.oracle_knn.restype = c.c_longlong
    lib.oracle_orca_line.argtypes = [_F64P, _F64P, c.c_double, c.c_double, c.c_int, c.c_int,
                                     _F64P, _F64P, _F64P]
    lib.oracle_orca_line.restype = c.c_int
    lib.oracle_lp2.argtypes = [_F64P, c.c_int, c.c_double, _F64P, c.c_int, _F64P]
    lib.oracle_lp2.restype = c.c_int
    lib.oracle_solve.argtypes = [_F64P, c.c_int, c.c_double, _F64P, _F64P]
    lib.oracle_solve.restype = c.c_int
    lib.oracle_solve_counted.argtypes = [_F64P, c.c_int, c.c_double, _F64P, _F64P,
                                         np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")]
    lib.oracle_solve_counted.restype = c.c_int
    lib.oracle_step.argtypes = ([c.c_int] + [_F64P] * 7 + [c.c_double, c.c_int, c.c_double,
                                c.c_int, c.c_int, c.c_void_p, c.c_void_p, c.c_void_p, c.c_int,
                                c.c_int, _F64P, _F64P, c.c_void_p, c.c_void_p, c.c_void_p,
                                c.c_void_p, c.c_int, c.c_void_p])
    lib.oracle_step.restype = c.c_int
    lib.oracle_step_obstacles.argtypes = lib.oracle_step.argtypes + [c.c_int, c.c_void_p, c.c_double,
                                                                     c.c_int, c.c_void_p]
    lib.oracle_step_obstacles.restype = c.c_int
    lib.oracle_lp_sensitivity.argtypes = [_F64P, c.c_int, c.c_int, c.c_double, _F64P, _F64P]
    lib.oracle_lp_sensitivity.restype = c.c_double
    lib.oracle_solve_fixed.argtypes = [_F64P, c.c_int, c.c_int, c.c_double, _F64P, _F64P]
    lib.oracle_solve_fixed.restype = c.c_int
    lib.oracle_obstacle_line.argtypes = [_F64P, c.c_double, _F64P, c.c_double, c.c_double, _F64P]
    lib.oracle_obstacle_line.restype = c.c_int
    lib.oracle_arrived.argtypes = [c.c_int, _F32P, _F32P, _F32P, _I32P]
    lib.oracle_spawn.argtypes = [c.c_int, _F32P, _F32P, _F32P, c.c_int, _F32P, _F32P, _F32P,
                                 c.c_float, _I32P]
    lib.oracle_spawn.restype = c.c_int
    lib.oracle_arrived.restype = c.c_int
    lib.oracle_max_threads.argtypes = []
    lib.oracle_max_threads.restype = c.c_int
    return lib


class use_library:
    """Context manager: route this module's calls to another build of the oracle source
    (the mutation tests compile deliberately broken copies and check that the pins fail)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self._saved = _load()
        _lib = None
        _lib = _bind(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def grid(pos, cell_size: float, max_cells: int):
    """Spatial bins of Fig. 2 (FP32): returns (grid_f=[xmin, ymin, s, 1/s], grid_i=[gx, gy])."""
    pos = np.ascontiguousarray(pos, dtype=np.float32).reshape(-1)
    gf = np.zeros(4, np.float32)
    gi = np.zeros(2, np.int32)
    r = _load().oracle_grid(pos, pos.size // 2, float(cell_size), int(max_cells), gf, gi)
    if r != 0:
        raise ValueError(f"oracle_grid failed ({r})")
    return gf, gi


def cells(pos, gf, gi) -> np.ndarray:
    pos = np.ascontiguousarray(pos, dtype=np.float32).reshape(-1)
    out = np.zeros(pos.size // 2, np.uint32)
    _load().oracle_cells(pos, pos.size // 2, np.ascontiguousarray(gf, np.float32),
                         np.ascontiguousarray(gi, np.int32), out)
    return out


def knn(pos, neighbor_dist: float, k: int, mode: int = 0, gf=None, gi=None):
    """Neighbour sets (Fig. 2 filter + k nearest by (d^2, index)), FP32 decisions.

    Returns (nbr int32[n, k] padded with -1, d2 float32[n, k], candidates scanned)."""
    pos = np.ascontiguousarray(pos, dtype=np.float32).reshape(-1)
    n = pos.size // 2
    nbr = np.zeros(n * k, np.int32)
    d2 = np.zeros(n * k, np.float32)
    if mode == 1:
        gf = np.ascontiguousarray(gf, np.float32)
        gi = np.ascontiguousarray(gi, np.int32)
    scanned = _load().oracle_knn(pos, n, float(neighbor_dist), int(k), int(mode), _ptr(gf),
                                 _ptr(gi), nbr, d2)
    if scanned < 0:
        raise ValueError("oracle_knn failed")
    return nbr.reshape(n, k), d2.reshape(n, k), int(scanned)


def orca_line(a, b, tau: float, dt: float, ia: int = 0, ib: int = 1):
    """Half-plane ORCA_{a|b} (Fig. 1).  a, b = (px, py, vx, vy, r).

    Returns (line [Px, Py, dx, dy], u [ux, uy], branch, margin); branch 0 cutoff circle,
    1 left leg, 2 right leg, 3 overlapping agents."""
    line = np.zeros(4)
    u = np.zeros(2)
    m = np.zeros(1)
    br = _load().oracle_orca_line(np.asarray(a, np.float64), np.asarray(b, np.float64),
                                  float(tau), float(dt), int(ia), int(ib), line, u, m)
    return line, u, int(br), float(m[0])


def lp2(lines, V: float, o, dir_opt: bool = False):
    """Incremental 2-D LP (Section 3).  Returns (index of failing line or n, x)."""
    lines = np.ascontiguousarray(lines, np.float64).reshape(-1)
    x = np.zeros(2)
    r = _load().oracle_lp2(lines, lines.size // 4, float(V), np.asarray(o, np.float64),
                           int(bool(dir_opt)), x)
    return int(r), x


def solve(lines, V: float, o):
    """LP2 then, if infeasible, the least-penetration LP3.  Returns (lp3_used, x)."""
    lines = np.ascontiguousarray(lines, np.float64).reshape(-1)
    x = np.zeros(2)
    r = _load().oracle_solve(lines, lines.size // 4, float(V), np.asarray(o, np.float64), x)
    return bool(r), x


def solve_counted(lines, V: float, o):
    """As solve, also returning the LP's operation counts as a dict (lp1_calls,
    lp1_bounds, lp_checks, bisectors, lp3_problem_lines)."""
    lines = np.ascontiguousarray(lines, np.float64).reshape(-1)
    x = np.zeros(2)
    counts = np.zeros(5, np.int64)
    r = _load().oracle_solve_counted(lines, lines.size // 4, float(V), np.asarray(o, np.float64),
                                     x, counts)
    if r < 0:
        raise ValueError("oracle_solve_counted: bad arguments")
    names = ("lp1_calls", "lp1_bounds", "lp_checks", "bisectors", "lp3_problem_lines")
    return bool(r), x, dict(zip(names, (int(c) for c in counts)))


def lp_sensitivity(lines, V: float, o, nobst: int = 0):
    """Conditioning of the velocity selection (LP2, then LP3) for FP32 parity: the largest
    move of the selected velocity (max-norm) when one half-plane at a time is shifted
    along its normal by +-4 FP32 ulps of max(|offset|, V) or turned by +-2^-22 rad.
    Returns (sens, x) with x the unperturbed selection."""
    lines = np.ascontiguousarray(lines, np.float64).reshape(-1)
    x = np.zeros(2)
    s = _load().oracle_lp_sensitivity(lines, lines.size // 4, int(nobst), float(V),
                                      np.asarray(o, np.float64), x)
    if s < 0:
        raise ValueError("oracle_lp_sensitivity: bad arguments")
    return float(s), x


def step(pos, vel, goal, radius, max_speed, pref_speed, time_horizon, neighbor_dist: float,
         max_neighbors: int, dt: float, knn_mode: int = 1, fp64_knn: bool = False,
         gf=None, gi=None, nthreads: int | None = None, subset=None,
         sensitivity: bool = False, obstacles=None, obstacle_time_horizon: float = 2.0,
         max_obstacle_neighbors: int = 4):
    """One synchronous ORCA step (Sections 2-3) in FP64.

    ``obstacles``: optional static segments, float[m, 4] (x1, y1, x2, y2); each agent
    takes the ``max_obstacle_neighbors`` nearest reachable ones as hard half-planes (see
    the C source) and the result gains ``obst`` (int32[rows, max_obstacle_neighbors]).

    Arrays are promoted to float64.  With ``subset`` (agent indices) only those agents are
    stepped -- their neighbours are still searched among all agents -- and output row q
    belongs to agent subset[q].  Returns a dict with pos, vel (float64[rows, 2]), nbr
    (int32[rows, k]), lp3 (bool[rows]), margin (float64[rows]), sens (float64[rows], the
    LP's sensitivity to FP32-sized perturbations of its half-planes, when
    ``sensitivity``) and operation counters (COUNTER_NAMES)."""
    d = lambda a: np.ascontiguousarray(np.asarray(a, np.float64).reshape(-1))
    pos, vel, goal = d(pos), d(vel), d(goal)
    radius, max_speed, pref_speed, time_horizon = d(radius), d(max_speed), d(pref_speed), d(time_horizon)
    n = pos.size // 2
    k = int(max_neighbors)
    if subset is not None:
        subset = np.ascontiguousarray(subset, np.int32)
        rows = subset.size
    else:
        rows = n
    pos_out = np.zeros(max(2 * rows, 2))
    vel_out = np.zeros(max(2 * rows, 2))
    nbr = np.zeros(max(rows * k, 1), np.int32)
    status = np.zeros(max(rows, 1), np.int32)
    margin = np.zeros(max(rows, 1))
    counters = np.zeros(8, np.int64)
    sens = np.zeros(max(rows, 1))
    if gf is not None:
        gf = np.ascontiguousarray(gf, np.float32)
        gi = np.ascontiguousarray(gi, np.int32)
    common = (n, pos, vel, goal, radius, max_speed, pref_speed, time_horizon,
              float(neighbor_dist), k, float(dt), int(knn_mode), int(bool(fp64_knn)),
              _ptr(gf), _ptr(gi), _ptr(subset), int(rows), int(nthreads or max_threads()),
              pos_out, vel_out, _ptr(nbr), _ptr(status), _ptr(margin), _ptr(counters),
              int(bool(sensitivity)), _ptr(sens))
    obst = None
    if obstacles is None:
        r = _load().oracle_step(*common)
    else:
        seg = np.ascontiguousarray(np.asarray(obstacles, np.float64).reshape(-1))
        ko = int(max_obstacle_neighbors)
        obst = np.full(max(rows * max(ko, 1), 1), -1, np.int32)
        r = _load().oracle_step_obstacles(*common, seg.size // 4, _ptr(seg),
                                          float(obstacle_time_horizon), ko, _ptr(obst))
    if r != 0:
        raise ValueError(f"oracle_step failed ({r})")
    out = {
        "pos": pos_out[: 2 * rows].reshape(rows, 2), "vel": vel_out[: 2 * rows].reshape(rows, 2),
        "nbr": nbr[: rows * k].reshape(rows, k), "lp3": status[:rows].astype(bool),
        "margin": margin[:rows], "sens": sens[:rows],
        "counters": dict(zip(COUNTER_NAMES, (int(c) for c in counters))),
    }
    if obst is not None:
        ko = max(int(max_obstacle_neighbors), 1)
        out["obst"] = obst[: rows * ko].reshape(rows, ko)
    return out


# operation counts of oracle_step, summed over the stepped agents: candidates scanned,
# half-planes built, LP1 calls (LP2 and inside LP3), agents that needed LP3, LP1 bounds
# evaluated, LP2/LP3 violation checks, LP3 bisectors formed, and the lines of LP3's
# projected problems (a problem for line i, 0-based, takes that line and the i before it)
COUNTER_NAMES = ("scanned", "lines", "lp1_calls", "lp3_agents", "lp1_bounds", "lp_checks",
                 "bisectors", "lp3_problem_lines")


def obstacle_line(p, r, seg, time_horizon: float, dt: float):
    """Obstacle half-plane of an agent at p with radius r against segment seg (x1, y1,
    x2, y2): ((Px, Py, dx, dy), overlapping)."""
    line4 = np.zeros(4)
    ov = _load().oracle_obstacle_line(np.asarray(p, np.float64), float(r),
                                      np.asarray(seg, np.float64), float(time_horizon), float(dt), line4)
    return line4, bool(ov)


def solve_fixed(lines, nobst: int, V: float, o):
    """LP2 then LP3 with the first nobst lines hard (static obstacles); lines: [n, 4]."""
    lines = np.ascontiguousarray(np.asarray(lines, np.float64).reshape(-1))
    x = np.zeros(2)
    r = _load().oracle_solve_fixed(lines, lines.size // 4, int(nobst), float(V),
                                   np.asarray(o, np.float64), x)
    if r < 0:
        raise ValueError("oracle_solve_fixed failed")
    return x, bool(r)


def arrived(pos, goal, radius) -> np.ndarray:
    """Which agents have reached their goal (Section 4: they leave the simulation):
    |goal - p| <= radius, decided in FP32 (bool[n])."""
    pos = np.ascontiguousarray(np.asarray(pos, np.float32).reshape(-1))
    goal = np.ascontiguousarray(np.asarray(goal, np.float32).reshape(-1))
    radius = np.ascontiguousarray(np.asarray(radius, np.float32).reshape(-1))
    n = radius.size
    out = np.zeros(max(n, 1), np.int32)
    _load().oracle_arrived(n, pos, goal, radius, out)
    return out[:n].astype(bool)


def spawn(pos, vel, radius, cand_pos, cand_radius, cand_vmax, window: float) -> np.ndarray:
    """Which candidates may enter (Section 4: spawned without overlap within a time window
    set by size and speed): a candidate at rest conflicts with a present agent j when
    |p_c - p_j| <= r_c + r_j + (V_c + |v_j|) T, and with an earlier accepted candidate c'
    when |p_c - p_c'| <= r_c + r_c' + (V_c + V_c') T; decided in FP32 (bool[m])."""
    f = lambda a: np.ascontiguousarray(np.asarray(a, np.float32).reshape(-1))  # noqa: E731
    pos, vel, radius = f(pos), f(vel), f(radius)
    cand_pos, cand_radius, cand_vmax = f(cand_pos), f(cand_radius), f(cand_vmax)
    n, m = radius.size, cand_radius.size
    out = np.zeros(max(m, 1), np.int32)
    _load().oracle_spawn(n, pos if n else np.zeros(2, np.float32), vel if n else np.zeros(2, np.float32),
                         radius if n else np.zeros(1, np.float32), m,
                         cand_pos if m else np.zeros(2, np.float32),
                         cand_radius if m else np.zeros(1, np.float32),
                         cand_vmax if m else np.zeros(1, np.float32), float(np.float32(window)), out)
    return out[:m].astype(bool)


def remove_arrived(scene):
    """The scene without the agents that have arrived, and the kept agents' indices."""
    keep = np.flatnonzero(~arrived(scene.pos, scene.goal, scene.radius))
    out = scene.copy()
    for name in ("pos", "vel", "goal", "radius", "max_speed", "pref_speed", "time_horizon"):
        setattr(out, name, np.ascontiguousarray(getattr(scene, name)[keep]))
    return out, keep


def step_scene(scene, **kw):
    """oracle step on a ``scenarios.Scene``'s current state."""
    obs = getattr(scene, "obstacles", None)
    if obs is not None and "obstacles" not in kw:
        kw = dict(kw, obstacles=obs, obstacle_time_horizon=scene.obstacle_time_horizon,
                  max_obstacle_neighbors=scene.max_obstacle_neighbors)
    return step(scene.pos, scene.vel, scene.goal, scene.radius, scene.max_speed,
                scene.pref_speed, scene.time_horizon, scene.neighbor_dist,
                scene.max_neighbors, scene.dt, **kw)
