"""Seeded synthetic crowd generators.

This module only draws initial agent states and per-agent parameters; it holds none
of the ORCA step's arithmetic (no preferred velocity, no cells, no half-planes, no
LP).  The GPU path, the CPU oracle, the tests and the benchmark all start from the
arrays produced here, so both sides of every parity check consume identical FP32
values.

The workloads stand in for the paper's test cases (Section 4): the two-way crossing
(two crowds in opposite bands, each heading for the far side) and the N-way
crossing, whose limit is the circle swap (every agent heads for its antipode).
The paper uses no public dataset; all inputs here are synthetic.

Every array is float32, length ``n`` (or ``2n`` for interleaved x/y pairs).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Scene:
    """One crowd: FP32 agent state plus the scene-wide ORCA parameters.

    pos, vel, goal: float32[n, 2] (x, y interleaved in memory).
    radius, max_speed, pref_speed, time_horizon: float32[n].
    neighbor_dist (r_obs of Fig. 2), max_neighbors, dt: scene-wide.
    """

    name: str
    pos: np.ndarray
    vel: np.ndarray
    goal: np.ndarray
    radius: np.ndarray
    max_speed: np.ndarray
    pref_speed: np.ndarray
    time_horizon: np.ndarray
    neighbor_dist: float
    max_neighbors: int
    dt: float
    steps: int
    # static obstacles (optional): float32[m, 4] segments (x1, y1, x2, y2), their time
    # horizon, and the obstacle half-planes kept per agent
    obstacles: np.ndarray | None = None
    obstacle_time_horizon: float = 2.0
    max_obstacle_neighbors: int = 4

    def __post_init__(self):
        # scene parameters are FP32 values, the precision the GPU receives them in, so
        # that both sides of a parity check start from identical numbers
        self.neighbor_dist = float(np.float32(self.neighbor_dist))
        self.dt = float(np.float32(self.dt))
        self.obstacle_time_horizon = float(np.float32(self.obstacle_time_horizon))
        if self.obstacles is not None:
            self.obstacles = _f32(np.asarray(self.obstacles).reshape(-1, 4))

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def arrays(self):
        return (self.pos, self.vel, self.goal, self.radius, self.max_speed,
                self.pref_speed, self.time_horizon)

    def copy(self) -> "Scene":
        return dataclasses.replace(self, **{f: getattr(self, f).copy() for f in
                                            ("pos", "vel", "goal", "radius", "max_speed",
                                             "pref_speed", "time_horizon")})


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _full(n, v) -> np.ndarray:
    return np.full(n, v, dtype=np.float32)


def circle_swap(n: int = 1024, circle_radius: float = 100.0, agent_radius: float = 0.5,
                max_speed: float = 2.0, neighbor_dist: float = 15.0, max_neighbors: int = 10,
                time_horizon: float = 10.0, dt: float = 0.25, steps: int = 100) -> Scene:
    """Agents evenly spaced on a circle, each heading for the antipodal point.

    Agent i sits at angle 2*pi*i/n; its goal is the point opposite.  With 1,024 agents
    on a 100 m circle the arc spacing (0.614 m) is below the radius sum (1.0 m), so
    neighbours start in contact.  Initial velocity is zero; preferred speed equals the
    maximum speed.
    """
    ang = 2.0 * np.pi * np.arange(n, dtype=np.float64) / max(n, 1)
    pos = np.stack([circle_radius * np.cos(ang), circle_radius * np.sin(ang)], axis=1)
    pos = _f32(pos)
    return Scene("circle_swap", pos, np.zeros_like(pos), _f32(-pos), _full(n, agent_radius),
                 _full(n, max_speed), _full(n, max_speed), _full(n, time_horizon),
                 neighbor_dist, max_neighbors, dt, steps)


def bidirectional(n: int = 524288, seed: int = 1909, side: float | None = None,
                  neighbor_dist: float = 10.0, max_neighbors: int = 10,
                  time_horizon: float = 5.0, dt: float = 1.0 / 60.0, steps: int = 600,
                  radius_range=(0.3, 0.5), speed_range=(1.2, 1.6)) -> Scene:
    """Two-way crossing: two equal crowds in opposite bands of an open square.

    Half the agents are uniform in the left quarter-width band, half in the right one;
    each agent's goal is the same point shifted by three quarters of the side towards
    the far side.  At 524,288 agents the square is 1 km (density ~1.05 agents/m^2 in
    the bands).  For other counts the side scales with sqrt(n) so the density stays
    the same.  radius ~ U[0.3, 0.5] m, max speed = preferred speed ~ U[1.2, 1.6] m/s.
    Initial velocity is zero.
    """
    rng = np.random.default_rng(seed)
    if side is None:
        side = 1000.0 * math.sqrt(n / 524288.0)
    band = 0.25 * side
    h = n // 2
    x = np.empty(n)
    x[:h] = rng.uniform(0.0, band, h)
    x[h:] = rng.uniform(side - band, side, n - h)
    y = rng.uniform(0.0, side, n)
    gx = np.where(np.arange(n) < h, x + 0.75 * side, x - 0.75 * side)
    pos = _f32(np.stack([x, y], axis=1))
    goal = _f32(np.stack([gx, y], axis=1))
    radius = _f32(rng.uniform(radius_range[0], radius_range[1], n))
    speed = _f32(rng.uniform(speed_range[0], speed_range[1], n))
    return Scene("bidirectional", pos, np.zeros_like(pos), goal, radius, speed, speed.copy(),
                 _full(n, time_horizon), neighbor_dist, max_neighbors, dt, steps)


def dense(n: int = 2097152, seed: int = 1910, side: float | None = None,
          neighbor_dist: float = 8.0, max_neighbors: int = 20, time_horizon: float = 4.0,
          dt: float = 1.0 / 60.0, steps: int = 300, agent_radius: float = 0.4,
          max_speed: float = 1.5) -> Scene:
    """Dense stress: agents and goals uniform in a square (2 km at 2,097,152 agents).

    For other counts the side scales with sqrt(n) (density ~0.52 agents/m^2).
    """
    rng = np.random.default_rng(seed)
    if side is None:
        side = 2000.0 * math.sqrt(n / 2097152.0)
    pos = _f32(rng.uniform(0.0, side, (n, 2)))
    goal = _f32(rng.uniform(0.0, side, (n, 2)))
    return Scene("dense", pos, np.zeros_like(pos), goal, _full(n, agent_radius),
                 _full(n, max_speed), _full(n, max_speed), _full(n, time_horizon),
                 neighbor_dist, max_neighbors, dt, steps)


def jitter_velocities(scene: Scene, seed: int, scale: float = 1.0) -> Scene:
    """Return a copy whose velocities are random (|v| <= scale * max_speed).

    Used by parity tests so that every half-plane branch (cutoff, both legs,
    collision) occurs from the first step.
    """
    rng = np.random.default_rng(seed)
    s = scene.copy()
    ang = rng.uniform(0.0, 2.0 * np.pi, s.n)
    mag = rng.uniform(0.0, scale, s.n) * s.max_speed.astype(np.float64)
    s.vel = _f32(np.stack([mag * np.cos(ang), mag * np.sin(ang)], axis=1))
    return s


def scene_by_name(name: str, n: int | None = None, seed: int | None = None) -> Scene:
    """The three single-scene workloads by name, optionally rescaled to ``n`` agents."""
    if name == "circle_swap":
        return circle_swap(n or 1024)
    if name == "bidirectional":
        return bidirectional(n or 524288, seed=1909 if seed is None else seed)
    if name == "dense":
        return dense(n or 2097152, seed=1910 if seed is None else seed)
    raise ValueError(f"unknown scene {name!r}")


@dataclasses.dataclass
class Batch:
    """Independent scenes advanced together.  Agent arrays are the scenes' arrays
    concatenated scene after scene; ``offsets[s]:offsets[s+1]`` are scene s's agents."""

    scenes: list

    @property
    def n(self) -> int:
        return int(sum(s.n for s in self.scenes))

    @property
    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum([s.n for s in self.scenes])]).astype(np.int64)

    def arrays(self):
        cols = list(zip(*[s.arrays() for s in self.scenes]))
        return tuple(np.ascontiguousarray(np.concatenate(c, axis=0)) for c in cols)

    def scene_params(self, cell_size: float = 0.0):
        """(count, max_neighbors, neighbor_dist, dt, cell_size) per scene."""
        return [(s.n, s.max_neighbors, s.neighbor_dist, s.dt, cell_size) for s in self.scenes]

    @property
    def max_neighbors(self) -> int:
        return max(s.max_neighbors for s in self.scenes)


def batched(n_scenes: int = 256, seed: int = 1912, lo: int = 500, hi: int = 50000) -> Batch:
    """Scenes of uneven size: counts round(exp(U[ln lo, ln hi])); each scene is, with equal
    probability, a circle swap (the 1,024-agent circle's parameters, radius scaled so the
    spacing on the circle is unchanged) or a bidirectional flow (the 524,288-agent flow's
    parameters, side scaled with sqrt(count)).  Scene s's flow uses seed + s."""
    rng = np.random.default_rng(seed)
    counts = np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), n_scenes))).astype(int)
    kinds = rng.integers(0, 2, n_scenes)
    scenes = []
    for s, (c, kind) in enumerate(zip(counts, kinds)):
        if kind == 0:
            scenes.append(circle_swap(int(c), circle_radius=100.0 * c / 1024.0))
        else:
            scenes.append(bidirectional(int(c), seed=seed + 1 + s))
    return Batch(scenes)


def differentiable(n: int = 16384, seed: int = 1913, dt: float = 0.1, steps: int = 64) -> Scene:
    """Bidirectional flow for differentiable rollouts: the 524,288-agent flow's parameters
    (r_obs 10 m, k 10, tau 5 s, radius U[0.3, 0.5] m, speed U[1.2, 1.6] m/s) at ``n`` agents
    with dt = 0.1 s, 64 steps.  The preferred speed is 90% of the maximum so that the
    preferred velocity lies inside the speed disc."""
    sc = bidirectional(n, seed=seed, dt=dt, steps=steps)
    sc.pref_speed = _f32(sc.max_speed * np.float32(0.9))
    return sc


def perturbed_parameters(scene: Scene, seed: int):
    """Target parameters: preferred speed x U[0.9, 1.1], radius x U[0.9, 1.1], time horizon
    x U[0.8, 1.2], per agent.  Returns (pref_speed, radius, time_horizon), float32."""
    rng = np.random.default_rng(seed)
    n = scene.n
    return (_f32(scene.pref_speed * rng.uniform(0.9, 1.1, n)),
            _f32(scene.radius * rng.uniform(0.9, 1.1, n)),
            _f32(scene.time_horizon * rng.uniform(0.8, 1.2, n)))


def patch(scene: Scene, m: int, seed: int = 0) -> Scene:
    """The m agents nearest a random agent of ``scene``, as a scene of their own."""
    rng = np.random.default_rng(seed)
    c = scene.pos[rng.integers(scene.n)].astype(np.float64)
    idx = np.sort(np.argsort(((scene.pos - c) ** 2).sum(1))[:m])
    s = scene.copy()
    for f in ("pos", "vel", "goal", "radius", "max_speed", "pref_speed", "time_horizon"):
        setattr(s, f, np.ascontiguousarray(getattr(scene, f)[idx]))
    return s


# ----------------------------------------------------------------------------------
# The paper's own test cases (Section 4): crowds spawned without overlap in start
# regions, each agent heading for its own goal in an associated end region.  The paper
# gives the agent parameters and the crowd layout in words only; the region sizes, the
# spawn density and the ORCA parameters below are readings (stated in the docstrings).
# ----------------------------------------------------------------------------------

def spawn_without_overlap(rng, lo, hi, radius, clearance, max_tries: int = 200) -> np.ndarray:
    """Positions uniform in the box [lo, hi) (lo, hi: float64[m, 2] per agent) such that
    no two agents are closer than radius_i + radius_j + clearance_i + clearance_j, by
    rejection sampling in agent order (a grid over the boxes finds the agents already
    placed nearby).  Raises if an agent finds no free spot in ``max_tries`` draws."""
    m = radius.shape[0]
    reach = 2.0 * float(np.max(radius + clearance)) if m else 1.0
    cells: dict = {}
    pos = np.zeros((m, 2))
    span = radius + clearance
    for i in range(m):
        for _ in range(max_tries):
            p = lo[i] + rng.random(2) * (hi[i] - lo[i])
            cx, cy = int(math.floor(p[0] / reach)), int(math.floor(p[1] / reach))
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for j in cells.get((cx + dx, cy + dy), ()):
                        if (p[0] - pos[j, 0]) ** 2 + (p[1] - pos[j, 1]) ** 2 < (span[i] + span[j]) ** 2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                pos[i] = p
                cells.setdefault((cx, cy), []).append(i)
                break
        else:
            raise ValueError(f"agent {i}: no free spawn spot after {max_tries} draws")
    return pos


def _crossing_parameters(rng, m: int, heterogeneous: bool):
    """Section 4's agent parameters.  Equal agents: radius 0.5 m, desired speed 1 m/s,
    maximum 1.33 m/s.  Varied agents: radius 0.5, 0.75 or 1 m and, independently, desired
    speed 1, 1.33 or 2 m/s, each with probability 1/3; maximum = 1.25 x desired."""
    if not heterogeneous:
        return _full(m, 0.5), _full(m, 1.0), _full(m, 1.33)
    radius = _f32(rng.choice([0.5, 0.75, 1.0], m))
    pref = _f32(rng.choice([1.0, 1.33, 2.0], m))
    return radius, pref, _f32(1.25 * pref.astype(np.float64))


def _region_boxes(centres, side):
    c = np.asarray(centres, np.float64)
    return c - 0.5 * side, c + 0.5 * side


def _region_side(radius, pref, dt, groups, coverage):
    """Side of square start regions in which the agents' spawn discs (radius plus one
    step of travel) cover ``coverage`` of the area, for the most crowded group."""
    disc = math.pi * (radius.astype(np.float64) + pref.astype(np.float64) * dt) ** 2
    need = max(float(disc[g].sum()) for g in groups) if len(radius) else 1.0
    return math.sqrt(need / coverage)


def two_way_crossing(n: int = 2500, heterogeneous: bool = False, seed: int = 1914,
                     coverage: float = 0.3, neighbor_dist: float = 10.0, max_neighbors: int = 10,
                     time_horizon: float = 5.0, dt: float = 0.1, steps: int = 3000) -> Scene:
    """Two-way crossing (Section 4, Figs. 3-4): two crowds of n/2; each crowd's start
    region is the other's end region, so they pass through each other.  Readings: square
    regions in which the spawn discs (radius plus one step of travel at the desired speed,
    the spawn clearance) cover 30% of the area (0.27 agents/m^2 for equal agents), centred
    one side length either side of the origin on the x axis; goals uniform in the end
    region; r_obs 10 m, k 10, tau 5 s, dt 0.1 s (the paper does not state its ORCA
    parameters)."""
    rng = np.random.default_rng(seed)
    h = n // 2
    radius, pref, vmax = _crossing_parameters(rng, n, heterogeneous)
    side = _region_side(radius, pref, dt, [slice(0, h), slice(h, n)], coverage)
    centre = np.array([[-side, 0.0]] * h + [[side, 0.0]] * (n - h)).reshape(-1, 2)
    lo, hi = _region_boxes(centre, side)
    pos = spawn_without_overlap(rng, lo, hi, radius.astype(np.float64), pref.astype(np.float64) * dt)
    glo, ghi = _region_boxes(-centre, side)
    goal = glo + rng.random((n, 2)) * (ghi - glo)
    name = "two_way_varied" if heterogeneous else "two_way"
    return Scene(name, _f32(pos), np.zeros((n, 2), np.float32), _f32(goal), radius, vmax, pref,
                 _full(n, time_horizon), neighbor_dist, max_neighbors, dt, steps)


class SpawnSource:
    """People waiting to enter a crowd during the run: their start boxes, goals and
    parameters.  ``candidates(rng)`` draws a uniform position in every waiting person's
    start box (float32 arrays in waiting order); ``admit(mask)`` removes the admitted ones
    (mask: bool over the same order)."""

    def __init__(self, lo, hi, goal, radius, max_speed, pref_speed, time_horizon):
        self.lo, self.hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
        self.goal, self.radius, self.max_speed = goal, radius, max_speed
        self.pref_speed, self.time_horizon = pref_speed, time_horizon

    @property
    def n(self) -> int:
        return int(self.radius.shape[0])

    def candidates(self, rng):
        pos = _f32(self.lo + rng.random(self.lo.shape) * (self.hi - self.lo))
        return (pos, self.goal, self.radius, self.max_speed, self.pref_speed, self.time_horizon)

    def admit(self, mask):
        keep = ~np.asarray(mask, bool)
        self.lo, self.hi, self.goal = self.lo[keep], self.hi[keep], self.goal[keep]
        self.radius, self.max_speed = self.radius[keep], self.max_speed[keep]
        self.pref_speed, self.time_horizon = self.pref_speed[keep], self.time_horizon[keep]


def two_way_stream(n: int = 2500, heterogeneous: bool = False, seed: int = 1916,
                   coverage: float = 0.3, dt: float = 0.1):
    """The two-way crossing's people entering during the run (Section 4: people are spawned
    at random locations of their start region where they overlap nobody within a time
    period based on size and speed): the crossing's regions, goals and parameters, with
    nobody present at the start.  Returns (empty Scene with the crossing's ORCA parameters,
    SpawnSource of the n people)."""
    rng = np.random.default_rng(seed)
    h = n // 2
    radius, pref, vmax = _crossing_parameters(rng, n, heterogeneous)
    side = _region_side(radius, pref, dt, [slice(0, h), slice(h, n)], coverage)
    centre = np.array([[-side, 0.0]] * h + [[side, 0.0]] * (n - h)).reshape(-1, 2)
    lo, hi = _region_boxes(centre, side)
    glo, ghi = _region_boxes(-centre, side)
    goal = _f32(glo + rng.random((n, 2)) * (ghi - glo))
    tau = _full(n, 5.0)
    z2, z1 = np.zeros((0, 2), np.float32), np.zeros(0, np.float32)
    empty = Scene("two_way_stream", z2, z2, z2, z1, z1, z1, z1, 10.0, 10, dt, 0)
    return empty, SpawnSource(lo, hi, goal, radius, vmax, pref, tau)


def eight_way_crossing(n: int = 10000, seed: int = 1915, coverage: float = 0.3,
                       neighbor_dist: float = 10.0, max_neighbors: int = 10,
                       time_horizon: float = 5.0, dt: float = 0.1, steps: int = 4000) -> Scene:
    """Eight-way crossing (Section 4, Fig. 5): eight crowds of n/8 whose start regions sit
    at 45-degree steps around a circle; each crowd's end region is the one 135 degrees
    further round, so the crowds cross near the centre and turn into a vortex.  Readings:
    square regions sized as in two_way_crossing, centred on a circle of radius twice the
    side (neighbouring regions do not touch); goals uniform in the end region; the equal
    agents of the two-way case; spawn clearance and ORCA parameters as two_way_crossing."""
    rng = np.random.default_rng(seed)
    m = n // 8
    counts = [m + (1 if c < n - 8 * m else 0) for c in range(8)]
    starts = np.cumsum([0] + counts)
    radius, pref, vmax = _crossing_parameters(rng, n, False)
    side = _region_side(radius, pref, dt, [slice(starts[c], starts[c + 1]) for c in range(8)],
                        coverage)
    rc = 2.0 * side
    ang = np.repeat(np.arange(8) * (math.pi / 4.0), counts)
    centre = rc * np.stack([np.cos(ang), np.sin(ang)], 1)
    gang = ang + 3.0 * math.pi / 4.0
    gcentre = rc * np.stack([np.cos(gang), np.sin(gang)], 1)
    lo, hi = _region_boxes(centre, side)
    pos = spawn_without_overlap(rng, lo, hi, radius.astype(np.float64), pref.astype(np.float64) * dt)
    glo, ghi = _region_boxes(gcentre, side)
    goal = glo + rng.random((n, 2)) * (ghi - glo)
    return Scene("eight_way", _f32(pos), np.zeros((n, 2), np.float32), _f32(goal), radius, vmax,
                 pref, _full(n, time_horizon), neighbor_dist, max_neighbors, dt, steps)


def bottleneck(n: int = 2000, seed: int = 1916, door: float = 2.4, coverage: float = 0.3,
               neighbor_dist: float = 10.0, max_neighbors: int = 10, time_horizon: float = 5.0,
               dt: float = 0.1, steps: int = 1500, obstacle_time_horizon: float = 2.0) -> Scene:
    """A room emptying through a door (static obstacles; not in the paper's experiments):
    a wall along x = 0 with a door of width ``door`` around y = 0, and the room's side
    walls.  Agents (r 0.4 m, desired speed 1.3 m/s, maximum 1.6) spawn without overlap in
    a square room left of the wall, sized like the crossings' start regions (spawn discs
    cover 30%), and head for goals past the door: within the door's width across, so that
    an agent pressed against the wall slides towards the door, and spread from 10 m to a
    room side beyond it, so that arrivals do not crowd one spot."""
    rng = np.random.default_rng(seed)
    radius = _full(n, 0.4)
    pref = _full(n, 1.3)
    vmax = _full(n, 1.6)
    side = _region_side(radius, pref, dt, [slice(0, n)], coverage)
    h = 0.5 * side + 1.0
    segs = np.array([[0.0, -h, 0.0, -0.5 * door], [0.0, 0.5 * door, 0.0, h],
                     [-side - 5.0, -h, 0.0, -h], [-side - 5.0, h, 0.0, h]], np.float32)
    lo = np.tile([[-2.0 - side, -0.5 * side]], (n, 1))
    hi = np.tile([[-2.0, 0.5 * side]], (n, 1))
    pos = spawn_without_overlap(rng, lo, hi, radius.astype(np.float64), pref.astype(np.float64) * dt)
    goal = np.stack([rng.uniform(10.0, 10.0 + side, n), rng.uniform(-0.4, 0.4, n) * door], 1)
    return Scene("bottleneck", _f32(pos), np.zeros((n, 2), np.float32), _f32(goal), radius, vmax,
                 pref, _full(n, time_horizon), neighbor_dist, max_neighbors, dt, steps,
                 obstacles=segs, obstacle_time_horizon=obstacle_time_horizon,
                 max_obstacle_neighbors=4)
