"""Host logic of the autotuner against a fake context whose step time is a known function of
the cell edge and launch shape (no GPU, no library)."""
import math

import numpy as np
import pytest

from paper_1908_10107_gb300 import autotune
from paper_1908_10107_gb300 import scenarios as S


class FakeSim:
    """Step time = a bowl in the cell edge (minimum at ``best_edge``) plus a per-shape cost,
    with optional noise; records what the tuner asked for."""

    def __init__(self, best_edge, shape_ms, noise=0.0, seed=0):
        self.ctx = object()
        self.best_edge = best_edge
        self.shape_ms = shape_ms
        self.edge = 1.0
        self.shape = (128, 1)
        self.noise = noise
        self.rng = np.random.default_rng(seed)
        self.steps = 0
        self.reloads = 0
        self.between_calls = 0
        self.profiling = False

    def set_scene(self, sc):
        self.reloads += 1

    def step(self, n):
        self.steps += n

    def time_ms(self):
        t = 0.3 + 0.05 * math.log(self.edge / self.best_edge) ** 2 + self.shape_ms[self.shape]
        return t * (1.0 + self.noise * self.rng.standard_normal())


@pytest.fixture
def fake(monkeypatch):
    def make(best_edge, shape_ms, noise=0.0):
        sim = FakeSim(best_edge, shape_ms, noise)
        ab = autotune.abi
        monkeypatch.setattr(ab, "orca_profile", lambda ctx, on: setattr(sim, "profiling", on))
        monkeypatch.setattr(ab, "orca_set_cell_size", lambda ctx, s: setattr(sim, "edge", s))
        monkeypatch.setattr(ab, "orca_set_launch", lambda ctx, t, g: setattr(sim, "shape", (t, g)))
        monkeypatch.setattr(ab, "orca_profile_read",
                            lambda ctx: np.array([0.0, 0.0, sim.time_ms()]))
        return sim
    return make


SHAPE_MS = {(64, 1): 0.01, (128, 1): 0.0, (256, 1): 0.03, (64, 4): 0.02, (128, 4): 0.04,
            (256, 4): 0.05, (64, 32): 0.015, (128, 32): 0.025}


def test_expected_kth_distance_uniform():
    # uniform density rho over a square: sqrt(k / (pi rho))
    rng = np.random.default_rng(0)
    pos = rng.uniform(0, 400, size=(40000, 2))
    rho = 40000 / 400.0 ** 2
    assert autotune.expected_kth_distance(pos, 10) == pytest.approx(math.sqrt(10 / (math.pi * rho)),
                                                                    rel=0.02)


def test_cell_size_picks_the_minimum(fake):
    sc = S.bidirectional(2000, seed=3)
    rk = autotune.expected_kth_distance(sc.pos, sc.max_neighbors)
    sim = fake(1.2 * rk, SHAPE_MS)
    flushes = []
    r = autotune.tune_cell_size(sim, sc, cache_path=None, between=lambda: flushes.append(1))
    assert r["cell_size"] == pytest.approx(float(np.float32(1.2 * rk)))
    assert sim.edge == r["cell_size"] and not sim.profiling
    assert len(r["timings_ms"]) == len(autotune.FACTORS)
    # one flush per timed step: the sweep plus two alternating re-timings of two candidates
    assert len(flushes) == autotune.STEPS * (len(autotune.FACTORS) + 4)


def test_refine_breaks_near_ties_by_retiming(fake):
    sim = fake(1.0, SHAPE_MS)
    calls = []

    def make_reload(c):
        return lambda: calls.append(c)

    # the sweep ranked "b" first by noise; the re-timing (true times a < b) decides
    sim.time_ms = lambda: {"a": 1.0, "b": 1.01, "c": 2.0}[calls[-1]]
    best = autotune._refine(sim, {"a": 1.02, "b": 1.0, "c": 2.0}, make_reload, 3, None)
    assert best == "a" and set(calls) == {"a", "b"} and len(calls) == 4


def test_launch_shape_picks_the_minimum(fake):
    sim = fake(1.0, SHAPE_MS)
    r = autotune.tune_launch(sim, lambda: sim.set_scene(None))
    assert r["shape"] == (128, 1) and sim.shape == (128, 1)
    assert set(r["timings_ms"]) == {f"{a}x{b}" for a, b in autotune.SHAPES}


def test_cache_round_trip(fake, tmp_path):
    sc = S.bidirectional(2000, seed=4)
    rk = autotune.expected_kth_distance(sc.pos, sc.max_neighbors)
    sim = fake(0.8 * rk, SHAPE_MS)
    path = str(tmp_path / "tune.json")
    first = autotune.tune_cell_size(sim, sc, cache_path=path)
    steps = sim.steps
    again = autotune.tune_cell_size(sim, sc, cache_path=path)
    assert again["cached"] and not first["cached"]
    assert again["cell_size"] == first["cell_size"] and sim.steps == steps
