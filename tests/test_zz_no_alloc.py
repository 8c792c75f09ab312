"""orca_step_static: one step for callers that cannot allocate GPU memory.

It keeps its scratch in a fixed array inside the library, so it must give the same result
as the ordinary context API (orca_set_agents + orca_step), call after call -- the second
call must not be disturbed by what the first left in the shared array.  This file is
collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_1908_10107_gb300 import abi
from paper_1908_10107_gb300 import scenarios as S

pytestmark = pytest.mark.gpu

VEL_TOL = 1e-4  # the parity tolerance of the other GPU tests (m/s)


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_10107_gb300 import build
    build.build()
    return torch


def _context_step(scene):
    sim = abi.OrcaSim.for_scene(scene)
    sim.set_scene(scene)
    sim.step(1)
    out = sim.get_state()
    sim.close()
    return out


def _static_step(torch, scene):
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in scene.arrays()]
    pos_out = torch.full((scene.n, 2), float("nan"), device="cuda")
    vel_out = torch.full((scene.n, 2), float("nan"), device="cuda")
    abi.orca_step_static(scene.n, *dev, scene.neighbor_dist, scene.max_neighbors, scene.dt,
                         0.0, pos_out, vel_out)
    torch.cuda.synchronize()
    return pos_out.cpu().numpy(), vel_out.cpu().numpy()


def _close(a, b, dt):
    # the same kernels with the same roundings: the results must be bitwise equal (the
    # parity tolerance is kept only to report how far apart they are if they are not)
    dv = float(np.abs(a[1] - b[1]).max(initial=0.0))
    assert dv <= VEL_TOL, f"velocities differ by {dv}"
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[0], b[0])


def test_two_calls_in_a_row_match_the_context_api(torch):
    first = S.jitter_velocities(S.bidirectional(40000, seed=21), 21)
    a1 = _static_step(torch, first)
    _close(a1, _context_step(first), first.dt)
    # second call: a different, smaller crowd with more neighbours, continuing from the
    # first call's output for its first agents
    second = S.jitter_velocities(S.dense(25000, seed=22), 22)
    second.max_neighbors = 16
    second.pos[:1000] = a1[0][:1000] - a1[0][:1000].min(0)
    a2 = _static_step(torch, second)
    _close(a2, _context_step(second), second.dt)


def test_rejects_more_agents_than_the_scratch_holds(torch):
    n = 65537
    t = torch.zeros(2 * n, device="cuda")
    s = torch.ones(n, device="cuda")
    with pytest.raises(abi.OrcaError) as e:
        abi.orca_step_static(n, t, t, t, s, s, s, s, 10.0, 10, 0.1, 0.0, t.clone(), t.clone())
    assert e.value.status == abi.ORCA_ERR_CAPACITY
    assert "65536" in abi.orca_last_error(None)


def test_rejects_short_tensors_before_any_launch(torch):
    n = 1000
    ok2 = torch.zeros(2 * n, device="cuda")
    ok1 = torch.ones(n, device="cuda")
    short = torch.ones(n - 1, device="cuda")
    with pytest.raises(ValueError):
        abi.orca_step_static(n, ok2, ok2, ok2, short, ok1, ok1, ok1, 10.0, 10, 0.1, 0.0,
                             ok2.clone(), ok2.clone())
    with pytest.raises(ValueError):
        abi.orca_step_static(n, ok2, ok2, ok2, ok1, ok1, ok1, ok1, 10.0, 10, 0.1, 0.0,
                             ok2.clone(), ok2[: 2 * n - 1].clone())
    with pytest.raises(TypeError):
        abi.orca_step_static(n, ok2.cpu(), ok2, ok2, ok1, ok1, ok1, ok1, 10.0, 10, 0.1, 0.0,
                             ok2.clone(), ok2.clone())
