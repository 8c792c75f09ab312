"""Hand-written adjoint of the ORCA step and of checkpointed rollouts, against FP64 central
finite differences of the oracle.

The step is piecewise smooth: the adjoint holds neighbour sets and every branch fixed.  A
finite difference whose +-h runs cross a branch (h and h/2 disagree by more than 1e-4
relative) is flagged non-differentiable and excluded; the rest must agree with the GPU
gradient within 1e-3 relative (FP32 adjoint along the FP32 trajectory against FP64 finite
differences).  Beyond the 1e-3 two allowances, neither a fraction of the largest gradient
large enough to hide an error: the finite difference's own error (twice the change of the
central difference from h to h/2), and the FP32 rounding of a gradient summed from terms
up to the largest gradient's size (1e-6 of it: ~100 terms of 6e-8 relative).  The FP64
instantiation of the same adjoint is held to finite differences without the FP32
allowance (test_gpu_adjoint_fp64.py).
"""
import numpy as np
import pytest

import oracle
from paper_1908_10107_gb300 import abi
from paper_1908_10107_gb300 import scenarios as S

pytestmark = pytest.mark.gpu

REL = 1e-3


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_10107_gb300 import build
    build.build()
    return torch


def gpu_grads(torch, sc, W, T, C):
    """GPU gradients of L = sum_t sum_i W[t,i].p_i(t) (t = 1..T)."""
    sim = abi.OrcaSim.for_scene(sc)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in sc.arrays()]
    sim.set_agents(*dev)
    nbytes = abi.orca_rollout_workspace_size(sim.ctx, T, C)
    raw = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    off = (-raw.data_ptr()) % 256
    ws = raw[off: off + nbytes]
    traj = torch.empty((T, sc.n, 2), device="cuda")
    abi.orca_rollout_forward(sim.ctx, T, C, traj, ws)
    g = [torch.empty(sc.n, device="cuda") for _ in range(3)]
    gp0 = torch.empty((sc.n, 2), device="cuda")
    gv0 = torch.empty((sc.n, 2), device="cuda")
    abi.orca_rollout_backward(sim.ctx, torch.from_numpy(W).float().cuda(), g[0], g[1], g[2], gp0, gv0, ws)
    torch.cuda.synchronize()
    out = dict(pref=g[0].cpu().numpy(), radius=g[1].cpu().numpy(), tau=g[2].cpu().numpy(),
               pos0=gp0.cpu().numpy(), vel0=gv0.cpu().numpy(), traj=traj.cpu().numpy())
    sim.close()
    return out


def oracle_loss(sc, W, T, fp64_knn, **override):
    """Sum_t W[t].p(t) of an FP64 oracle rollout with some inputs replaced (float64)."""
    a = dict(pos=sc.pos.astype(np.float64), vel=sc.vel.astype(np.float64),
             goal=sc.goal.astype(np.float64), radius=sc.radius.astype(np.float64),
             max_speed=sc.max_speed.astype(np.float64), pref_speed=sc.pref_speed.astype(np.float64),
             time_horizon=sc.time_horizon.astype(np.float64))
    a.update(override)
    pos, vel = a.pop("pos"), a.pop("vel")
    L = 0.0
    for t in range(T):
        r = oracle.step(pos, vel, neighbor_dist=sc.neighbor_dist, max_neighbors=sc.max_neighbors,
                        dt=sc.dt, knn_mode=0, fp64_knn=fp64_knn, **a)
        pos, vel = r["pos"], r["vel"]
        L += float((W[t] * pos).sum())
    return L


def fd(sc, W, T, key, agent, comp=None, fp64_knn=False, rel_h=1e-6):
    """Central difference of the FP64 oracle loss, and whether the loss is smooth there:
    the forward and backward one-sided differences agree (a kink -- a branch crossed
    inside the stencil -- makes them differ, while the central difference would silently
    average them) and the central differences at h and h/2 agree."""
    name = {"pref": "pref_speed", "radius": "radius", "tau": "time_horizon", "pos0": "pos",
            "vel0": "vel"}[key]
    base = getattr(sc, name).astype(np.float64)
    x0 = base[agent] if comp is None else base[agent, comp]

    def L(dx):
        arr = base.copy()
        if comp is None:
            arr[agent] = x0 + dx
        else:
            arr[agent, comp] = x0 + dx
        return oracle_loss(sc, W, T, fp64_knn, **{name: arr})

    h = rel_h * max(abs(x0), 1.0)
    f0, fp, fm, fp2, fm2 = L(0.0), L(h), L(-h), L(h / 2), L(-h / 2)
    central, central2 = (fp - fm) / (2 * h), (fp2 - fm2) / h
    fwd, bwd = (fp - f0) / h, (f0 - fm) / h
    err = abs(central - central2)
    # a branch crossed inside the stencil changes the slope by a sizeable fraction;
    # curvature changes it by about h f'' (h ~ 1e-6 relative)
    slope = max(abs(fwd), abs(bwd))
    smooth = (abs(fwd - bwd) <= 1e-2 * slope + 1e-7 and
              err <= 1e-4 * max(abs(central), 1e-3))
    return central, err, smooth


def inside_disc(sc, factor=0.9):
    """Preferred speed below the maximum, so the preferred velocity is not on the disc's
    boundary (where the selected velocity has a kink in the preferred speed)."""
    sc = sc.copy()
    sc.pref_speed = (sc.max_speed * np.float32(factor)).astype(np.float32)
    return sc


def check(torch, sc, T, C, agents, keys=("pref", "radius", "tau"), seed=0, fp64_for_state=True):
    W = np.random.default_rng(seed).standard_normal((T, sc.n, 2))
    g = gpu_grads(torch, sc, W, T, C)
    checked = excluded = 0
    for key in keys:
        scale = np.abs(g[key]).max() + 1e-12
        comps = [None] if key in ("pref", "radius", "tau") else [0, 1]
        for a in agents:
            for comp in comps:
                want, err, smooth = fd(sc, W, T, key, a, comp,
                                       fp64_knn=fp64_for_state and comp is not None)
                got = g[key][a] if comp is None else g[key][a, comp]
                if not smooth:
                    excluded += 1
                    continue
                assert abs(got - want) <= REL * abs(want) + 2 * err + 1e-6 * scale, \
                    (key, a, comp, got, want, err, scale)
                checked += 1
    return checked, excluded


def test_one_step_adjoint_matches_fd(torch):
    sc = inside_disc(S.jitter_velocities(S.bidirectional(600, seed=31), 31))
    agents = list(range(0, sc.n, 37))
    checked, excluded = check(torch, sc, T=1, C=1, agents=agents,
                              keys=("pref", "radius", "tau", "pos0", "vel0"))
    assert checked > 60 and excluded <= 0.1 * (checked + excluded)


def test_one_step_adjoint_circle(torch):
    sc = inside_disc(S.jitter_velocities(S.circle_swap(256), 32, scale=0.5))
    checked, excluded = check(torch, sc, T=1, C=1, agents=list(range(0, 256, 13)),
                              keys=("pref", "radius", "tau", "vel0"))
    assert checked > 30


def test_rollout_adjoint_matches_fd(torch):
    sc = inside_disc(S.jitter_velocities(S.bidirectional(300, seed=33), 33, scale=0.3))
    checked, excluded = check(torch, sc, T=6, C=4, agents=list(range(0, sc.n, 29)))
    assert checked > 15 and excluded <= 0.2 * (checked + excluded)


def test_checkpoint_spacing_does_not_change_gradients(torch):
    sc = S.bidirectional(2000, seed=34)
    W = np.random.default_rng(1).standard_normal((10, sc.n, 2))
    a = gpu_grads(torch, sc, W, 10, 1)
    b = gpu_grads(torch, sc, W, 10, 4)
    c = gpu_grads(torch, sc, W, 10, 10)
    np.testing.assert_array_equal(a["traj"], c["traj"])
    for key in ("pref", "radius", "tau", "pos0", "vel0"):
        scale = np.abs(a[key]).max()
        np.testing.assert_allclose(a[key], b[key], atol=1e-5 * scale)
        np.testing.assert_allclose(a[key], c[key], atol=1e-5 * scale)


def test_recording_forward_pass_gives_the_same_gradients(torch):
    """ckpt_every = 0: the forward pass records every step and the backward pass re-runs
    nothing; the recorded steps are the same arithmetic as the re-run ones, so trajectory
    and gradients are bitwise those of the checkpointed modes."""
    sc = S.jitter_velocities(S.bidirectional(3000, seed=36), 36)
    W = np.random.default_rng(4).standard_normal((11, sc.n, 2))
    rec = gpu_grads(torch, sc, W, 11, 0)
    for C in (1, 4):
        ck = gpu_grads(torch, sc, W, 11, C)
        for key in ("traj", "pref", "radius", "tau", "pos0", "vel0"):
            np.testing.assert_array_equal(rec[key], ck[key])
    assert np.abs(rec["radius"]).max() > 0


def test_autograd_function(torch):
    from paper_1908_10107_gb300 import adjoint
    sc = S.bidirectional(1500, seed=35)
    sim = abi.OrcaSim.for_scene(sc)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in sc.arrays()]
    pos0, vel0, goal, radius, vmax, pref, tau = dev
    target = adjoint.rollout(sim, pos0, vel0, goal, radius * 1.05, vmax, pref * 0.95, tau, 12, 4).detach()
    for t in (radius, pref, tau, pos0, vel0):
        t.requires_grad_(True)
    traj = adjoint.rollout(sim, pos0, vel0, goal, radius, vmax, pref, tau, 12, 4)
    loss = adjoint.mse_trajectory_loss(traj, target)
    loss.backward()
    # the same gradients through the C ABI with dL/dp = 2 (p - target) / (T n)
    W = (2.0 * (traj.detach() - target) / (12 * sc.n)).cpu().numpy()
    g = gpu_grads(torch, sc, W, 12, 4)
    for t, key in ((radius, "radius"), (pref, "pref"), (tau, "tau"), (pos0, "pos0"), (vel0, "vel0")):
        scale = np.abs(g[key]).max()
        np.testing.assert_allclose(t.grad.cpu().numpy(), g[key], atol=1e-5 * scale + 1e-12)
    assert float(loss.detach()) > 0 and np.abs(radius.grad.cpu().numpy()).max() > 0


def test_gradients_are_bitwise_reproducible(torch):
    """What an agent's half-planes give its neighbours is summed in a fixed order (a sorted
    transposed neighbour list), not by atomics: two backward passes agree bit for bit."""
    sc = S.differentiable(4096)
    W = np.random.default_rng(3).standard_normal((12, sc.n, 2))
    a = gpu_grads(torch, sc, W, 12, 4)
    b = gpu_grads(torch, sc, W, 12, 4)
    for key in ("pref", "radius", "tau", "pos0", "vel0"):
        np.testing.assert_array_equal(a[key], b[key])
