"""Batched ensemble (extension row a9): instances of uneven size advanced by
persistent launches over a shared work list, captured in a CUDA graph,
with an autotuned work-item size. Every instance must match its solo run:
the first time step bit for bit, the states to rounding (the persistent
kernels inline the same per-cell device functions inside a loop over work
items, where the compiler may hoist a product out of the loop and then not
contract it into an FMA); and the ensemble's own results must not depend
on the tile size or on whether the step is graph-replayed (bit for bit)."""
import math

import numpy as np
import pytest

from paper_2508_19911_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_19911_gb300 import gks
    gks.lib()
    return torch, torch.device("cuda:0"), gks


def small_instances():
    """Uneven 2D and 3D instances with different physics."""
    out = []
    rng = np.random.default_rng(7)
    Q, G, grid = wl.double_shear_layer(32, 48, amp=0.05)
    out.append((Q, G, grid, dict(mu=1e-3)))
    Q, G, grid = wl.double_shear_layer(64, 32, amp=0.01, Ma=0.5)
    out.append((Q, G, grid, dict(mu=1e-4)))
    st = np.stack([rng.uniform(0.1, 1.5, 4), rng.uniform(-1, 1, 4), rng.uniform(-1, 1, 4),
                   rng.uniform(0.05, 1.5, 4)], axis=1)
    Q, G, grid = wl.riemann_quadrants(32, 32, states=st, amp=0.02, seed=3)
    out.append((Q, G, grid, dict(mu=0.0, inviscid=True)))
    Q, G, grid = wl.taylor_green((12, 10, 8))
    out.append((Q, G, grid, dict(mu=1.0 / 1600)))
    Q, G, grid = wl.double_sod(48)
    out.append((Q, G, grid, dict(mu=0.0, inviscid=True, Pr=1.0)))
    return out


def build(env, insts, precision):
    torch, dev, gks = env
    spec = [dict(n=g.n, L=g.L, **ph) for _, _, g, ph in insts]
    e = gks.Ensemble(spec, precision=precision)
    for i, (Q, G, _, _) in enumerate(insts):
        q, gg = e.views(i)
        q.copy_(torch.tensor(Q, device=dev))
        gg.copy_(torch.tensor(G, device=dev))
    return e


def solo_steps(env, Q, G, grid, ph, precision, steps):
    """Solo run one step at a time; returns the state and the dt list."""
    torch, dev, gks = env
    s = gks.Solver(gks.Config(n=grid.n, L=grid.L, scheme="cgks5", precision=precision, **ph))
    Qd, Gd = torch.tensor(Q, device=dev), torch.tensor(G, device=dev)
    dts = [s.step(Qd, Gd, nsteps=1) for _ in range(steps)]
    return Qd, Gd, dts


def grouped_err(a, b):
    """max over (density, momentum vector, energy) of the max-norm error
    relative to that group's max-norm (the parity metric of the GPU tests)."""
    groups = ((0,), (1, 2, 3), (4,))
    errs = []
    for gidx in groups:
        x, y = a[list(gidx)], b[list(gidx)]
        errs.append(float((x - y).abs().max() / y.abs().max().clamp_min(1e-300)))
    return max(errs)


@pytest.mark.parametrize("precision,tol,tol_t", [("fp64", 1e-12, 1e-12), ("mixed", 1e-6, 1e-9)])
def test_instances_match_their_solo_runs(env, precision, tol, tol_t):
    torch, dev, gks = env
    insts = small_instances()
    e = build(env, insts, precision)
    e.step(1, graph=False)
    t1 = e.times()
    e.step(2, graph=True)
    t = e.times()
    for i, (Q, G, grid, ph) in enumerate(insts):
        Qs, Gs, dts = solo_steps(env, Q, G, grid, ph, precision, 3)
        q, gg = e.views(i)
        assert t1[i] == dts[0], i                      # first dt: same state, same reduction
        assert t[i] == pytest.approx(sum(dts), rel=tol_t), i
        eq = grouped_err(q, Qs)
        eg = float((gg - Gs).abs().max() / Gs.abs().max().clamp_min(1e-300))
        print(f"instance {i} {precision}: state err {eq:.2e}, gradient err {eg:.2e}")
        assert eq < tol, (i, eq)
        assert eg < 100 * tol, (i, eg)


def test_graph_and_tile_size_do_not_change_results(env):
    torch, dev, gks = env
    insts = small_instances()
    runs = []
    for tile, graph in ((256, False), (4096, True), (1000, True)):
        e = build(env, insts, "mixed")
        e.set_tile(tile)
        e.step(2, graph=graph)
        runs.append((e.Q.clone(), e.G.clone()))
        e.close()
    for Q, G in runs[1:]:
        assert torch.equal(Q, runs[0][0]) and torch.equal(G, runs[0][1])


def test_autotune_keeps_state_and_times(env):
    torch, dev, gks = env
    insts = small_instances()
    e = build(env, insts, "fp64")
    e.step(1)
    Q0, G0, t0 = e.Q.clone(), e.G.clone(), e.times()
    tile, ms = e.autotune()
    assert tile in (256, 512, 1024, 2048, 4096, 8192) and ms > 0
    assert torch.equal(e.Q, Q0) and torch.equal(e.G, G0)
    assert np.array_equal(e.times(), t0)


def test_time_stop_per_instance(env):
    torch, dev, gks = env
    insts = small_instances()
    e = build(env, insts, "fp64")
    e.step(50, t_stop=1e-2, graph=True)
    np.testing.assert_allclose(e.times(), 1e-2, rtol=1e-14)


def test_ensemble_dump_equals_solo_dumps(env):
    torch, dev, gks = env
    insts = small_instances()
    e = build(env, insts, "mixed")
    e.step(2)
    x, chi, y = e.dump()
    for i, (Q, G, grid, ph) in enumerate(insts):
        s = gks.Solver(gks.Config(n=grid.n, L=grid.L, scheme="cgks5", precision="mixed", **ph))
        q, gg = e.views(i)
        xs, chis, ys = s.indicator_dump(q.contiguous(), gg.contiguous())
        o, c = e.offsets[i], e.offsets[i + 1] - e.offsets[i]
        assert torch.equal(x[:, 5 * o: 5 * (o + c)], xs)
        assert torch.equal(chi[5 * o: 5 * (o + c)], chis)
        assert torch.equal(y[5 * o: 5 * (o + c)], ys)


def test_set_tile_right_after_an_asynchronous_step(env):
    """set_tile rebuilds the work list while the previous step's persistent
    kernels may still run on the ensemble's stream: the result must equal a
    run with a host synchronisation in between."""
    torch, dev, gks = env
    insts = small_instances()
    runs = []
    for sync in (True, False):
        e = build(env, insts, "fp64")
        e.set_tile(512)
        e.step(2, graph=False)
        if sync:
            torch.cuda.synchronize()
        e.set_tile(2048)
        e.step(2, graph=False)
        torch.cuda.synchronize()
        runs.append((e.Q.clone(), e.G.clone()))
        e.close()
    assert torch.equal(runs[0][0], runs[1][0]) and torch.equal(runs[0][1], runs[1][1])


@pytest.mark.parametrize("precision,tol,tol_t", [("fp64", 1e-13, 1e-12), ("mixed", 1e-6, 1e-8)])
def test_single_launch_step_equals_the_per_phase_launches(env, precision, tol, tol_t):
    """Mode 1 (one persistent launch per step, phases separated by grid-wide
    barriers) against mode 0 (one persistent launch per phase): the same
    device code in another kernel, so the same first dt and states equal to
    rounding (the single-launch kernel's translation unit contracts the
    mixed reconstruction's multiply-adds, which the per-phase one does not;
    the later dt follow the states: 4e-10 apart after 4 mixed steps)."""
    torch, dev, gks = env
    insts = small_instances()
    res = []
    for mode in (0, 1):
        e = build(env, insts, precision)
        e.set_mode(mode)
        assert e.mode == mode
        e.step(1, graph=False)
        t1 = e.times()
        e.step(3, graph=True)
        res.append((t1, e.times(), e.Q.clone(), e.G.clone()))
        e.close()
    assert np.array_equal(res[0][0], res[1][0])
    np.testing.assert_allclose(res[1][1], res[0][1], rtol=tol_t)
    q0, q1 = res[0][2], res[1][2]
    assert float((q1 - q0).abs().max() / q0.abs().max()) < tol


def test_barrier_wait_runs_out_and_the_device_stays_usable(env):
    """Two blocks wait at a barrier for a third that never arrives: their
    bounded waits give up after 0.2 s and report a timeout (no hang, no
    fault); an ensemble step afterwards runs normally."""
    torch, dev, gks = env
    assert gks.barrier_timeout_check(0.2) == -4  # GKS_ERR_TIMEOUT
    insts = small_instances()[:2]
    e = build(env, insts, "fp64")
    e.step(2, graph=True)
    t = e.times()
    assert np.all(t > 0)
