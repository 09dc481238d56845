"""Batched ensemble (extension row a9) against the FP64 CPU oracle: every
instance of an uneven ensemble, advanced by the persistent graph-replayed
kernels, equals the oracle's run of that instance alone, element by
element within 1e-11 (the parity metric of the single-grid tests); and the
64-instance workload of the ensemble benchmark, sampled: every instance's
first time step against the oracle's, and the smallest instances' states
after one step element by element."""
import numpy as np
import pytest

import oracle
from paper_2508_19911_gb300 import workloads as wl
from test_gpu_parity import GROUPS, state_err

pytestmark = pytest.mark.gpu

TOL = 1e-11


def grad_err(a, ref, Q, h):
    """Parity metric of a gradient field: max |a - ref| over cells against
    max |ref| + max |Q| / h of its physical group. A cell-averaged gradient
    is a sum of interface values over h (Gauss's theorem), so its rounding
    is relative to |Q|/h: a field that is uniform up to tiny variations (the
    density of a shear layer after one step, 4e-6 against a rounding floor
    of 1e-13) has gradients made of that rounding, and its own maximum is no
    scale for them."""
    worst = 0.0
    for g in GROUPS:
        sc = np.abs(ref[g]).max() + np.abs(Q[g]).max() / h
        worst = max(worst, float(np.abs(a[g] - ref[g]).max() / sc))
    return worst


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_19911_gb300 import gks
    gks.lib()
    return torch, torch.device("cuda:0"), gks


def oracle_params(grid, ph):
    return oracle.params(n=grid.n, L=grid.L, scheme=1, nonlinear=1, mu0=ph.get("mu", 1.0 / 1600),
                         inviscid=int(bool(ph.get("inviscid", False))), Pr=ph.get("Pr", 0.72))


def build(env, insts):
    torch, dev, gks = env
    e = gks.Ensemble([dict(n=g.n, L=g.L, **ph) for _, _, g, ph in insts], precision="fp64")
    for i, (Q, G, _, _) in enumerate(insts):
        q, gg = e.views(i)
        q.copy_(torch.tensor(Q, device=dev))
        gg.copy_(torch.tensor(G, device=dev))
    return e


def test_uneven_ensemble_matches_the_oracle_per_instance(env):
    """Double shear layers and four-quadrant Riemann problems from 16^2 to
    48^2 cells (non-square) and a small 3D Taylor-Green grid, FP64, five
    steps (one eager, four graph-replayed): states, gradients and each
    instance's clock against oracle.run of that instance."""
    rng = np.random.default_rng(11)
    insts = []
    Q, G, grid = wl.double_shear_layer(16, 24, amp=0.05)
    insts.append((Q, G, grid, dict(mu=1e-3)))
    Q, G, grid = wl.double_shear_layer(48, 32, amp=0.02, Ma=0.5)
    insts.append((Q, G, grid, dict(mu=1e-4)))
    for nx, ny, seed in ((32, 16, 3), (24, 48, 4)):
        st = np.stack([rng.uniform(0.3, 1.5, 4), rng.uniform(-1, 1, 4), rng.uniform(-1, 1, 4),
                       rng.uniform(0.2, 1.5, 4)], axis=1)
        Q, G, grid = wl.riemann_quadrants(nx, ny, states=st, amp=0.02, seed=seed)
        insts.append((Q, G, grid, dict(mu=0.0, inviscid=True)))
    Q, G, grid = wl.taylor_green((12, 10, 8))
    insts.append((Q, G, grid, dict(mu=1.0 / 1600)))
    e = build(env, insts)
    e.step(1, graph=False)
    e.step(4, graph=True)
    t = e.times()
    for i, (Q, G, grid, ph) in enumerate(insts):
        Qo, Go = Q.copy(), G.copy()
        to, _ = oracle.run(oracle_params(grid, ph), Qo, Go, nsteps=5)
        q, gg = e.views(i)
        eq = state_err(q.cpu().numpy(), Qo)
        eg = grad_err(gg.cpu().numpy(), Go, Qo, min(grid.h))
        print(f"instance {i} {grid.n}: state {eq:.2e} gradient {eg:.2e}")
        assert eq < TOL and eg < TOL, (i, eq, eg)
        assert t[i] == pytest.approx(to, rel=1e-13), i
    e.close()


def test_sixty_four_instance_ensemble_sampled_against_the_oracle(env):
    """The ensemble benchmark's workload (64 seeded 2D instances, 64^2 to
    512^2): after one graph-replayed step every instance's clock equals the
    oracle's time step for its initial state, and the three smallest
    instances' states equal the oracle's one-step run within 1e-11."""
    insts = wl.ensemble_instances(64, seed0=2000)
    e = build(env, insts)
    e.step(1, graph=True)
    t = e.times()
    for i, (Q, G, grid, ph) in enumerate(insts):
        assert t[i] == pytest.approx(oracle.dt(oracle_params(grid, ph), Q), rel=1e-13), i
    sizes = [g.n[0] * g.n[1] for _, _, g, _ in insts]
    for i in np.argsort(sizes, kind="stable")[:3]:
        Q, G, grid, ph = insts[i]
        Qo, Go = Q.copy(), G.copy()
        oracle.run(oracle_params(grid, ph), Qo, Go, nsteps=1)
        q, gg = e.views(int(i))
        eq = state_err(q.cpu().numpy(), Qo)
        eg = grad_err(gg.cpu().numpy(), Go, Qo, min(grid.h))
        print(f"instance {i} {grid.n}: state {eq:.2e} gradient {eg:.2e}")
        assert eq < TOL and eg < TOL, (int(i), eq, eg)
    e.close()
