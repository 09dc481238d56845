"""GPU parity of CGKS-5th with the line-averaged derivatives as the target
cell's own data (Sec. 3.1-3.2, the set S^0; reading R17) against the FP64
CPU oracle, through the C-ABI (gks_reconstruct_lines, gks_step_lines,
gks_lines_gradients).

Ragged periodic grids (9 x 8 x 7 cells: several warps, a ragged tail in
every axis; uniform, and stretched along x and y) from a perturbed
Taylor-Green state whose lines carry their own seeded perturbation. FP64 results must agree with the oracle within 1e-11
relative to each physical group's magnitude (lines: plus max|Q|/h, their
rounding scale, as for the gradients of the averaged-gradient form).
"""
import numpy as np
import pytest

import oracle
from paper_2508_19911_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-11
GROUPS = ([0], [1, 2, 3], [4])


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_19911_gb300 import gks
    gks.lib()
    return torch, torch.device("cuda:0")


def case(n=(9, 8, 7), amp=0.02, seed=47):
    Q, G, grid, L = wl.taylor_green(n, Ma=0.3, lines=True)
    Q, G = wl.perturb(Q, G, amp=amp, seed=seed)
    rng = np.random.default_rng(seed + 1)
    scale = np.abs(L).reshape(5, -1).max(axis=1)[:, None, None, None, None]
    L = L + amp * scale * rng.standard_normal(L.shape)
    return Q, np.ascontiguousarray(L), grid


def stretched_case(n=(9, 8, 7), amp=0.005, seed=53):
    """The same state on a periodic box whose x and y cells are stretched
    (0.7-1.3 of the mean size)."""
    edges = (wl.stretched_edges(n[0], 2 * np.pi, 0.3), wl.stretched_edges(n[1], 2 * np.pi, -0.25),
             np.linspace(0.0, 2 * np.pi, n[2] + 1))
    Q, G, grid, L = wl.taylor_green(edges=edges, Ma=0.3, lines=True)
    Q, G = wl.perturb(Q, G, amp=amp, seed=seed)
    rng = np.random.default_rng(seed + 1)
    scale = np.abs(L).reshape(5, -1).max(axis=1)[:, None, None, None, None]
    L = L + amp * scale * rng.standard_normal(L.shape)
    return Q, np.ascontiguousarray(L), grid


def solver(grid, **kw):
    from paper_2508_19911_gb300 import gks
    return gks.Solver(gks.Config(n=grid.n, L=grid.L, **kw))


def oparams(grid, nonlinear=True, **kw):
    return oracle.params(n=grid.n, L=grid.L, scheme=1, nonlinear=int(nonlinear), **kw)


def group_err(a, ref, extra=0.0):
    worst = 0.0
    for g in GROUPS:
        sc = np.abs(ref[g]).max() + (extra[g] if np.ndim(extra) else extra)
        worst = max(worst, float(np.abs(a[g] - ref[g]).max() / (sc if sc > 0 else 1.0)))
    return worst


@pytest.mark.parametrize("nonlinear", [False, True])
def test_face_states_from_lines_match_oracle(torch_dev, nonlinear):
    torch, dev = torch_dev
    Q, L, grid = case()
    s = solver(grid, nonlinear=nonlinear)
    fs = s.reconstruct_lines(torch.tensor(Q, device=dev), torch.tensor(L, device=dev))
    ref = oracle.face_states_b(oparams(grid, nonlinear), Q, L)
    got = fs.cpu().numpy().transpose(0, 2, 1, 3).reshape(6, 20, -1)
    ref = ref.transpose(0, 2, 1, 3).reshape(6, 20, -1)
    scale = np.abs(ref).max(axis=2, keepdims=True)
    scale = np.where(scale == 0, 1.0, scale)
    err = float(np.max(np.abs(got - ref) / scale))
    assert err < TOL, err


@pytest.mark.parametrize("nonlinear", [False, True])
def test_ten_steps_with_lines_match_oracle(torch_dev, nonlinear):
    torch, dev = torch_dev
    Q, L, grid = case(amp=0.005)
    s = solver(grid, nonlinear=nonlinear)
    Qd, Ld = torch.tensor(Q, device=dev), torch.tensor(L, device=dev)
    t = torch.zeros(1, dtype=torch.float64, device=dev)
    dt_gpu = s.step_lines(Qd, Ld, nsteps=10, t=t)
    assert s.status() == 0
    Qo, Lo = Q.copy(), L.copy()
    t_o, dt_o = oracle.run_b(oparams(grid, nonlinear), Qo, Lo, nsteps=10)
    assert abs(dt_gpu - dt_o) <= 1e-12 * dt_o
    assert abs(float(t.item()) - t_o) <= 1e-12 * t_o
    assert group_err(Qd.cpu().numpy(), Qo) < TOL
    h = min(grid.L[a] / grid.n[a] for a in range(3))
    qscale = np.abs(Qo).reshape(5, -1).max(axis=1) / h
    Lg = Ld.cpu().numpy()
    for v in range(5):
        sc = np.abs(Lo[v]).max() + qscale[v]
        assert np.abs(Lg[v] - Lo[v]).max() / sc < TOL, v


@pytest.mark.parametrize("nonlinear", [False, True])
def test_lines_on_a_stretched_periodic_grid_match_oracle(torch_dev, nonlinear):
    """Face states and 10 steps on a stretched periodic mesh (each
    neighbour's gradient taken in its own index coordinates)."""
    torch, dev = torch_dev
    Q, L, grid = stretched_case()
    s = solver(grid, nonlinear=nonlinear, spacing=grid.spacing)
    P = oparams(grid, nonlinear, spacing=grid.spacing)
    fs = s.reconstruct_lines(torch.tensor(Q, device=dev), torch.tensor(L, device=dev))
    ref = oracle.face_states_b(P, Q, L).transpose(0, 2, 1, 3).reshape(6, 20, -1)
    got = fs.cpu().numpy().transpose(0, 2, 1, 3).reshape(6, 20, -1)
    scale = np.abs(ref).max(axis=2, keepdims=True)
    scale = np.where(scale == 0, 1.0, scale)
    assert float(np.max(np.abs(got - ref) / scale)) < TOL
    Qd, Ld = torch.tensor(Q, device=dev), torch.tensor(L, device=dev)
    s.step_lines(Qd, Ld, nsteps=10)
    assert s.status() == 0
    Qo, Lo = Q.copy(), L.copy()
    oracle.run_b(P, Qo, Lo, nsteps=10)
    assert group_err(Qd.cpu().numpy(), Qo) < TOL
    h = min(float(w.min()) for w in grid.spacing)
    qscale = np.abs(Qo).reshape(5, -1).max(axis=1) / h
    Lg = Ld.cpu().numpy()
    for v in range(5):
        assert np.abs(Lg[v] - Lo[v]).max() / (np.abs(Lo[v]).max() + qscale[v]) < TOL, v


def test_uniform_flow_with_lines_is_bitwise_steady(torch_dev):
    torch, dev = torch_dev
    nx, ny, nz = 5, 6, 4
    rho, U, V, W, p = 1.3, 0.2, -0.3, 0.1, 0.9
    Q = np.zeros((5, nz, ny, nx))
    Q[0], Q[1], Q[2], Q[3] = rho, rho * U, rho * V, rho * W
    Q[4] = p / 0.4 + 0.5 * rho * (U * U + V * V + W * W)
    from paper_2508_19911_gb300 import gks
    s = gks.Solver(gks.Config(n=(nx, ny, nz), L=(1.0, 1.3, 0.7), mu=1e-3))
    Qd = torch.tensor(Q, device=dev)
    Ld = torch.zeros(5, 12, nz, ny, nx, dtype=torch.float64, device=dev)
    s.step_lines(Qd, Ld, nsteps=3)
    assert torch.equal(Qd.cpu(), torch.tensor(Q))
    assert bool((Ld == 0).all())


def test_lines_gradients_are_the_line_means(torch_dev):
    torch, dev = torch_dev
    Q, L, grid = case()
    s = solver(grid)
    G = s.lines_gradients(torch.tensor(L, device=dev)).cpu().numpy()
    ref = L.reshape((5, 3, 4) + L.shape[2:]).mean(axis=2)
    np.testing.assert_allclose(G, ref, rtol=1e-15, atol=1e-15 * np.abs(L).max())


def test_lines_need_an_fp64_cgks5_periodic_context(torch_dev):
    torch, dev = torch_dev
    from paper_2508_19911_gb300 import gks
    Q, L, grid = case(n=(4, 4, 4))
    Qd, Ld = torch.tensor(Q, device=dev), torch.tensor(L, device=dev)
    for kw in (dict(precision="mixed"), dict(scheme="gks2"), dict(bc=("symmetry", "periodic", "periodic"))):
        s = solver(grid, **kw)
        with pytest.raises(gks.GksError) as e:
            s.step_lines(Qd, Ld, nsteps=1)
        assert e.value.code == gks.GKS_ERR_STATE
