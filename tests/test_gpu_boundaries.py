"""GPU parity of the general-grid kernels (symmetry / outflow boundaries,
stretched meshes; Sec. 3.2, last paragraph) against the FP64 CPU oracle,
through the C-ABI.

Every case runs on a ragged grid whose axes mix the three boundary kinds
and a stretched spacing, from a perturbed Taylor-Green state (the normal
velocity of the vortex vanishes on its symmetry planes x, y = 0, pi, so the
octant boxes below are physical). FP64 results must agree with the oracle
within 1e-11 relative to each physical group's magnitude (gradients: plus
max|Q|/h, their rounding scale by Gauss's theorem); mixed precision within
1e-5 relative L2 of the per-cell kinetic energy of the FP64 path.
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


def case(n=(9, 8, 7), bc=("symmetry", "outflow", "periodic"), amp=0.02, seed=31):
    """Perturbed Taylor-Green vortex on [0, pi] x [0, pi] x [0, 2 pi],
    x and y stretched."""
    edges = (wl.stretched_edges(n[0], np.pi, 0.35), wl.stretched_edges(n[1], np.pi, -0.25),
             np.linspace(0.0, 2 * np.pi, n[2] + 1))
    Q, G, grid = wl.taylor_green(edges=edges, Ma=0.3)
    Q, G = wl.perturb(Q, G, amp=amp, seed=seed)
    return Q, G, grid, bc


BCN = {"periodic": 0, "symmetry": 1, "outflow": 2}


def make(torch_dev, grid, bc, **kw):
    from paper_2508_19911_gb300 import gks
    return gks.Solver(gks.Config(n=grid.n, L=grid.L, bc=bc, spacing=grid.spacing, **kw))


def oparams(grid, bc, scheme="cgks5", nonlinear=True, **kw):
    return oracle.params(n=grid.n, L=grid.L, scheme=1 if scheme == "cgks5" else 0,
                         nonlinear=int(nonlinear), bc=tuple(BCN[b] for b in bc),
                         spacing=grid.spacing, **kw)


def state_err(a, ref):
    worst = 0.0
    for g in GROUPS:
        sc = np.abs(ref[g]).max()
        worst = max(worst, float(np.abs(a[g] - ref[g]).max() / (sc if sc > 0 else 1.0)))
    return worst


def grad_err(a, ref, Q, h):
    worst = 0.0
    for g in GROUPS:
        sc = np.abs(ref[g]).max() + np.abs(Q[g]).max() / h
        worst = max(worst, float(np.abs(a[g] - ref[g]).max() / sc))
    return worst


@pytest.mark.parametrize("scheme", ["gks2", "cgks5"])
def test_face_states_match_oracle_on_a_general_grid(torch_dev, scheme):
    torch, dev = torch_dev
    Q, G, grid, bc = case()
    cg = scheme == "cgks5"
    for nonlinear in (False, True):
        s = make(torch_dev, grid, bc, scheme=scheme, nonlinear=nonlinear)
        fs = s.reconstruct(torch.tensor(Q, device=dev),
                           torch.tensor(G, device=dev) if cg else None).cpu().numpy()
        ref = oracle.face_states(oparams(grid, bc, scheme, nonlinear), Q, G if cg else None)
        got = fs.transpose(0, 2, 1, 3).reshape(6, 20, -1)
        ref = ref.transpose(0, 2, 1, 3).reshape(6, 20, -1)
        scale = np.abs(ref).max(axis=2, keepdims=True)
        scale = np.where(scale == 0, 1.0, scale)
        err = float(np.max(np.abs(got - ref) / scale))
        assert err < TOL, (nonlinear, err)


@pytest.mark.parametrize("scheme", ["gks2", "cgks5"])
def test_boundary_face_records_match_oracle(torch_dev, scheme):
    """gks_flux on a grid with symmetry and outflow axes: the low boundary
    faces (cell and mirror ghost) and the high boundary records that follow
    the 90 x cells records."""
    torch, dev = torch_dev
    Q, G, grid, bc = case(bc=("symmetry", "outflow", "symmetry"))
    cg = scheme == "cgks5"
    P = oparams(grid, bc, scheme)
    fs = oracle.face_states(P, Q, G if cg else None)
    dt = 0.004
    _, _, faces, fhi = oracle.stage(P, Q, G if cg else None, dt, boundary=True)
    s = make(torch_dev, grid, bc, scheme=scheme)
    n = Q[0].size
    np_ = oracle.n_plane(P)
    assert s.flux_bytes() == 8 * 90 * (n + np_)
    got = s.flux(torch.tensor(fs, device=dev), torch.tensor([dt], dtype=torch.float64, device=dev))
    got = got.cpu().numpy()
    rec, rhi = got[:90 * n].reshape(3, 30, n), got[90 * n:].reshape(3, 30, np_)
    nq = 30 if cg else 10
    for d in range(3):
        ref = faces[d, :nq]
        scale = np.abs(ref).max(axis=1, keepdims=True)
        scale = np.where(scale == 0, 1.0, scale)
        assert np.max(np.abs(rec[d, :nq] - ref) / scale) < TOL, d
        if bc[d] != "periodic":
            m = {0: grid.n[1] * grid.n[2], 1: grid.n[0] * grid.n[2], 2: grid.n[0] * grid.n[1]}[d]
            assert np.max(np.abs(rhi[d, :nq, :m] - fhi[d, :nq, :m]) / scale) < TOL, d


@pytest.mark.parametrize("scheme,nonlinear", [("gks2", True), ("cgks5", False), ("cgks5", True)])
def test_twenty_steps_match_oracle_on_a_general_grid(torch_dev, scheme, nonlinear):
    """The 20-step FP64 gate on a stretched grid with a symmetry, an outflow
    and a periodic axis."""
    torch, dev = torch_dev
    Q, G, grid, bc = case(amp=0.005)
    cg = scheme == "cgks5"
    s = make(torch_dev, grid, bc, scheme=scheme, nonlinear=nonlinear)
    Qd = torch.tensor(Q, device=dev)
    Gd = torch.tensor(G, device=dev) if cg else None
    s.step(Qd, Gd, nsteps=20)
    assert s.status() == 0
    Qo, Go = Q.copy(), (G.copy() if cg else None)
    oracle.run(oparams(grid, bc, scheme, nonlinear), Qo, Go, nsteps=20)
    assert state_err(Qd.cpu().numpy(), Qo) < TOL
    if cg:
        h = min(float(w.min()) for w in grid.spacing)
        assert grad_err(Gd.cpu().numpy(), Go, Qo, h) < TOL


@pytest.mark.parametrize("scheme", ["gks2", "cgks5"])
def test_octant_box_matches_oracle_and_conserves(torch_dev, scheme):
    """The Taylor-Green octant with six symmetry planes on a stretched mesh:
    oracle parity after 10 steps; mass and energy conserved to round-off."""
    torch, dev = torch_dev
    n = 8
    e = wl.stretched_edges(2 * n, 2 * np.pi, 0.3)[:n + 1]
    Q, G, grid = wl.taylor_green(edges=(e, e, e))
    bc = ("symmetry",) * 3
    cg = scheme == "cgks5"
    s = make(torch_dev, grid, bc, scheme=scheme)
    Qd = torch.tensor(Q, device=dev)
    Gd = torch.tensor(G, device=dev) if cg else None
    d0 = s.diagnostics(Qd, Gd)
    s.step(Qd, Gd, nsteps=10)
    d1 = s.diagnostics(Qd, Gd)
    Qo, Go = Q.copy(), (G.copy() if cg else None)
    oracle.run(oparams(grid, bc, scheme), Qo, Go, nsteps=10)
    assert state_err(Qd.cpu().numpy(), Qo) < TOL
    for slot in (5, 9):  # sum of rho and rho E times the cell volumes
        assert abs(d1[slot] - d0[slot]) <= 1e-13 * abs(d0[slot])
    ref = oracle.diagnostics(oparams(grid, bc, scheme), Qo, Go)
    np.testing.assert_allclose(d1, ref, rtol=1e-11, atol=1e-14 * np.abs(ref).max())


def test_time_step_matches_oracle_on_a_stretched_grid(torch_dev):
    torch, dev = torch_dev
    Q, G, grid, bc = case()
    for kw in (dict(mu=1.0 / 1600), dict(mu=0.2), dict(inviscid=True)):
        s = make(torch_dev, grid, bc, scheme="gks2", **kw)
        dt = s.compute_dt(torch.tensor(Q, device=dev)).item()
        okw = dict(kw)
        if "mu" in okw:
            okw["mu0"] = okw.pop("mu")
        if "inviscid" in okw:
            okw["inviscid"] = int(okw["inviscid"])
        ref = oracle.dt(oparams(grid, bc, "gks2", **okw), Q)
        assert dt == pytest.approx(ref, rel=1e-14), kw


def test_diagnostics_match_oracle_on_a_general_grid(torch_dev):
    torch, dev = torch_dev
    Q, G, grid, bc = case()
    for scheme in ("cgks5", "gks2"):
        cg = scheme == "cgks5"
        s = make(torch_dev, grid, bc, scheme=scheme, mu=1e-3, mu_law=1)
        d = s.diagnostics(torch.tensor(Q, device=dev), torch.tensor(G, device=dev) if cg else None)
        ref = oracle.diagnostics(oparams(grid, bc, scheme, mu0=1e-3, mu_law=1), Q, G if cg else None)
        np.testing.assert_allclose(d, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


def test_uniform_flow_along_walls_is_bitwise_steady_on_gpu(torch_dev):
    torch, dev = torch_dev
    edges = (wl.stretched_edges(6, 1.0, 0.4), wl.stretched_edges(5, 1.3, -0.3),
             np.linspace(0.0, 0.7, 5))
    grid = wl.grid_from_edges(edges)
    Q = np.zeros((5, 4, 5, 6))
    Q[0], Q[1], Q[2], Q[3] = 1.3, 0.0, -0.3, 0.1
    Q[4] = 0.9 / 0.4 + 0.5 * (0.3 ** 2 + 0.1 ** 2) / 1.3
    G = np.zeros((5, 3, 4, 5, 6))
    for scheme in ("gks2", "cgks5"):
        for prec in ("fp64", "mixed"):
            s = make(torch_dev, grid, ("symmetry", "outflow", "periodic"), scheme=scheme,
                     precision=prec, mu=1e-3)
            Qd, Gd = torch.tensor(Q, device=dev), torch.tensor(G, device=dev)
            s.step(Qd, Gd if scheme == "cgks5" else None, nsteps=3)
            assert np.array_equal(Qd.cpu().numpy(), Q), (scheme, prec)
            assert np.array_equal(Gd.cpu().numpy(), G), (scheme, prec)


@pytest.mark.parametrize("scheme", ["gks2", "cgks5"])
def test_mixed_precision_on_a_general_grid(torch_dev, scheme):
    """Mixed precision against the FP64 path on the same general grid:
    per-cell kinetic energy within 1e-5 relative L2 after 20 steps."""
    torch, dev = torch_dev
    Q, G, grid, bc = case(n=(16, 14, 12), amp=0.002)
    cg = scheme == "cgks5"
    out = {}
    for prec in ("fp64", "mixed"):
        s = make(torch_dev, grid, bc, scheme=scheme, precision=prec)
        Qd = torch.tensor(Q, device=dev)
        Gd = torch.tensor(G, device=dev) if cg else None
        s.step(Qd, Gd, nsteps=20)
        assert s.status() == 0
        q = Qd.cpu().numpy()
        out[prec] = 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2) / q[0]
    err = np.linalg.norm(out["mixed"] - out["fp64"]) / np.linalg.norm(out["fp64"])
    assert err < 1e-5, err


def test_slabs_equal_the_whole_grid_with_a_z_wall(torch_dev):
    """z-slabs on a grid whose z axis is a symmetry plane pair: the last
    slab computes the high-z boundary faces; bit for bit the whole-grid
    result."""
    torch, dev = torch_dev
    Q, G, grid, _ = case(n=(6, 5, 11))
    bc = ("outflow", "periodic", "symmetry")
    res = []
    for planes in (0, 3):
        s = make(torch_dev, grid, bc, scheme="cgks5", slab_planes=planes)
        Qd, Gd = torch.tensor(Q, device=dev), torch.tensor(G, device=dev)
        s.step(Qd, Gd, nsteps=2)
        res.append((Qd.cpu().numpy(), Gd.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_general_grid_rejects_the_indicator(torch_dev):
    from paper_2508_19911_gb300 import gks
    Q, G, grid, bc = case()
    with pytest.raises(gks.GksError):
        make(torch_dev, grid, bc, scheme="cgks5", precision="mixed", indicator=True)
