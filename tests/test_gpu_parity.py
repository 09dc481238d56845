"""GPU parity of the CUDA path (through the C-ABI) against the FP64 CPU
oracle, element by element on the same seeded inputs.

Tolerance: the FP64 path must agree with the oracle within 1e-11 relative:
states are measured against the largest magnitude of their physical group
(density, momentum vector, energy; see state_err), intermediate quantities
(face states, fluxes) per component against that component's largest
magnitude.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2508_19911_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_19911_gb300 import gks
    gks.lib()
    return torch, torch.device("cuda:0")


def solver(torch_dev, grid, **kw):
    from paper_2508_19911_gb300 import gks
    return gks.Solver(gks.Config(n=grid.n, L=grid.L, **kw))


def oparams(grid, **kw):
    m = {"cgks5": 1, "gks2": 0}
    kw = dict(kw)
    kw.pop("precision", None)  # the oracle is FP64 only
    if "scheme" in kw:
        kw["scheme"] = m[kw["scheme"]]
    if "mu" in kw:
        kw["mu0"] = kw.pop("mu")
    if "nonlinear" in kw:
        kw["nonlinear"] = int(kw["nonlinear"])
    if "inviscid" in kw:
        kw["inviscid"] = int(kw["inviscid"])
    return oracle.params(n=grid.n, L=grid.L, **kw)


def rel_err(a, ref, keep):
    """max over cells of |a - ref| / max|ref|, per leading index (keep axes)."""
    axes = tuple(range(keep, ref.ndim))
    scale = np.abs(ref).max(axis=axes, keepdims=True)
    scale = np.where(scale == 0, 1.0, scale)
    return float(np.max(np.abs(a - ref) / scale))


GROUPS = ([0], [1, 2, 3], [4])  # density, momentum, total energy


def state_err(a, ref):
    """Parity metric of a state (Q [5,...] or gradQ [5,3,...]): max |a - ref|
    over cells, divided by the largest |ref| of the quantity's physical
    group -- density, the three momentum components together, energy
    (for gradQ also all three axes together). A momentum component that
    is zero in exact arithmetic (rho W of the Taylor-Green vortex, rho V
    and rho W of a 1D tube) carries only rounding noise and cannot be its
    own scale."""
    worst = 0.0
    for g in GROUPS:
        sc = np.abs(ref[g]).max()
        sc = sc if sc > 0 else 1.0
        worst = max(worst, float(np.abs(a[g] - ref[g]).max() / sc))
    return worst


# ---------------------------------------------------------------------------
def random_states(rng, n, jump=0.5, grad=2.0, gamma=1.4):
    """Seeded face-frame state pairs (W, dW/dn, dW/dt1, dW/dt2)."""
    def one(base=None):
        if base is None:
            rho = rng.uniform(0.3, 3.0, n)
            vel = rng.uniform(-2.0, 2.0, (3, n))
            p = rng.uniform(0.3, 3.0, n)
        else:
            rho0, vel0, p0 = base
            rho = rho0 * np.exp(rng.uniform(-jump, jump, n))
            vel = vel0 + rng.uniform(-jump, jump, (3, n))
            p = p0 * np.exp(rng.uniform(-jump, jump, n))
        dprim = rng.normal(scale=grad, size=(3, 5, n))
        S = np.zeros((20, n))
        S[0] = rho
        S[1:4] = rho * vel
        S[4] = p / (gamma - 1) + 0.5 * rho * (vel ** 2).sum(0)
        for j in range(3):
            dr, du, dv, dw, dp = dprim[j]
            dvel = np.stack([du, dv, dw])
            S[5 + 5 * j + 0] = dr
            S[5 + 5 * j + 1:5 + 5 * j + 4] = vel * dr + rho * dvel
            S[5 + 5 * j + 4] = dp / (gamma - 1) + 0.5 * (vel ** 2).sum(0) * dr + rho * (vel * dvel).sum(0)
        return S, (rho, vel, p)

    sl, base = one()
    sr, _ = one(base)
    return sl, sr


FLUX_CASES = [
    dict(name="viscous", kw=dict(mu=1e-3), dt=1e-3),
    dict(name="viscous-sutherland", kw=dict(mu=2e-3, mu_law=1, T_ref=0.7), dt=2e-3),
    dict(name="inviscid", kw=dict(inviscid=True), dt=5e-3),
    dict(name="tau-zero", kw=dict(inviscid=True, eps_tau=0.0, C_tau=0.0), dt=5e-3),
    dict(name="large-tau", kw=dict(mu=0.5), dt=1e-3),
    dict(name="monatomic", kw=dict(gamma=5.0 / 3.0, mu=1e-3, Pr=2.0 / 3.0), dt=1e-3),
]


@pytest.mark.parametrize("case", FLUX_CASES, ids=[c["name"] for c in FLUX_CASES])
def test_flux_points_match_oracle(torch_dev, case):
    torch, dev = torch_dev
    rng = np.random.default_rng(hash(case["name"]) % 2 ** 32)
    gamma = case["kw"].get("gamma", 1.4)
    n = 300
    sl, sr = random_states(rng, n, gamma=gamma)
    sl[:, :20] = sr[:, :20]  # a few continuous states (l = r)
    grid = wl.Grid((4, 4, 4), (1.0, 1.0, 1.0))
    s = solver(torch_dev, grid, scheme="cgks5", **case["kw"])
    dt = torch.tensor([case["dt"]], dtype=torch.float64, device=dev)
    out = s.flux_points(torch.tensor(sl, device=dev), torch.tensor(sr, device=dev), dt)
    got = out.cpu().numpy()
    P = oparams(grid, scheme="cgks5", **case["kw"])
    ref = np.stack([oracle.flux_gp(P, sl[:, i], sr[:, i], case["dt"]) for i in range(n)], axis=1)
    err = rel_err(got, ref, 1)
    assert err < TOL, err
    assert s.status() == 0


def run_parity(torch_dev, Q, G, grid, steps, **kw):
    torch, dev = torch_dev
    s = solver(torch_dev, grid, **kw)
    cg = kw["scheme"] == "cgks5"
    Qd = torch.tensor(Q, device=dev)
    Gd = torch.tensor(G, device=dev) if cg else None
    s.step(Qd, Gd, nsteps=steps)
    Qo, Go = Q.copy(), (G.copy() if cg else None)
    oracle.run(oparams(grid, **kw), Qo, Go, nsteps=steps)
    eq = state_err(Qd.cpu().numpy(), Qo)
    eg = state_err(Gd.cpu().numpy(), Go) if cg else 0.0
    return eq, eg, s


def test_flux_points_empty_input(torch_dev):
    """No Gauss points: the call succeeds without work (empty tensors,
    whose data pointers may be null)."""
    torch, dev = torch_dev
    Q, G, grid = wl.taylor_green(4)
    s = solver(torch_dev, grid, scheme="cgks5")
    empty = torch.zeros(20, 0, dtype=torch.float64, device=dev)
    dt = torch.full((1,), 1e-3, dtype=torch.float64, device=dev)
    out = s.flux_points(empty, empty.clone(), dt)
    assert out.shape == (30, 0)
    assert s.status() == 0


@pytest.mark.parametrize("scheme", ["gks2", "cgks5"])
def test_face_states_match_oracle(torch_dev, scheme):
    torch, dev = torch_dev
    Q, G, grid = wl.taylor_green((9, 8, 7))
    Q, G = wl.perturb(Q, G, amp=0.02, seed=3)
    for nonlinear in (False, True):
        s = solver(torch_dev, grid, scheme=scheme, nonlinear=nonlinear)
        cg = scheme == "cgks5"
        fs = s.reconstruct(torch.tensor(Q, device=dev), torch.tensor(G, device=dev) if cg else None)
        ref = oracle.face_states(oparams(grid, scheme=scheme, nonlinear=nonlinear), Q, G if cg else None)
        got = fs.cpu().numpy()
        # scale per (face, component)
        err = rel_err(got.transpose(0, 2, 1, 3).reshape(6, 20, -1),
                      ref.transpose(0, 2, 1, 3).reshape(6, 20, -1), 2)
        assert err < TOL, (nonlinear, err)


@pytest.mark.parametrize("scheme", ["gks2", "cgks5"])
def test_face_fluxes_match_oracle(torch_dev, scheme):
    torch, dev = torch_dev
    Q, G, grid = wl.taylor_green((8, 8, 8))
    Q, G = wl.perturb(Q, G, amp=0.02, seed=4)
    cg = scheme == "cgks5"
    P = oparams(grid, scheme=scheme, nonlinear=True)
    fs = oracle.face_states(P, Q, G if cg else None)
    dt = 0.01
    _, _, faces = oracle.stage(P, Q, G if cg else None, dt)
    s = solver(torch_dev, grid, scheme=scheme, nonlinear=True)
    got = s.flux(torch.tensor(fs, device=dev), torch.tensor([dt], dtype=torch.float64, device=dev))
    got = got.cpu().numpy()
    nq = 30 if cg else 10
    err = rel_err(got[:, :nq], faces[:, :nq], 2)
    assert err < TOL, err


def test_time_step_matches_oracle(torch_dev):
    torch, dev = torch_dev
    Q, G, grid = wl.taylor_green((10, 12, 6))
    Q, G = wl.perturb(Q, G, amp=0.05, seed=5)
    for kw in (dict(mu=1.0 / 1600), dict(mu=0.2), dict(inviscid=True), dict(mu=0.05, mu_law=1)):
        s = solver(torch_dev, grid, scheme="gks2", **kw)
        dt = s.compute_dt(torch.tensor(Q, device=dev)).item()
        ref = oracle.dt(oparams(grid, scheme="gks2", **kw), Q)
        assert dt == pytest.approx(ref, rel=1e-14), kw


@pytest.mark.parametrize("scheme,nonlinear", [("gks2", True), ("gks2", False), ("cgks5", False),
                                              ("cgks5", True)])
def test_tgv16_twenty_steps_match_oracle(torch_dev, scheme, nonlinear):
    """The parity gate: Taylor-Green vortex 16^3, Ma 0.1, Re 1600, Pr 0.72,
    CFL 0.3, FP64, 20 steps, within 1e-11, for both schemes, linear (as the
    subsonic case of Sec. 4.1 runs them) and nonlinear (GKS-2nd with its
    limiter, CGKS-5th with GENO)."""
    Q, G, grid = wl.taylor_green(16)
    eq, eg, s = run_parity(torch_dev, Q, G, grid, 20, scheme=scheme, nonlinear=nonlinear)
    assert eq < TOL and eg < TOL, (eq, eg)
    assert s.status() == 0


@pytest.mark.parametrize("scheme", ["gks2", "cgks5"])
def test_linear_variant_and_ragged_grid_match_oracle(torch_dev, scheme):
    Q, G, grid = wl.taylor_green((7, 9, 11))
    Q, G = wl.perturb(Q, G, amp=0.03, seed=6)
    for nonlinear in (False, True):
        eq, eg, _ = run_parity(torch_dev, Q, G, grid, 3, scheme=scheme, nonlinear=nonlinear)
        assert eq < TOL and eg < TOL, (nonlinear, eq, eg)


@pytest.mark.parametrize("n", [(1, 1, 1), (2, 3, 1), (3, 2, 2)])
@pytest.mark.parametrize("scheme", ["gks2", "cgks5"])
def test_grids_smaller_than_the_stencil_match_oracle(torch_dev, scheme, n):
    """Periodic grids with fewer cells per axis than the stencil spans: the
    face and edge neighbours alias onto the same cells (on 1 x 1 x 1 every
    neighbour is the cell itself); nonlinear, 3 steps within 1e-11."""
    Q, G, grid = wl.taylor_green(n)
    Q, G = wl.perturb(Q, G, amp=0.03, seed=11)
    eq, eg, s = run_parity(torch_dev, Q, G, grid, 3, scheme=scheme, nonlinear=True)
    assert eq < TOL and eg < TOL, (eq, eg)
    assert s.status() == 0
    # the mixed-precision kernels on the same aliasing stencils: within the
    # mixed path's stated bound (1e-5) of the FP64 oracle
    eq, eg, s = run_parity(torch_dev, Q, G, grid, 3, scheme=scheme, nonlinear=True,
                           precision="mixed")
    assert eq < 1e-5 and eg < 1e-5, (eq, eg)
    assert s.status() == 0


@pytest.mark.parametrize("scheme", ["gks2", "cgks5"])
def test_step_on_host_buffers_equals_device_step(torch_dev, scheme):
    """gks_step_host (state in pinned host memory, copied by the library)
    gives the bits of gks_step on device buffers, including the time
    control (the last step clamped to t_stop, then no-op steps)."""
    torch, dev = torch_dev
    Q, G, grid = wl.taylor_green((12, 10, 8))
    Q, G = wl.perturb(Q, G, amp=0.02, seed=8)
    cg = scheme == "cgks5"
    s = solver(torch_dev, grid, scheme=scheme)
    Qd = torch.tensor(Q, device=dev)
    Gd = torch.tensor(G, device=dev) if cg else None
    t = torch.zeros(1, dtype=torch.float64, device=dev)
    dt0 = s.compute_dt(Qd).item()
    t_stop = 2.5 * dt0
    s.step(Qd, Gd, nsteps=4, t_stop=t_stop, t=t)
    s2 = solver(torch_dev, grid, scheme=scheme)
    Qp = torch.tensor(Q).pin_memory()
    Gp = torch.tensor(G).pin_memory() if cg else None
    th = s2.step_host(Qp, Gp, nsteps=4, t_stop=t_stop, t=0.0)
    assert th == t.item() and abs(th - t_stop) <= 1e-15 * t_stop
    assert np.array_equal(Qp.numpy(), Qd.cpu().numpy())
    if cg:
        assert np.array_equal(Gp.numpy(), Gd.cpu().numpy())
    s2.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_linear_cgks_taylor_green_energy_decays(torch_dev, precision):
    """The linear CGKS-5th (the paper's choice for the subsonic vortex,
    Sec. 4.1) over 1500 steps of the Taylor-Green vortex at 32^3 (t ~ 8):
    the kinetic energy never rises by more than 1e-6 of itself between
    samples 100 steps apart (viscous decay; the weakly compressible flow
    moves a little energy back and forth). With unit least-squares weights
    in Eq. compact-big-5 a grid-scale mode grew after ~1000 steps and the
    energy rose to many times its initial value."""
    torch, dev = torch_dev
    Q, G, grid = wl.taylor_green(32)
    s = solver(torch_dev, grid, scheme="cgks5", nonlinear=False, precision=precision)
    Qd, Gd = torch.tensor(Q, device=dev), torch.tensor(G, device=dev)
    ek = [s.diagnostics(Qd, Gd)[0]]
    for _ in range(15):
        s.step(Qd, Gd, nsteps=100)
        ek.append(s.diagnostics(Qd, Gd)[0])
    ek = np.array(ek)
    assert np.all(ek[1:] <= ek[:-1] * (1 + 1e-6)), ek
    assert ek[-1] < 0.9 * ek[0], ek
    s.close()


@pytest.mark.parametrize("scheme", ["gks2", "cgks5"])
def test_sod_tube_matches_oracle(torch_dev, scheme):
    """Quasi-1D grid (ny = nz = 1), discontinuous data, inviscid collision
    time: exercises the limiter / GENO weights and the numerical part of
    tau; 10 steps."""
    Q, G, grid = wl.double_sod(64)
    eq, eg, _ = run_parity(torch_dev, Q, G, grid, 10, scheme=scheme, nonlinear=True,
                           inviscid=True, Pr=1.0)
    assert eq < TOL and eg < TOL, (eq, eg)


@pytest.mark.parametrize("scheme", ["cgks5", "gks2"])
def test_supersonic_tgv_sutherland_matches_oracle(torch_dev, scheme):
    """Sec. 4.2's supersonic Taylor-Green vortex (Ma 2, Re 1600, Pr 0.7,
    Sutherland viscosity), both nonlinear schemes, 12^3, 4 steps."""
    Q, G, grid = wl.taylor_green_supersonic(12)
    U0 = math.sqrt(1.4) * 2.0
    eq, eg, _ = run_parity(torch_dev, Q, G, grid, 4, scheme=scheme, nonlinear=True,
                           mu=U0 / 1600, mu_law=1, Pr=0.7)
    assert eq < TOL and eg < TOL, (eq, eg)


def test_gks2_taylor_green_dissipation_onset(torch_dev):
    """Sec. 4.1's dissipation rate at t = 0 on the GPU path (parity-proven
    against the oracle above): GKS-2nd, linear as the paper runs it, 128^3;
    -dE_k/dt(0) from the quadratic through E_k after 0..3 steps equals
    mu <|omega|^2> = 0.75 mu0 within 5% (the second-order scheme's own
    dissipation adds 6% at 128^3 and, falling like h^2, under 2% at 256^3)."""
    torch, dev = torch_dev
    Q, G, grid = wl.taylor_green(256)
    s = solver(torch_dev, grid, scheme="gks2", nonlinear=False)
    Qd = torch.tensor(Q, device=dev)
    t = torch.zeros(1, dtype=torch.float64, device=dev)
    ts, E = [0.0], [s.diagnostics(Qd)[0]]
    for _ in range(3):
        s.step(Qd, None, nsteps=1, t=t)
        ts.append(float(t.item()))
        E.append(s.diagnostics(Qd)[0])
    rate = -np.polyfit(ts, E, 2)[1]
    assert rate == pytest.approx(0.75 / 1600, rel=0.05), rate / (0.75 / 1600)


def test_diagnostics_match_oracle(torch_dev):
    torch, dev = torch_dev
    Q, G, grid = wl.taylor_green((12, 10, 8))
    Q, G = wl.perturb(Q, G, amp=0.02, seed=8)
    for scheme in ("cgks5", "gks2"):
        s = solver(torch_dev, grid, scheme=scheme, mu=1e-3, mu_law=1)
        cg = scheme == "cgks5"
        d = s.diagnostics(torch.tensor(Q, device=dev), torch.tensor(G, device=dev) if cg else None)
        ref = oracle.diagnostics(oparams(grid, scheme=scheme, mu=1e-3, mu_law=1), Q, G if cg else None)
        np.testing.assert_allclose(d, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("scheme", ["gks2", "cgks5"])
def test_uniform_flow_is_bitwise_steady_on_gpu(torch_dev, scheme):
    torch, dev = torch_dev
    grid = wl.Grid((6, 5, 4), (1.0, 1.3, 0.7))
    Q = np.zeros((5, 4, 5, 6))
    Q[0], Q[1], Q[2], Q[3] = 1.3, 0.2, -0.3, 0.1
    Q[4] = 0.9 / 0.4 + 0.5 * (0.2 ** 2 + 0.3 ** 2 + 0.1 ** 2) / 1.3
    G = np.zeros((5, 3, 4, 5, 6))
    s = solver(torch_dev, grid, scheme=scheme, mu=1e-3)
    Qd, Gd = torch.tensor(Q, device=dev), torch.tensor(G, device=dev)
    s.step(Qd, Gd if scheme == "cgks5" else None, nsteps=3)
    assert np.array_equal(Qd.cpu().numpy(), Q)
    assert np.array_equal(Gd.cpu().numpy(), G)


def test_conservation_on_gpu(torch_dev):
    torch, dev = torch_dev
    Q, G, grid = wl.taylor_green((16, 12, 8))
    Q, G = wl.perturb(Q, G, amp=0.05, seed=9)
    s = solver(torch_dev, grid, scheme="cgks5")
    Qd, Gd = torch.tensor(Q, device=dev), torch.tensor(G, device=dev)
    s0 = [math.fsum(Q[v].ravel()) for v in range(5)]
    s.step(Qd, Gd, nsteps=4)
    Qn = Qd.cpu().numpy()
    s1 = [math.fsum(Qn[v].ravel()) for v in range(5)]
    scale = [math.fsum(np.abs(Qn[v]).ravel()) for v in range(5)]
    for a, b, c in zip(s0, s1, scale):
        assert abs(a - b) <= 4e-13 * c


def test_time_control_and_argument_errors(torch_dev):
    torch, dev = torch_dev
    from paper_2508_19911_gb300 import gks
    Q, G, grid = wl.taylor_green(8)
    s = solver(torch_dev, grid, scheme="cgks5")
    Qd, Gd = torch.tensor(Q, device=dev), torch.tensor(G, device=dev)
    t = torch.zeros(1, dtype=torch.float64, device=dev)
    # stop exactly at t_stop, then further steps are no-ops
    dt0 = s.compute_dt(Qd).item()
    s.step(Qd, Gd, nsteps=5, t_stop=1.5 * dt0, t=t)
    assert t.item() == pytest.approx(1.5 * dt0, rel=1e-15)
    Qc, Gc = Qd.clone(), Gd.clone()
    s.step(Qd, Gd, nsteps=3, t_stop=1.5 * dt0, t=t)
    assert torch.equal(Qc, Qd) and torch.equal(Gc, Gd)
    s.step(Qd, Gd, nsteps=0)
    assert torch.equal(Qc, Qd)
    with pytest.raises(gks.GksError) as e:
        s.step(Qd, None, nsteps=1)
    assert e.value.code == gks.GKS_ERR_ARG
    # a non-physical state raises through the status word, without a fault
    Qbad = Qd.clone()
    Qbad[0, 0, 0, 0] = -1.0
    with pytest.raises(gks.GksError) as e:
        s.step(Qbad, Gd.clone(), nsteps=1)
    assert e.value.code == gks.GKS_ERR_NONPHYSICAL
    s.status()  # clears
