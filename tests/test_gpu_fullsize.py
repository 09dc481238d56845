"""Parity at the benchmark's full sizes (Taylor-Green 128^3 and 256^3,
CGKS-5th, in the launch configuration the benchmark times): sampled
outputs that the oracle computes one by one, and properties that hold at
any size.

After two GPU steps (a generic state), for a few hundred sampled cells
including the corners where the stencils wrap around the periodic box:
the face states of the reconstruction kernel against the oracle's
reconstruction of those cells; the face records of the flux kernel against
the oracle's flux on the same face states; the time step against the
oracle's; and conservation of the cell-average sums over a step.
Face records are compared the way they enter the update (Sec. 3.4, Eq.
deri-t-f): F^n dt + F_t dt^2/2 and Q + dQ/dt dt, so an error in F_t is
weighted by dt/2 against the scale of F^n and one in dQ/dt by dt against
the scale of Q, each over the groups density, momentum, energy (the
grouped parity metric). Bounds: FP64 1e-11; the mixed path 1e-5, its
FP32-level bound (the face states are FP32 offsets)."""
import numpy as np
import pytest

import oracle
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


def sample_cells(n, m, seed):
    nx, ny, nz = n
    corners = [i + nx * (j + ny * k) for i in (0, nx - 1) for j in (0, ny - 1) for k in (0, nz - 1)]
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([corners, rng.choice(nx * ny * nz, m, replace=False)]))


def left_of(c, d, n):
    nx, ny, nz = n
    i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
    if d == 0:
        i = (i - 1) % nx
    elif d == 1:
        j = (j - 1) % ny
    else:
        k = (k - 1) % nz
    return i + nx * (j + ny * k)


def to_face_frame_values(fs_cols, Qh_cols, mixed):
    """Mixed face states hold FP32 offsets from the cell's FP64 average:
    restore W = Q0 + offset (face-frame component c of variable v)."""
    out = fs_cols.astype(np.float64)
    if mixed:
        for f in range(6):
            d = f // 2
            for c in range(5):
                v = c if c in (0, 4) else 1 + (d + c - 1) % 3
                out[f, :, c, :] += Qh_cols[v][None, :]
    return out


def scaled_err(a, b, axes):
    scale = np.abs(b).max(axis=axes, keepdims=True)
    return float(np.max(np.abs(a - b) / np.where(scale == 0, 1.0, scale)))


def record_err(got, want, dt):
    """max over the record blocks and groups of the update-weighted error:
    F^n, F_t dt/2 against the F^n scale; Q, dQ/dt dt against the Q scale."""
    g = got.reshape(-1, 6, 5)
    w = want.reshape(-1, 6, 5)
    worst = 0.0
    for gi in ([0], [1, 2, 3], [4]):
        for val, der in ((0, 1), (2, 3), (4, 5)):
            scale = np.abs(w[:, val, gi]).max()
            scale = scale if scale > 0 else 1.0
            fac = 0.5 * dt if val == 0 else dt
            worst = max(worst, np.abs(g[:, val, gi] - w[:, val, gi]).max() / scale,
                        fac * np.abs(g[:, der, gi] - w[:, der, gi]).max() / scale)
    return float(worst)


@pytest.mark.parametrize("N,precision", [(128, "fp64"), (128, "mixed"), (256, "mixed")])
def test_full_size_sampled_parity(env, N, precision):
    torch, dev, gks = env
    mixed = precision == "mixed"
    tol = 1e-5 if mixed else 1e-11
    Q, G, grid = wl.taylor_green(N)
    s = gks.Solver(gks.Config(n=grid.n, L=grid.L, scheme="cgks5", precision=precision))
    Qd, Gd = torch.tensor(Q, device=dev), torch.tensor(G, device=dev)
    del Q, G
    s.step(Qd, Gd, nsteps=2)
    Qh, Gh = Qd.cpu().numpy(), Gd.cpu().numpy()
    n = grid.n
    ncell = n[0] * n[1] * n[2]
    P = oracle.params(n=n, L=grid.L, mu0=1.0 / 1600, scheme=1, nonlinear=1)

    # time step
    dtd = s.compute_dt(Qd)
    dt_gpu = float(dtd.item())
    assert dt_gpu == pytest.approx(oracle.dt(P, Qh), rel=1e-13)

    # reconstruction: sampled cells
    cells = sample_cells(n, 300, seed=N)
    fs = s.reconstruct(Qd, Gd)
    idx = torch.tensor(cells, device=dev)
    Qflat = Qh.reshape(5, ncell)
    own = to_face_frame_values(fs[..., idx].cpu().numpy(), Qflat[:, cells], mixed)
    ref = np.moveaxis(oracle.face_states_at(P, Qh, Gh, cells), 0, -1)  # [6][4][20][m]
    err_fs = scaled_err(own, ref, axes=(1, 3))
    assert err_fs < tol, err_fs

    # flux: the faces of the sampled cells, on the GPU's own face states
    frec = s.flux(fs, dtd, Q=Qd)
    got, want = [], []
    for d in range(3):
        lefts = np.array([left_of(c, d, n) for c in cells])
        li = torch.tensor(lefts, device=dev)
        sl = to_face_frame_values(fs[..., li].cpu().numpy(), Qflat[:, lefts], mixed)[2 * d + 1]
        sr = own[2 * d]
        rec = frec[d][:, idx].cpu().numpy()                  # [30][m]
        for m in range(cells.size):
            want.append(oracle.face_record(P, d, sl[:, :, m], sr[:, :, m], dt_gpu))
            got.append(rec[:, m])
    got, want = np.array(got), np.array(want)                  # [3m][30]
    err_fl = record_err(got, want, dt_gpu)
    assert err_fl < tol, err_fl

    # conservation over one more step (periodic box: sums move by rounding only)
    s0 = Qd.sum(dim=(1, 2, 3))
    a0 = Qd.abs().sum(dim=(1, 2, 3))
    s.step(Qd, Gd, nsteps=1)
    s1 = Qd.sum(dim=(1, 2, 3))
    drift = float(((s1 - s0).abs() / a0).max())
    assert drift < 1e-12, drift
    print(f"full size {N}^3 {precision}: face states {err_fs:.2e}, face records {err_fl:.2e}, "
          f"sum drift {drift:.2e}")
