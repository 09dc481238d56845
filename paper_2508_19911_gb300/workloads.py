"""Seeded synthetic initial data for the CGKS-5th / GKS-2nd hot path.

This module is input generation only: it builds cell averages Q and
cell-averaged gradients G of analytic initial conditions (numpy, host side)
and holds none of the method's arithmetic. Both the CUDA library's tests and
the CPU oracle consume its arrays.

Layouts (float64, C order, x fastest):
    Q [5][nz][ny][nx]      (rho, rho U, rho V, rho W, rho E)
    G [5][3][nz][ny][nx]   d/dx, d/dy, d/dz of each conserved variable

Every field below is a finite sum of separable products f(x) g(y) h(z), so
its cell average is a sum of products of 1D cell averages (6-point
Gauss-Legendre per cell, i.e. the 6x6x6 tensor rule evaluated exactly) and
its cell-averaged gradient follows from Gauss's theorem: the x-component is
(average over the +x face - average over the -x face)/h_x, which for a
separable term is (f(x_{i+1/2}) - f(x_{i-1/2}))/h_x times the 1D averages of
the other two factors.

Workloads:
  * Taylor-Green vortex (Sec. 4.1): on [0, 2 pi]^3, rho = 1 (or the paper's
    density), p = p0 + rho0 U0^2 (cos 2x + cos 2y)(cos 2z + 2)/16 with
    p0 = rho0 U0^2/(gamma Ma^2);
  * supersonic Taylor-Green vortex (Sec. 4.2);
  * smooth advection rho = 1 + 0.2 sin(x + y + z), U = V = W = 1, p = 1;
  * periodic double Sod tube on [0, 2] along x;
  * decaying isotropic turbulence (random solenoidal field with spectrum
    E(k) ~ k^4 exp(-2 (k/k0)^2), seeded phases), built spectrally;
  * a seeded cell-wise perturbation of any of the above.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GL_X, _GL_W = np.polynomial.legendre.leggauss(6)


@dataclass
class Grid:
    n: tuple[int, int, int]
    L: tuple[float, float, float]
    origin: tuple[float, float, float] = (0.0, 0.0, 0.0)
    # stretched mesh: the n[d] + 1 face coordinates of each axis (None:
    # uniform cells of size L/n)
    edges: tuple | None = None

    @property
    def h(self):
        return tuple(self.L[d] / self.n[d] for d in range(3))

    def faces(self, d):
        if self.edges is not None:
            return np.asarray(self.edges[d], dtype=float)
        return self.origin[d] + self.h[d] * np.arange(self.n[d] + 1)

    def widths(self, d):
        """Cell sizes along axis d."""
        if self.edges is not None:
            return np.diff(self.faces(d))
        return np.full(self.n[d], self.h[d])

    @property
    def spacing(self):
        """Per-axis cell sizes for a stretched mesh, else (None, None, None)."""
        if self.edges is None:
            return (None, None, None)
        return tuple(self.widths(d) for d in range(3))


def stretched_edges(n, length, amp, x0=0.0):
    """Face coordinates x(s) = x0 + length (s + amp sin(2 pi s)/(2 pi)),
    s = 0, 1/n, ..., 1: a smooth periodic stretching (|amp| < 1), cells
    (1 - amp)..(1 + amp) times the mean, mirror-symmetric about the middle."""
    s = np.arange(n + 1) / n
    return x0 + length * (s + amp * np.sin(2 * np.pi * s) / (2 * np.pi))


def grid_from_edges(edges):
    edges = tuple(np.asarray(e, dtype=float) for e in edges)
    n = tuple(len(e) - 1 for e in edges)
    L = tuple(float(e[-1] - e[0]) for e in edges)
    return Grid(n, L, tuple(float(e[0]) for e in edges), edges)


def _avg1(f, grid: Grid, d: int):
    """Cell averages of f along axis d (6-point Gauss-Legendre per cell)."""
    xf = grid.faces(d)
    lo, hi = xf[:-1], xf[1:]
    mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
    pts = mid[:, None] + half[:, None] * _GL_X[None, :]
    return (f(pts) * _GL_W[None, :]).sum(axis=1) * 0.5


def _dif1(f, grid: Grid, d: int):
    """(f(x_{i+1/2}) - f(x_{i-1/2}))/h_i along axis d."""
    xf = grid.faces(d)
    v = f(xf)
    if grid.edges is None:
        return (v[1:] - v[:-1]) / grid.h[d]
    return (v[1:] - v[:-1]) / grid.widths(d)


# A separable field is a list of (coef, fx, fy, fz) with fi callables.
def _one(x):
    return np.ones_like(x)


def _mul(a, b):
    out = []
    for ca, ax, ay, az in a:
        for cb, bx, by, bz in b:
            out.append((ca * cb,
                        (lambda x, f=ax, g=bx: f(x) * g(x)),
                        (lambda y, f=ay, g=by: f(y) * g(y)),
                        (lambda z, f=az, g=bz: f(z) * g(z))))
    return out


def _scale(a, s):
    return [(c * s, fx, fy, fz) for c, fx, fy, fz in a]


def _const(c):
    return [(c, _one, _one, _one)]


def _eval(terms, grid: Grid):
    """Cell averages and cell-averaged gradients of a separable field."""
    nx, ny, nz = grid.n
    avg = np.zeros((nz, ny, nx))
    grad = np.zeros((3, nz, ny, nx))
    for c, fx, fy, fz in terms:
        ax, ay, az = _avg1(fx, grid, 0), _avg1(fy, grid, 1), _avg1(fz, grid, 2)
        dx, dy, dz = _dif1(fx, grid, 0), _dif1(fy, grid, 1), _dif1(fz, grid, 2)
        avg += c * np.einsum("k,j,i->kji", az, ay, ax)
        grad[0] += c * np.einsum("k,j,i->kji", az, ay, dx)
        grad[1] += c * np.einsum("k,j,i->kji", az, dy, ax)
        grad[2] += c * np.einsum("k,j,i->kji", dz, ay, ax)
    return avg, grad


def _lines(terms, grid: Grid):
    """Line-averaged derivatives of a separable field, [12][nz][ny][nx]:
    entry 4a + k is (f(x_a + h_a/2) - f(x_a - h_a/2))/h_a along the line
    parallel to axis a through the cell at the tangential position of face
    Gauss point k (offsets +-h/(2 sqrt 3) from the cell centre on axes
    (a+1) % 3, bit 0 of k, and (a+2) % 3, bit 1)."""
    nx, ny, nz = grid.n
    gq = 0.5 / np.sqrt(3.0)
    out = np.zeros((12, nz, ny, nx))
    for c, fx, fy, fz in terms:
        f = (fx, fy, fz)
        for a in range(3):
            for k in range(4):
                parts = [None, None, None]
                parts[a] = _dif1(f[a], grid, a)
                for ax, bit in (((a + 1) % 3, k & 1), ((a + 2) % 3, k & 2)):
                    xf = grid.faces(ax)
                    mid = 0.5 * (xf[:-1] + xf[1:])
                    parts[ax] = f[ax](mid + (gq if bit else -gq) * grid.widths(ax))
                out[4 * a + k] += c * np.einsum("k,j,i->kji", parts[2], parts[1], parts[0])
    return out


def _conserved(grid, rho, u, v, w, p, gamma, lines=False):
    """Conserved separable fields from separable primitive fields; with
    lines=True also their line-averaged derivatives [5][12][...]."""
    mx, my, mz = _mul(rho, u), _mul(rho, v), _mul(rho, w)
    kin = _scale(_mul(rho, _mul(u, u) + _mul(v, v) + _mul(w, w)), 0.5)
    en = _scale(p, 1.0 / (gamma - 1.0)) + kin
    Q = np.zeros((5,) + tuple(reversed(grid.n)))
    G = np.zeros((5, 3) + tuple(reversed(grid.n)))
    L = np.zeros((5, 12) + tuple(reversed(grid.n))) if lines else None
    for q, terms in enumerate((rho, mx, my, mz, en)):
        Q[q], G[q] = _eval(terms, grid)
        if lines:
            L[q] = _lines(terms, grid)
    return (Q, G, L) if lines else (Q, G)


def taylor_green(n=16, *, Ma=0.1, gamma=1.4, rho0=1.0, U0=1.0, L=1.0,
                 rho_form="uniform", edges=None, lines=False):
    """Subsonic Taylor-Green vortex (Sec. 4.1) on [0, 2 pi L]^3.

    rho_form = "uniform": rho = rho0, p = p0 + rho0 U0^2/16 (...)(...);
    rho_form = "paper":   rho and p both scaled by 1 + gamma Ma^2/16 (...)(...).
    edges: face coordinates per axis (a stretched mesh or a sub-box such as
    the octant [0, pi L]^3 bounded by the vortex's symmetry planes); n is
    then ignored.
    """
    nn = (n, n, n) if np.isscalar(n) else tuple(n)
    grid = Grid(nn, (2 * np.pi * L,) * 3) if edges is None else grid_from_edges(edges)
    p0 = rho0 * U0 * U0 / (gamma * Ma * Ma)
    s, c = (lambda x: np.sin(x / L)), (lambda x: np.cos(x / L))
    c2 = lambda x: np.cos(2 * x / L)
    u = [(U0, s, c, c)]
    v = [(-U0, c, s, c)]
    w = [(0.0, _one, _one, _one)]
    fluct = [(1.0, c2, _one, c2), (2.0, c2, _one, _one), (1.0, _one, c2, c2), (2.0, _one, c2, _one)]
    if rho_form == "uniform":
        rho = _const(rho0)
        p = _const(p0) + _scale(fluct, rho0 * U0 * U0 / 16.0)
    elif rho_form == "paper":
        rel = _const(1.0) + _scale(fluct, gamma * Ma * Ma / 16.0)
        rho = _scale(rel, rho0)
        p = _scale(rel, p0)
    else:
        raise ValueError(rho_form)
    if lines:
        Q, G, Ls = _conserved(grid, rho, u, v, w, p, gamma, lines=True)
        return Q, G, grid, Ls
    Q, G = _conserved(grid, rho, u, v, w, p, gamma)
    return Q, G, grid


def taylor_green_supersonic(n=16, *, Ma=2.0, gamma=1.4, rho0=1.0, p0=1.0, L=1.0):
    """High-speed Taylor-Green vortex (Sec. 4.2): U0 = sqrt(gamma) Ma,
    rho and p scaled by 1 + (cos 2x + cos 2y)(cos 2z + 2)/16."""
    nn = (n, n, n) if np.isscalar(n) else tuple(n)
    grid = Grid(nn, (2 * np.pi * L,) * 3)
    U0 = np.sqrt(gamma) * Ma
    s, c = (lambda x: np.sin(x / L)), (lambda x: np.cos(x / L))
    c2 = lambda x: np.cos(2 * x / L)
    fluct = [(1.0, c2, _one, c2), (2.0, c2, _one, _one), (1.0, _one, c2, c2), (2.0, _one, c2, _one)]
    rel = _const(1.0) + _scale(fluct, 1.0 / 16.0)
    Q, G = _conserved(grid, _scale(rel, rho0), [(U0, s, c, c)], [(-U0, c, s, c)],
                      _const(0.0), _scale(rel, p0), gamma)
    return Q, G, grid


def advection(n=16, *, amp=0.2, gamma=1.4, vel=(1.0, 1.0, 1.0), p=1.0,
              dims=3, t=0.0, edges=None, lines=False):
    """rho = 1 + amp sin(x + y + z - (U + V + W) t) (dims = 3) or
    rho = 1 + amp sin(x + y - (U + V) t) on an n x n x 1 grid (dims = 2,
    W = 0, the z extent one cell of size 2 pi/n), uniform velocity and
    pressure; t > 0 gives the exact translated solution."""
    if dims == 2:
        grid = (Grid((n, n, 1), (2 * np.pi, 2 * np.pi, 2 * np.pi / n)) if edges is None
                else grid_from_edges(edges))
        vel = (vel[0], vel[1], 0.0)
        ph = -(vel[0] + vel[1]) * t
        s = lambda x: np.sin(x + ph)
        c = lambda x: np.cos(x + ph)
        sxyz = [(1.0, s, np.cos, _one), (1.0, c, np.sin, _one)]
    else:
        nn = (n, n, n) if np.isscalar(n) else tuple(n)
        grid = Grid(nn, (2 * np.pi,) * 3) if edges is None else grid_from_edges(edges)
        ph = -(vel[0] + vel[1] + vel[2]) * t
        s = lambda x: np.sin(x + ph)
        c = lambda x: np.cos(x + ph)
        sxyz = [(1.0, s, np.cos, np.cos), (1.0, c, np.sin, np.cos),
                (1.0, c, np.cos, np.sin), (-1.0, s, np.sin, np.sin)]
    rho = _const(1.0) + _scale(sxyz, amp)
    if lines:
        Q, G, Ls = _conserved(grid, rho, _const(vel[0]), _const(vel[1]), _const(vel[2]),
                              _const(p), gamma, lines=True)
        return Q, G, grid, Ls
    Q, G = _conserved(grid, rho, _const(vel[0]), _const(vel[1]), _const(vel[2]),
                      _const(p), gamma)
    return Q, G, grid


def double_sod(nx=200, *, gamma=1.4, high=(1.0, 1.0), low=(0.125, 0.1)):
    """Periodic double shock tube on [0, 2] along x (ny = nz = 1): the high
    state (rho, p) inside [0.5, 1.5], the low state outside, at rest.
    nx must be a multiple of 4 so that the jumps sit on cell faces."""
    if nx % 4:
        raise ValueError("nx must be a multiple of 4")
    h = 2.0 / nx
    grid = Grid((nx, 1, 1), (2.0, h, h))
    x = (np.arange(nx) + 0.5) * h
    inside = (x > 0.5) & (x < 1.5)
    rho = np.where(inside, high[0], low[0])
    p = np.where(inside, high[1], low[1])
    Q = np.zeros((5, 1, 1, nx))
    Q[0, 0, 0] = rho
    Q[4, 0, 0] = p / (gamma - 1.0)
    G = np.zeros((5, 3, 1, 1, nx))
    return Q, G, grid


def isotropic_turbulence(n=32, *, Mt=0.5, k0=8.0, seed=101, gamma=1.4,
                         rho0=1.0, c0=1.0):
    """Decaying compressible isotropic turbulence on [0, 2 pi]^3.

    Solenoidal velocity with energy spectrum E(k) = A k^4 exp(-2 (k/k0)^2),
    random phases from ``seed``, u_rms = Mt c0/sqrt(3), rho = rho0 and
    uniform temperature (p = rho0 c0^2/gamma). The field is built in Fourier
    space; its exact cell averages and cell-averaged gradients follow from
    the sinc factors of each mode. rho E uses the cell averages of the
    velocity (a definition of this synthetic initial condition).
    Returns Q, G, grid and a dict with u_rms and the Taylor microscale of
    the discrete field.
    """
    rng = np.random.default_rng(seed)
    h = 2 * np.pi / n
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    kk_safe = np.where(kk == 0, 1.0, kk)
    # random complex vector field, projected onto the solenoidal subspace
    a = rng.standard_normal((3, n, n, n)) + 1j * rng.standard_normal((3, n, n, n))
    kvec = np.stack([kx, ky, kz])
    a -= kvec * (np.sum(kvec * a, axis=0) / kk_safe ** 2)[None]
    spec = kk ** 4 * np.exp(-2.0 * (kk / k0) ** 2)
    # no energy in the Nyquist planes (their sign of k is ambiguous, which
    # would break the solenoidal projection of the real field)
    nyq = (np.abs(kx) >= n // 2) | (np.abs(ky) >= n // 2) | (np.abs(kz) >= n // 2)
    spec[nyq] = 0.0
    # amplitude so that the shell energy follows spec: |u_k|^2 ~ E(k)/(4 pi k^2)
    amp = np.sqrt(spec / (4 * np.pi * kk_safe ** 2))
    amp[kk == 0] = 0.0
    norm = np.sqrt(np.sum(np.abs(a) ** 2, axis=0))
    norm = np.where(norm == 0, 1.0, norm)
    uk = a / norm[None] * amp[None]
    # real field (take the real part of the inverse transform), then scale
    u = np.real(np.fft.ifftn(uk, axes=(1, 2, 3)))
    u -= u.mean(axis=(1, 2, 3), keepdims=True)
    urms_target = Mt * c0 / np.sqrt(3.0)
    u *= urms_target / np.sqrt(np.mean(u ** 2))
    uk = np.fft.fftn(u, axes=(1, 2, 3))
    # cell averages: multiply each mode by prod_d sinc(k_d h/2)
    sinc = lambda t: np.sinc(t / np.pi)
    filt = sinc(kx * h / 2) * sinc(ky * h / 2) * sinc(kz * h / 2)
    ubar = np.real(np.fft.ifftn(uk * filt[None], axes=(1, 2, 3)))
    # cell-averaged derivative along d: i k_d times the filter
    dbar = np.zeros((3, 3, n, n, n))
    for d, kd in enumerate((kx, ky, kz)):
        dbar[:, d] = np.real(np.fft.ifftn(uk * (1j * kd * filt)[None], axes=(1, 2, 3)))
    p0 = rho0 * c0 * c0 / gamma
    Q = np.zeros((5, n, n, n))
    G = np.zeros((5, 3, n, n, n))
    Q[0] = rho0
    for d in range(3):
        Q[1 + d] = rho0 * ubar[d]
        G[1 + d] = rho0 * dbar[d]
    Q[4] = p0 / (gamma - 1.0) + 0.5 * rho0 * np.sum(ubar ** 2, axis=0)
    for d in range(3):
        G[4, d] = rho0 * np.sum(ubar * dbar[:, d], axis=0)
    # Taylor microscale of the discrete (point) field: lambda^2 = <u^2>/<(du/dx)^2>
    dudx = np.real(np.fft.ifftn(1j * kx * uk[0]))
    lam_t = np.sqrt(np.mean(u[0] ** 2) / np.mean(dudx ** 2))
    grid = Grid((n, n, n), (2 * np.pi,) * 3)
    return Q, G, grid, {"u_rms": urms_target, "taylor_lambda": float(lam_t),
                        "p0": p0}


def double_shear_layer(nx=64, ny=64, *, amp=0.05, Ma=0.3, gamma=1.4, delta=np.pi / 15):
    """Periodic double shear layer on [0, 2 pi]^2 (nz = 1): U = tanh((y -
    pi/2)/delta) for y <= pi and tanh((3 pi/2 - y)/delta) above, V = amp
    sin x, rho = 1, p from Ma with U0 = 1."""
    h = 2 * np.pi / nx
    grid = Grid((nx, ny, 1), (2 * np.pi, 2 * np.pi, h))

    def u_of_y(y):
        return np.where(y <= np.pi, np.tanh((y - np.pi / 2) / delta),
                        np.tanh((3 * np.pi / 2 - y) / delta))

    p0 = 1.0 / (gamma * Ma * Ma)
    Q, G = _conserved(grid, _const(1.0), [(1.0, _one, u_of_y, _one)],
                      [(amp, np.sin, _one, _one)], _const(0.0), _const(p0), gamma)
    return Q, G, grid


def riemann_quadrants(nx=64, ny=64, *, states, amp=0.01, seed=0, gamma=1.4):
    """Periodic four-quadrant Riemann problem on [0, 1]^2 (nz = 1): states[q]
    = (rho, u, v, p) for the quadrants q = (x > 1/2) + 2 (y > 1/2), cell
    averages (the jumps sit on cell faces for even nx, ny) with a seeded
    cell-wise relative noise of amplitude amp on rho."""
    if nx % 2 or ny % 2:
        raise ValueError("nx, ny must be even")
    rng = np.random.default_rng(seed)
    grid = Grid((nx, ny, 1), (1.0, 1.0, 1.0 / nx))
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    q = (x[None, :] > 0.5).astype(int) + 2 * (y[:, None] > 0.5).astype(int)
    st = np.asarray(states, dtype=float)
    rho = st[q, 0] * (1.0 + amp * rng.uniform(-1, 1, q.shape))
    u, v, p = st[q, 1], st[q, 2], st[q, 3]
    Q = np.zeros((5, 1, ny, nx))
    Q[0, 0] = rho
    Q[1, 0] = rho * u
    Q[2, 0] = rho * v
    Q[4, 0] = p / (gamma - 1) + 0.5 * rho * (u * u + v * v)
    G = np.zeros((5, 3, 1, ny, nx))
    return Q, G, grid


def ensemble_instances(count=64, seed0=2000, sizes=(64, 128, 256, 512), max_rho_ratio=5.0):
    """Seeded ensemble of 2D instances: the first half periodic double shear
    layers (Ma 0.3, Re 1e4), the second half four-quadrant Riemann problems
    (inviscid collision time) with quadrant states drawn per seed
    (rho in [0.1, 1.5], p in [0.05, 1.5], u, v in [-1, 1]), drawn again from
    the same generator until the density ratio between the quadrants is at
    most ``max_rho_ratio`` (the scheme has no positivity limiter: unconstrained
    draws with ratios of 5.7 to 11 became non-physical within 20 steps); nx,
    ny drawn from ``sizes``, perturbation amplitude log-uniform in
    [1e-3, 1e-1]. Returns a list of (Q, G, grid, physics dict)."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        nx, ny = int(rng.choice(sizes)), int(rng.choice(sizes))
        amp = float(10 ** rng.uniform(-3, -1))
        if i < count // 2:
            Q, G, grid = double_shear_layer(nx, ny, amp=amp)
            phys = dict(mu=1.0 / 1e4, inviscid=False)
        else:
            while True:
                st = np.stack([rng.uniform(0.1, 1.5, 4), rng.uniform(-1, 1, 4),
                               rng.uniform(-1, 1, 4), rng.uniform(0.05, 1.5, 4)], axis=1)
                if st[:, 0].max() <= max_rho_ratio * st[:, 0].min():
                    break
            Q, G, grid = riemann_quadrants(nx, ny, states=st, amp=amp, seed=seed0 + i)
            phys = dict(mu=0.0, inviscid=True)
        out.append((Q, G, grid, phys))
    return out


def perturb(Q, G=None, *, amp=1e-2, seed=0):
    """Seeded cell-wise relative perturbation of every field (keeps rho and
    p positive for amp << 1). Returns new arrays."""
    rng = np.random.default_rng(seed)
    Qp = Q * (1.0 + amp * rng.uniform(-1.0, 1.0, Q.shape))
    Gp = None
    if G is not None:
        scale = np.abs(G).max(axis=(2, 3, 4), keepdims=True) + 1e-3
        Gp = G + amp * scale * rng.uniform(-1.0, 1.0, G.shape)
    return Qp, Gp
