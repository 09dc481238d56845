"""Pins of the oracle's non-periodic boundaries and stretched meshes
(Sec. 3.2, last paragraph: every cell mapped to one reference cell;
readings R15, R16).

* The Taylor-Green vortex is mirror-symmetric about the planes x, y, z = 0
  and pi (the normal velocity odd, everything else even), so the octant
  [0, pi]^3 with symmetry planes on all six sides must evolve exactly as
  the first octant of the periodic [0, 2 pi]^3 run, on a uniform and on a
  mirror-symmetric stretched mesh.
* A closed box of symmetry planes conserves mass and energy to round-off.
* A uniform flow parallel to the symmetry planes and through the outflow
  boundaries stays uniform bit for bit on a stretched mesh.
* Reference-cell mapping: a quartic in the index coordinates of a
  stretched mesh (cell i covers index values [i, i + 1], mapped linearly
  onto the physical cell) is reproduced exactly, values and physical
  derivatives; GKS-2nd reproduces linear ones.
"""
import math

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

from paper_2508_19911_gb300 import workloads

GX, GW = leggauss(4)


def _group_err(A, B):
    """Largest difference relative to each physical group's magnitude
    (density, momentum vector, energy; gradients with all three axes)."""
    groups = [[0], [1, 2, 3], [4]]
    worst = 0.0
    for g in groups:
        scale = np.abs(B[g]).max() + 1e-300
        worst = max(worst, np.abs(A[g] - B[g]).max() / scale)
    return worst


def _grad_err(GA, GB, QB, h):
    """Gradient differences against max|G| + max|Q|/h per group (Gauss's
    theorem: a gradient is interface values over h, so rounding of the
    values, not of the gradient, sets its noise)."""
    groups = [[0], [1, 2, 3], [4]]
    worst = 0.0
    for g in groups:
        scale = np.abs(GB[g]).max() + np.abs(QB[g]).max() / h
        worst = max(worst, np.abs(GA[g] - GB[g]).max() / scale)
    return worst


def _octant(Q, n):
    return Q[..., :n, :n, :n]


@pytest.mark.parametrize("scheme,nonlinear", [(1, 1), (0, 1), (1, 0)])
@pytest.mark.parametrize("stretch", [0.0, 0.3])
def test_octant_with_symmetry_planes_equals_the_periodic_vortex(orc, scheme, nonlinear, stretch):
    n, steps = 6, 3
    full_edges = workloads.stretched_edges(2 * n, 2 * np.pi, stretch)
    Qf, Gf, gf = workloads.taylor_green(edges=(full_edges,) * 3)
    Qo, Go, go = workloads.taylor_green(edges=(full_edges[:n + 1],) * 3)
    np.testing.assert_array_equal(Qo, _octant(Qf, n))
    sp_f = gf.spacing if stretch else (None,) * 3
    sp_o = go.spacing if stretch else (None,) * 3
    Pf = orc.params(n=gf.n, L=gf.L, scheme=scheme, nonlinear=nonlinear, spacing=sp_f)
    Po = orc.params(n=go.n, L=go.L, scheme=scheme, nonlinear=nonlinear, spacing=sp_o,
                    bc=(orc.BC_SYMMETRY,) * 3)
    Gf_ = Gf if scheme else None
    Go_ = Go if scheme else None
    tf, _ = orc.run(Pf, Qf, Gf_, nsteps=steps)
    to, _ = orc.run(Po, Qo, Go_, nsteps=steps)
    assert abs(tf - to) <= 1e-14 * tf
    assert _group_err(Qo, _octant(Qf, n)) < 1e-12
    if scheme:
        h = min(float(np.min(w)) for w in go.spacing)
        assert _grad_err(Go, _octant(Gf, n), Qo, h) < 1e-12


@pytest.mark.parametrize("scheme", [0, 1])
def test_closed_box_conserves_mass_and_energy(orc, scheme):
    n = 6
    edges = (workloads.stretched_edges(n, np.pi, 0.4), workloads.stretched_edges(n, np.pi, -0.2),
             np.linspace(0.0, np.pi, n + 1))
    Q, G, g = workloads.taylor_green(edges=edges, Ma=0.3)
    Q, G = workloads.perturb(Q, G, amp=1e-2, seed=3)
    P = orc.params(n=g.n, L=g.L, scheme=scheme, spacing=g.spacing, bc=(1, 1, 1))
    vol = np.einsum("k,j,i->kji", *[g.widths(a) for a in (2, 1, 0)])
    m0 = [np.sum(Q[v] * vol) for v in (0, 4)]
    orc.run(P, Q, G if scheme else None, nsteps=5)
    m1 = [np.sum(Q[v] * vol) for v in (0, 4)]
    for a, b in zip(m0, m1):
        assert abs(b - a) <= 1e-13 * abs(a)
    d = orc.diagnostics(P, Q, G if scheme else None)
    assert abs(d[5] - m1[0]) <= 1e-13 * m1[0] and abs(d[9] - m1[1]) <= 1e-13 * m1[1]


@pytest.mark.parametrize("scheme", [0, 1])
def test_uniform_flow_along_the_walls_is_preserved_bitwise(orc, scheme):
    nx, ny, nz = 5, 6, 4
    edges = (workloads.stretched_edges(nx, 1.0, 0.5), workloads.stretched_edges(ny, 2.0, -0.4),
             np.linspace(0.0, 1.0, nz + 1))
    g = workloads.grid_from_edges(edges)
    rho, U, V, W, p = 1.3, 0.0, 0.4, -0.25, 0.9
    Q = np.zeros((5, nz, ny, nx))
    Q[0], Q[1], Q[2], Q[3] = rho, rho * U, rho * V, rho * W
    Q[4] = p / 0.4 + 0.5 * rho * (U * U + V * V + W * W)
    G = np.zeros((5, 3, nz, ny, nx))
    Q0 = Q.copy()
    # x: symmetry planes (no normal velocity); y: outflow; z: periodic
    P = orc.params(n=g.n, L=g.L, scheme=scheme, spacing=g.spacing, bc=(1, 2, 0), mu0=1e-2)
    orc.run(P, Q, G if scheme else None, nsteps=3)
    np.testing.assert_array_equal(Q, Q0)
    if scheme:
        assert np.all(G == 0.0)


def _index_poly_fields(rng, n, spacing, deg):
    """Cell averages and physical cell-averaged gradients of random
    polynomials of the index coordinates (cell i: index values [i, i + 1])."""
    expo = [(a, b, c) for a in range(deg + 1) for b in range(deg + 1 - a)
            for c in range(deg + 1 - a - b)]
    coef = rng.normal(size=(5, len(expo)))
    nodes = [np.arange(m)[:, None] + 0.5 + 0.5 * GX[None, :] for m in n]

    def avg1(ax, e):  # 1D average of s^e over each index cell
        return (nodes[ax] ** e * GW[None, :]).sum(axis=1) * 0.5

    Q = np.zeros((5, n[2], n[1], n[0]))
    G = np.zeros((5, 3, n[2], n[1], n[0]))
    for v in range(5):
        for (a, b, c), cf in zip(expo, coef[v]):
            Ax, Ay, Az = avg1(0, a), avg1(1, b), avg1(2, c)
            Q[v] += cf * np.einsum("k,j,i->kji", Az, Ay, Ax)
            if a:
                G[v, 0] += cf * a * np.einsum("k,j,i->kji", Az, Ay, avg1(0, a - 1) / spacing[0])
            if b:
                G[v, 1] += cf * b * np.einsum("k,j,i->kji", Az, avg1(1, b - 1) / spacing[1], Ax)
            if c:
                G[v, 2] += cf * c * np.einsum("k,j,i->kji", avg1(2, c - 1) / spacing[2], Ay, Ax)
    return expo, coef, Q, G


def _poly_at(expo, cf, x, deriv=None):
    s = 0.0
    for (a, b, c), v in zip(expo, cf):
        e = [a, b, c]
        if deriv is not None:
            if e[deriv] == 0:
                continue
            v = v * e[deriv]
            e[deriv] -= 1
        s += v * x[0] ** e[0] * x[1] ** e[1] * x[2] ** e[2]
    return s


@pytest.mark.parametrize("scheme,nonlinear,deg", [(1, 0, 4), (1, 1, 4), (0, 1, 1)])
def test_index_polynomials_are_reproduced_on_a_stretched_mesh(orc, scheme, nonlinear, deg):
    rng = np.random.default_rng(21 + scheme + 2 * nonlinear)
    n = (9, 8, 7)
    spacing = tuple(np.diff(workloads.stretched_edges(m, 1.0 + a, amp))
                    for a, (m, amp) in enumerate(zip(n, (0.45, -0.3, 0.2))))
    expo, coef, Q, G = _index_poly_fields(rng, n, spacing, deg)
    Q[0] += 10.0  # positive density and energy for GENO's floor (not needed otherwise)
    Q[4] += 10.0
    P = orc.params(n=n, L=tuple(float(s.sum()) for s in spacing), scheme=scheme,
                   nonlinear=nonlinear, spacing=spacing)
    cells = [(i, j, k) for i in range(2, n[0] - 2) for j in range(2, n[1] - 2)
             for k in range(2, n[2] - 2)]
    ids = [(k * n[1] + j) * n[0] + i for i, j, k in cells]
    out = orc.face_states_at(P, Q, G if scheme else None, ids)
    ngp = 4 if scheme else 1
    g = 0.5 / math.sqrt(3)
    exp = np.zeros_like(out)
    for s, (i, j, k) in enumerate(cells):
        h = (spacing[0][i], spacing[1][j], spacing[2][k])
        for f in range(6):
            d = f // 2
            axes = [d, (d + 1) % 3, (d + 2) % 3]
            for kk in range(ngp):
                x = [i + 0.5, j + 0.5, k + 0.5]
                x[d] += 0.5 if f % 2 else -0.5
                if ngp == 4:
                    x[(d + 1) % 3] += g if kk & 1 else -g
                    x[(d + 2) % 3] += g if kk & 2 else -g
                for c in range(5):
                    v = 1 + axes[c - 1] if 1 <= c <= 3 else c
                    exp[s, f, kk, c] = _poly_at(expo, coef[v], x) + (10.0 if v in (0, 4) else 0.0)
                    for jj in range(3):
                        exp[s, f, kk, 5 + 5 * jj + c] = _poly_at(expo, coef[v], x, axes[jj]) / h[axes[jj]]
    vals, ders = exp[..., :5], exp[..., 5:]
    np.testing.assert_allclose(out[..., :5], vals, rtol=0, atol=1e-12 * np.abs(vals).max())
    np.testing.assert_allclose(out[..., 5:], ders, rtol=0, atol=1e-11 * np.abs(ders).max())
