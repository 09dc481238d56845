"""Pins of the oracle's reconstructions (Sec. 3.2 CGKS-5th, Sec. 3.3
GKS-2nd): exact reproduction of polynomials, GENO's misfit against an
independent constrained least-squares solve, chi on smooth and
discontinuous data, and the nonlinear weights' limits."""
import itertools
import math

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

FACE = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
EDGE = [(-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 1, 0), (-1, 0, -1), (1, 0, -1),
        (-1, 0, 1), (1, 0, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1), (0, 1, 1)]
GX, GW = leggauss(4)


class Poly:
    """Polynomial in physical coordinates relative to the target cell centre."""

    def __init__(self, coef):
        self.coef = coef  # dict (a, b, c) -> value

    def __call__(self, x, y, z):
        return sum(v * x ** a * y ** b * z ** c for (a, b, c), v in self.coef.items())

    def d(self, j):
        out = {}
        for e, v in self.coef.items():
            if e[j] > 0:
                e2 = list(e)
                e2[j] -= 1
                out[tuple(e2)] = out.get(tuple(e2), 0.0) + v * e[j]
        return Poly(out)


def random_poly(rng, deg, scale=1.0):
    coef = {}
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                coef[(a, b, c)] = rng.normal() * scale
    return Poly(coef)


def cell_avg(P, o, h):
    """Exact cell average (4-point Gauss-Legendre per axis) over the cell at
    integer offset o, cell sizes h."""
    xs = [(o[j] + 0.5 * GX) * h[j] for j in range(3)]
    X, Y, Z = np.meshgrid(*xs, indexing="ij")
    W = GW[:, None, None] * GW[None, :, None] * GW[None, None, :] / 8.0
    return float(np.sum(W * P(X, Y, Z)))


def data_vector(P, h):
    """The 63-entry CGKS-5th data vector of the target cell for a field P."""
    q0 = cell_avg(P, (0, 0, 0), h)
    d = np.zeros(63)
    for m, o in enumerate(FACE):
        d[m] = cell_avg(P, o, h) - q0
        for j in range(3):
            d[18 + 3 * m + j] = h[j] * cell_avg(P.d(j), o, h)
    for n, o in enumerate(EDGE):
        d[6 + n] = cell_avg(P, o, h) - q0
        ax = [j for j in range(3) if o[j] != 0]
        ez = [j for j in range(3) if o[j] == 0][0]
        da = h[ax[0]] * cell_avg(P.d(ax[0]), o, h)
        db = h[ax[1]] * cell_avg(P.d(ax[1]), o, h)
        d[36 + 2 * n] = (o[ax[0]] * da - o[ax[1]] * db) / math.sqrt(2)
        d[36 + 2 * n + 1] = h[ez] * cell_avg(P.d(ez), o, h)
    for j in range(3):
        d[60 + j] = h[j] * cell_avg(P.d(j), (0, 0, 0), h)
    return q0, d


def gauss_point(f, k):
    d = f // 2
    g = 0.5 / math.sqrt(3)
    x = [0.0, 0.0, 0.0]
    x[d] = 0.5 if f % 2 else -0.5
    x[(d + 1) % 3] = g if k & 1 else -g
    x[(d + 2) % 3] = g if k & 2 else -g
    return x


def expected_face_states(polys, h):
    """Face-frame states (value, d/dn, d/dt1, d/dt2) of five fields."""
    out = np.zeros((6, 4, 20))
    for f in range(6):
        d = f // 2
        axes = [d, (d + 1) % 3, (d + 2) % 3]
        for k in range(4):
            xn = gauss_point(f, k)
            xp = [xn[j] * h[j] for j in range(3)]
            for c in range(5):
                v = 1 + axes[c - 1] if 1 <= c <= 3 else c
                out[f, k, c] = polys[v](*xp)
                for j in range(3):
                    out[f, k, 5 + 5 * j + c] = polys[v].d(axes[j])(*xp)
    return out


@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (0.3, 0.5, 0.7)])
def test_linear_cgks_reproduces_quartics(orc, h):
    rng = np.random.default_rng(4)
    polys = [random_poly(rng, 4) for _ in range(5)]
    q0, d = zip(*[data_vector(P, h) for P in polys])
    out, chi = orc.recon5_cell(np.array(q0), np.concatenate(d), h, nonlinear=0)
    exp = expected_face_states(polys, h)
    scale = np.abs(exp).max()
    np.testing.assert_allclose(out, exp, rtol=0, atol=1e-11 * scale)
    assert np.all(chi == 1.0)


def test_nonlinear_cgks_reproduces_linear_data_with_chi_one(orc):
    rng = np.random.default_rng(8)
    h = (0.2, 0.25, 0.3)
    polys = [random_poly(rng, 1) for _ in range(5)]
    q0, d = zip(*[data_vector(P, h) for P in polys])
    out, chi = orc.recon5_cell(np.array(q0), np.concatenate(d), h, nonlinear=1)
    np.testing.assert_allclose(chi, 1.0, rtol=0, atol=1e-12)
    exp = expected_face_states(polys, h)
    np.testing.assert_allclose(out, exp, rtol=0, atol=1e-12 * np.abs(exp).max())


def test_nonlinear_cgks_reproduces_quartics_with_chi_one(orc):
    """Data sampled from any quartic are met exactly by P4 (the least-squares
    misfit is zero), so GENO keeps the linear reconstruction: chi = 1 to
    rounding and the face states are the quartic's own values and
    derivatives, for any cell aspect ratio."""
    rng = np.random.default_rng(14)
    h = (0.3, 0.5, 0.7)
    polys = [random_poly(rng, 4) for _ in range(5)]
    q0, d = zip(*[data_vector(P, h) for P in polys])
    out, chi = orc.recon5_cell(np.array(q0), np.concatenate(d), h, nonlinear=1)
    np.testing.assert_allclose(chi, 1.0, rtol=0, atol=1e-12)
    exp = expected_face_states(polys, h)
    np.testing.assert_allclose(out, exp, rtol=0, atol=1e-11 * np.abs(exp).max())


def test_chi_collapses_across_a_step(orc):
    """A jump between the target cell and its +x neighbours: chi -> 0 and
    the values stay within the data range (ENO-like behaviour)."""
    h = (1.0, 1.0, 1.0)
    step = Poly({})
    q0 = np.ones(5)
    d = np.zeros((5, 63))
    for m, o in enumerate(FACE):
        d[:, m] = 1.0 if o[0] > 0 else 0.0
    for n, o in enumerate(EDGE):
        d[:, 6 + n] = 1.0 if o[0] > 0 else 0.0
    out, chi = orc.recon5_cell(q0, d.ravel(), h, nonlinear=1)
    assert np.all(chi < 1e-2)
    vals = out[:, :, 0]
    assert vals.min() > 1.0 - 0.02 and vals.max() < 2.0 + 0.02


def _sine_data(hh):
    """Data vector of f = sin(1 + x + 2y + 3z) through its Taylor polynomial
    of degree 10 (exact to rounding on the 3x3x3 block for h <= 0.02)."""
    coef = {}
    for a in range(11):
        for b in range(11 - a):
            for c in range(11 - a - b):
                n = a + b + c
                coef[(a, b, c)] = math.sin(1 + n * math.pi / 2) * 2 ** b * 3 ** c / (
                    math.factorial(a) * math.factorial(b) * math.factorial(c))
    return data_vector(Poly(coef), (hh, hh, hh))


def test_geno_misfit_falls_with_the_eighth_power_of_h(orc):
    """The least-squares residual of a smooth field is its quintic Taylor
    remainder, O(h^4) relative to the derivative data, so the misfit sigma
    falls like h^8: halving h divides it by at least 2^7 (2^8 in the limit),
    and 1 - chi = O(sigma) is negligible on resolved smooth data."""
    sig = []
    for hh in (0.04, 0.02, 0.01):
        q0, d = _sine_data(hh)
        sig.append(orc.geno_misfit(np.full(5, q0), np.tile(d, 5))[0])
    r1, r2 = sig[0] / sig[1], sig[1] / sig[2]
    assert r1 > 2 ** 7 and r2 > 2 ** 7, (sig, r1, r2)
    _, chi = orc.recon5_cell(np.full(5, _sine_data(0.04)[0]), np.tile(_sine_data(0.04)[1], 5),
                             (0.04,) * 3, nonlinear=1)
    assert np.all(chi > 1.0 - 1e-7)  # 1 - chi ~ sigma/5e-4 = 8e-9 here


def test_geno_misfit_matches_an_independent_least_squares_solve(orc):
    """sigma = |W (B a - d_B)|^2 / (|d_C|^2 + |W d_B|^2 + (0.01 S)^2 + eps),
    with a the constrained least-squares quartic of Eq. compact-big-5 (row
    weights 1, 0.1 for the edge tangential derivatives, 1): here a comes from
    the KKT system built from the test's own rows, and S from the cell's
    magnitudes (rho; rho E; sqrt(rho rho E) for the momenta). Random data
    vectors with random magnitudes; a wrong weight, row, norm or floor fails."""
    C, WB, w = _ls_rows(0.1)
    n, m = 34, 18
    K = np.zeros((n + m, n + m))
    K[:n, :n] = WB.T @ WB
    K[:n, n:] = C.T
    K[n:, :n] = C
    rng = np.random.default_rng(21)
    for trial in range(4):
        q0 = np.array([rng.uniform(0.5, 2.0), rng.normal(), rng.normal(), rng.normal(),
                       rng.uniform(1.0, 5.0)])
        scale = 10.0 ** rng.uniform(-3, 0, 5)
        d = rng.normal(size=(5, 63)) * scale[:, None]
        got = orc.geno_misfit(q0, d.ravel())
        for v in range(5):
            dC, dB = d[v, :18], d[v, 18:]
            rhs = np.concatenate([WB.T @ (w * dB), dC])
            a = np.linalg.solve(K, rhs)[:n]
            res = WB @ a - w * dB
            S = q0[0] if v == 0 else q0[4] if v == 4 else math.sqrt(abs(q0[0] * q0[4]))
            sig = res @ res / (dC @ dC + (w * dB) @ (w * dB) + (0.01 * S) ** 2 + 1e-15)
            assert got[v] == pytest.approx(sig, rel=1e-9), (trial, v)


def test_chi_is_one_on_a_resolved_taylor_green_vortex(orc):
    """GENO keeps the high-order reconstruction where the flow is smooth and
    resolved (Sec. 3.2): on the Taylor-Green vortex with 64 cells per
    velocity wavelength, chi >= 1 - 1e-3 in every cell and variable,
    including the cells at its degenerate critical points (where the
    velocity is locally cubic, u ~ xyz)."""
    from paper_2508_19911_gb300 import workloads as wl
    Q, G, grid = wl.taylor_green(64)
    P = orc.params(n=grid.n, L=grid.L, scheme=1, nonlinear=1)
    chi = orc.chi_field(P, Q, G)
    assert chi.min() >= 1.0 - 1e-3, chi.min()


def _step_cells(normal, offset, n=10, s=12):
    """Cell averages and Gauss-theorem cell-averaged gradients (sub-cell
    midpoint sampling, s^3 per cell, s^2 per face) of the unit step
    H(normal . x - offset) on an n^3 grid with h = 1: the data a discontinuity
    leaves in a CGKS-5th state."""
    t = (np.arange(s) + 0.5) / s
    nv = np.asarray(normal, float)
    Q = np.zeros((n, n, n))
    G = np.zeros((3, n, n, n))
    f = lambda X, Y, Z: (nv[0] * X + nv[1] * Y + nv[2] * Z > offset).astype(float)
    for k in range(n):
        for j in range(n):
            for i in range(n):
                X, Y, Z = np.meshgrid(i + t, j + t, k + t, indexing="ij")
                Q[k, j, i] = f(X, Y, Z).mean()
                base = [i + t, j + t, k + t]
                for ax in range(3):
                    lo, hi = list(base), list(base)
                    lo[ax] = np.array([float([i, j, k][ax])])
                    hi[ax] = np.array([float([i, j, k][ax] + 1)])
                    G[ax, k, j, i] = (f(*np.meshgrid(*hi, indexing="ij")).mean() -
                                      f(*np.meshgrid(*lo, indexing="ij")).mean())
    return Q, G


@pytest.mark.parametrize("normal,offset", [((1, 0, 0), 5.3), ((1, 1, 0), 10.2),
                                           ((1, 1, 1), 15.1), ((1, 0.3, 0), 6.6)])
def test_chi_collapses_in_cells_a_discontinuity_cuts(orc, normal, offset):
    """GENO falls back to the sub-stencil reconstruction at a discontinuity
    (Sec. 3.2): a unit step in the density (on a uniform background) along
    a plane of several orientations. In every interior cell the plane cuts
    through its middle (centre within 0.3 h of the plane), chi <= 1e-3."""
    n = 10
    Qs, Gs = _step_cells(normal, offset, n)
    Q = np.zeros((5, n, n, n))
    G = np.zeros((5, 3, n, n, n))
    Q[0] = 1.0 + Qs
    G[0] = Gs
    Q[4] = 2.5
    P = orc.params(n=(n, n, n), L=(float(n),) * 3, scheme=1, nonlinear=1)
    chi = orc.chi_field(P, Q, G)[0].reshape(n, n, n)
    idx = np.arange(n) + 0.5
    K, J, I = np.meshgrid(idx, idx, idx, indexing="ij")
    nv = np.asarray(normal, float)
    dist = (nv[0] * I + nv[1] * J + nv[2] * K - offset) / np.linalg.norm(nv)
    inner = (I > 2) & (I < n - 2) & (J > 2) & (J < n - 2) & (K > 2) & (K < n - 2)
    cut = inner & (np.abs(dist) <= 0.3)
    assert cut.sum() >= 4
    assert chi[cut].max() <= 1e-3, chi[cut].max()


def test_gks2_reconstruction(orc):
    rng = np.random.default_rng(12)
    h = (0.5, 0.4, 0.3)
    # linear data: exact, limiter inactive
    polys = [random_poly(rng, 1) for _ in range(5)]
    q7 = np.zeros((7, 5))
    for v, P in enumerate(polys):
        q7[0, v] = cell_avg(P, (0, 0, 0), h)
        for m, o in enumerate(FACE):
            q7[m + 1, v] = cell_avg(P, o, h)
    for nl in (0, 1):
        out, phi = orc.recon2_cell(q7.ravel(), h, nonlinear=nl)
        np.testing.assert_allclose(phi, 1.0, rtol=0, atol=1e-12)
        for f in range(6):
            d = f // 2
            axes = [d, (d + 1) % 3, (d + 2) % 3]
            xf = [0.0, 0.0, 0.0]
            xf[d] = (0.5 if f % 2 else -0.5) * h[d]
            for c in range(5):
                v = 1 + axes[c - 1] if 1 <= c <= 3 else c
                assert out[f, c] == pytest.approx(polys[v](*xf), rel=1e-12, abs=1e-12)
                for j in range(3):
                    assert out[f, 5 + 5 * j + c] == pytest.approx(polys[v].d(axes[j])(0, 0, 0), rel=1e-11)
    # random data, linear variant: central-difference gradient
    q7 = rng.uniform(0.5, 1.5, (7, 5))
    out, _ = orc.recon2_cell(q7.ravel(), h, nonlinear=0)
    b = np.array([(q7[2] - q7[1]) / 2, (q7[4] - q7[3]) / 2, (q7[6] - q7[5]) / 2])  # [axis][var]
    assert out[1, 0] == pytest.approx(q7[0, 0] + 0.5 * b[0, 0], rel=1e-14)
    assert out[1, 5] == pytest.approx(b[0, 0] / h[0], rel=1e-13)
    # a step activates the limiter; with eps^2 = h^3 small against the jump
    # the face values stay (almost) inside the data range
    q7 = np.ones((7, 5))
    q7[2] = 3.0
    out, phi = orc.recon2_cell(q7.ravel(), (0.1, 0.1, 0.1), nonlinear=1)
    assert np.all(phi < 0.01)
    assert out[:, 0].max() <= 3.0 and out[:, 0].min() >= 0.99


# ---- the least-squares matrix of Eq. compact-big-5, from its definition ----
BASIS5 = [(i, j, d - i - j) for d in range(1, 5) for i in range(d, -1, -1)
          for j in range(d - i, -1, -1)]  # monomials by degree, x exponent first


def _mean1(o, n):
    """mean of t^n over [o - 1/2, o + 1/2]"""
    return ((o + 0.5) ** (n + 1) - (o - 0.5) ** (n + 1)) / (n + 1)


def _mean_mono(o, e):
    if min(e) < 0:
        return 0.0
    return (_mean1(o[0], e[0]) * _mean1(o[1], e[1]) * _mean1(o[2], e[2]) /
            (math.factorial(e[0]) * math.factorial(e[1]) * math.factorial(e[2])))


def _ls_rows(w_edge):
    """Constraint rows C (neighbour averages of the zero-mean basis) and the
    weighted derivative rows W B (face neighbours' gradients, the edge
    neighbours' two tangential derivatives, the own gradient), in the data
    order of the C-ABI's gks_recon_matrix."""
    def dmean(o, e, j):
        e2 = list(e)
        e2[j] -= 1
        return _mean_mono(o, e2)
    C = np.array([[_mean_mono(o, e) - _mean_mono((0, 0, 0), e) for e in BASIS5]
                  for o in FACE + EDGE])
    rows, w = [], []
    for o in FACE:
        for j in range(3):
            rows.append([dmean(o, e, j) for e in BASIS5])
            w.append(1.0)
    for o in EDGE:
        a, b = [j for j in range(3) if o[j]]
        ez = [j for j in range(3) if not o[j]][0]
        rows.append([(o[a] * dmean(o, e, a) - o[b] * dmean(o, e, b)) / math.sqrt(2)
                     for e in BASIS5])
        rows.append([dmean(o, e, ez) for e in BASIS5])
        w += [w_edge, w_edge]
    for j in range(3):
        rows.append([dmean((0, 0, 0), e, j) for e in BASIS5])
        w.append(1.0)
    return C, np.array(w)[:, None] * np.array(rows), np.array(w)


def test_recon_matrix_is_the_weighted_constrained_least_squares_solution(orc):
    """Eq. compact-big-5 with the row weights h1 = h3 = 1, h2 = 0.1 (edge
    tangential derivatives): for each data column, the quartic whose
    neighbour averages match exactly and whose weighted derivative residual
    is least. Solved here through its KKT system, independently of the
    oracle's elimination; a wrong weight, sign or row order fails."""
    C, WB, w = _ls_rows(0.1)
    n, m = 34, 18
    K = np.zeros((n + m, n + m))
    K[:n, :n] = WB.T @ WB
    K[:n, n:] = C.T
    K[n:, :n] = C
    R = np.zeros((34, 63))
    for col in range(63):
        rhs = np.zeros(n + m)
        if col < 18:
            rhs[n + col] = 1.0
        else:
            rhs[:n] = WB.T[:, col - 18] * w[col - 18]
        R[:, col] = np.linalg.solve(K, rhs)[:n]
    got = orc.recon5_matrix()
    assert np.abs(got - R).max() <= 1e-10 * np.abs(R).max(), np.abs(got - R).max()


def test_edge_weight_is_near_the_condition_number_minimum():
    """The reading of h2: the edge rows' weight 0.1 lies within 1% of the
    smallest 2-norm condition number of the weighted least-squares system
    on the null space of the exact constraints (weights of the other rows
    1), which unit weights exceed by more than 5x."""
    def cond(we):
        C, WB, _ = _ls_rows(we)
        _, s, vt = np.linalg.svd(C)
        Z = vt[np.sum(s > 1e-12):].T
        sv = np.linalg.svd(WB @ Z, compute_uv=False)
        return sv[0] / sv[-1]
    grid = np.linspace(0.02, 1.0, 99)
    best = min(cond(x) for x in grid)
    assert cond(0.1) <= 1.01 * best, (cond(0.1), best)
    assert cond(1.0) > 5 * cond(0.1)


def _vk_smooth_min(y, e):
    """Venkatakrishnan's limiter as the smooth minimum of (1, y) in the
    ratio y = Delta_+ / Delta_2 of the admissible to the unlimited
    increment, with the smoothing e = eps^2 / Delta_2^2:
    phi = (y^2 + 2 y + e) / (y^2 + y + 2 + e)."""
    return (y * y + 2.0 * y + e) / (y * y + y + 2.0 + e)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_venkatakrishnan_limiter_interior_values(orc, seed):
    """The limiter of Sec. 3.3 away from its limits: a cell with neighbours
    only along x (central gradient b = (q_+ - q_-)/2), so that the two x
    faces carry the unlimited increments +-b/2 and the admissible ones
    max - q0 and min - q0 (the y and z faces have none: phi = 1 there).
    phi0 = the smaller of the two faces' smooth minima, with eps^2 = h^3
    (reading R9); both signs of the increment are covered by each draw."""
    rng = np.random.default_rng(seed)
    for _ in range(5):
        h = 10.0 ** rng.uniform(-2.0, -0.3)
        a, b = rng.uniform(-1.0, 1.0, 2)
        q7 = np.zeros((7, 5))
        q7[1, :] = a        # -x neighbour
        q7[2, :] = b        # +x neighbour
        _, phi = orc.recon2_cell(q7.ravel(), (h, h, h), nonlinear=1)
        grad = 0.5 * (b - a)
        qmax, qmin = max(0.0, a, b), min(0.0, a, b)
        e2 = h ** 3
        want = 1.0
        for d2 in (0.5 * grad, -0.5 * grad):  # the +x and -x faces
            if d2 == 0.0:
                continue
            dp = qmax if d2 > 0 else qmin
            want = min(want, _vk_smooth_min(dp / d2, e2 / (d2 * d2)))
        np.testing.assert_allclose(phi, want, rtol=1e-13, atol=0)
