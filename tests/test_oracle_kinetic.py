"""Pins of the oracle's kinetic part (Sec. 2 of the paper) against
brute-force quadrature, closed forms and the Navier-Stokes limit.

None of these tests reuses the oracle's arithmetic: moments come from
velocity-space quadrature (tests/kinetic_quadrature.py), linear solves from
numpy, time integrals from Gauss-Legendre quadrature in t, and the
Navier-Stokes fluxes from the textbook Chapman-Enskog expressions.
"""
import math

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

from kinetic_quadrature import Maxwellian, apsi, psi


def cons(rho, U, V, W, p, gamma=1.4):
    return np.array([rho, rho * U, rho * V, rho * W,
                     p / (gamma - 1) + 0.5 * rho * (U * U + V * V + W * W)])


def cons_grad(prim, dprim, gamma=1.4):
    """Gradients of conserved variables from primitive gradients.
    prim = (rho, U, V, W, p); dprim[j] = d/dx_j of (rho, U, V, W, p)."""
    rho, U, V, W, p = prim
    out = np.zeros((3, 5))
    for j in range(3):
        dr, dU, dV, dW, dp = dprim[j]
        out[j] = [dr, U * dr + rho * dU, V * dr + rho * dV, W * dr + rho * dW,
                  dp / (gamma - 1) + 0.5 * (U * U + V * V + W * W) * dr
                  + rho * (U * dU + V * dV + W * dW)]
    return out


def euler_flux(Wc, j, gamma=1.4):
    """Euler flux along axis j of a conserved state (complex-safe)."""
    rho = Wc[0]
    vel = [Wc[1] / rho, Wc[2] / rho, Wc[3] / rho]
    p = (gamma - 1) * (Wc[4] - 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2))
    un = vel[j]
    F = [rho * un, Wc[1] * un, Wc[2] * un, Wc[3] * un, (Wc[4] + p) * un]
    F[1 + j] = F[1 + j] + p
    return np.array(F)


def jacobian(Wc, j, gamma=1.4):
    """Complex-step Jacobian dF_j/dW (exact to rounding)."""
    h = 1e-30
    J = np.zeros((5, 5))
    for k in range(5):
        Wp = Wc.astype(complex)
        Wp[k] += 1j * h
        J[:, k] = euler_flux(Wp, j, gamma).imag / h
    return J


def state(sl_W, dW):
    return np.concatenate([sl_W, dW[0], dW[1], dW[2]])


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0, 4.0 / 3.0])
@pytest.mark.parametrize("half", [0, 1, -1])
def test_moment_matrices_match_quadrature(orc, gamma, half):
    rng = np.random.default_rng(11)
    extras = [lambda u, v, w: 1.0, lambda u, v, w: u, lambda u, v, w: v,
              lambda u, v, w: w, lambda u, v, w: u * u, lambda u, v, w: u * v,
              lambda u, v, w: u * w]
    for _ in range(3):
        rho, p = rng.uniform(0.5, 2.0, 2)
        U, V, W = rng.uniform(-1.5, 1.5, 3)
        M = Maxwellian(cons(rho, U, V, W, p, gamma), gamma)
        for which, ex in enumerate(extras):
            G = orc.moment_matrix(U, V, W, M.lam, M.N, half, which)

            def fn(u, v, w, s, ex=ex):
                ps = psi(u, v, w, s)
                return ex(u, v, w) * ps[:, None] * ps[None, :]

            Gq = M.integrate(fn, half) / rho
            scale = np.abs(Gq).max()
            np.testing.assert_allclose(G, Gq, rtol=1e-11, atol=1e-12 * scale)


def test_slope_solves_moment_system(orc):
    rng = np.random.default_rng(5)
    for _ in range(5):
        prim = (rng.uniform(0.5, 2), *rng.uniform(-1, 1, 3), rng.uniform(0.5, 2))
        Wc = cons(*prim)
        dW = rng.normal(size=5)
        a = orc.slope(Wc, dW)
        M = Maxwellian(Wc)
        back = M.integrate(lambda u, v, w, s: apsi(a, u, v, w, s) * psi(u, v, w, s))
        np.testing.assert_allclose(back, dW, rtol=1e-11, atol=1e-12)


# ---------------------------------------------------------------------------
def test_uniform_equilibrium_gives_euler_flux(orc):
    rng = np.random.default_rng(2)
    for _ in range(4):
        prim = (rng.uniform(0.5, 2), *rng.uniform(-1, 1, 3), rng.uniform(0.5, 2))
        Wc = cons(*prim)
        s = state(Wc, np.zeros((3, 5)))
        P = orc.params(mu0=1e-3)
        out = orc.flux_gp(P, s, s, 1e-2)
        F = euler_flux(Wc, 0)
        np.testing.assert_allclose(out[:5], F, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(out[5:10], 0.0, atol=1e-10)
        for blk in (10, 20):
            np.testing.assert_allclose(out[blk:blk + 5], Wc, rtol=1e-14)
            np.testing.assert_allclose(out[blk + 5:blk + 10], 0.0, atol=1e-12)


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
@pytest.mark.parametrize("Pr", [1.0, 0.72])
def test_chapman_enskog_limit_is_navier_stokes(orc, gamma, Pr):
    """l = r smooth data, dt = 100 tau: F^n equals the Euler flux plus the
    BGK Navier-Stokes stress (bulk term 2/(N+3)) and Fourier heat flux
    c_p mu/Pr dT/dx; F_t^n and dQ/dt equal the Euler time derivatives."""
    rng = np.random.default_rng(7)
    N = (5 - 3 * gamma) / (gamma - 1)
    cp = gamma / (gamma - 1)
    for _ in range(4):
        prim = np.array([rng.uniform(0.6, 1.8), *rng.uniform(-0.8, 0.8, 3), rng.uniform(0.6, 1.8)])
        dprim = rng.normal(scale=0.3, size=(3, 5))
        Wc = cons(*prim, gamma=gamma)
        dW = cons_grad(prim, dprim, gamma)
        s = state(Wc, dW)
        mu = 1e-3
        rho, U, V, W, p = prim
        tau = mu / p
        P = orc.params(gamma=gamma, Pr=Pr, mu0=mu, C_tau=10.0)
        out = orc.flux_gp(P, s, s, 100 * tau)
        vel = np.array([U, V, W])
        du = dprim[:, 1:4].T  # du[i][j] = dU_i/dx_j
        div = np.trace(du)
        sig = mu * (du + du.T) - mu * 2.0 / (N + 3) * div * np.eye(3)
        T = p / rho
        dTdx = (dprim[0, 4] - T * dprim[0, 0]) / rho
        F = euler_flux(Wc, 0, gamma)
        F[1:4] -= sig[0]
        F[4] += -sig[0] @ vel - cp * mu / Pr * dTdx
        np.testing.assert_allclose(out[:5], F, rtol=1e-10, atol=1e-12)
        dtW = -sum(jacobian(Wc, j, gamma) @ dW[j] for j in range(3))
        for blk in (10, 20):
            np.testing.assert_allclose(out[blk:blk + 5], Wc, rtol=1e-13)
            np.testing.assert_allclose(out[blk + 5:blk + 10], dtW, rtol=1e-10, atol=1e-11)
        if Pr == 1.0:
            Ft = jacobian(Wc, 0, gamma) @ dtW
            np.testing.assert_allclose(out[5:10], Ft, rtol=1e-8, atol=1e-9)


# ---------------------------------------------------------------------------
def _brute_fbar(sl, sr, *, gamma, Pr, mu0, C, eps, inviscid, dt, T):
    """Eq. flux integrated over [0, T] by quadrature in velocity and time,
    with every slope solved from quadrature moment matrices."""
    Wl, Wr = sl[:5], sr[:5]
    dWl, dWr = sl[5:].reshape(3, 5), sr[5:].reshape(3, 5)
    Ml, Mr = Maxwellian(Wl, gamma), Maxwellian(Wr, gamma)

    def mmat(M, half=0):
        return M.integrate(lambda u, v, w, s: psi(u, v, w, s)[:, None] * psi(u, v, w, s)[None, :], half)

    def slopes(M, dW):
        return [np.linalg.solve(mmat(M) / M.rho, dW[j] / M.rho) for j in range(3)]

    def compat(M, a):
        rhs = M.integrate(lambda u, v, w, s: (apsi(a[0], u, v, w, s) * u + apsi(a[1], u, v, w, s) * v
                                              + apsi(a[2], u, v, w, s) * w) * psi(u, v, w, s))
        return np.linalg.solve(mmat(M), -rhs)

    al, ar = slopes(Ml, dWl), slopes(Mr, dWr)
    Al, Ar = compat(Ml, al), compat(Mr, ar)
    W0 = (Ml.integrate(lambda u, v, w, s: psi(u, v, w, s), +1)
          + Mr.integrate(lambda u, v, w, s: psi(u, v, w, s), -1))
    dW0 = np.array([Ml.integrate(lambda u, v, w, s: apsi(al[j], u, v, w, s) * psi(u, v, w, s), +1)
                    + Mr.integrate(lambda u, v, w, s: apsi(ar[j], u, v, w, s) * psi(u, v, w, s), -1)
                    for j in range(3)])
    M0 = Maxwellian(W0, gamma)
    ab = slopes(M0, dW0)
    Ab = compat(M0, ab)
    dpr = abs((Ml.p - Mr.p) / (Ml.p + Mr.p))
    tau = (eps * dt + C * dpr * dt) if inviscid else (mu0 / M0.p + C * dpr * dt)
    U0, V0, Wv0 = M0.U, M0.V, M0.Wv

    def heat(u, v, w, s):
        return 0.5 * (u - U0) * ((u - U0) ** 2 + (v - V0) ** 2 + (w - Wv0) ** 2 + s)

    def dirslope(a, u, v, w, s):
        return apsi(a[0], u, v, w, s) * u + apsi(a[1], u, v, w, s) * v + apsi(a[2], u, v, w, s) * w

    # each term of Eq. flux as (Maxwellian, half, polynomial factor)
    terms = [
        [(M0, 0, lambda u, v, w, s: 1.0)],
        [(M0, 0, lambda u, v, w, s: dirslope(ab, u, v, w, s))],
        [(M0, 0, lambda u, v, w, s: apsi(Ab, u, v, w, s))],
        [(Ml, +1, lambda u, v, w, s: 1.0), (Mr, -1, lambda u, v, w, s: 1.0)],
        [(Ml, +1, lambda u, v, w, s: dirslope(al, u, v, w, s)),
         (Mr, -1, lambda u, v, w, s: dirslope(ar, u, v, w, s))],
        [(Ml, +1, lambda u, v, w, s: apsi(Al, u, v, w, s)),
         (Mr, -1, lambda u, v, w, s: apsi(Ar, u, v, w, s))],
    ]
    X, Y, Z = [], [], []
    for parts in terms:
        x = y = z = 0.0
        for M, half, fac in parts:
            x = x + M.integrate(lambda u, v, w, s: u * fac(u, v, w, s) * psi(u, v, w, s), half)
            y = y + M.integrate(lambda u, v, w, s: fac(u, v, w, s) * psi(u, v, w, s), half)
            z = z + M.integrate(lambda u, v, w, s: heat(u, v, w, s) * fac(u, v, w, s)
                                * np.ones_like(u * v * w * s), half)
        X.append(x)
        Y.append(y)
        Z.append(z)
    tx, tw = leggauss(60)
    t = 0.5 * T * (tx + 1)
    wt = 0.5 * T * tw
    if tau > 0:
        e = np.exp(-t / tau)
        fns = [1 - e, (t + tau) * e - tau, t - tau + tau * e, e, -(tau + t) * e, -tau * e]
    else:
        fns = [np.ones_like(t), 0 * t, t, 0 * t, 0 * t, 0 * t]
    c = [np.sum(wt * f) for f in fns]
    Fb = sum(ci * xi for ci, xi in zip(c, X))
    Wb = sum(ci * yi for ci, yi in zip(c, Y))
    q = sum(ci * zi for ci, zi in zip(c, Z))
    FbPr = Fb.copy()
    FbPr[4] += (1 / Pr - 1) * q
    return Fb, Wb, FbPr, tau, W0


@pytest.mark.parametrize("inviscid", [1, 0])
def test_time_integrated_flux_matches_brute_force(orc, inviscid):
    rng = np.random.default_rng(23 + inviscid)
    gamma, Pr, mu0, C, eps = 1.4, 0.72, 2e-3, 10.0, 0.05
    for trial in range(2):
        pl = np.array([1.0, 0.3, -0.2, 0.1, 1.0]) + rng.uniform(-0.1, 0.1, 5)
        pr = np.array([0.8, 0.25, -0.1, 0.15, 0.85]) + rng.uniform(-0.1, 0.1, 5)
        sl = state(cons(*pl), cons_grad(pl, rng.normal(scale=0.5, size=(3, 5))))
        sr = state(cons(*pr), cons_grad(pr, rng.normal(scale=0.5, size=(3, 5))))
        dt = 0.01
        P = orc.params(gamma=gamma, Pr=Pr, mu0=mu0, C_tau=C, eps_tau=eps, inviscid=inviscid)
        for T in (dt, dt / 2):
            got = orc.fbar(P, sl, sr, dt, T)
            Fb, Wb, FbPr, tau, W0 = _brute_fbar(sl, sr, gamma=gamma, Pr=Pr, mu0=mu0, C=C,
                                                eps=eps, inviscid=inviscid, dt=dt, T=T)
            assert got[15] == pytest.approx(tau, rel=1e-12)
            scale = np.abs(FbPr).max()
            np.testing.assert_allclose(got[0:5], Fb, rtol=1e-10, atol=1e-12 * scale)
            np.testing.assert_allclose(got[5:10], Wb, rtol=1e-10, atol=1e-12 * np.abs(Wb).max())
            np.testing.assert_allclose(got[10:15], FbPr, rtol=1e-10, atol=1e-12 * scale)
            np.testing.assert_allclose(got[16], W0[0], rtol=1e-12)


def test_linearised_flux_reproduces_fbar(orc):
    """dt F^n + dt^2/2 F_t^n = Fbar(dt) for the linearisation in time."""
    rng = np.random.default_rng(3)
    pl = np.array([1.0, 0.2, 0.1, -0.1, 1.0])
    pr = np.array([0.7, 0.1, 0.0, 0.05, 0.6])
    sl = state(cons(*pl), cons_grad(pl, rng.normal(scale=0.5, size=(3, 5))))
    sr = state(cons(*pr), cons_grad(pr, rng.normal(scale=0.5, size=(3, 5))))
    for inviscid in (0, 1):
        P = orc.params(mu0=1e-3, inviscid=inviscid)
        dt = 0.02
        out = orc.flux_gp(P, sl, sr, dt)
        fb = orc.fbar(P, sl, sr, dt, dt)
        np.testing.assert_allclose(dt * out[:5] + 0.5 * dt * dt * out[5:10], fb[10:15],
                                   rtol=1e-12, atol=1e-15)


def test_mirror_symmetry_of_flux(orc):
    """Reflecting x -> -x swaps the sides and flips normal velocity and
    normal derivatives: the mass, tangential-momentum and energy fluxes
    change sign, the normal-momentum flux does not."""
    rng = np.random.default_rng(9)
    pl = np.array([1.0, 0.3, 0.2, -0.1, 1.0])
    pr = np.array([0.6, -0.2, 0.1, 0.3, 0.5])
    dl = rng.normal(scale=0.5, size=(3, 5))
    dr = rng.normal(scale=0.5, size=(3, 5))
    sl = state(cons(*pl), cons_grad(pl, dl))
    sr = state(cons(*pr), cons_grad(pr, dr))

    def mirror(prim, dprim):
        p2 = prim.copy()
        p2[1] = -p2[1]
        d2 = dprim.copy()
        d2[:, 1] = -d2[:, 1]   # U flips sign
        d2[0] = -d2[0]         # d/dx flips sign
        return state(cons(*p2), cons_grad(p2, d2))

    P = orc.params(mu0=1e-3)
    a = orc.flux_gp(P, sl, sr, 0.01)
    b = orc.flux_gp(P, mirror(pr, dr), mirror(pl, dl), 0.01)
    sgn = np.array([-1, 1, -1, -1, -1.0])
    np.testing.assert_allclose(b[:5], sgn * a[:5], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(b[5:10], sgn * a[5:10], rtol=1e-9, atol=1e-11)
    # interface values swap sides and the normal momentum flips
    flip = np.array([1, -1, 1, 1, 1.0])
    np.testing.assert_allclose(b[20:25], flip * a[10:15], rtol=1e-12)
    np.testing.assert_allclose(b[10:15], flip * a[20:25], rtol=1e-12)


def test_small_tau_is_continuous_with_zero_tau(orc):
    pl = np.array([1.0, 0.2, 0.1, -0.1, 1.0])
    pr = np.array([0.9, 0.15, 0.1, -0.05, 0.95])
    rng = np.random.default_rng(1)
    sl = state(cons(*pl), cons_grad(pl, rng.normal(scale=0.3, size=(3, 5))))
    sr = state(cons(*pr), cons_grad(pr, rng.normal(scale=0.3, size=(3, 5))))
    P0 = orc.params(inviscid=1, eps_tau=0.0, C_tau=0.0)
    P1 = orc.params(inviscid=1, eps_tau=1e-9, C_tau=0.0)
    a = orc.flux_gp(P0, sl, sr, 0.01)
    b = orc.flux_gp(P1, sl, sr, 0.01)
    np.testing.assert_allclose(a[:10], b[:10], rtol=1e-6, atol=1e-8)


def test_interface_values_blend(orc):
    """Sec. 3.4 update model of the interface values: with
    e = exp(-dt/tau0), tau0 = C |p_l - p_r|/(p_l + p_r) dt,
    Q^s = (1-e) W0 + e W_s and dQ^s/dt = (1-e) dW0/dt + e dW_s/dt, where
    the time derivatives are the Euler ones (-sum_j J_j dW/dx_j) of the
    interface equilibrium and of each one-sided state."""
    rng = np.random.default_rng(31)
    pl = np.array([1.0, 0.3, -0.2, 0.1, 1.0])
    pr = np.array([0.7, 0.1, 0.1, -0.2, 0.55])
    dWl = cons_grad(pl, rng.normal(scale=0.5, size=(3, 5)))
    dWr = cons_grad(pr, rng.normal(scale=0.5, size=(3, 5)))
    sl, sr = state(cons(*pl), dWl), state(cons(*pr), dWr)
    dt, C = 0.01, 10.0
    P = orc.params(mu0=1e-3, C_tau=C)
    out = orc.flux_gp(P, sl, sr, dt)
    Ml, Mr = Maxwellian(cons(*pl)), Maxwellian(cons(*pr))
    W0 = (Ml.integrate(lambda u, v, w, s: psi(u, v, w, s), +1)
          + Mr.integrate(lambda u, v, w, s: psi(u, v, w, s), -1))

    def slopes(M, dW):
        mm = M.integrate(lambda u, v, w, s: psi(u, v, w, s)[:, None] * psi(u, v, w, s)[None, :]) / M.rho
        return [np.linalg.solve(mm, dW[j] / M.rho) for j in range(3)]

    al, ar = slopes(Ml, dWl), slopes(Mr, dWr)
    dW0 = np.array([Ml.integrate(lambda u, v, w, s: apsi(al[j], u, v, w, s) * psi(u, v, w, s), +1)
                    + Mr.integrate(lambda u, v, w, s: apsi(ar[j], u, v, w, s) * psi(u, v, w, s), -1)
                    for j in range(3)])
    dtW0 = -sum(jacobian(W0, j) @ dW0[j] for j in range(3))
    dtWl = -sum(jacobian(cons(*pl), j) @ dWl[j] for j in range(3))
    dtWr = -sum(jacobian(cons(*pr), j) @ dWr[j] for j in range(3))
    e = math.exp(-1.0 / (C * abs(pl[4] - pr[4]) / (pl[4] + pr[4])))
    assert 0.05 < e < 0.95
    np.testing.assert_allclose(out[10:15], (1 - e) * W0 + e * cons(*pl), rtol=1e-12)
    np.testing.assert_allclose(out[20:25], (1 - e) * W0 + e * cons(*pr), rtol=1e-12)
    np.testing.assert_allclose(out[15:20], (1 - e) * dtW0 + e * dtWl, rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(out[25:30], (1 - e) * dtW0 + e * dtWr, rtol=1e-10, atol=1e-11)
