"""Brute-force velocity-space quadrature of Maxwellian moments.

Used by the CPU tests to pin the oracle's analytic moment recursions:
u by Gauss-Hermite (full line) or Gauss-Legendre on the half line,
v and w by Gauss-Hermite, the internal energy s = xi^2 of N internal
degrees of freedom by generalized Gauss-Laguerre (the integral over the
N-dimensional xi space of F(xi^2) times the normalised Gaussian reduces to
sum_i w_i F(x_i/lam)/Gamma(N/2) with Laguerre parameter N/2 - 1).
Nothing here calls the oracle.
"""
import math

import numpy as np
from numpy.polynomial.hermite import hermgauss
from numpy.polynomial.legendre import leggauss
from scipy.special import roots_genlaguerre

_HX, _HW = hermgauss(40)
_LX, _LW = leggauss(400)


class Maxwellian:
    def __init__(self, W, gamma=1.4):
        W = np.asarray(W, float)
        self.rho = W[0]
        self.U, self.V, self.Wv = W[1] / W[0], W[2] / W[0], W[3] / W[0]
        self.p = (gamma - 1.0) * (W[4] - 0.5 * self.rho * (self.U ** 2 + self.V ** 2 + self.Wv ** 2))
        self.lam = self.rho / (2.0 * self.p)
        self.N = (5.0 - 3.0 * gamma) / (gamma - 1.0)

    def _u_nodes(self, half):
        s = 1.0 / math.sqrt(self.lam)
        if half == 0:
            return self.U + _HX * s, _HW / math.sqrt(math.pi)
        if half > 0:
            a, b = 0.0, max(self.U + 18 * s, 0.0)
        else:
            a, b = min(self.U - 18 * s, 0.0), 0.0
        x = 0.5 * (a + b) + 0.5 * (b - a) * _LX
        g = math.sqrt(self.lam / math.pi) * np.exp(-self.lam * (x - self.U) ** 2)
        return x, 0.5 * (b - a) * _LW * g

    def integrate(self, fn, half=0):
        """rho * <fn(u, v, w, s)> over the full space or a half space in u.
        fn receives broadcastable node arrays and returns an array whose
        last four axes are (u, v, w, s)."""
        u, wu = self._u_nodes(half)
        s1 = 1.0 / math.sqrt(self.lam)
        hx, hw = hermgauss(12)
        v = self.V + hx * s1
        w = self.Wv + hx * s1
        wv = ww = hw / math.sqrt(math.pi)
        if self.N > 0:
            xs, ws = roots_genlaguerre(6, self.N / 2.0 - 1.0)
            s = xs / self.lam
            wsn = ws / math.gamma(self.N / 2.0)
        else:
            s, wsn = np.zeros(1), np.ones(1)
        U = u[:, None, None, None]
        V = v[None, :, None, None]
        Wn = w[None, None, :, None]
        S = s[None, None, None, :]
        vals = np.asarray(fn(U, V, Wn, S), float)
        wt = (wu[:, None, None, None] * wv[None, :, None, None] *
              ww[None, None, :, None] * wsn[None, None, None, :])
        return self.rho * np.sum(vals * wt, axis=(-4, -3, -2, -1))


def psi(u, v, w, s):
    """Collision invariants stacked on a leading axis of length 5."""
    one = np.ones(np.broadcast_shapes(np.shape(u), np.shape(v), np.shape(w), np.shape(s)))
    return np.stack([one, u * one, v * one, w * one, 0.5 * (u * u + v * v + w * w + s) * one])


def apsi(a, u, v, w, s):
    """a . psi for a 5-vector a."""
    p = psi(u, v, w, s)
    return np.tensordot(np.asarray(a, float), p, axes=(0, 0))
