"""Pins of the oracle's indicator network: the loss against closed forms
(special weights where the network reduces to a hand-computable value) and
the gradient against central finite differences of that loss."""
import math

import numpy as np

D = 63


def shape(orc):
    npar = orc.lib().orc_mlp_nparams()
    H = (npar - 1) // (D + 2)
    assert H * D + 2 * H + 1 == npar
    return npar, H


def unpack(p, H):
    return p[:H * D].reshape(H, D), p[H * D:H * D + H], p[H * D + H:H * D + 2 * H], p[-1]


def softplus(z):
    return max(z, 0.0) + math.log1p(math.exp(-abs(z)))


def test_loss_closed_forms(orc):
    npar, H = shape(orc)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(D, 5))
    # W1 = 0: every hidden unit is relu(b1), the logit is the same for all samples
    p = np.zeros(npar)
    W1, b1, w2, _ = unpack(p, H)
    b1[:] = np.linspace(-1.0, 1.0, H)
    w2[:] = np.linspace(0.5, -0.25, H)
    p[-1] = 0.3
    logit = float(np.maximum(b1, 0.0) @ w2) + 0.3
    y = np.array([1.0, 0.0, 1.0, 0.0, 0.0])
    nw = 2.5
    expect = np.mean([(1.0 if yy else nw) * (softplus(logit) - yy * logit) for yy in y])
    loss, _ = orc.mlp_loss_grad(p, x, y, neg_weight=nw)
    assert abs(loss - expect) < 1e-14
    # one hidden unit that reads entry 7: logit = w2_0 relu(x7 / max|x|) + b2
    p = np.zeros(npar)
    W1, b1, w2, _ = unpack(p, H)
    W1[0, 7] = 1.0
    w2[0] = 2.0
    p[-1] = -0.5
    x = np.zeros((D, 2))
    x[7, 0], x[3, 0] = 0.5, -2.0      # x7 / max|x| = 0.25
    x[7, 1], x[9, 1] = -1.0, 0.5      # relu(-1) = 0
    y = np.array([1.0, 1.0])
    l0 = softplus(2.0 * 0.25 - 0.5) - (2.0 * 0.25 - 0.5)
    l1 = softplus(-0.5) - (-0.5)
    loss, _ = orc.mlp_loss_grad(p, x, y, neg_weight=1.0)
    assert abs(loss - 0.5 * (l0 + l1)) < 1e-14


def test_mlp_gradient_matches_finite_differences(orc):
    npar, H = shape(orc)
    rng = np.random.default_rng(3)
    params = rng.normal(scale=0.3, size=npar)
    n = 40
    x = rng.normal(size=(D, n)) * rng.uniform(0.01, 10, n)  # varied scales
    y = (rng.uniform(size=n) > 0.4).astype(float)
    loss, grad = orc.mlp_loss_grad(params, x, y, neg_weight=3.0)
    assert np.isfinite(loss) and loss > 0
    h = 1e-6
    idx = list(rng.choice(npar, 60, replace=False)) + [npar - 1, H * D, H * D + H]
    for p in idx:
        e = np.zeros(npar)
        e[p] = h
        lp, _ = orc.mlp_loss_grad(params + e, x, y, neg_weight=3.0)
        lm, _ = orc.mlp_loss_grad(params - e, x, y, neg_weight=3.0)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[p]) <= 1e-7 + 1e-6 * abs(fd), (p, fd, grad[p])


def test_mlp_scale_invariance(orc):
    """The network sees x / max|x|: scaling a sample leaves the loss unchanged."""
    npar, _ = shape(orc)
    rng = np.random.default_rng(4)
    params = rng.normal(scale=0.3, size=npar)
    x = rng.normal(size=(D, 10))
    y = np.ones(10)
    a, _ = orc.mlp_loss_grad(params, x, y)
    b, _ = orc.mlp_loss_grad(params, 1e3 * x, y)
    assert abs(a - b) < 1e-12
