"""Learned smoothness indicator: training data from the method itself,
training on the GPU with the library's own kernels, evaluation.

The network predicts, per (cell, conserved variable), whether GENO's chi
would be 1 (within ``label_eps``), i.e. whether the CGKS-5th nonlinear
reconstruction reduces to the linear quartic; where it is confident
(sigmoid >= theta) the mixed-precision reconstruction skips the nonlinear
weights, everywhere else it runs them. Host code here only chooses
workloads and hyper-parameters; dumps, loss, gradients and Adam steps run
in libgks (gks_indicator_dump, gks_mlp_train).
"""
from __future__ import annotations

import math

import numpy as np

from . import gks
from . import workloads as wl

# label: GENO's chi within LABEL_EPS of 1; loss weight of label-0 samples;
# skip threshold on the network's sigmoid output (chosen on held-out data:
# 0.9 skipped 47% of the smooth samples but 5% of the others, 0.99 almost
# nothing; 0.97 in between keeps the false skips near 1%)
LABEL_EPS = 1e-3
NEG_WEIGHT = 1.0
THETA = 0.97


D = 63


def hidden_units() -> int:
    """Hidden width of the library's network (from its parameter count)."""
    return (gks.mlp_nparams() - 1) // (D + 2)


def init_params(seed: int = 0) -> np.ndarray:
    """He-initialised hidden layer, small output layer (float32)."""
    rng = np.random.default_rng(seed)
    H = hidden_units()
    W1 = rng.normal(scale=math.sqrt(2.0 / D), size=(H, D))
    b1 = np.zeros(H)
    w2 = rng.normal(scale=math.sqrt(1.0 / H), size=H)
    b2 = np.zeros(1)
    p = np.concatenate([W1.ravel(), b1, w2, b2]).astype(np.float32)
    assert p.size == gks.mlp_nparams()
    return p


def _snapshot_cases(n: int, seed: int):
    """(name, Q, G, grid, config kwargs, steps before the dump)."""
    cases = []
    Q, G, grid = wl.taylor_green(n)
    cases.append(("tgv", Q, G, grid, dict(mu=1.0 / 1600), (0, 8)))
    Q, G, grid = wl.taylor_green_supersonic(n)
    cases.append(("tgv_ma2", Q, G, grid, dict(mu=math.sqrt(1.4) * 2 / 1600, mu_law=1, Pr=0.7), (6,)))
    # shocklets (Mt = 1) with a spectrum peak of 8 cells per wavelength
    # (under-resolved: GENO active almost everywhere)
    Q, G, grid, _ = wl.isotropic_turbulence(n, Mt=1.0, k0=max(2.0, n / 8), seed=seed)
    cases.append(("hit_mt1", Q, G, grid, dict(mu=2e-3), (0, 6)))
    # Mt = 0.5 with 32 cells per peak wavelength (the resolution of the
    # 256^3, k0 = 8 turbulence workload)
    Q, G, grid, _ = wl.isotropic_turbulence(n, Mt=0.5, k0=n / 32, seed=seed + 7)
    cases.append(("hit_res", Q, G, grid, dict(mu=1e-3), (0, 10)))
    Q, G, grid = wl.double_sod(4 * n)
    cases.append(("sod", Q, G, grid, dict(inviscid=True, Pr=1.0), (10, 40)))
    return cases


def dump_set(device, n: int = 32, seed: int = 101):
    """Dump (x [63][M], chi [M], parts) from smooth, shocked and
    discontinuous flows advanced by the mixed-precision CGKS-5th solver;
    parts maps "workload@step" to its slice of the samples."""
    import torch
    xs, chis, parts, m = [], [], {}, 0
    for name, Q, G, grid, kw, snaps in _snapshot_cases(n, seed):
        s = gks.Solver(gks.Config(n=grid.n, L=grid.L, scheme="cgks5", precision="mixed", **kw))
        Qd = torch.tensor(Q, device=device)
        Gd = torch.tensor(G, device=device)
        done = 0
        for k in snaps:
            if k > done:
                try:
                    s.step(Qd, Gd, nsteps=k - done)
                except gks.GksError as e:
                    raise RuntimeError(f"training workload {name} at step {k}: {e}") from e
                done = k
            x, chi, _ = s.indicator_dump(Qd, Gd)
            xs.append(x)
            chis.append(chi.reshape(-1))
            parts[f"{name}@{k}"] = slice(m, m + chi.numel())
            m += chi.numel()
        s.close()
    xe, ce = ensemble_dump(device, seed0=seed + 1899)
    xs.append(xe)
    chis.append(ce)
    parts["ensemble"] = slice(m, m + ce.numel())
    return torch.cat(xs, dim=1).contiguous(), torch.cat(chis).contiguous(), parts


def labels(chi, label_eps: float = LABEL_EPS):
    """y = 1 where GENO's chi is within label_eps of 1 (skipping GENO there
    changes each face value by at most label_eps |P4 - P1|)."""
    return (chi >= 1.0 - label_eps).float()


def training_set(device, n: int = 32, seed: int = 101, label_eps: float = LABEL_EPS):
    """(x [63][M], y [M], label-1 fraction per workload)."""
    x, chi, parts = dump_set(device, n, seed)
    y = labels(chi, label_eps)
    stats = {k: float(y[sl].mean().item()) for k, sl in parts.items()}
    return x, y, stats


def ensemble_dump(device, count: int = 8, sizes=(32, 64), steps=(4, 12), seed0: int = 2000):
    """Data vectors and chi from a batched ensemble of 2D double shear
    layers and four-quadrant Riemann problems (the ensemble workload at
    reduced size), dumped by gks_ensemble_dump after each of ``steps``."""
    import torch
    insts = wl.ensemble_instances(count, seed0=seed0, sizes=sizes)
    spec = [dict(n=g.n, L=g.L, **ph) for _, _, g, ph in insts]
    e = gks.Ensemble(spec, precision="mixed")
    for i, (Q, G, _, _) in enumerate(insts):
        q, gg = e.views(i)
        q.copy_(torch.tensor(Q, device=device))
        gg.copy_(torch.tensor(G, device=device))
    xs, chis = [], []
    done = 0
    for k in steps:
        e.step(k - done)
        done = k
        x, chi, _ = e.dump()
        xs.append(x)
        chis.append(chi.reshape(-1))
    e.times()  # raises if any instance became non-physical
    e.close()
    return torch.cat(xs, dim=1).contiguous(), torch.cat(chis).contiguous()


def train(x, y, *, epochs: int = 8, batch: int = 4096, lr: float = 3e-3,
          neg_weight: float = NEG_WEIGHT, seed: int = 0):
    """Train a fresh network on (x, y) with the library's kernels."""
    import torch
    params = torch.tensor(init_params(seed), device=x.device)
    hist = gks.mlp_train(params, x, y, epochs=epochs, batch=batch, lr=lr,
                         neg_weight=neg_weight, seed=seed)
    return params, hist


def predict_logits(params, x):
    """Logits of the network for the samples x [63][M] (torch, for evaluation)."""
    import torch
    H = hidden_units()
    p = params.float()
    W1 = p[: H * D].view(H, D)
    b1 = p[H * D: H * D + H]
    w2 = p[H * D + H: H * D + 2 * H]
    b2 = p[-1]
    xh = x / (x.abs().amax(dim=0, keepdim=True) + 1e-30)
    h = torch.relu(W1 @ xh + b1[:, None])
    return (w2 @ h) + b2


def evaluate(params, x, y, theta: float = THETA):
    """Classification of the skip decision: skip rate on label-1 samples and
    false-skip rate on label-0 samples (where GENO is needed)."""
    import torch
    logit = predict_logits(params, x)
    skip = logit >= math.log(theta / (1.0 - theta)) if theta < 1 else torch.zeros_like(y, dtype=torch.bool)
    pos = y > 0.5
    neg = ~pos
    return {
        "skip_rate_on_smooth": float(skip[pos].float().mean().item()) if pos.any() else float("nan"),
        "false_skip_rate": float(skip[neg].float().mean().item()) if neg.any() else 0.0,
        "label_1_fraction": float(pos.float().mean().item()),
        "samples": int(y.numel()),
    }
