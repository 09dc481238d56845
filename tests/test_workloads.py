"""Properties of the seeded synthetic inputs (input generation only)."""
import numpy as np

from paper_2508_19911_gb300 import workloads as wl


def test_isotropic_turbulence_is_solenoidal_and_seeded():
    Q, G, grid, info = wl.isotropic_turbulence(32, Mt=0.5, k0=8, seed=101)
    # exact cell-averaged velocity gradients of a solenoidal field
    div = G[1, 0] + G[2, 1] + G[3, 2]
    assert np.abs(div).max() < 1e-12 * np.abs(G[1:4]).max()
    # Taylor microscale of the discrete field near 2/k0 = 0.25
    assert abs(info["taylor_lambda"] - 0.25) < 0.02
    # zero mean momentum, uniform density, reproducible
    assert np.abs(Q[1:4].mean(axis=(1, 2, 3))).max() < 1e-14
    assert np.all(Q[0] == 1.0)
    Q2, _, _, _ = wl.isotropic_turbulence(32, Mt=0.5, k0=8, seed=101)
    Q3, _, _, _ = wl.isotropic_turbulence(32, Mt=0.5, k0=8, seed=102)
    assert np.array_equal(Q, Q2) and not np.array_equal(Q, Q3)


def test_advection_exact_solution_is_a_translation():
    Q0, _, grid = wl.advection(12, dims=2)
    Q1, _, _ = wl.advection(12, dims=2, t=2 * np.pi / 2.0)  # (U + V) t = 2 pi: one period
    np.testing.assert_allclose(Q1, Q0, atol=1e-13)


def test_ensemble_instances_are_seeded_and_bounded():
    a = wl.ensemble_instances(6, seed0=2000, sizes=(8, 16))
    b = wl.ensemble_instances(6, seed0=2000, sizes=(8, 16))
    for (Qa, Ga, ga, pa), (Qb, Gb, gb, pb) in zip(a, b):
        assert ga.n == gb.n and pa == pb
        assert np.array_equal(Qa, Qb) and np.array_equal(Ga, Gb)
        assert ga.n[2] == 1 and ga.n[0] in (8, 16) and ga.n[1] in (8, 16)
        assert np.all(Qa[0] > 0)
    # Riemann half: quadrant density ratio within the bound (noise aside)
    for Q, G, g, ph in a[3:]:
        assert ph["inviscid"]
        assert Q[0].max() <= 5.0 * Q[0].min() * 1.25
