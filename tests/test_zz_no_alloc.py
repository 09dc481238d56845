"""gks_diagnostics_noalloc: the diagnostics entry point that allocates no
device memory, for callers that cannot (a monitor sampling a running
simulation that has filled the GPU, code that holds device pointers but no
gks_ctx). It must agree with gks_diagnostics, call after call, while its
scratch lives in a static device array shared by all calls.

This file is collected last on purpose; it passes run alone in a fresh
process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2508_19911_gb300 import workloads as wl


def _call(L, Qd, Gd, grid, gamma, mu, mu_law, T_ref, out, stream):
    return L.gks_diagnostics_noalloc(
        ctypes.c_void_p(Qd.data_ptr()),
        ctypes.c_void_p(Gd.data_ptr()) if Gd is not None else None,
        grid.n[0], grid.n[1], grid.n[2], grid.L[0], grid.L[1], grid.L[2],
        gamma, mu, mu_law, T_ref, ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(stream.cuda_stream))


def test_rejects_grids_beyond_the_cell_limit():
    from paper_2508_19911_gb300 import gks
    L = gks.lib()
    out = ctypes.c_void_p(8)  # never dereferenced: the size check comes first
    q = ctypes.c_void_p(8)
    rc = L.gks_diagnostics_noalloc(q, None, 2048, 2048, 1024, 1.0, 1.0, 1.0, 1.4, 1e-3, 0, 1.0,
                                   out, None)  # 2^32 cells
    assert rc == gks.GKS_ERR_ARG
    rc = L.gks_diagnostics_noalloc(q, None, 0, 8, 8, 1.0, 1.0, 1.0, 1.4, 1e-3, 0, 1.0, out, None)
    assert rc == gks.GKS_ERR_ARG


@pytest.mark.gpu
def test_noalloc_diagnostics_match_the_context_entry_point_and_the_oracle_twice():
    """Two calls in a row on each grid (they share the static scratch) equal
    gks_diagnostics bit for bit and the CPU oracle within 1e-12. The 128^3
    grid uses all 608 reduction blocks, more than the final block has
    threads, so its strided loop over the partial results runs."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_19911_gb300 import gks
    L = gks.lib()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    cases = [
        ("cgks5", wl.taylor_green((40, 36, 33)), dict(mu=1.0 / 1600, mu_law=0, T_ref=1.0)),
        ("gks2", wl.taylor_green_supersonic((21, 20, 19)), dict(mu=0.002, mu_law=1, T_ref=1.0)),
        ("cgks5", wl.taylor_green(128), dict(mu=1.0 / 1600, mu_law=1, T_ref=1.0)),
    ]
    for scheme, (Q, G, grid), phys in cases:
        Q, G = wl.perturb(Q, G, amp=0.02, seed=11)
        cg = scheme == "cgks5"
        s = gks.Solver(gks.Config(n=grid.n, L=grid.L, scheme=scheme, **phys), stream)
        Qd = torch.tensor(Q, device=dev)
        Gd = torch.tensor(G, device=dev) if cg else None
        ref = s.diagnostics(Qd, Gd)
        P = oracle.params(n=grid.n, L=grid.L, scheme=1 if cg else 0, mu0=phys["mu"],
                          mu_law=phys["mu_law"], T_ref=phys["T_ref"])
        want = oracle.diagnostics(P, Q, G if cg else None)
        for _ in range(2):  # two calls in a row share the static scratch
            out = torch.full((12,), float("nan"), dtype=torch.float64, device=dev)
            rc = _call(L, Qd, Gd, grid, 1.4, phys["mu"], phys["mu_law"], phys["T_ref"], out, stream)
            assert rc == gks.GKS_OK
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.array_equal(got, ref), (got, ref)
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14 * np.abs(want).max())
        s.close()
