"""z-slab execution of gks_step (large grids whose face-state buffer does not
fit next to the state): reconstruction and flux run slab by slab, each slab
also reconstructing the plane below it. Every cell and face is computed by
the same kernels as in whole-grid mode, so the results must be identical bit
for bit, whatever the slab size (including a remainder slab and slabs of
one plane)."""
import numpy as np
import pytest

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


def run(env, scheme, precision, slab_planes, steps=3):
    torch, dev, gks = env
    Q, G, grid = wl.taylor_green((12, 10, 9))
    Q, G = wl.perturb(Q, G, amp=0.03, seed=17)
    cg = scheme == "cgks5"
    s = gks.Solver(gks.Config(n=grid.n, L=grid.L, scheme=scheme, precision=precision,
                              slab_planes=slab_planes))
    Qd = torch.tensor(Q, device=dev)
    Gd = torch.tensor(G, device=dev) if cg else None
    s.step(Qd, Gd, nsteps=steps)
    return s, Qd, Gd


@pytest.mark.parametrize("scheme,precision", [("cgks5", "fp64"), ("cgks5", "mixed"),
                                              ("gks2", "fp64"), ("gks2", "mixed")])
@pytest.mark.parametrize("planes", [1, 2, 4, 9, 20])
def test_slabs_equal_whole_grid(env, scheme, precision, planes):
    torch, dev, gks = env
    _, Qw, Gw = run(env, scheme, precision, 0)
    _, Qs, Gs = run(env, scheme, precision, planes)
    assert torch.equal(Qw, Qs)
    if Gw is not None:
        assert torch.equal(Gw, Gs)


def test_slab_context_needs_caller_buffer(env):
    torch, dev, gks = env
    import ctypes
    s, Qd, Gd = run(env, "cgks5", "fp64", 2, steps=0)
    # the context's own buffer holds one slab: reconstructing the whole grid
    # into it is refused (GKS_ERR_STATE)
    rc = gks.lib().gks_reconstruct(s.ctx, ctypes.c_void_p(Qd.data_ptr()),
                                   ctypes.c_void_p(Gd.data_ptr()), None)
    assert rc == gks.GKS_ERR_STATE
    fs = s.reconstruct(Qd, Gd)   # a whole-grid buffer of the caller's: allowed
    assert fs.shape[-1] == Qd[0].numel()
