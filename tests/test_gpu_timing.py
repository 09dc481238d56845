"""gks_kernel_timing / gks_kernel_times: the per-kernel device time that the
benchmark reports for its roofline, recorded inside the timed steps. The
launch counts follow the step's structure, the times are positive, and the
recording changes no result."""
import numpy as np
import pytest

from paper_2508_19911_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("slab_planes", [0, 4])
def test_kernel_times_count_every_launch_and_change_nothing(slab_planes):
    torch = pytest.importorskip("torch")
    from paper_2508_19911_gb300 import gks
    dev = torch.device("cuda:0")
    Q, G, grid = wl.taylor_green(16)
    out = []
    for timed in (False, True):
        s = gks.Solver(gks.Config(n=grid.n, L=grid.L, scheme="cgks5", slab_planes=slab_planes))
        Qd, Gd = torch.tensor(Q, device=dev), torch.tensor(G, device=dev)
        if timed:
            s.kernel_timing(True)
        s.step(Qd, Gd, nsteps=2)
        if timed:
            t = s.kernel_times()
            slabs = 1 if s.slab_planes == 0 else -(-16 // s.slab_planes)
            assert t["recon"][1] == t["flux"][1] == 2 * 2 * slabs
            assert t["update"][1] == 4 and t["dt"][1] == 2
            assert all(ms > 0 for ms, _ in t.values())
            s.kernel_timing(False)
            s.step(Qd, Gd, nsteps=0)
            assert s.kernel_times() == t  # stopped: nothing new recorded
        out.append((Qd.cpu().numpy(), Gd.cpu().numpy()))
        s.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
