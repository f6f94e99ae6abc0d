"""Lead + RGF solve captured in a CUDA graph (GraphSolve) against eager calls.

The captured sequence runs the decimation a fixed number of steps with converged points masked
on the device (no host synchronisation); its results must equal the eager call with early
stopping, and replays after in-place input updates must follow the new inputs."""
import numpy as np
import pytest

from workloads import make_device

torch = pytest.importorskip("torch")
negf = pytest.importorskip("paper_1510_04686_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    negf._build.build()
    negf.library()


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_matches_eager(prec):
    N, b = 6, 24
    dev = make_device(N, b, 808)
    D = negf.Device(torch.as_tensor(dev.D[None], device="cuda"),
                    torch.as_tensor(dev.T[None], device="cuda"))
    E = torch.as_tensor(np.linspace(-1.2, 1.4, 9), device="cuda")
    st = torch.zeros(9, dtype=torch.int32, device="cuda")
    opt = negf.options(precision=prec)
    lead = negf.lead_selfenergy(D, E, st, opt)
    ref = negf.rgf_solve(D, E, st, lead["sigma_R"], lead["sigma_L"], opt)
    g = negf.GraphSolve(D, E, st, opt, sr_steps=60)
    out = g.replay()
    torch.cuda.synchronize()
    for k in ("density", "current", "transmission"):
        assert torch.equal(out[k], ref[k]), k
    assert torch.equal(g.lead["iters"], lead["iters"])
    # new energies written in place, replayed
    E.copy_(torch.as_tensor(np.linspace(-0.8, 0.9, 9), device="cuda"))
    out = g.replay()
    lead2 = negf.lead_selfenergy(D, E, st, opt)
    ref2 = negf.rgf_solve(D, E, st, lead2["sigma_R"], lead2["sigma_L"], opt)
    torch.cuda.synchronize()
    for k in ("density", "current", "transmission"):
        assert torch.equal(out[k], ref2[k]), k
