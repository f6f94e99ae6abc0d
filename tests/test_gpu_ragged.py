"""Ragged block sizes (alloy samples with different cross-sections) through solve_ragged, which
stacks systems of equal (N, b) and runs the groups on concurrent streams, against one call per
system and the oracle."""
import numpy as np
import pytest

import oracle as O
from workloads import make_device

torch = pytest.importorskip("torch")
negf = pytest.importorskip("paper_1510_04686_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    negf._build.build()
    negf.library()


@pytest.mark.parametrize("prec", [0, 1])
def test_ragged_groups_match_single_calls(prec):
    specs = [(5, 24, 1), (5, 40, 2), (5, 24, 3), (4, 16, 4), (5, 40, 5)]
    devs = [make_device(N, b, 7000 + s, ge_frac=0.1) for (N, b, s) in specs]
    Es = [np.linspace(-1.0 + 0.1 * j, 1.0, 3 + j) for j in range(len(specs))]
    systems = [(torch.as_tensor(d.D, device="cuda"), torch.as_tensor(d.T, device="cuda"),
                torch.as_tensor(E, device="cuda")) for d, E in zip(devs, Es)]
    opt = negf.options(precision=prec)
    out = negf.solve_ragged(systems, opt)
    torch.cuda.synchronize()
    tol = 1e-9 if prec == 0 else 1e-6
    for d, E, r in zip(devs, Es, out):
        refs = [O.solve_point(d.D, d.T, e, 1e-6, None) for e in E]
        scale = max(np.abs(x["density"]).max() for x in refs)
        for p, x in enumerate(refs):
            assert np.abs(r["density"][p].cpu().numpy() - x["density"]).max() <= tol * scale
            assert abs(float(r["transmission"][p]) - x["transmission"]) <= tol * max(1.0, abs(x["transmission"]))


@pytest.mark.parametrize("prec", [0, 1])
def test_ragged_graph_replay_matches_oracle_per_block_size(prec):
    """The whole ragged batch (three block sizes, one of them shared by two samples, uneven
    energy counts) in one captured CUDA graph: every system's points match the oracle, equal
    solve_ragged run with the same fixed decimation, and a replay after the energies were
    changed in place follows the new energies."""
    specs = [(5, 40, 1), (5, 24, 2), (5, 56, 3), (5, 24, 4)]
    devs = [make_device(N, b, 7100 + s, ge_frac=0.1) for (N, b, s) in specs]
    Es = [np.linspace(-1.1 + 0.1 * j, 1.2, 4 + j) for j in range(len(specs))]
    systems = [(torch.as_tensor(d.D, device="cuda"), torch.as_tensor(d.T, device="cuda"),
                torch.as_tensor(E, device="cuda")) for d, E in zip(devs, Es)]
    opt = negf.options(precision=prec)
    rg = negf.RaggedGraph(systems, opt, sr_steps=60)
    out = rg.replay()
    ref = negf.solve_ragged(systems, negf.options(precision=prec, sr_host_check=0,
                                                  sr_max_iter=60))
    torch.cuda.synchronize()
    tol = 1e-9 if prec == 0 else 1e-6
    for d, E, r, q in zip(devs, Es, out, ref):
        for k in ("density", "current", "transmission"):
            assert torch.equal(r[k], q[k]), k
        assert int(r["status"].abs().sum()) == 0 and int(r["lead_status"].abs().sum()) == 0
        refs = [O.solve_point(d.D, d.T, e, 1e-6, None) for e in E]
        scale = max(np.abs(x["density"]).max() for x in refs)
        for p, x in enumerate(refs):
            assert np.abs(r["density"][p].cpu().numpy() - x["density"]).max() <= tol * scale
            assert abs(float(r["transmission"][p]) - x["transmission"]) <= \
                tol * max(1.0, abs(x["transmission"]))
    # new energies in place
    E2 = [np.linspace(-0.7, 0.8 + 0.05 * j, len(E)) for j, E in enumerate(Es)]
    for (_, _, Et), e in zip(systems, E2):
        Et.copy_(torch.as_tensor(e, device="cuda"))
    out = rg.replay()
    torch.cuda.synchronize()
    for d, E, r in zip(devs, E2, out):
        for p, e in enumerate(E):
            x = O.solve_point(d.D, d.T, e, 1e-6, None)
            assert abs(float(r["transmission"][p]) - x["transmission"]) <= \
                tol * max(1.0, abs(x["transmission"]))
