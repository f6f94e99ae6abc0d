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
