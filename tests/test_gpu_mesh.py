"""Non-uniform energy meshes on the GPU: the interpolating Born update against the oracle, and an
adaptively refined mesh of a small resonant device whose points and energy integrals match the
oracle's at the same energies."""
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


def _t(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


@pytest.mark.parametrize("mix", [1.0, 0.4])
def test_scba_step_mesh_matches_oracle(mix):
    rng = np.random.default_rng(31)
    n_k, n_E, n_orb = 2, 57, 9
    E = np.sort(rng.uniform(-0.5, 0.5, n_E))
    dGR = rng.normal(size=(n_k, n_E, n_orb)) + 1j * rng.normal(size=(n_k, n_E, n_orb))
    dGL = 1j * rng.random((n_k, n_E, n_orb))
    wk = np.array([0.4, 0.6])
    sR0 = rng.normal(size=(n_E, n_orb)) * 1e-3 + 0j
    sL0 = 1j * rng.random((n_E, n_orb)) * 1e-3
    args = (0.01, 0.02, 0.06, 0.11)
    refR, refL, d_ref = O.scba_step_mesh(dGR, dGL, wk, E, *args, sR0, sL0, mix=mix)
    sR, sL = _t(sR0), _t(sL0)
    d = negf.scba_step_mesh(_t(dGR), _t(dGL), _t(wk), _t(E), sR, sL, *args, mix=mix)
    torch.cuda.synchronize()
    assert np.abs(sR.cpu().numpy() - refR).max() < 1e-15
    assert np.abs(sL.cpu().numpy() - refL).max() < 1e-15
    assert abs(float(d) - d_ref) < 1e-15


def test_adaptive_mesh_points_and_integrals_match_oracle():
    """A 5-slab, b = 24 device with eta = 1e-4 (sharp resonances): the mesh refined on T, slab
    electrons and bond currents; every point equals the oracle at the same energy (FP64 form,
    1e-9) and the mesh's trapezoid integrals equal the oracle's on that mesh."""
    dev = make_device(5, 24, 515)
    d = negf.Device(_t(dev.D[None]), _t(dev.T[None]))
    opt = negf.options(precision=negf.PREC_FP64, eta_lead=1e-4, eta_device=1e-4)
    r = negf.adaptive_energy_mesh(d, 0, opt, -1.0, 0.5, n_init=17, tol=1e-3, max_points=600)
    E, w = r["E"], r["w"]
    assert np.all(np.diff(E) > 0) and abs(w.sum() - 1.5) < 1e-13 and len(E) > 17
    # the mesh is not uniform: refined where the integrands vary fastest
    assert np.diff(E).min() <= 0.25 * np.diff(E).max()
    refs = [O.solve_point(dev.D, dev.T, float(e), 1e-4, None) for e in E]
    scale = max(np.abs(x["density"]).max() for x in refs)
    for p, x in enumerate(refs[::7]):
        q = 7 * p
        assert np.abs(r["density"][q] - x["density"]).max() <= 1e-9 * scale
        assert abs(r["transmission"][q] - x["transmission"]) <= 1e-9 * max(1.0, x["transmission"])
    n_ref = O.integrate([x["density"] for x in refs], w)
    assert np.abs(O.integrate(r["density"], w) - n_ref).max() <= 1e-9 * np.abs(n_ref).max()
