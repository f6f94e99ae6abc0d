"""Parity of the CUDA path (through the C ABI) with the CPU oracle, FP64 form.

Per-point outputs are compared element by element; the energy-integrated density and current
are held to the stated bar rel. err <= 1e-6 (infinity norm relative to the oracle's).
"""
import numpy as np
import pytest

import oracle as O
from workloads import make_device, chain_device, config_workload, energy_grid_linspace

torch = pytest.importorskip("torch")
negf = pytest.importorskip("paper_1510_04686_gb300")

pytestmark = pytest.mark.gpu
KT = O.KT_300K


@pytest.fixture(scope="module", autouse=True)
def _lib():
    negf._build.build()
    negf.library()


def _cuda(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def gpu_solve(Hds, Hus, E, sys, opt, V=None, scatR=None, scatL=None, e_idx=None, diag=False):
    Hd = _cuda(np.stack(Hds), torch.complex128)
    Hu = _cuda(np.stack(Hus), torch.complex128) if Hds[0].shape[0] > 1 else None
    dev = negf.Device(Hd, Hu)
    Et = _cuda(E, torch.float64)
    st = _cuda(sys, torch.int32)
    lead = negf.lead_selfenergy(dev, Et, st, opt)
    kw = {}
    if V is not None:
        kw["V"] = _cuda(V, torch.float64)
    if scatR is not None:
        kw["scat_R"] = _cuda(scatR, torch.complex128)
        kw["scat_L"] = _cuda(scatL, torch.complex128)
    if e_idx is not None:
        kw["e_idx"] = _cuda(e_idx, torch.int32)
    out = negf.rgf_solve(dev, Et, st, lead["sigma_R"], lead["sigma_L"], opt, diag=diag, **kw)
    torch.cuda.synchronize()
    res = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in out.items()}
    res["lead"] = {k: v.cpu().numpy() for k, v in lead.items()}
    return res


def oracle_solve(Hds, Hus, E, sys, eta, eta_lead, V=None, scatR=None, scatL=None, e_idx=None):
    outs = []
    for p, (e, s) in enumerate(zip(E, sys)):
        N, b = Hds[s].shape[0], Hds[s].shape[1]
        row = (e_idx[p] if e_idx is not None else p)
        sR = scatR[row].reshape(N, b) if scatR is not None else None
        sL = scatL[row].reshape(N, b) if scatL is not None else None
        outs.append(O.solve_point(Hds[s], Hus[s], e, eta, V, eta_lead=eta_lead, sR=sR, sL=sL))
    return outs


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _le(err, bound):
    # inclusive, so that exact zeros (e.g. no source on an N = 1 device) pass
    return err <= bound


def test_lead_selfenergy_matches_oracle():
    devs = [make_device(5, 8, 101), make_device(5, 8, 102)]
    E = np.array([-2.1, -0.7, 0.05, 0.9, 1.6, 2.8])
    sys = np.array([0, 1, 0, 1, 0, 1])
    opt = negf.options()
    r = gpu_solve([d.D for d in devs], [d.T for d in devs], E, sys, opt)
    for p, (e, s) in enumerate(zip(E, sys)):
        lo = O.lead_self_energies(devs[s].D, devs[s].T, e, 1e-6, 0.1, -0.1, KT)
        assert _rel(r["lead"]["sigma_R"][p, 0], lo["sigL"]) < 1e-9
        assert _rel(r["lead"]["sigma_R"][p, 1], lo["sigR"]) < 1e-9
        assert _rel(r["lead"]["sigma_L"][p, 0], lo["lesL"]) < 1e-9
        assert _rel(r["lead"]["sigma_L"][p, 1], lo["lesR"]) < 1e-9
        assert abs(int(r["lead"]["iters"][p, 0]) - lo["itL"]) <= 1
        assert r["lead"]["status"][p] == 0


@pytest.mark.parametrize("N,b", [(1, 6), (2, 3), (6, 8), (4, 33)])
def test_rgf_matches_oracle(N, b):
    devs = [make_device(N, b, 200 + N + b), make_device(N, b, 300 + N + b, ge_frac=0.3)]
    E = np.array([-1.9, -0.33, 0.02, 0.41, 1.27])
    sys = np.array([0, 1, 1, 0, 1])
    V = np.random.default_rng(1).uniform(-0.3, 0.3, (N, b))
    opt = negf.options()
    r = gpu_solve([d.D for d in devs], [d.T for d in devs], E, sys, opt, V=V, diag=True)
    ref = oracle_solve([d.D for d in devs], [d.T for d in devs], E, sys, 1e-6, 1e-6, V=V)
    # roundoff is judged against each quantity's scale over all points of the batch
    dscale = max(np.abs(o["density"]).max() for o in ref)
    rscale = max(np.abs(o["diagGR"]).max() for o in ref)
    lscale = max(np.abs(o["diagGL"]).max() for o in ref)
    for p, o in enumerate(ref):
        assert r["status"][p] == 0
        assert _le(np.abs(r["density"][p] - o["density"]).max(), 1e-9 * dscale)
        assert _le(np.abs(r["diagGR"][p] - o["diagGR"]).max(), 1e-9 * rscale)
        assert _le(np.abs(r["diagGL"][p] - o["diagGL"]).max(), 1e-9 * lscale)
        assert abs(r["transmission"][p] - o["transmission"]) < 1e-8 * max(1.0, abs(o["transmission"]))
        if N > 1:
            assert _le(np.abs(r["current"][p] - o["current"]).max(), 1e-9 * lscale)


def test_rgf_blocked_inverse_path():
    # b = 130 does not fit one CTA's shared memory in FP64 and takes the panel path
    N, b = 3, 130
    dev = make_device(N, b, 77)
    E = np.array([-0.5, 0.3, 1.1])
    opt = negf.options()
    r = gpu_solve([dev.D], [dev.T], E, np.zeros(3, int), opt, diag=True)
    ref = oracle_solve([dev.D], [dev.T], E, [0, 0, 0], 1e-6, 1e-6)
    rscale = max(np.abs(o["diagGR"]).max() for o in ref)
    dscale = max(np.abs(o["density"]).max() for o in ref)
    for p, o in enumerate(ref):
        assert np.abs(r["diagGR"][p] - o["diagGR"]).max() <= 1e-9 * rscale
        assert np.abs(r["density"][p] - o["density"]).max() <= 1e-9 * dscale
        assert abs(r["transmission"][p] - o["transmission"]) < 1e-8


def test_rgf_with_scattering_rows():
    N, b = 4, 6
    dev = make_device(N, b, 88)
    E = np.array([-0.8, -0.1, 0.6, 0.9])
    rng = np.random.default_rng(2)
    n_rows = 3
    gam = 0.04 * rng.random((n_rows, N * b))
    scatR = 0.01 * rng.normal(size=(n_rows, N * b)) - 1j * gam
    scatL = 1j * 0.6 * 2 * gam
    e_idx = np.array([2, 0, 1, 2])
    opt = negf.options()
    r = gpu_solve([dev.D], [dev.T], E, np.zeros(4, int), opt, scatR=scatR, scatL=scatL,
                  e_idx=e_idx, diag=True)
    ref = oracle_solve([dev.D], [dev.T], E, [0] * 4, 1e-6, 1e-6, scatR=scatR, scatL=scatL,
                       e_idx=e_idx)
    dscale = max(np.abs(o["density"]).max() for o in ref)
    lscale = max(np.abs(o["diagGL"]).max() for o in ref)
    for p, o in enumerate(ref):
        assert np.abs(r["density"][p] - o["density"]).max() <= 1e-9 * dscale
        assert np.abs(r["current"][p] - o["current"]).max() <= 1e-9 * lscale


def test_chain_transmission_on_gpu():
    ch = chain_device(6, 0.0, 1.0)
    E = np.array([-2.5, -1.7, -0.3, 0.6, 1.95, 2.2])
    opt = negf.options(eta_lead=1e-9, eta_device=0.0)
    r = gpu_solve([ch.D], [ch.T], E, np.zeros(len(E), int), opt)
    expect = (np.abs(E) < 2.0).astype(float)
    assert np.abs(r["transmission"] - expect).max() < 1e-6
    # Landauer: every bond carries (f_L - f_R) T
    df = O.fermi(E, 0.1, KT) - O.fermi(E, -0.1, KT)
    assert np.abs(r["current"] - (df * r["transmission"])[:, None]).max() < 1e-9


def test_chunking_is_invisible():
    N, b = 5, 7
    dev = make_device(N, b, 99)
    E = np.linspace(-1.5, 1.5, 7)
    a = gpu_solve([dev.D], [dev.T], E, np.zeros(7, int), negf.options(chunk=3))
    c = gpu_solve([dev.D], [dev.T], E, np.zeros(7, int), negf.options())
    assert np.array_equal(a["density"], c["density"])
    assert np.array_equal(a["current"], c["current"])


def test_fp64_is_deterministic():
    N, b = 6, 20
    dev = make_device(N, b, 5)
    E = np.linspace(-1.0, 1.0, 5)
    a = gpu_solve([dev.D], [dev.T], E, np.zeros(5, int), negf.options())
    c = gpu_solve([dev.D], [dev.T], E, np.zeros(5, int), negf.options())
    for k in ("density", "current", "transmission"):
        assert np.array_equal(a[k], c[k])


def test_decimation_cap_reports_not_converged():
    dev = make_device(4, 5, 6)
    E = np.array([0.1, 0.2])
    r = gpu_solve([dev.D], [dev.T], E, np.zeros(2, int), negf.options(sr_max_iter=1))
    assert np.all(r["lead"]["status"] & 1)
    assert np.all(r["lead"]["iters"] == 1)


def test_config0_integrated_parity():
    """The small ballistic workload: N = 20, b = 40, 64 energies in [-3, 3], eta = 1e-6, one
    k-point."""
    w = config_workload(0)
    dev = w["device"]
    E, wE = w["E"], w["wE"]
    opt = negf.options()
    r = gpu_solve([dev.D], [dev.T], E, np.zeros(len(E), int), opt)
    ref = oracle_solve([dev.D], [dev.T], E, [0] * len(E), 1e-6, 1e-6)
    n_ref = O.integrate([o["density"] for o in ref], wE)
    j_ref = O.integrate([o["current"] for o in ref], wE)
    n_gpu = O.integrate(r["density"], wE)
    j_gpu = O.integrate(r["current"], wE)
    assert _rel(n_gpu, n_ref) < 1e-6
    assert _rel(j_gpu, j_ref) < 1e-6
    T_ref = np.array([o["transmission"] for o in ref])
    assert np.abs(r["transmission"] - T_ref).max() < 1e-6 * max(1.0, np.abs(T_ref).max())
    assert np.all(r["status"] == 0)


def test_integrate_matches_oracle():
    rng = np.random.default_rng(3)
    vals = rng.normal(size=(9, 13))
    w = rng.random(9)
    grp = np.array([0, 1, 0, 2, 1, 0, 2, 2, 1])
    out = negf.integrate(_cuda(vals, torch.float64), _cuda(w, torch.float64),
                         _cuda(grp, torch.int32), 3).cpu().numpy()
    for g in range(3):
        m = grp == g
        assert np.allclose(out[g], O.integrate(vals[m], w[m]), rtol=1e-14, atol=1e-15)


def test_scba_step_matches_oracle():
    rng = np.random.default_rng(4)
    n_k, n_E, n_orb, sh, n0 = 3, 40, 11, 5, 0.1089
    dGR = rng.normal(size=(n_k, n_E, n_orb)) + 1j * rng.normal(size=(n_k, n_E, n_orb))
    dGL = 1j * rng.random((n_k, n_E, n_orb))
    wk = rng.random(n_k)
    oldR = rng.normal(size=(n_E, n_orb)) + 1j * rng.normal(size=(n_E, n_orb))
    oldL = 1j * rng.random((n_E, n_orb))
    for mix in (1.0, 0.3):
        sR = _cuda(oldR, torch.complex128)
        sL = _cuda(oldL, torch.complex128)
        d = negf.scba_step(_cuda(dGR, torch.complex128), _cuda(dGL, torch.complex128),
                           _cuda(wk, torch.float64), sR, sL, 0.01, 0.02, sh, n0, mix)
        eR, eL, ed = O.scba_step(dGR, dGL, wk, 0.01, 0.02, sh, n0, oldR, oldL, mix)
        assert np.abs(sR.cpu().numpy() - eR).max() < 1e-14 * np.abs(eR).max()
        assert np.abs(sL.cpu().numpy() - eL).max() < 1e-14 * np.abs(eL).max()
        assert abs(float(d.cpu()) - ed) < 1e-13 * ed
